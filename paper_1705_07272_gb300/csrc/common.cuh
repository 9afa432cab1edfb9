// Shared declarations of the sm_103a Haar phase-shift library: the plan,
// per-shift parameter records and small device helpers.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "../../include/haarshift.h"

namespace hs {

// Per-shift record built in FP64 by the set-up kernel (the per-launch
// construction of the shift's mixing weights; the "rotation input pass" of
// Sec. "Experimental results").
struct ShiftParam {
  int kx, ky;                // integer part of the translation (kx in [0,W), ky in [0,period))
  float wx0, wx1, wy0, wy1;  // bilinear weights: g = wy0 (wx0 F[i-ky][j-kx] + wx1 F[i-ky][j-kx-1])
                             //                    + wy1 (wx0 F[i-ky-1][j-kx] + wx1 F[i-ky-1][j-kx-1])
  uint32_t perm_mask;        // bit l (1..n): level l is a signed permutation; bit n+1: scaling
  int order;                 // translations: record y's `order` is the shift that CTA row y of the
                             // 8 x 8-block batch kernel takes (shifts grouped by column phase)
  float R[9];                // rotation p' = R p (row-major), float32
  float a_px;                // rotations: a / dphi - 1/2 for R = Ry(a) Rx(b) Ry(c) (picks anchor columns)
  float pad2[2];
};
static_assert(sizeof(ShiftParam) == 80, "ShiftParam layout");

struct Geometry {
  int H, W, C, n, q;
  int T, Lt;                 // tile side and the number of levels done inside a tile
  int tiles_r, tiles_c, n_tiles;
  int boundary;
  long long N;               // H * W
};

// Tile side: 64 x 64 output tiles unless that leaves too few CTAs for the
// machine (small maps with few shifts), then 32 x 32.
static inline int choose_tile(int H, int W, int C, int S) {
  const long long t64 = (H >= 64) ? (long long)(H / 64) * (W / 64) : 1;
  return (t64 * C * S >= 640) ? 64 : 32;
}

static inline Geometry make_geometry(int H, int W, int C, int boundary, int tile = 64) {
  Geometry g;
  g.H = H; g.W = W; g.C = C; g.boundary = boundary;
  int n = 0;
  while ((1 << n) < H) ++n;
  g.n = n;
  g.q = W / H;
  g.T = H < tile ? H : tile;
  int lt = 0;
  while ((1 << lt) < g.T) ++lt;
  g.Lt = lt;
  g.tiles_r = H / g.T;
  g.tiles_c = W / g.T;
  g.n_tiles = g.tiles_r * g.tiles_c;
  g.N = (long long)H * W;
  return g;
}

}  // namespace hs

struct haar_shift_plan_s {
  haar_shift_desc_t desc;
  hs::Geometry geo;          // of the map the shift runs on (the level-k scaling image for start_level k)
  int K;                     // coefficients written per (s, c)
  long long cin_stride;      // floats between the channels of coeffs_in (the full map's N)
  double pscale;             // translation scale 2^-start_level
  int device;
  // workspace (device)
  float* pix;                // [C][H][W] pixel map synthesised per launch
  float* pixE;               // translation batches: the map extended to [C][pixE_H][pixE_W] (rows past the
                             // poles mirrored half a turn, one period plus a window's rows; columns wrapped
                             // plus a window's width), so that every tile's source window is one TMA box
  int pixE_H, pixE_W;
  float* trig;               // rotation tables of the map: see trig_floats()
  float* rtab;               // rotation kinds: per-rotation tables [max_shifts][rot_table_float4s] float4
  hs::ShiftParam* prm;       // [max_shifts]
  float* means;              // [max_shifts][C][n_tiles] (or [max_shifts][C][H W / 256] for the KSC kernel)
  size_t means_cap;          // floats in means
  unsigned* counters;        // [max_shifts]
  void* light;               // shade_batch lighting [max_shifts * C * K] (x2 planes for BF16_HILO)
  size_t light_elems;        // elements per plane
  int* status;               // device status word (0 = fine)
  float* chain_ws;           // ROTATE_CHAIN: [max_shifts][C][4][N] derivative fields, rotations, angle tables
};

namespace hs {

// Rotation tables of a map (plan->trig): [H] float4 (sin theta_i hi, lo,
// cos theta_i hi, lo), then [W] float4 (sin phi_j hi, lo, cos phi_j hi, lo),
// built in FP64.
__host__ __device__ __forceinline__ long long trig_floats(int H, int W) { return 4LL * (H + W); }
// Per-rotation tables (float4): sin/cos psi_j [W], sin/cos alpha_m [W], rows [2H].
__host__ __device__ __forceinline__ long long rot_table_float4s(int H, int W) { return 2LL * W + 2LL * H; }
// Pixel map floats the set-up synthesises: rotations read an interleaved map
// [ceil(C/3)][H][W][8] (each texel holds three channels at columns j and j+1).
__host__ __device__ __forceinline__ long long pix_floats(int kind, int H, int W, int C) {
  const long long N = (long long)H * W;
  return (kind == HAAR_SHIFT_ROTATE || kind == HAAR_SHIFT_ROTATE_EULER) ? 8LL * N * ((C + 2) / 3) : N * C;
}

// atan2(y, x) in [-pi, pi]: reduction to t = min(|x|, |y|) / max(|x|, |y|)
// in [0, 1], atan(t) = t P(t^2) with P of degree 7 (Lawson's minimax fit,
// tests/atan_fit.py: |error| < 1.5e-7 rad when evaluated in FP32), then the
// reflections atan(y/x) = pi/2 - atan(x/y) and the half-plane x < 0.  (0, 0)
// gives 0.
__device__ __forceinline__ float rot_atan2(float y, float x) {
  const float ax = fabsf(x), ay = fabsf(y);
  const float mx = fmaxf(ax, ay), mn = fminf(ax, ay);
  const float t = (mx > 0.0f) ? __fdividef(mn, mx) : 0.0f;
  const float u = t * t;
  constexpr float P[8] = {9.999993356e-01f, -3.332986071e-01f, 1.994656467e-01f, -1.390862427e-01f, 9.642182932e-02f, -5.591211863e-02f, 2.186280589e-02f, -4.054523135e-03f};
  float p = P[7];
#pragma unroll
  for (int i = 6; i >= 0; --i) p = fmaf(p, u, P[i]);
  float r = t * p;
  if (ay > ax) r = 1.57079632679f - r;
  if (x < 0.0f) r = 3.14159265359f - r;
  return copysignf(r, y);
}

// Programmatic dependent launch: a kernel launched this way may be scheduled
// while the previous kernel of the stream finishes its last CTAs (which call
// pdl_trigger() once their outputs are final, or exit); it calls pdl_wait()
// before it reads anything that kernel wrote.  Without a dependency (first
// kernel, or a plain launch before it) both are no-ops.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
static inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                                     cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Paired FP32 arithmetic of sm_100+ (fma.rn.f32x2): two lanes of a 64-bit
// register pair per instruction, each rounded like fmaf.
__device__ __forceinline__ unsigned long long f2_dup(float a) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %1};" : "=l"(r) : "f"(a));
  return r;
}
__device__ __forceinline__ unsigned long long f2_fma(unsigned long long a, unsigned long long b,
                                                     unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ unsigned long long f2_add(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ unsigned long long f2_shfl_xor(unsigned long long a, int o) {
  return __shfl_xor_sync(0xffffffffu, a, o);
}

__device__ __forceinline__ unsigned long long f2_mul(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ unsigned long long f2_pack(float x, float y) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(x), "f"(y));
  return r;
}
__device__ __forceinline__ float2 u2f(unsigned long long a) {
  float2 f;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(f.x), "=f"(f.y) : "l"(a));
  return f;
}

// status helpers (abi.cu)
haar_status_t set_error(haar_status_t st, const char* fmt, ...);
void clear_error();
haar_status_t cuda_check(cudaError_t e, const char* what);
bool injected(const char* entry);

// launchers (shift.cu)
// translation plans whose batches run the 8 x 8-block kernel from the extended map
bool tr8_tma_plan(const haar_shift_desc_t& d, const Geometry& g, int K, int max_shifts);
haar_status_t launch_setup(haar_shift_plan_s* p, const float* coeffs_in, const double* params, const void* out,
                           int S, cudaStream_t st);
haar_status_t launch_shift(haar_shift_plan_s* p, const float* coeffs_in, int S, void* out,
                           cudaStream_t st);
haar_status_t launch_trig(haar_shift_plan_s* p, cudaStream_t st);
haar_status_t launch_chain(haar_shift_plan_s* p, const double* params, int S, void* out,
                           cudaStream_t st);                                           // chain.cu
size_t chain_ws_floats(const Geometry& g, int S);                                      // chain.cu
haar_status_t launch_normal_rotations(int V, const float* nrm, double* params, cudaStream_t st);  // triple.cu
haar_status_t launch_triple(int H, int W, int C, int V, const float* light, const float* brdf, long long sb,
                            const float* vis, long long sv, float* out, float* work, cudaStream_t st);
long long triple_work_floats(int H, int W, int C);
long long shade_triple_work_floats(int H, int W, int C);
haar_status_t launch_rasterize(int V, const float* pos, int T, const int32_t* tris, const float* M, int width,
                               int height, float* screen, unsigned long long* zbuf, int32_t* tri_id, float* bary,
                               cudaStream_t st);                                     // raster.cu
haar_status_t launch_shade_pixels(int width, int height, int C, int V, int T, const int32_t* tri_id,
                                  const float* bary, const int32_t* tris, const float* rad, const float* bg,
                                  float* img, cudaStream_t st);
haar_status_t launch_shade_triple(int H, int W, int C, int V, const float* light, const float* brdf_local,
                                  const double* params, const float* vis, long long sv, float* out, float* work,
                                  cudaStream_t st);
bool ksc_eligible(const haar_shift_desc_t& d, const Geometry& g, int S);
size_t ksc_means_floats(const Geometry& g, int S);
size_t ksc_smem_floats(long long n16, int planes);
haar_status_t launch_forward(int H, int W, int batch, const float* maps, float* coeffs,
                             float scale, cudaStream_t st);
haar_status_t launch_inverse(int H, int W, int batch, const float* coeffs, float* maps,
                             cudaStream_t st);

// launchers (shade.cu)
haar_status_t launch_shade_dense_f32(const float* T, int V, int K, const float* L, int ldl,
                                     int ncols, float* R, cudaStream_t st);
haar_status_t launch_shade_csr_f32(const float* vals, const uint16_t* idx, const int32_t* rowptr,
                                   int V, const float* L, int NL, int ncols, float* R, cudaStream_t st);
haar_status_t launch_shade_bincsr_f16(const __half* vals, const uint32_t* idx, const uint8_t* bin_of,
                                      int V, int bins, int K, int S, int C, const float* L,
                                      long long NL, bool vec4, float* R, cudaStream_t st);
haar_status_t launch_shade_gcsr_f32(const float* vals, const uint16_t* idx, const int32_t* gptr, int V,
                                    const float* L, int NL, int ncols, float* R, int* status, cudaStream_t st);
haar_status_t launch_gcsr_pack(int V, int N, const int32_t* rowptr, const uint16_t* idx, const float* vals,
                               int32_t* gptr, uint16_t* gidx, float* gvals, cudaStream_t st);
haar_status_t launch_view_bins(int V, int S, int bins, const float* pos, const float* nrm,
                               const float* cams, const float* bin_dirs, uint8_t* bin_of,
                               cudaStream_t st);

// tensor-core contraction (gemm_tc.cu)
haar_status_t launch_shade_dense_bf16_tc(const __nv_bfloat16* T, int V, int K,
                                         const __nv_bfloat16* Lhi, const __nv_bfloat16* Llo,
                                         int ncols, float* R, int* status, cudaStream_t st);

}  // namespace hs
