// Transport surrogate on sm_103a: a 4 x 256 GELU MLP that maps a vertex's
// position, normal and view direction to its Haar transport coefficients at a
// fixed index set, with BF16 tensor-core (tcgen05) forward and backward
// GEMMs, FP32 accumulation, FP32 master weights and Adam, and an inference
// path whose last hidden layer's epilogue performs the double product with
// the shifted lighting directly (the output layer folded into the lighting).
//
// Encoding (9 inputs): x, then sin(w_f x), cos(w_f x) for w_f = pi 2^(f/2),
// f = 0..15 (297 features, zero-padded to 320).  GELU in its tanh form.  Flat parameter layout:
// W1[256][320] b1[256] W2[256][256] b2 W3 b3 W4 b4 Wo[512][256] bo[512].
#include <math.h>
#include <string.h>

#include <new>

#include "tc.cuh"

namespace hs {
namespace mlpk {

constexpr int N_RAW = 9, N_FREQ = 16, N_IN = 320, WIDTH = 256, N_OUT = 512, N_LAYERS = 5;
constexpr int THREADS = 192;

__host__ __device__ constexpr int fan_in(int l) { return l == 0 ? N_IN : WIDTH; }
__host__ __device__ constexpr int fan_out(int l) { return l == N_LAYERS - 1 ? N_OUT : WIDTH; }
__host__ __device__ inline long long w_off(int l) {
  long long o = 0;
  for (int i = 0; i < l; ++i) o += (long long)fan_out(i) * fan_in(i) + fan_out(i);
  return o;
}
__host__ __device__ inline long long b_off(int l) { return w_off(l) + (long long)fan_out(l) * fan_in(l); }
constexpr long long N_PARAMS = (long long)WIDTH * N_IN + WIDTH + 3LL * (WIDTH * WIDTH + WIDTH) +
                               (long long)N_OUT * WIDTH + N_OUT;

enum Epi { EPI_F32 = 0, EPI_BIAS_GELU = 1, EPI_GELU_BWD = 2, EPI_SHADE = 3 };

struct EpiArgs {
  int M, N;
  const float* bias;
  float* out_f32;          // EPI_F32: out[m][n]; EPI_BIAS_GELU: pre-activation z (optional)
  int ld_f32;
  __nv_bfloat16* out_bf16; // EPI_BIAS_GELU: gelu(z); EPI_GELU_BWD: dz
  int ld_bf16;
  const float* zprev;      // EPI_GELU_BWD: pre-activation of the layer below
  int ld_zprev;
  const float* weff;       // EPI_SHADE: [groups][N][C]
  const float* beff;       // EPI_SHADE: [groups][C]
  int rows_per_group, groups, C, row0;
  float* radiance;         // EPI_SHADE: R[v][s][c], row m + row0 = s * rows_per_group + v
  float* split_ws;         // EPI_F32 split-K partial sums [splits][M][N] (null: no split)
  long long split_ws_floats;
};

// GELU in its tanh form (Hendrycks and Gimpel 2016), with the hardware tanh
// approximation (tanh.approx.f32, relative error ~2^-11, below the bf16
// rounding of the stored activations).
__device__ __forceinline__ float tanh_fast(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
constexpr float kGeluA = 0.79788456080286536f;   // sqrt(2 / pi)
constexpr float kGeluB = 0.044715f;
__device__ __forceinline__ float gelu(float z) {
  const float t = tanh_fast(kGeluA * fmaf(kGeluB * z, z * z, z));
  return 0.5f * z * (1.0f + t);
}
// GELU of two values in one register pair (paired FP32 arithmetic; the two
// tanh go through the SFU one by one)
__device__ __forceinline__ unsigned long long gelu2(unsigned long long z) {
  const unsigned long long u = f2_mul(z, z);
  const unsigned long long t = f2_fma(u, f2_dup(kGeluA * kGeluB), f2_dup(kGeluA));   // A (1 + B z^2)
  const float2 arg = u2f(f2_mul(t, z));                                                 // A (z + B z^3)
  const unsigned long long th = f2_pack(tanh_fast(arg.x), tanh_fast(arg.y));
  const unsigned long long hz = f2_mul(z, f2_dup(0.5f));
  return f2_fma(hz, th, hz);                                                            // z (1 + tanh) / 2
}
__device__ __forceinline__ float gelu_grad(float z) {
  const float t = tanh_fast(kGeluA * fmaf(kGeluB * z, z * z, z));
  return 0.5f * (1.0f + t) + 0.5f * z * (1.0f - t * t) * kGeluA * fmaf(3.0f * kGeluB, z * z, 1.0f);
}

struct __align__(8) GBars {
  uint64_t full[tc::MAX_STAGES];
  uint64_t empty[tc::MAX_STAGES];
  uint64_t tfull;
  uint64_t drain;
  uint32_t tmem_base;
  int abort_flag;
};

// C[M][N] = A[M][K] . B[N][K]^T, one 128 x BN tile per CTA; warp 0 TMA
// producer, warp 1 MMA issuer, warps 2-5 epilogue.
template <int EPI>
__global__ void __launch_bounds__(THREADS, 1)
k_gemm(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, int K, int BN,
       int STAGES, int tmem_cols, EpiArgs e, int* status) {
  // split-K: CTA z accumulates k-blocks [z * kbs, (z + 1) * kbs); EPI_F32 adds
  // its partial sums atomically into a zeroed output
  using namespace tc;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  __shared__ GBars bars;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  const uint32_t a_bytes = BM * BK * 2, b_bytes = (uint32_t)BN * BK * 2;
  const uint32_t stage_bytes = a_bytes + b_bytes;
  const int kbs = (K / BK + gridDim.z - 1) / gridDim.z;
  const int kb0 = blockIdx.z * kbs;
  const int kblocks = min(kbs, K / BK - kb0);
  const int tm = blockIdx.x, tn = blockIdx.y;
  volatile int* abort_flag = &bars.abort_flag;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(smem_u32(&bars.full[s]), 1);
      mbar_init(smem_u32(&bars.empty[s]), 1);
    }
    mbar_init(smem_u32(&bars.tfull), 1);
    mbar_init(smem_u32(&bars.drain), 1);
    bars.abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&bars.tmem_base)),
                 "r"(tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = bars.tmem_base;

  if (warp == 0) {
    if (lane == 0) {
      int issued[MAX_STAGES];
      uint32_t issued_phase[MAX_STAGES];
      for (int i = 0; i < MAX_STAGES; ++i) { issued[i] = 0; issued_phase[i] = 0; }
      int stage = 0;
      uint32_t phase = 0;
      for (int kb = 0; kb < kblocks; ++kb) {
        if (!mbar_wait(smem_u32(&bars.empty[stage]), phase ^ 1u, status, abort_flag)) break;
        const uint32_t sa = base + stage * stage_bytes;
        const uint32_t fb = smem_u32(&bars.full[stage]);
        mbar_arrive_tx(fb, stage_bytes);
        tma_load_2d(sa, &mapA, (kb0 + kb) * BK, tm * BM, fb);
        tma_load_2d(sa + a_bytes, &mapB, (kb0 + kb) * BK, tn * BN, fb);
        issued[stage] = 1;
        issued_phase[stage] = phase;
        if (++stage == STAGES) { stage = 0; phase ^= 1u; }
      }
      for (int i = 0; i < STAGES; ++i) {
        if (!issued[i]) continue;
        const unsigned long long t0 = gtimer();
        while (!mbar_try(smem_u32(&bars.full[i]), issued_phase[i]) && gtimer() - t0 < TIMEOUT_NS) {
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = make_idesc(BM, BN);
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      for (int kb = 0; kb < kblocks; ++kb) {
        if (!mbar_wait(smem_u32(&bars.full[stage]), phase, status, abort_flag)) { ok = false; break; }
        fence_after();
        const uint32_t sa = base + stage * stage_bytes;
#pragma unroll
        for (int k = 0; k < BK / UMMA_K; ++k)
          mma_bf16(tmem, make_desc(sa + k * UMMA_K * 2), make_desc(sa + a_bytes + k * UMMA_K * 2), idesc,
                   (kb | k) != 0 ? 1u : 0u);
        mma_commit(smem_u32(&bars.empty[stage]));
        if (++stage == STAGES) { stage = 0; phase ^= 1u; }
      }
      if (ok) mma_commit(smem_u32(&bars.tfull));
      mma_commit(smem_u32(&bars.drain));
      const unsigned long long t0 = gtimer();
      while (!mbar_try(smem_u32(&bars.drain), 0) && gtimer() - t0 < TIMEOUT_NS) {
      }
    }
  } else {
    const int quarter = warp & 3;
    const int m = tm * BM + quarter * 32 + lane;
    // bf16 outputs are staged per warp (32 rows x BN, rows padded by 16 bytes)
    // in the stage ring, free once the accumulator is complete, and written
    // back one row per warp instruction (coalesced)
    const uint32_t pitch = (uint32_t)BN * 2 + 16;
    uint8_t* stage = smem_raw + (base - smem_u32(smem_raw)) + (size_t)quarter * 32 * pitch;
    if (mbar_wait(smem_u32(&bars.tfull), 0, status, abort_flag)) {
      fence_after();
      const uint32_t t_row = tmem + ((uint32_t)(quarter * 32) << 16);
      float acc_c[4] = {0.f, 0.f, 0.f, 0.f};
      int grp = 0;
      if (EPI == EPI_SHADE) grp = (m + e.row0) / e.rows_per_group;
      const bool row_ok = m < e.M;
      for (int c0 = 0; c0 < BN; c0 += 16) {
        float v[16];
        tmem_ld16(t_row + (uint32_t)c0, v);
        const int n0 = tn * BN + c0;
        if (EPI == EPI_F32) {
          if (row_ok && gridDim.z > 1) {
            float* dst = e.split_ws + ((long long)blockIdx.z * e.M + m) * e.N + n0;
            for (int i = 0; i < 16; ++i)
              if (n0 + i < e.N) dst[i] = v[i];
          } else if (row_ok) {
            float* dst = e.out_f32 + (long long)m * e.ld_f32 + n0;
            if (n0 + 16 <= e.N && (e.ld_f32 & 3) == 0) {
#pragma unroll
              for (int i = 0; i < 16; i += 4)
                *reinterpret_cast<float4*>(dst + i) =
                    make_float4(v[i] + (e.bias ? e.bias[n0 + i] : 0.f), v[i + 1] + (e.bias ? e.bias[n0 + i + 1] : 0.f),
                                v[i + 2] + (e.bias ? e.bias[n0 + i + 2] : 0.f), v[i + 3] + (e.bias ? e.bias[n0 + i + 3] : 0.f));
            } else {
              for (int i = 0; i < 16; ++i)
                if (n0 + i < e.N) dst[i] = v[i] + (e.bias ? e.bias[n0 + i] : 0.0f);
            }
          }
        } else if (EPI == EPI_BIAS_GELU || EPI == EPI_GELU_BWD) {
          uint32_t packed[8];
#pragma unroll
          for (int i = 0; i < 16; i += 2) {
            float h0, h1;
            if (EPI == EPI_BIAS_GELU) {
              const float z0 = v[i] + e.bias[min(n0 + i, e.N - 1)];
              const float z1 = v[i + 1] + e.bias[min(n0 + i + 1, e.N - 1)];
              if (e.out_f32 && row_ok) {
                if (n0 + i < e.N) e.out_f32[(long long)m * e.ld_f32 + n0 + i] = z0;
                if (n0 + i + 1 < e.N) e.out_f32[(long long)m * e.ld_f32 + n0 + i + 1] = z1;
              }
              h0 = gelu(z0);
              h1 = gelu(z1);
            } else {
              const float* zp = e.zprev + (long long)(row_ok ? m : 0) * e.ld_zprev;
              h0 = v[i] * gelu_grad(zp[min(n0 + i, e.N - 1)]);
              h1 = v[i + 1] * gelu_grad(zp[min(n0 + i + 1, e.N - 1)]);
            }
            __nv_bfloat162 hb = __floats2bfloat162_rn(h0, h1);
            packed[i >> 1] = *reinterpret_cast<uint32_t*>(&hb);
          }
          uint4* sp = reinterpret_cast<uint4*>(stage + (size_t)lane * pitch + (size_t)c0 * 2);
          sp[0] = make_uint4(packed[0], packed[1], packed[2], packed[3]);
          sp[1] = make_uint4(packed[4], packed[5], packed[6], packed[7]);
        } else {  // EPI_SHADE: fold gelu(z) against the per-group effective output weights
          const float* W = e.weff + (long long)grp * e.N * e.C;
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const int n = n0 + i;
            if (n < e.N) {
              const float h = gelu(v[i] + e.bias[n]);
#pragma unroll
              for (int c = 0; c < 4; ++c)
                if (c < e.C) acc_c[c] = fmaf(h, __ldg(W + (long long)n * e.C + c), acc_c[c]);
            }
          }
        }
      }
      if (EPI == EPI_BIAS_GELU || EPI == EPI_GELU_BWD) {
        __syncwarp();
        const int ncol = min(BN, e.N - tn * BN);            // valid columns of this tile (multiple of 8)
        for (int r = 0; r < 32; ++r) {
          const int mr = tm * BM + quarter * 32 + r;
          if (mr >= e.M) break;
          for (int cb = lane * 8; cb < ncol; cb += 256)
            *reinterpret_cast<uint4*>(e.out_bf16 + (long long)mr * e.ld_bf16 + tn * BN + cb) =
                *reinterpret_cast<const uint4*>(stage + (size_t)r * pitch + (size_t)cb * 2);
        }
      }
      if (EPI == EPI_SHADE && row_ok) {
        const int row = m + e.row0;
        const int s = row / e.rows_per_group, vv = row - s * e.rows_per_group;
        for (int c = 0; c < e.C; ++c)
          e.radiance[((long long)vv * e.groups + s) * e.C + c] = acc_c[c] + e.beff[s * e.C + c];
      }
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols));
  }
}

// -------------------------------------------------------------- helper kernels

// Encoding layout: [p, n] (6); per f: sin(w_f [p, n]) (6), cos(w_f [p, n]) (6);
// 2 zeros (columns 0..199 depend on the vertex alone); view w (3); per f:
// sin(w_f w) (3), cos(w_f w) (3) (columns 200..298); zeros to 320.
constexpr int N_VCOLS = 200;

// sin and cos of omega_f x for f = 0..15: omega_0 x = pi x and omega_1 x =
// pi sqrt(2) x directly, the rest by the double-angle identities
// (omega_{f+2} = 2 omega_f): sin 2a = 2 sin a cos a, cos 2a = (c - s)(c + s).
// The doubled angles are exact (no FP32 rounding of a large argument); the
// recurrence's error grows 2x per step, to ~1e-5 at f = 15, far below the
// bfloat16 rounding of the stored features.
__device__ __forceinline__ void sincos_ladder(float x, float (&sv)[N_FREQ], float (&cv)[N_FREQ]) {
  sincosf(3.14159265358979323846f * x, &sv[0], &cv[0]);
  sincosf(4.44288293815836624702f * x, &sv[1], &cv[1]);
#pragma unroll
  for (int f = 2; f < N_FREQ; ++f) {
    const float sa = sv[f - 2], ca = cv[f - 2];
    sv[f] = 2.0f * sa * ca;
    cv[f] = (ca - sa) * (ca + sa);
  }
}

// lane r < 6 encodes component r of [p, n]
__device__ __forceinline__ void encode_vertex_part(const float pn[6], __nv_bfloat16* out, int lane) {
  if (lane < 6) {
    float sv[N_FREQ], cv[N_FREQ];
    sincos_ladder(pn[lane], sv, cv);
#pragma unroll
    for (int f = 0; f < N_FREQ; ++f) {
      out[6 + 12 * f + lane] = __float2bfloat16_rn(sv[f]);
      out[12 + 12 * f + lane] = __float2bfloat16_rn(cv[f]);
    }
    out[lane] = __float2bfloat16_rn(pn[lane]);
  }
  if (lane < 2) out[198 + lane] = __float2bfloat16_rn(0.0f);
}

// lane r < 3 encodes component r of the view direction w
__device__ __forceinline__ void encode_view_part(const float w[3], __nv_bfloat16* out, int lane) {
  if (lane < 3) {
    float sv[N_FREQ], cv[N_FREQ];
    sincos_ladder(w[lane], sv, cv);
#pragma unroll
    for (int f = 0; f < N_FREQ; ++f) {
      out[203 + 6 * f + lane] = __float2bfloat16_rn(sv[f]);
      out[206 + 6 * f + lane] = __float2bfloat16_rn(cv[f]);
    }
    out[200 + lane] = __float2bfloat16_rn(w[lane]);
  }
  for (int j = 299 + lane; j < N_IN; j += 32) out[j] = __float2bfloat16_rn(0.0f);
}

__device__ __forceinline__ void encode_row(const float raw[N_RAW], __nv_bfloat16* out, int lane) {
  encode_vertex_part(raw, out, lane);
  encode_view_part(raw + 6, out, lane);
}

// X[b][320] from raw inputs [b][9]
__global__ void k_encode_raw(const float* __restrict__ raw, int B, __nv_bfloat16* __restrict__ X) {
  const int b = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (b >= B) return;
  float r[N_RAW];
  for (int i = 0; i < N_RAW; ++i) r[i] = raw[(long long)b * N_RAW + i];
  encode_row(r, X + (long long)b * N_IN, threadIdx.x & 31);
}

// X[row][320] for rows row0.. of the (s, v) grid, row = s * V + v:
// raw = (pos[v], nrm[v], normalize(cam[s] - pos[v]))
__global__ void k_encode_scene(const float* __restrict__ pos, const float* __restrict__ nrm,
                               const float* __restrict__ cams, int V, long long row0, int rows,
                               __nv_bfloat16* __restrict__ X) {
  const int r = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (r >= rows) return;
  const long long row = row0 + r;
  const int s = (int)(row / V), v = (int)(row - (long long)s * V);
  float raw[N_RAW];
  for (int i = 0; i < 3; ++i) {
    raw[i] = pos[3 * v + i];
    raw[3 + i] = nrm[3 * v + i];
  }
  float wx = cams[3 * s] - raw[0], wy = cams[3 * s + 1] - raw[1], wz = cams[3 * s + 2] - raw[2];
  const float inv = rsqrtf(wx * wx + wy * wy + wz * wz);
  raw[6] = wx * inv; raw[7] = wy * inv; raw[8] = wz * inv;
  encode_row(raw, X + (long long)r * N_IN, threadIdx.x & 31);
}

// out[c][r] = in[r][c] (bf16), 32 x 32 tiles
__global__ void k_transpose(const __nv_bfloat16* __restrict__ in, int R, int C, __nv_bfloat16* __restrict__ out) {
  __shared__ __nv_bfloat16 t[32][34];
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int r = r0 + i, c = c0 + threadIdx.x;
    if (r < R && c < C) t[i][threadIdx.x] = in[(long long)r * C + c];
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int c = c0 + i, r = r0 + threadIdx.x;
    if (r < R && c < C) out[(long long)c * R + r] = t[threadIdx.x][i];
  }
}

// out[m][n] (row stride ld) = bias[n] + sum_z ws[z][m][n], fixed order
__global__ void k_split_reduce(const float* __restrict__ ws, int splits, int M, int N, const float* __restrict__ bias,
                               float* __restrict__ out, int ld) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= (long long)M * N) return;
  const int m = (int)(i / N), n = (int)(i - (long long)m * N);
  float acc = bias ? bias[n] : 0.0f;
  for (int z = 0; z < splits; ++z) acc += ws[(long long)z * M * N + i];
  out[(long long)m * ld + n] = acc;
}

// dOut = bf16(2 (out - y) / (B N)); loss += mean((out - y)^2)
__global__ void k_mse(const float* __restrict__ out, const float* __restrict__ y, long long n, float inv_n,
                      __nv_bfloat16* __restrict__ dout, float* loss) {
  float acc = 0.0f;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float d = out[i] - y[i];
    acc = fmaf(d, d, acc);
    dout[i] = __float2bfloat16_rn(2.0f * d * inv_n);
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ float part[32];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.0f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += part[w];
    atomicAdd(loss, s * inv_n);
  }
}

// db[n] = sum_b dz[b][n]
// Bias gradients db[n] = sum_b dz[b][n] in two deterministic passes: block
// (x, y) sums rows [y R, (y + 1) R) of 32 columns into part[y][n] (8 row
// strides per column, then a fixed-order add), and one thread per column
// adds the P parts in order.
__global__ void k_colsum_part(const __nv_bfloat16* __restrict__ dz, int B, int N, int R, float* __restrict__ part) {
  const int n = blockIdx.x * 32 + (threadIdx.x & 31);
  const int sub = threadIdx.x >> 5;
  const int r0 = blockIdx.y * R, r1 = min(B, r0 + R);
  float acc = 0.0f;
  if (n < N)
#pragma unroll 4
    for (int b = r0 + sub; b < r1; b += 8) acc += __bfloat162float(dz[(long long)b * N + n]);
  __shared__ float red[8][32];
  red[sub][threadIdx.x & 31] = acc;
  __syncthreads();
  if (sub == 0 && n < N) {
    float t = 0.0f;
    for (int q = 0; q < 8; ++q) t += red[q][threadIdx.x & 31];
    part[(long long)blockIdx.y * N + n] = t;
  }
}

__global__ void k_colsum_final(const float* __restrict__ part, int P, int N, float* __restrict__ db) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float t = 0.0f;
  for (int q = 0; q < P; ++q) t += part[(long long)q * N + n];
  db[n] = t;
}

// One Adam step; the step count lives on the device (read here, advanced by
// k_pack) so captured training steps replay correctly.
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, long long n, float lr, float b1, float b2, float eps,
                       const int* __restrict__ step) {
  const float t = (float)(*step + 1);
  const float c1 = 1.0f - powf(b1, t), c2 = 1.0f - powf(b2, t);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// bf16 copies of every weight matrix ([out][in]) and of its transpose ([in][out])
__global__ void k_pack(const float* __restrict__ p, __nv_bfloat16* __restrict__ wb, __nv_bfloat16* __restrict__ wt,
                       int* step, int advance) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (advance && i == 0) *step += 1;
  long long off = 0;
  for (int l = 0; l < N_LAYERS; ++l) {
    const long long sz = (long long)fan_out(l) * fan_in(l);
    if (i < sz) {
      const int o = (int)(i / fan_in(l)), in = (int)(i - (long long)o * fan_in(l));
      const __nv_bfloat16 x = __float2bfloat16_rn(p[w_off(l) + i]);
      wb[off + i] = x;
      wt[off + (long long)in * fan_out(l) + o] = x;
      return;
    }
    i -= sz;
    off += sz;
  }
}

// Output layer folded into the lighting, per group s:
//   Weff[s][i][c] = sum_j Wo[j][i] sigma_j L(s, c, idx_j)
//   beff[s][c]    = sum_j (mu_j + sigma_j bo_j) L(s, c, idx_j)
// Block (s, ib) computes i in [32 ib, 32 ib + 32): lane = i, warp = a slice of j.
__global__ void __launch_bounds__(256) k_fold(const float* __restrict__ p, const float* __restrict__ mu,
                                              const float* __restrict__ sigma, const int* __restrict__ idx,
                                              const float* __restrict__ L, long long st_s, long long st_c,
                                              long long st_k, int S, int C, float* __restrict__ weff,
                                              float* __restrict__ beff) {
  const int s = blockIdx.x, ib = blockIdx.y;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float* Wo = p + w_off(N_LAYERS - 1);
  const float* bo = p + b_off(N_LAYERS - 1);
  __shared__ float sl[N_OUT][4];
  __shared__ float part[8][32][4];
  for (int j = threadIdx.x; j < N_OUT; j += blockDim.x)
    for (int c = 0; c < 4; ++c)
      sl[j][c] = (c < C) ? sigma[j] * L[s * st_s + c * st_c + (long long)idx[j] * st_k] : 0.0f;
  __syncthreads();
  const int i = ib * 32 + lane;
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  for (int j = warp * (N_OUT / 8); j < (warp + 1) * (N_OUT / 8); ++j) {
    const float w = Wo[(long long)j * WIDTH + i];
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[c] = fmaf(w, sl[j][c], acc[c]);
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) part[warp][lane][c] = acc[c];
  __syncthreads();
  if (warp == 0) {
    for (int c = 0; c < C; ++c) {
      float t = 0.0f;
      for (int w8 = 0; w8 < 8; ++w8) t += part[w8][lane][c];
      weff[((long long)s * WIDTH + i) * C + c] = t;
    }
  }
  if (ib == 0 && threadIdx.x < C) {
    const int c = threadIdx.x;
    float t = 0.0f;
    for (int j = 0; j < N_OUT; ++j) {
      const float lj = L[s * st_s + c * st_c + (long long)idx[j] * st_k];
      t = fmaf(mu[j] + sigma[j] * bo[j], lj, t);
    }
    beff[s * C + c] = t;
  }
}

// ----------------------------------------------------------- fused surrogate shading
// Persistent, one CTA per SM, 18 warps, one 128-row tile at a time (rows are
// (shift, vertex) pairs, row = s * V + v):
//   warp 0     TMA producer: the weight k-blocks [256 x 64] of W1..W4 into a
//              3-stage ring, in the order the MMAs use them, tile after tile;
//   warp 1     TMEM allocator and MMA issuer (M = 128, N = 256, K = 16);
//   warps 2-17 encode the tile into the activation buffer (the 200
//              per-vertex columns copied from a table, the view columns
//              computed), then each layer's epilogue: bias + GELU, written
//              back as the next layer's bf16 A operand in the same
//              128-byte-swizzled K-major layout the tensor core reads; the
//              last layer's epilogue takes the double product with the output
//              layer folded into the lighting; the 4 column groups of a TMEM
//              lane quarter meet in shared memory (an mbarrier per quarter) and
//              group 0 adds them in a fixed order and writes the radiance.
//              Activations never leave the SM.
constexpr int F_EPI = 16;                    // epilogue warps: 4 per TMEM lane quarter
constexpr int F_RPW = tc::BM / F_EPI;        // rows each epilogue warp encodes
constexpr int F_COLS = WIDTH / (F_EPI / 4);  // columns each epilogue warp takes per layer
constexpr int F_THREADS = 64 + 32 * F_EPI;
constexpr int F_STAGES = 3;
constexpr uint32_t F_ACT_BYTES = 5 * 16384;  // 128 rows x 320 bf16
constexpr uint32_t F_W_BYTES = 256 * 128;    // one weight k-block [256 x 64] bf16

struct __align__(8) FBars {
  uint64_t wfull[F_STAGES], wempty[F_STAGES];
  uint64_t tfull, drain;
  uint64_t kready[5];              // k-block j of the next MMA's A operand is written (by all epilogue warps)
  uint64_t red[4];                 // per lane quarter: the 4 column groups' partial radiance are in
  uint32_t tmem_base;
  int abort_flag;
};

struct FusedArgs {
  int V, S, C;
  long long rows;
  const __nv_bfloat16* vfeat;  // [V][200]
  const float* pos;            // [V][3]
  const float* cams;           // [S][3]
  const float* params;         // flat parameters (biases)
  const float* weff;           // [S][256][C]
  const float* beff;           // [S][C]
  float* radiance;             // [V][S][C]
};

// byte offset of element (r, c) in the activation buffer: k-block c/64 is a
// [128 rows x 128 B] tile, rows in 1024-byte groups of 8, 16-byte chunk
// (c % 64) / 8 stored at chunk ^ (r % 8)
__device__ __forceinline__ uint32_t act_off(int r, int c) {
  const int ch = (c & 63) >> 3;
  return (uint32_t)((c >> 6) * 16384 + (r >> 3) * 1024 + (r & 7) * 128 + ((ch ^ (r & 7)) << 4) + ((c & 7) << 1));
}

__global__ void __launch_bounds__(F_THREADS, 1)
k_mlp_fused(const __grid_constant__ CUtensorMap w0, const __grid_constant__ CUtensorMap w1,
            const __grid_constant__ CUtensorMap w2, const __grid_constant__ CUtensorMap w3, FusedArgs f,
            int* status) {
  using namespace tc;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  __shared__ FBars bars;
  __shared__ int rinfo[F_EPI][F_RPW][2];
  __shared__ float rview[F_EPI][F_RPW][3];
  __shared__ __align__(16) float sbias[3][WIDTH];        // hidden-layer biases 1..3 (the last one folds into beff)
  __shared__ __align__(16) float sbias3[WIDTH];          // bias of the 4th hidden layer
  // per epilogue warp: its column group of the folded output layer for the
  // tile's (at most two) shifts, so that no barrier across warps is needed
  __shared__ __align__(16) float sweff[F_EPI][2][F_COLS][4];
  // per lane quarter: the partial radiance of column groups 1..3 for group 0
  __shared__ __align__(16) float sred[4][3][32][4];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  uint8_t* act = smem_raw + (base - smem_u32(smem_raw));
  const uint32_t act_s = base;
  const uint32_t ring = base + F_ACT_BYTES;
  const long long n_tiles = (f.rows + BM - 1) / BM;
  volatile int* abort_flag = &bars.abort_flag;

  if (threadIdx.x == 0) {
    for (int i = 0; i < F_STAGES; ++i) {
      mbar_init(smem_u32(&bars.wfull[i]), 1);
      mbar_init(smem_u32(&bars.wempty[i]), 1);
    }
    mbar_init(smem_u32(&bars.tfull), 1);
    for (int i = 0; i < 5; ++i) mbar_init(smem_u32(&bars.kready[i]), F_EPI);
    for (int i = 0; i < 4; ++i) mbar_init(smem_u32(&bars.red[i]), 3);
    mbar_init(smem_u32(&bars.drain), 1);
    bars.abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(&bars.tmem_base)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  for (int i = threadIdx.x; i < 4 * WIDTH; i += blockDim.x) {
    const int l = i / WIDTH, j = i - l * WIDTH;
    const float bv = f.params[b_off(l) + j];
    if (l < 3) sbias[l][j] = bv; else sbias3[j] = bv;
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = bars.tmem_base;

  if (warp == 0) {
    if (lane == 0) {
      int issued[F_STAGES];
      uint32_t issued_phase[F_STAGES];
      for (int i = 0; i < F_STAGES; ++i) { issued[i] = 0; issued_phase[i] = 0; }
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      for (long long t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
        for (int l = 0; l < 4 && ok; ++l) {
          const CUtensorMap* map = (l == 0) ? &w0 : (l == 1) ? &w1 : (l == 2) ? &w2 : &w3;
          const int nk = (l == 0) ? 5 : 4;
          for (int kb = 0; kb < nk; ++kb) {
            if (!mbar_wait(smem_u32(&bars.wempty[stage]), phase ^ 1u, status, abort_flag)) { ok = false; break; }
            const uint32_t fb = smem_u32(&bars.wfull[stage]);
            mbar_arrive_tx(fb, F_W_BYTES);
            tma_load_2d(ring + stage * F_W_BYTES, map, kb * BK, 0, fb);
            issued[stage] = 1;
            issued_phase[stage] = phase;
            if (++stage == F_STAGES) { stage = 0; phase ^= 1u; }
          }
        }
      }
      for (int i = 0; i < F_STAGES; ++i) {
        if (!issued[i]) continue;
        const unsigned long long t0 = gtimer();
        while (!mbar_try(smem_u32(&bars.wfull[i]), issued_phase[i]) && gtimer() - t0 < TIMEOUT_NS) {
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = make_idesc(BM, 256);
      int stage = 0;
      uint32_t phase = 0;
      uint32_t kpar = 0u;                                // bit j: parity of the next completion of kready[j]
      bool ok = true;
      for (long long t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
        for (int l = 0; l < 4 && ok; ++l) {
          // layers alternate between two accumulators, so that a layer's MMAs
          // run while the epilogue still reads the previous layer's; each
          // k-block starts as soon as the epilogue warps have written it
          const uint32_t acc = tmem + (uint32_t)((l & 1) * 256);
          const int nk = (l == 0) ? 5 : 4;
          for (int kb = 0; kb < nk; ++kb) {
            if (!mbar_wait(smem_u32(&bars.kready[kb]), (kpar >> kb) & 1u, status, abort_flag)) { ok = false; break; }
            kpar ^= 1u << kb;
            fence_after();
            if (!mbar_wait(smem_u32(&bars.wfull[stage]), phase, status, abort_flag)) { ok = false; break; }
            fence_after();
            const uint32_t wa = ring + stage * F_W_BYTES;
#pragma unroll
            for (int k = 0; k < BK / UMMA_K; ++k)
              mma_bf16(acc, make_desc(act_s + kb * 16384 + k * UMMA_K * 2), make_desc(wa + k * UMMA_K * 2), idesc,
                       (kb | k) != 0 ? 1u : 0u);
            mma_commit(smem_u32(&bars.wempty[stage]));
            if (++stage == F_STAGES) { stage = 0; phase ^= 1u; }
          }
          if (ok) mma_commit(smem_u32(&bars.tfull));
        }
      }
      mma_commit(smem_u32(&bars.drain));
      const unsigned long long t0 = gtimer();
      while (!mbar_try(smem_u32(&bars.drain), 0) && gtimer() - t0 < TIMEOUT_NS) {
      }
    }
  } else {
    const int wid = warp - 2;                 // 0..F_EPI-1
    const int q = warp & 3;                   // TMEM lane quarter
    const int cg = wid >> 2;                  // column group: columns [cg F_COLS, (cg + 1) F_COLS)
    long long step = 0;
    long long it = 0;                         // tiles done (phase of the reduction barrier)
    bool ok = true;
    // this warp's column group of a tile's folded output layer (the tile's
    // rows span at most two shifts)
    auto load_weff = [&](long long t) {
      const long long row0 = t * BM;
      const int s_lo = (int)(row0 / f.V);
      const int s_hi = (int)((row0 + BM - 1 < f.rows ? row0 + BM - 1 : f.rows - 1) / f.V);
      __syncwarp();
      for (int i = lane; i < 2 * F_COLS; i += 32) {
        // local column j = 16 kb + m is layer column 64 kb + 16 cg + m
        const int k = i / F_COLS, j = i - k * F_COLS;
        const int col = 64 * (j >> 4) + 16 * cg + (j & 15);
        const float* W = f.weff + ((long long)(k ? s_hi : s_lo) * WIDTH + col) * f.C;
        float4 w4 = make_float4(0.f, 0.f, 0.f, 0.f);
        w4.x = W[0];
        if (f.C > 1) w4.y = W[1];
        if (f.C > 2) w4.z = W[2];
        if (f.C > 3) w4.w = W[3];
        *reinterpret_cast<float4*>(&sweff[wid][k][j][0]) = w4;
      }
      __syncwarp();
    };
    // encode F_RPW rows of a tile per warp into the activation buffer (row
    // info first, then many independent loads per lane: lanes sweep (row,
    // chunk) pairs), then release its 5 k-blocks to the MMA warp
    auto encode = [&](long long t) {
      const long long row0 = t * BM;
      const int r0 = wid * F_RPW;
      if (lane < F_RPW) {
        const long long row = row0 + r0 + lane;
        int sr = -1, vr = 0;
        float w0 = 0.f, w1 = 0.f, w2 = 0.f;
        if (row < f.rows) {
          sr = (int)(row / f.V);
          vr = (int)(row - (long long)sr * f.V);
          const float wx = __ldg(f.cams + 3 * sr) - __ldg(f.pos + 3 * vr);
          const float wy = __ldg(f.cams + 3 * sr + 1) - __ldg(f.pos + 3 * vr + 1);
          const float wz = __ldg(f.cams + 3 * sr + 2) - __ldg(f.pos + 3 * vr + 2);
          const float inv = rsqrtf(wx * wx + wy * wy + wz * wz);
          w0 = wx * inv; w1 = wy * inv; w2 = wz * inv;
        }
        rinfo[wid][lane][0] = sr;
        rinfo[wid][lane][1] = vr;
        rview[wid][lane][0] = w0;
        rview[wid][lane][1] = w1;
        rview[wid][lane][2] = w2;
      }
      __syncwarp();
#pragma unroll 4
      for (int e = lane; e < F_RPW * 25; e += 32) {
        const int i = e / 25, ch = e - i * 25;
        const int sr = rinfo[wid][i][0];
        uint4 val = make_uint4(0, 0, 0, 0);
        if (sr >= 0) val = __ldg(reinterpret_cast<const uint4*>(f.vfeat + (long long)rinfo[wid][i][1] * N_VCOLS) + ch);
        *reinterpret_cast<uint4*>(act + act_off(r0 + i, 8 * ch)) = val;
      }
      // view features: one lane per (row, component), all 16 frequencies by the ladder
      if (lane < F_RPW * 3) {
        const int i = lane / 3, rr = lane - i * 3;
        float sv[N_FREQ], cv[N_FREQ];
        sincos_ladder(rview[wid][i][rr], sv, cv);
        const bool live = rinfo[wid][i][0] >= 0;
#pragma unroll
        for (int fq = 0; fq < N_FREQ; ++fq) {
          *reinterpret_cast<__nv_bfloat16*>(act + act_off(r0 + i, 203 + 6 * fq + rr)) =
              __float2bfloat16_rn(live ? sv[fq] : 0.0f);
          *reinterpret_cast<__nv_bfloat16*>(act + act_off(r0 + i, 206 + 6 * fq + rr)) =
              __float2bfloat16_rn(live ? cv[fq] : 0.0f);
        }
      }
      for (int e = lane; e < F_RPW * 24; e += 32) {    // raw view (3) and the zero pad (21)
        const int i = e / 24, j = e - i * 24;
        const float x = (j < 3 && rinfo[wid][i][0] >= 0) ? rview[wid][i][j] : 0.0f;
        *reinterpret_cast<__nv_bfloat16*>(act + act_off(r0 + i, (j < 3) ? 200 + j : 296 + j)) = __float2bfloat16_rn(x);
      }
      fence_before();
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0)
        for (int j = 0; j < 5; ++j) mbar_arrive(smem_u32(&bars.kready[j]));
    };
    if (blockIdx.x < n_tiles) {
      load_weff(blockIdx.x);
      encode(blockIdx.x);
    }
    for (long long t = blockIdx.x; t < n_tiles && ok; t += gridDim.x, ++it) {
      const long long row0 = t * BM;
      const int s_lo = (int)(row0 / f.V);
      // ---- layers
      const int r = q * 32 + lane;
      const long long row = row0 + r;
      const bool row_ok = row < f.rows;
      for (int l = 0; l < 4; ++l, ++step) {
        if (!mbar_wait(smem_u32(&bars.tfull), (uint32_t)(step & 1), status, abort_flag)) { ok = false; break; }
        fence_after();
        // the last layer's MMAs have read the activation buffer: encode the
        // next tile now, so that its first layer runs on the tensor cores
        // while this epilogue computes the tile's radiance
        if (l == 3 && t + gridDim.x < n_tiles) encode(t + gridDim.x);
        const float* bias = (l < 3) ? sbias[l] : sbias3;
        float acc_c[4] = {0.f, 0.f, 0.f, 0.f};
        int s = 0;
        if (l == 3 && row_ok) s = (int)(row / f.V);
        const float(*Wt)[4] = sweff[wid][(l == 3 && s != s_lo) ? 1 : 0];   // column 64 kb + 16 cg + m at [16 kb + m]
        const uint32_t acc_t = tmem + (uint32_t)((l & 1) * 256) + ((uint32_t)(q * 32) << 16);
        // the warp's 16 columns of each k-block in turn: the next layer's MMA
        // on k-block kb can start once all epilogue warps have written it
        for (int kb = 0; kb < 4; ++kb) {
          const int c0 = 64 * kb + 16 * cg;
          float v[16];
          tmem_ld16(acc_t + (uint32_t)c0, v);
          if (l < 3) {
            uint32_t pk[8];
#pragma unroll
            for (int i = 0; i < 16; i += 2) {
              const float2 b2 = *reinterpret_cast<const float2*>(bias + c0 + i);
              const float2 h = u2f(gelu2(f2_add(f2_pack(v[i], v[i + 1]), f2_pack(b2.x, b2.y))));
              __nv_bfloat162 hb = __floats2bfloat162_rn(h.x, h.y);
              pk[i >> 1] = *reinterpret_cast<uint32_t*>(&hb);
            }
            *reinterpret_cast<uint4*>(act + act_off(r, c0)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
            *reinterpret_cast<uint4*>(act + act_off(r, c0 + 8)) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
            fence_before();
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&bars.kready[kb]));
          } else {
#pragma unroll
            for (int i = 0; i < 16; i += 2) {
              const float2 b2 = *reinterpret_cast<const float2*>(bias + c0 + i);
              const float2 h = u2f(gelu2(f2_add(f2_pack(v[i], v[i + 1]), f2_pack(b2.x, b2.y))));
              const float4 wa = *reinterpret_cast<const float4*>(Wt[16 * kb + i]);
              const float4 wb = *reinterpret_cast<const float4*>(Wt[16 * kb + i + 1]);
              acc_c[0] = fmaf(h.y, wb.x, fmaf(h.x, wa.x, acc_c[0]));
              acc_c[1] = fmaf(h.y, wb.y, fmaf(h.x, wa.y, acc_c[1]));
              acc_c[2] = fmaf(h.y, wb.z, fmaf(h.x, wa.z, acc_c[2]));
              acc_c[3] = fmaf(h.y, wb.w, fmaf(h.x, wa.w, acc_c[3]));
            }
          }
        }
        if (l == 3) {
          fence_before();
          // the 4 column groups of this lane quarter meet in group 0, which adds
          // them in a fixed order (deterministic) and writes the radiance
          if (cg > 0) {
            *reinterpret_cast<float4*>(&sred[q][cg - 1][lane][0]) = make_float4(acc_c[0], acc_c[1], acc_c[2], acc_c[3]);
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&bars.red[q]));
          } else {
            if (!mbar_wait(smem_u32(&bars.red[q]), (uint32_t)(it & 1), status, abort_flag)) { ok = false; break; }
            if (row_ok) {
              const int vv = (int)(row - (long long)s * f.V);
              for (int c = 0; c < f.C; ++c) {
                float tsum = acc_c[c];
#pragma unroll
                for (int g2 = 0; g2 < 3; ++g2) tsum += sred[q][g2][lane][c];
                f.radiance[((long long)vv * f.S + s) * f.C + c] = tsum + f.beff[s * f.C + c];
              }
            }
          }
        }
      }
      if (ok && t + gridDim.x < n_tiles) load_weff(t + gridDim.x);   // after this tile's last use of sweff
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
  }
}

// per-vertex part of the encoding: vfeat[v][0..199]
__global__ void k_vertex_features(const float* __restrict__ pos, const float* __restrict__ nrm, int V,
                                  __nv_bfloat16* __restrict__ vfeat) {
  const int v = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (v >= V) return;
  float pn[6];
  for (int i = 0; i < 3; ++i) {
    pn[i] = pos[3 * v + i];
    pn[3 + i] = nrm[3 * v + i];
  }
  encode_vertex_part(pn, vfeat + (long long)v * N_VCOLS, threadIdx.x & 31);
}

}  // namespace mlpk
}  // namespace hs

using namespace hs;
using namespace hs::mlpk;

struct haar_mlp_s {
  int max_batch, max_rows, max_groups;
  float* p;           // master parameters (flat, FP32)
  float* g;           // gradients (flat)
  float* m;           // Adam first moments
  float* v;           // Adam second moments
  __nv_bfloat16* wb;  // bf16 weights, [out][in] per layer
  __nv_bfloat16* wt;  // bf16 transposed weights, [in][out] per layer
  // training buffers (max_batch rows)
  __nv_bfloat16* X;   // [B][320]
  __nv_bfloat16* h[4];// [B][256]
  float* z[4];        // [B][256]
  float* out;         // [B][512]
  __nv_bfloat16* dout;// [B][512]
  __nv_bfloat16* dz;  // [B][256]
  __nv_bfloat16* dz2; // [B][256]
  __nv_bfloat16* tA;  // transpose scratch [512][B]
  __nv_bfloat16* tB;  // transpose scratch [320][B]
  float* loss;        // [1]
  int* step;          // [1] Adam step count
  float* split_ws;    // split-K partial sums of the weight gradients
  long long split_ws_floats;
  // inference buffers (max_rows rows)
  __nv_bfloat16* iX;  // [rows][320]
  __nv_bfloat16* ih0; // [rows][256]
  __nv_bfloat16* ih1; // [rows][256]
  float* weff;        // [groups][256][4]
  float* beff;        // [groups][4]
  int* status;
};

namespace hs {
namespace mlpk {

static size_t w_total() {
  size_t t = 0;
  for (int l = 0; l < N_LAYERS; ++l) t += (size_t)fan_out(l) * fan_in(l);
  return t;
}
static size_t wb_off(int l) {
  size_t t = 0;
  for (int i = 0; i < l; ++i) t += (size_t)fan_out(i) * fan_in(i);
  return t;
}

template <int EPI>
static haar_status_t gemm(const __nv_bfloat16* A, int M, const __nv_bfloat16* B, int N, int K, const EpiArgs& e,
                          int* status, cudaStream_t st) {
  using namespace tc;
  if (K % BK != 0) return set_error(HAAR_ERR_INVALID_ARG, "mlp gemm: K = %d is not a multiple of 64", K);
  int ntiles = (N + 255) / 256;
  const int mtiles = (M + BM - 1) / BM;
  if (EPI != EPI_SHADE && mtiles * ntiles < 152 && N >= 256) ntiles = (N + 127) / 128;   // more CTAs
  int BN = (N + ntiles - 1) / ntiles;
  BN = (BN + 15) / 16 * 16;
  if (EPI == EPI_SHADE && ntiles != 1) return set_error(HAAR_ERR_UNSUPPORTED, "mlp gemm: shade epilogue needs N <= 256");
  // split K for small outputs with long K (weight gradients: K = batch)
  int ksplit = 1;
  if (EPI == EPI_F32 && e.split_ws != nullptr) {
    const int tiles = mtiles * ((N + BN - 1) / BN);
    const int kb = K / BK;
    while (ksplit * 2 * tiles <= 2 * 152 && kb / (ksplit * 2) >= 4 && kb % (ksplit * 2) == 0 &&
           (long long)ksplit * 2 * M * N <= e.split_ws_floats) ksplit *= 2;
  }
  CUtensorMap mA, mB;
  if (!encode_2d(&mA, A, (uint64_t)K, (uint64_t)M, BK, BM) || !encode_2d(&mB, B, (uint64_t)K, (uint64_t)N, BK, (uint32_t)BN))
    return set_error(HAAR_ERR_CUDA, "mlp gemm: cuTensorMapEncodeTiled failed");
  if ((EPI == EPI_BIAS_GELU || EPI == EPI_GELU_BWD) && (N % 8) != 0)
    return set_error(HAAR_ERR_UNSUPPORTED, "mlp gemm: bf16 outputs need N %% 8 == 0");
  const size_t stage = (size_t)BM * BK * 2 + (size_t)BN * BK * 2;
  // two stages (two CTAs per SM overlap one's epilogue with the other's
  // main loop); the bf16 epilogue stages its rows in the same memory
  int stages = K / BK / ksplit < 2 ? 1 : 2;
  size_t ring = (size_t)stages * stage;
  const size_t staging = (size_t)4 * 32 * ((size_t)BN * 2 + 16);
  if (ring < staging) ring = staging;
  const size_t smem = ring + 1024;
  int tcols = 32;
  while (tcols < BN) tcols <<= 1;
  cudaError_t err = cudaFuncSetAttribute(k_gemm<EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return cuda_check(err, "cudaFuncSetAttribute(k_gemm)");
  dim3 grid((M + BM - 1) / BM, (N + BN - 1) / BN, ksplit);
  k_gemm<EPI><<<grid, THREADS, smem, st>>>(mA, mB, K, BN, stages, tcols, e, status);
  haar_status_t r = cuda_check(cudaGetLastError(), "k_gemm launch");
  if (r != HAAR_OK || ksplit == 1) return r;
  const long long n = (long long)M * N;
  k_split_reduce<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(e.split_ws, ksplit, M, N, e.bias, e.out_f32, e.ld_f32);
  return cuda_check(cudaGetLastError(), "k_split_reduce launch");
}

static EpiArgs epi(int M, int N) {
  EpiArgs e;
  memset(&e, 0, sizeof(e));
  e.M = M;
  e.N = N;
  return e;
}

// db = column sums of dz [B][N] through the partial-sum scratch ws (at least
// 64 N floats; the split-K scratch, free between the weight-gradient GEMMs)
static haar_status_t colsum(const __nv_bfloat16* dz, int B, int N, float* ws, float* db, cudaStream_t st) {
  const int P = B >= 64 * 128 ? 64 : (B + 127) / 128 > 0 ? (B + 127) / 128 : 1;
  const int R = (B + P - 1) / P;
  k_colsum_part<<<dim3((N + 31) / 32, P), 256, 0, st>>>(dz, B, N, R, ws);
  const haar_status_t r = cuda_check(cudaGetLastError(), "k_colsum_part launch");
  if (r != HAAR_OK) return r;
  k_colsum_final<<<(N + 255) / 256, 256, 0, st>>>(ws, P, N, db);
  return cuda_check(cudaGetLastError(), "k_colsum_final launch");
}

static haar_status_t transpose(const __nv_bfloat16* in, int R, int C, __nv_bfloat16* out, cudaStream_t st) {
  dim3 grid((C + 31) / 32, (R + 31) / 32), block(32, 8);
  k_transpose<<<grid, block, 0, st>>>(in, R, C, out);
  return cuda_check(cudaGetLastError(), "k_transpose launch");
}

#define HS_TRY(x)                   \
  do {                              \
    haar_status_t _r = (x);         \
    if (_r != HAAR_OK) return _r;   \
  } while (0)

// forward over B rows of encoded inputs in M->X; keeps z and h for backward
static haar_status_t forward(haar_mlp_s* M, int B, cudaStream_t st) {
  const __nv_bfloat16* in = M->X;
  for (int l = 0; l < 4; ++l) {
    EpiArgs e = epi(B, WIDTH);
    e.bias = M->p + b_off(l);
    e.out_f32 = M->z[l];
    e.ld_f32 = WIDTH;
    e.out_bf16 = M->h[l];
    e.ld_bf16 = WIDTH;
    HS_TRY(gemm<EPI_BIAS_GELU>(in, B, M->wb + wb_off(l), WIDTH, fan_in(l), e, M->status, st));
    in = M->h[l];
  }
  EpiArgs e = epi(B, N_OUT);
  e.bias = M->p + b_off(4);
  e.out_f32 = M->out;
  e.ld_f32 = N_OUT;
  return gemm<EPI_F32>(M->h[3], B, M->wb + wb_off(4), N_OUT, WIDTH, e, M->status, st);
}

static haar_status_t backward(haar_mlp_s* M, int B, const float* target, cudaStream_t st) {
  const long long n = (long long)B * N_OUT;
  k_mse<<<(unsigned)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024), 256, 0, st>>>(M->out, target, n, 1.0f / (float)n,
                                                                                  M->dout, M->loss);
  HS_TRY(cuda_check(cudaGetLastError(), "k_mse launch"));
  // output layer
  HS_TRY(transpose(M->dout, B, N_OUT, M->tA, st));
  HS_TRY(transpose(M->h[3], B, WIDTH, M->tB, st));
  {
    EpiArgs e = epi(N_OUT, WIDTH);
    e.out_f32 = M->g + w_off(4);
    e.ld_f32 = WIDTH;
    e.split_ws = M->split_ws;
    e.split_ws_floats = M->split_ws_floats;
    HS_TRY(gemm<EPI_F32>(M->tA, N_OUT, M->tB, WIDTH, B, e, M->status, st));
  }
  HS_TRY(colsum(M->dout, B, N_OUT, M->split_ws, M->g + b_off(4), st));
  {
    EpiArgs e = epi(B, WIDTH);
    e.out_bf16 = M->dz;
    e.ld_bf16 = WIDTH;
    e.zprev = M->z[3];
    e.ld_zprev = WIDTH;
    HS_TRY(gemm<EPI_GELU_BWD>(M->dout, B, M->wt + wb_off(4), WIDTH, N_OUT, e, M->status, st));
  }
  __nv_bfloat16* dz = M->dz;
  __nv_bfloat16* dz_next = M->dz2;
  for (int l = 3; l >= 0; --l) {
    const int fin = fan_in(l);
    const __nv_bfloat16* hin = (l == 0) ? M->X : M->h[l - 1];
    HS_TRY(transpose(dz, B, WIDTH, M->tA, st));
    HS_TRY(transpose(hin, B, fin, M->tB, st));
    EpiArgs e = epi(WIDTH, fin);
    e.out_f32 = M->g + w_off(l);
    e.ld_f32 = fin;
    e.split_ws = M->split_ws;
    e.split_ws_floats = M->split_ws_floats;
    HS_TRY(gemm<EPI_F32>(M->tA, WIDTH, M->tB, fin, B, e, M->status, st));
    HS_TRY(colsum(dz, B, WIDTH, M->split_ws, M->g + b_off(l), st));
    if (l > 0) {
      EpiArgs d = epi(B, WIDTH);
      d.out_bf16 = dz_next;
      d.ld_bf16 = WIDTH;
      d.zprev = M->z[l - 1];
      d.ld_zprev = WIDTH;
      HS_TRY(gemm<EPI_GELU_BWD>(dz, B, M->wt + wb_off(l), WIDTH, WIDTH, d, M->status, st));
      __nv_bfloat16* t = dz; dz = dz_next; dz_next = t;
    }
  }
  return HAAR_OK;
}

static haar_status_t pack(haar_mlp_s* M, cudaStream_t st, int advance) {
  const long long n = (long long)w_total();
  k_pack<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(M->p, M->wb, M->wt, M->step, advance);
  return cuda_check(cudaGetLastError(), "k_pack launch");
}

static haar_status_t encode_raw(haar_mlp_s* M, const float* raw, int B, cudaStream_t st) {
  k_encode_raw<<<(B + 7) / 8, 256, 0, st>>>(raw, B, M->X);
  return cuda_check(cudaGetLastError(), "k_encode_raw launch");
}

}  // namespace mlpk
}  // namespace hs

#define HS_ENTRY(name)                                              \
  if (injected(name)) return set_error(HAAR_ERR_INJECTED, "%s: injected fault", name)

static void mlp_free(haar_mlp_s* M) {
  if (!M) return;
  void* ptrs[] = {M->p, M->g, M->m, M->v, M->wb, M->wt, M->X, M->h[0], M->h[1], M->h[2], M->h[3], M->z[0],
                  M->z[1], M->z[2], M->z[3], M->out, M->dout, M->dz, M->dz2, M->tA, M->tB, M->loss, M->iX,
                  M->ih0, M->ih1, M->weff, M->beff, M->status, M->step, M->split_ws};
  for (void* q : ptrs) cudaFree(q);
  delete M;
}

extern "C" {

long long haar_mlp_param_count(void) { return N_PARAMS; }

haar_status_t haar_mlp_create(int max_batch, int max_rows, int max_groups, haar_mlp_t* out) {
  HS_ENTRY("haar_mlp_create");
  if (out == nullptr) return set_error(HAAR_ERR_INVALID_ARG, "haar_mlp_create: null output");
  *out = nullptr;
  if (max_batch < 128 || max_batch % 128 != 0 || max_batch > (1 << 22))
    return set_error(HAAR_ERR_INVALID_ARG, "haar_mlp_create: max_batch %d must be a multiple of 128", max_batch);
  if (max_rows < 128 || max_rows % 128 != 0 || max_groups < 1 || max_groups > 65535)
    return set_error(HAAR_ERR_INVALID_ARG, "haar_mlp_create: max_rows %d (multiple of 128), max_groups %d", max_rows,
                     max_groups);
  haar_mlp_s* M = new (std::nothrow) haar_mlp_s();
  if (!M) return set_error(HAAR_ERR_NOMEM, "haar_mlp_create: host allocation failed");
  memset(M, 0, sizeof(*M));
  M->max_batch = max_batch;
  M->max_rows = max_rows;
  M->max_groups = max_groups;
  const size_t B = max_batch, R = max_rows, P = N_PARAMS, WT = w_total();
  cudaError_t e = cudaSuccess;
#define ALLOC(ptr, bytes) \
  if (e == cudaSuccess) e = cudaMalloc((void**)&(ptr), (bytes))
  ALLOC(M->p, P * 4);
  ALLOC(M->g, P * 4);
  ALLOC(M->m, P * 4);
  ALLOC(M->v, P * 4);
  ALLOC(M->wb, WT * 2);
  ALLOC(M->wt, WT * 2);
  ALLOC(M->X, B * N_IN * 2);
  for (int l = 0; l < 4; ++l) {
    ALLOC(M->h[l], B * WIDTH * 2);
    ALLOC(M->z[l], B * WIDTH * 4);
  }
  ALLOC(M->out, B * N_OUT * 4);
  ALLOC(M->dout, B * N_OUT * 2);
  ALLOC(M->dz, B * WIDTH * 2);
  ALLOC(M->dz2, B * WIDTH * 2);
  ALLOC(M->tA, B * N_OUT * 2);
  ALLOC(M->tB, B * N_IN * 2);
  ALLOC(M->loss, 4);
  ALLOC(M->iX, R * N_IN * 2);
  ALLOC(M->ih0, R * WIDTH * 2);
  ALLOC(M->ih1, R * WIDTH * 2);
  ALLOC(M->weff, (size_t)max_groups * WIDTH * 4 * 4);
  ALLOC(M->beff, (size_t)max_groups * 4 * 4);
  ALLOC(M->status, 16);
  ALLOC(M->step, 16);
  M->split_ws_floats = (long long)(max_batch / 256 > 1 ? max_batch / 256 : 1) * N_OUT * WIDTH;
  ALLOC(M->split_ws, (size_t)M->split_ws_floats * 4);
#undef ALLOC
  if (e != cudaSuccess) {
    mlp_free(M);
    return set_error(HAAR_ERR_NOMEM, "haar_mlp_create: allocation failed: %s", cudaGetErrorString(e));
  }
  e = cudaMemset(M->p, 0, P * 4);
  if (e == cudaSuccess) e = cudaMemset(M->m, 0, P * 4);
  if (e == cudaSuccess) e = cudaMemset(M->v, 0, P * 4);
  if (e == cudaSuccess) e = cudaMemset(M->status, 0, 16);
  if (e == cudaSuccess) e = cudaMemset(M->loss, 0, 4);
  if (e == cudaSuccess) e = cudaMemset(M->step, 0, 16);
  if (e != cudaSuccess) {
    mlp_free(M);
    return cuda_check(e, "haar_mlp_create: cudaMemset");
  }
  *out = M;
  return HAAR_OK;
}

haar_status_t haar_mlp_destroy(haar_mlp_t M) {
  HS_ENTRY("haar_mlp_destroy");
  if (!M) return HAAR_OK;
  cudaError_t e = cudaDeviceSynchronize();
  mlp_free(M);
  return cuda_check(e, "haar_mlp_destroy: synchronise");
}

haar_status_t haar_mlp_set_params(haar_mlp_t M, const float* params, void* stream) {
  HS_ENTRY("haar_mlp_set_params");
  if (!M || !params) return set_error(HAAR_ERR_INVALID_ARG, "haar_mlp_set_params: null argument");
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(M->p, params, N_PARAMS * 4, cudaMemcpyDefault, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(M->m, 0, N_PARAMS * 4, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(M->v, 0, N_PARAMS * 4, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(M->step, 0, sizeof(int), st);
  if (e != cudaSuccess) return cuda_check(e, "haar_mlp_set_params");
  return pack(M, st, 0);
}

haar_status_t haar_mlp_get_params(haar_mlp_t M, float* params, void* stream) {
  HS_ENTRY("haar_mlp_get_params");
  if (!M || !params) return set_error(HAAR_ERR_INVALID_ARG, "haar_mlp_get_params: null argument");
  return cuda_check(cudaMemcpyAsync(params, M->p, N_PARAMS * 4, cudaMemcpyDefault, (cudaStream_t)stream),
                    "haar_mlp_get_params");
}

static haar_status_t check_batch(haar_mlp_t M, int B, const char* who) {
  if (!M) return set_error(HAAR_ERR_INVALID_ARG, "%s: null surrogate", who);
  if (B < 128 || B % 128 != 0 || B > M->max_batch)
    return set_error(HAAR_ERR_INVALID_ARG, "%s: batch %d must be a multiple of 128 in [128, %d]", who, B, M->max_batch);
  return HAAR_OK;
}

haar_status_t haar_mlp_forward(haar_mlp_t M, const float* raw, int B, float* out, void* stream) {
  HS_ENTRY("haar_mlp_forward");
  haar_status_t r = check_batch(M, B, "haar_mlp_forward");
  if (r != HAAR_OK) return r;
  if (!raw || !out) return set_error(HAAR_ERR_INVALID_ARG, "haar_mlp_forward: null pointer");
  cudaStream_t st = (cudaStream_t)stream;
  HS_TRY(encode_raw(M, raw, B, st));
  HS_TRY(forward(M, B, st));
  return cuda_check(cudaMemcpyAsync(out, M->out, (size_t)B * N_OUT * 4, cudaMemcpyDeviceToDevice, st),
                    "haar_mlp_forward: copy");
}

haar_status_t haar_mlp_grads(haar_mlp_t M, const float* raw, const float* target, int B, float* grads, float* loss,
                             void* stream) {
  HS_ENTRY("haar_mlp_grads");
  haar_status_t r = check_batch(M, B, "haar_mlp_grads");
  if (r != HAAR_OK) return r;
  if (!raw || !target) return set_error(HAAR_ERR_INVALID_ARG, "haar_mlp_grads: null pointer");
  cudaStream_t st = (cudaStream_t)stream;
  HS_TRY(cuda_check(cudaMemsetAsync(M->loss, 0, 4, st), "haar_mlp_grads: memset"));
  HS_TRY(encode_raw(M, raw, B, st));
  HS_TRY(forward(M, B, st));
  HS_TRY(backward(M, B, target, st));
  if (grads)
    HS_TRY(cuda_check(cudaMemcpyAsync(grads, M->g, N_PARAMS * 4, cudaMemcpyDeviceToDevice, st), "haar_mlp_grads: copy"));
  if (loss) HS_TRY(cuda_check(cudaMemcpyAsync(loss, M->loss, 4, cudaMemcpyDeviceToDevice, st), "haar_mlp_grads: loss"));
  return HAAR_OK;
}

haar_status_t haar_mlp_train_step(haar_mlp_t M, const float* raw, const float* target, int B, float lr, float* loss,
                                  void* stream) {
  HS_ENTRY("haar_mlp_train_step");
  haar_status_t r = check_batch(M, B, "haar_mlp_train_step");
  if (r != HAAR_OK) return r;
  if (!raw || !target) return set_error(HAAR_ERR_INVALID_ARG, "haar_mlp_train_step: null pointer");
  cudaStream_t st = (cudaStream_t)stream;
  HS_TRY(cuda_check(cudaMemsetAsync(M->loss, 0, 4, st), "haar_mlp_train_step: memset"));
  HS_TRY(encode_raw(M, raw, B, st));
  HS_TRY(forward(M, B, st));
  HS_TRY(backward(M, B, target, st));
  k_adam<<<1024, 256, 0, st>>>(M->p, M->g, M->m, M->v, N_PARAMS, lr, 0.9f, 0.999f, 1e-8f, M->step);
  HS_TRY(cuda_check(cudaGetLastError(), "k_adam launch"));
  HS_TRY(pack(M, st, 1));
  if (loss) HS_TRY(cuda_check(cudaMemcpyAsync(loss, M->loss, 4, cudaMemcpyDeviceToDevice, st), "haar_mlp_train_step: loss"));
  return HAAR_OK;
}

haar_status_t haar_mlp_shade(haar_mlp_t M, int V, int S, const float* pos, const float* nrm, const float* cams,
                             const float* mu, const float* sigma, const int32_t* idx, const float* lighting, int C,
                             long long st_s, long long st_c, long long st_k, float* radiance, void* stream) {
  HS_ENTRY("haar_mlp_shade");
  if (!M || !pos || !nrm || !cams || !mu || !sigma || !idx || !lighting || !radiance)
    return set_error(HAAR_ERR_INVALID_ARG, "haar_mlp_shade: null argument");
  if (V < 1 || S < 1 || S > M->max_groups || C < 1 || C > 4)
    return set_error(HAAR_ERR_INVALID_ARG, "haar_mlp_shade: V=%d S=%d (max %d) C=%d (1..4)", V, S, M->max_groups, C);
  cudaStream_t st = (cudaStream_t)stream;
  k_fold<<<dim3(S, WIDTH / 32), 256, 0, st>>>(M->p, mu, sigma, idx, lighting, st_s, st_c, st_k, S, C, M->weff,
                                              M->beff);
  HS_TRY(cuda_check(cudaGetLastError(), "k_fold launch"));
  const long long rows = (long long)V * S;
  if ((long long)V * N_VCOLS <= (long long)M->max_rows * N_IN) {
    // fused: per-vertex features once, then every layer on chip
    k_vertex_features<<<(V + 7) / 8, 256, 0, st>>>(pos, nrm, V, M->iX);
    HS_TRY(cuda_check(cudaGetLastError(), "k_vertex_features launch"));
    CUtensorMap wm[4];
    for (int l = 0; l < 4; ++l)
      if (!encode_2d(&wm[l], M->wb + wb_off(l), (uint64_t)fan_in(l), (uint64_t)WIDTH, tc::BK, WIDTH))
        return set_error(HAAR_ERR_CUDA, "haar_mlp_shade: cuTensorMapEncodeTiled failed");
    FusedArgs fa;
    fa.V = V;
    fa.S = S;
    fa.C = C;
    fa.rows = rows;
    fa.vfeat = M->iX;
    fa.pos = pos;
    fa.cams = cams;
    fa.params = M->p;
    fa.weff = M->weff;
    fa.beff = M->beff;
    fa.radiance = radiance;
    const size_t smem = F_ACT_BYTES + (size_t)F_STAGES * F_W_BYTES + 1024;
    cudaError_t e = cudaFuncSetAttribute(k_mlp_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_check(e, "cudaFuncSetAttribute(k_mlp_fused)");
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long tiles = (rows + 127) / 128;
    const int grid = (int)(tiles < sms ? tiles : sms);
    k_mlp_fused<<<grid, F_THREADS, smem, st>>>(wm[0], wm[1], wm[2], wm[3], fa, M->status);
    return cuda_check(cudaGetLastError(), "k_mlp_fused launch");
  }
  for (long long r0 = 0; r0 < rows; r0 += M->max_rows) {
    const int n = (int)((rows - r0) < M->max_rows ? (rows - r0) : M->max_rows);
    k_encode_scene<<<(n + 7) / 8, 256, 0, st>>>(pos, nrm, cams, V, r0, n, M->iX);
    HS_TRY(cuda_check(cudaGetLastError(), "k_encode_scene launch"));
    const __nv_bfloat16* in = M->iX;
    __nv_bfloat16* bufs[2] = {M->ih0, M->ih1};
    for (int l = 0; l < 3; ++l) {
      EpiArgs e = epi(n, WIDTH);
      e.bias = M->p + b_off(l);
      e.out_bf16 = bufs[l & 1];
      e.ld_bf16 = WIDTH;
      HS_TRY(gemm<EPI_BIAS_GELU>(in, n, M->wb + wb_off(l), WIDTH, fan_in(l), e, M->status, st));
      in = bufs[l & 1];
    }
    EpiArgs e = epi(n, WIDTH);
    e.bias = M->p + b_off(3);
    e.weff = M->weff;
    e.beff = M->beff;
    e.rows_per_group = V;
    e.groups = S;
    e.C = C;
    e.row0 = (int)r0;
    e.radiance = radiance;
    HS_TRY(gemm<EPI_SHADE>(in, n, M->wb + wb_off(3), WIDTH, WIDTH, e, M->status, st));
  }
  return HAAR_OK;
}

haar_status_t haar_mlp_status(haar_mlp_t M, int* out) {
  HS_ENTRY("haar_mlp_status");
  if (!M || !out) return set_error(HAAR_ERR_INVALID_ARG, "haar_mlp_status: null argument");
  cudaError_t e = cudaMemcpy(out, M->status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemset(M->status, 0, sizeof(int));
  return cuda_check(e, "haar_mlp_status");
}

}  // extern "C"
