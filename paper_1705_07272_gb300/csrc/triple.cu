// The paper's shading loop on the GPU (Sec. "Algorithmic optimization", Sec.
// "Experimental results": rotation input pass, rotation pass, triple integral
// pass).  The rotation pass is haar_shift; this file holds the rotation input
// pass (each vertex's normal -> rotation record) and the triple integral pass:
// the Haar triple product of lighting x rotated BRDF x visibility by the
// Tripling Coefficient Theorem (Sec. "Related work"), square by square:
//   out = sum_k a_k b_k c_k / H                                   (scaling)
//       + sum over squares Q of side B, types t in {H, V, D}:
//           (1/B) sum over the 6 orderings of (H, V, D) of a_t1 b_t2 c_t3
//           + a_t b_t m_c(Q) + a_t c_t m_b(Q) + b_t c_t m_a(Q)
// where m_x(Q) is factor x's mean over Q: the value of its coarser basis
// functions there.  Means follow top down: a child quadrant's mean is its
// parent's plus the parent's three details times their +-1/B signs.
#include <math.h>

#include "rotcoord.cuh"
#include "tc.cuh"

namespace hs {

// ---------------------------------------------------------------- rotation input pass

// R = Rx(-theta_N) Ry(-phi_N) from the unit normal without trigonometry:
// cos(phi) = n_z / rho, sin(phi) = n_x / rho, cos(theta) = n_y, sin(theta) =
// rho = sqrt(n_x^2 + n_z^2) (phi = 0 on the poles).  FP64: a per-frame record.
__global__ void k_normal_rotations(int V, const float* __restrict__ nrm, double* __restrict__ params) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= V) return;
  double x = nrm[3 * v], y = nrm[3 * v + 1], z = nrm[3 * v + 2];
  const double inv = 1.0 / sqrt(x * x + y * y + z * z);
  x *= inv;
  y *= inv;
  z *= inv;
  const double rho = sqrt(x * x + z * z);
  const double cp = rho > 0.0 ? z / rho : 1.0, sp = rho > 0.0 ? x / rho : 0.0;
  const double ct = y, st = rho;
  double* R = params + 9 * (long long)v;
  R[0] = cp;      R[1] = 0.0;  R[2] = -sp;
  R[3] = st * sp; R[4] = ct;   R[5] = st * cp;
  R[6] = ct * sp; R[7] = -st;  R[8] = ct * cp;
}

haar_status_t launch_normal_rotations(int V, const float* nrm, double* params, cudaStream_t st) {
  k_normal_rotations<<<(V + 255) / 256, 256, 0, st>>>(V, nrm, params);
  return cuda_check(cudaGetLastError(), "k_normal_rotations launch");
}

// ---------------------------------------------------------------- triple integral pass

struct TripleArgs {
  int H, W, n, q, N, Nm, V, C;
  const float* light;    // [C][N]
  const float* brdf;     // row v at brdf + v * sb
  const float* vis;      // row v at vis + v * sv
  long long sb, sv;
  float* out;            // [V][C]
  const float* ma;       // [C][Nm] lighting means, level n first
  const float4* pk;      // [Nm][C] per square: the lighting's (H, V, D) details and mean
  int* status;
};

// means of level l start at q (4^(n-l) - 1) / 3 = (g_l - q) / 3 with g_l the
// level's square count; the finest level's children are not needed
__device__ __forceinline__ int mean_off(int g, int q) { return (g - q) / 3; }

// child means of square k (row r, column col of a level with `cols` columns)
// from its mean m and details (h, v, d) of side B
__device__ __forceinline__ void put_children(float* M, int coff, int r, int col, int cols, float m, float h,
                                             float v, float d, float invB) {
  const int c2 = 2 * cols;
  float* p = M + coff + (2 * r) * c2 + 2 * col;
  p[0] = m + (-h - v + d) * invB;
  p[1] = m + (h - v - d) * invB;
  p[c2] = m + (-h + v - d) * invB;
  p[c2 + 1] = m + (h + v + d) * invB;
}

// One channel's lighting means over every square (a whole CTA, top down),
// then every square's (H, V, D, mean) packed as one float4 per channel.
__device__ void light_means(const TripleArgs& a, int ch, float* ma, float4* pk) {
  const float* L = a.light + (long long)ch * a.N;
  float* M = ma + (long long)ch * a.Nm;
  for (int k = threadIdx.x; k < a.q; k += blockDim.x) M[k] = L[k] / (float)a.H;
  __syncthreads();
  for (int l = a.n; l >= 2; --l) {
    const int g = a.q << (2 * (a.n - l)), cols = a.W >> l, moff = mean_off(g, a.q);
    const float invB = 1.0f / (float)(1 << l);
    for (int k = threadIdx.x; k < g; k += blockDim.x) {
      const int r = k / cols, col = k - r * cols;
      put_children(M, moff + g, r, col, cols, M[moff + k], L[g + k], L[2 * g + k], L[3 * g + k], invB);
    }
    __syncthreads();
  }
  for (int l = a.n; l >= 1; --l) {
    const int g = a.q << (2 * (a.n - l)), moff = mean_off(g, a.q);
    for (int k = threadIdx.x; k < g; k += blockDim.x)
      pk[(long long)(moff + k) * a.C + ch] = make_float4(L[g + k], L[2 * g + k], L[3 * g + k], M[moff + k]);
  }
}

// The lighting's means and packed squares, one CTA per channel; block 0 also
// clears the status word of the call.
__global__ void __launch_bounds__(256) k_triple_means(TripleArgs a, float* ma, float4* pk) {
  if (blockIdx.x == 0 && threadIdx.x == 0) *a.status = 0;
  light_means(a, blockIdx.x, ma, pk);
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(dst), "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

// One CTA per vertex: the squares are visited level by level from the
// coarsest, the factors' means for the next level written as they go.  With
// STAGED both factors' rows first arrive in shared memory by two bulk copies
// (one latency per vertex); without it (maps whose rows would leave too few
// CTAs per SM) each level's details are read straight from global memory,
// coalesced, and shared memory holds only the means.
template <int C, int T, bool STAGED>
__global__ void __launch_bounds__(T) k_triple(TripleArgs a) {
  extern __shared__ __align__(16) float sm[];
  float* mb = sm + (STAGED ? 2 * a.N : 0);   // [Nm] BRDF means
  float* mc = mb + a.Nm;                     // [Nm] visibility means
  __shared__ __align__(8) unsigned long long bar;
  __shared__ int abort_flag;
  __shared__ float red[T / 32][C];
  const int v = blockIdx.x, t = threadIdx.x;
  const float* sb = STAGED ? sm : a.brdf + (long long)v * a.sb;        // BRDF row
  const float* sc = STAGED ? sm + a.N : a.vis + (long long)v * a.sv;   // visibility row
  if (STAGED) {
    const uint32_t b32 = tc::smem_u32(&bar);
    if (t == 0) {
      abort_flag = 0;
      tc::mbar_init(b32, 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (t == 0) {
      const uint32_t bytes = (uint32_t)a.N * 4u;
      tc::mbar_arrive_tx(b32, 2u * bytes);
      bulk_g2s(tc::smem_u32(sm), a.brdf + (long long)v * a.sb, bytes, b32);
      bulk_g2s(tc::smem_u32(sm + a.N), a.vis + (long long)v * a.sv, bytes, b32);
    }
    bool ok = true;
    if (t < 32) ok = tc::mbar_wait(b32, 0, a.status, &abort_flag);   // one warp polls, the rest sleep
    if (!__syncthreads_and(ok)) {
      if (t < C) a.out[(long long)v * C + t] = __int_as_float(0x7fc00000);
      return;
    }
  }
  auto ld = [](const float* p, int i) { return STAGED ? p[i] : __ldg(p + i); };
  float acc[C];
#pragma unroll
  for (int ch = 0; ch < C; ++ch) acc[ch] = 0.0f;
  const float invH = 1.0f / (float)a.H;
  for (int k = t; k < a.q; k += T) {          // three scaling functions
    const float bk = ld(sb, k), ck = ld(sc, k), bc = bk * ck;
#pragma unroll
    for (int ch = 0; ch < C; ++ch) acc[ch] += __ldg(a.light + (long long)ch * a.N + k) * bc * invH;
    mb[k] = bk * invH;
    mc[k] = ck * invH;
  }
  __syncthreads();
  const int logW = 31 - __clz(a.W);
  for (int l = a.n; l >= 1; --l) {
    const int g = a.q << (2 * (a.n - l)), cols = a.W >> l, lc = logW - l, moff = mean_off(g, a.q);
    const float invB = 1.0f / (float)(1 << l);
    for (int k = t; k < g; k += T) {
      const float bH = ld(sb, g + k), bV = ld(sb, 2 * g + k), bD = ld(sb, 3 * g + k);
      const float cH = ld(sc, g + k), cV = ld(sc, 2 * g + k), cD = ld(sc, 3 * g + k);
      const float mbk = mb[moff + k], mck = mc[moff + k];
      // the factors' products that do not involve the lighting
      const float x1 = (bV * cD + bD * cV) * invB, x2 = (bH * cD + bD * cH) * invB, x3 = (bH * cV + bV * cH) * invB;
      const float yH = bH * mck + cH * mbk, yV = bV * mck + cV * mbk, yD = bD * mck + cD * mbk;
      const float bc = bH * cH + bV * cV + bD * cD;
      const float4* P = a.pk + (long long)(moff + k) * C;
#pragma unroll
      for (int ch = 0; ch < C; ++ch) {
        const float4 L4 = __ldg(P + ch);
        acc[ch] += L4.x * (x1 + yH) + L4.y * (x2 + yV) + L4.z * (x3 + yD) + bc * L4.w;
      }
      if (l > 1) {
        const int r = k >> lc, col = k & (cols - 1);
        put_children(mb, moff + g, r, col, cols, mbk, bH, bV, bD, invB);
        put_children(mc, moff + g, r, col, cols, mck, cH, cV, cD, invB);
      }
    }
    __syncthreads();
  }
  const int lane = t & 31, warp = t >> 5;
#pragma unroll
  for (int ch = 0; ch < C; ++ch) {
    float x = acc[ch];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) red[warp][ch] = x;
  }
  __syncthreads();
  if (t < C) {
    float x = 0.0f;
#pragma unroll
    for (int w = 0; w < T / 32; ++w) x += red[w][t];
    a.out[(long long)v * C + t] = x;
  }
}

// ---------------------------------------------------------------- fused rotation + triple integral

// The rotation pass and the triple integral pass in one kernel, one CTA per
// vertex.  The vertex's BRDF map is resampled under its rotation record
// (g(w) = f(R w), bilinear, SPHERE extension: the exact operator of
// haar_shift's rotations), 2 x 2 pixels per thread, straight into the first
// level of a bottom-up Haar analysis in shared memory.  Each square's BRDF
// details and mean (its scaling value / B) enter the same case sum as
// k_triple, with the visibility's details and top-down means.  Neither the
// rotated BRDF nor its pixels reach memory.
struct ShadeTripleArgs {
  TripleArgs t;
  const float* F;            // [H][W] the local BRDF map in pixels
  const float4* tab_t;       // [H] (sin, cos) of theta_i as float pairs (hi, lo, hi, lo)
  const float4* tab_p;       // [W] (sin, cos) of phi_j as float pairs
  const double* params;      // [V][9] rotation records
};

// Set-up: blocks 0..C-1 the lighting means, block C the BRDF's pixel map
// (inverse transform, top down in shared memory) and the angle tables.
__global__ void __launch_bounds__(256) k_shade_triple_setup(ShadeTripleArgs s, const float* brdf_local, float* F,
                                                           float4* tab_t, float4* tab_p) {
  const TripleArgs& a = s.t;
  if (blockIdx.x < (unsigned)gridDim.x - 1) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *a.status = 0;
    light_means(a, blockIdx.x, const_cast<float*>(a.ma), const_cast<float4*>(a.pk));
    return;
  }
  extern __shared__ __align__(16) float buf[];       // two planes of N floats
  float* X = buf;
  float* Y = buf + a.N;
  for (int k = threadIdx.x; k < a.q; k += blockDim.x) X[k] = brdf_local[k];
  __syncthreads();
  for (int l = a.n; l >= 1; --l) {                    // A_l [rows][cols] -> A_{l-1} [2 rows][2 cols]
    const int g = a.q << (2 * (a.n - l)), cols = a.W >> l;
    for (int k = threadIdx.x; k < g; k += blockDim.x) {
      const int r = k / cols, col = k - r * cols;
      const float A = X[k], h = brdf_local[g + k], v = brdf_local[2 * g + k], d = brdf_local[3 * g + k];
      float* o = Y + (2 * r) * (2 * cols) + 2 * col;
      o[0] = 0.5f * (A - h - v + d);
      o[1] = 0.5f * (A + h - v - d);
      o[2 * cols] = 0.5f * (A - h + v - d);
      o[2 * cols + 1] = 0.5f * (A + h + v + d);
    }
    __syncthreads();
    float* tmp = X;
    X = Y;
    Y = tmp;
  }
  for (int k = threadIdx.x; k < a.N; k += blockDim.x) F[k] = X[k];
  for (int i = threadIdx.x; i < a.H; i += blockDim.x) {
    double sv, cv;
    sincospi((i + 0.5) / a.H, &sv, &cv);
    const float sh = (float)sv, ch = (float)cv;
    tab_t[i] = make_float4(sh, (float)(sv - (double)sh), ch, (float)(cv - (double)ch));
  }
  for (int j = threadIdx.x; j < a.W; j += blockDim.x) {
    double sv, cv;
    sincospi(2.0 * (j + 0.5) / a.W, &sv, &cv);
    const float sh = (float)sv, ch = (float)cv;
    tab_p[j] = make_float4(sh, (float)(sv - (double)sh), ch, (float)(cv - (double)ch));
  }
}

// Per-vertex rotation tables in shared memory for rot_source (R = Ry(a)
// Rx(b) Ry(c) of the vertex's record): sin/cos(phi_j + c) [W], sin/cos(phi_m
// - a) [W] and the row products of b [2H], all float pairs, built from the
// map's FP64-derived pair tables and the record's angles by error-free
// products and sums.
struct RotTabs {
  float4* psi;
  float4* al;
  float4* row;
  float a_px;
};

__device__ void build_rot_tabs(const ShadeTripleArgs& s, const double* ang, const RotTabs& rt, int t, int T) {
  const TripleArgs& a = s.t;
  const RotAngles g = rot_angles(ang);
  for (int j = t; j < a.W; j += T) rot_col_entries(s.tab_p[j], g, rt.psi[j], rt.al[j]);
  for (int i = t; i < a.H; i += T) rot_row_entries(s.tab_t[i], g, rt.row[2 * i], rt.row[2 * i + 1]);
}

// The rotated BRDF at output pixel (i, j): the source position from
// rot_source (integer anchors plus float-pair offsets), bilinear with the
// SPHERE extension (one reflection across a pole at most).
__device__ __forceinline__ float rot_sample(const ShadeTripleArgs& s, const RotTabs& rt, int i, int j,
                                            float inv_dth, float inv_dph) {
  const TripleArgs& a = s.t;
  const RotSrc o = rot_source<false>(s.tab_t[i], rt.row[2 * i], rt.row[2 * i + 1], rt.psi[j], rt.al, s.tab_t,
                                     rt.a_px, inv_dth, inv_dph, a.H, a.W);
  int r0 = o.r, r1 = o.r + 1, s0 = 0, s1 = 0;
  if (r0 < 0) { r0 = 0; s0 = a.W >> 1; }
  if (r1 >= a.H) { r1 = a.H - 1; s1 = a.W >> 1; }
  const int m = a.W - 1;
  const float f00 = __ldg(s.F + r0 * a.W + ((o.c + s0) & m)), f01 = __ldg(s.F + r0 * a.W + ((o.c + 1 + s0) & m));
  const float f10 = __ldg(s.F + r1 * a.W + ((o.c + s1) & m)), f11 = __ldg(s.F + r1 * a.W + ((o.c + 1 + s1) & m));
  const float top = fmaf(o.fv, f01 - f00, f00), bot = fmaf(o.fv, f11 - f10, f10);
  return fmaf(o.fu, bot - top, top);
}

template <int C, int T>
__global__ void __launch_bounds__(T) k_shade_triple(ShadeTripleArgs s) {
  const TripleArgs& a = s.t;
  extern __shared__ __align__(16) float sm[];
  float* sc = sm;                      // [N] visibility row
  float* mc = sc + a.N;                // [Nm] visibility means, level n first
  float* sa = mc + a.Nm;               // [Nm] the rotated BRDF's scaling values A_l, same layout
  RotTabs rt;                          // [2W + 2H] float4 after them, 16-byte aligned
  rt.psi = reinterpret_cast<float4*>(sm + ((a.N + 2 * a.Nm + 3) & ~3));
  rt.al = rt.psi + a.W;
  rt.row = rt.al + a.W;
  __shared__ double ang[6];
  __shared__ __align__(8) unsigned long long bar;
  __shared__ int abort_flag;
  __shared__ float red[T / 32][C];
  const int v = blockIdx.x, t = threadIdx.x;
  const uint32_t b32 = tc::smem_u32(&bar);
  if (t == 0) {
    abort_flag = 0;
    tc::mbar_init(b32, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (t == 0) {
    tc::mbar_arrive_tx(b32, (uint32_t)a.N * 4u);
    bulk_g2s(tc::smem_u32(sc), a.vis + (long long)v * a.sv, (uint32_t)a.N * 4u, b32);
  }
  if (t == 0) {
    double R[9];
    for (int k = 0; k < 9; ++k) R[k] = s.params[9 * (long long)v + k];
    yxy_angles(R, ang);
  }
  __syncthreads();
  rt.a_px = (float)(atan2(ang[0], ang[1]) * (a.W / (2.0 * 3.14159265358979323846)) - 0.5);
  build_rot_tabs(s, ang, rt, t, T);
  const int logW = 31 - __clz(a.W);
  const float inv_dth = (float)a.H * 0.318309886183791f, inv_dph = (float)a.W * 0.159154943091895f;
  bool ok = true;
  if (t < 32) ok = tc::mbar_wait(b32, 0, a.status, &abort_flag);
  if (!__syncthreads_and(ok)) {
    if (t < C) a.out[(long long)v * C + t] = __int_as_float(0x7fc00000);
    return;
  }
  // visibility means, top down
  const float invH = 1.0f / (float)a.H;
  for (int k = t; k < a.q; k += T) mc[k] = sc[k] * invH;
  __syncthreads();
  for (int l = a.n; l >= 2; --l) {
    const int g = a.q << (2 * (a.n - l)), cols = a.W >> l, lc = logW - l, moff = mean_off(g, a.q);
    const float invB = 1.0f / (float)(1 << l);
    for (int k = t; k < g; k += T)
      put_children(mc, moff + g, k >> lc, k & (cols - 1), cols, mc[moff + k], sc[g + k], sc[2 * g + k],
                   sc[3 * g + k], invB);
    __syncthreads();
  }
  // the rotated BRDF analysed bottom up, with the case sum of every square;
  // level 1 resamples its 2 x 2 pixels itself (the pixels are never stored)
  float acc[C];
#pragma unroll
  for (int ch = 0; ch < C; ++ch) acc[ch] = 0.0f;
  for (int l = 1; l <= a.n; ++l) {
    const int g = a.q << (2 * (a.n - l)), cols = a.W >> l, lc = logW - l, moff = mean_off(g, a.q);
    const float invB = 1.0f / (float)(1 << l);
    const float* src = sa + moff + g;                 // A_{l-1}, [2 rows][2 cols] (l > 1)
    for (int k = t; k < g; k += T) {
      const int r = k >> lc, col = k & (cols - 1);
      float ta, tb, tc_, td;
      if (l == 1) {
        ta = rot_sample(s, rt, 2 * r, 2 * col, inv_dth, inv_dph);
        tb = rot_sample(s, rt, 2 * r, 2 * col + 1, inv_dth, inv_dph);
        tc_ = rot_sample(s, rt, 2 * r + 1, 2 * col, inv_dth, inv_dph);
        td = rot_sample(s, rt, 2 * r + 1, 2 * col + 1, inv_dth, inv_dph);
      } else {
        const float* c0 = src + (2 * r) * (2 * cols) + 2 * col;
        ta = c0[0];
        tb = c0[1];
        tc_ = c0[2 * cols];
        td = c0[2 * cols + 1];
      }
      const float A = 0.5f * (ta + tb + tc_ + td);
      const float bH = 0.5f * (tb + td - ta - tc_), bV = 0.5f * (tc_ + td - ta - tb), bD = 0.5f * (ta + td - tb - tc_);
      const float mbk = A * invB;
      const float cH = sc[g + k], cV = sc[2 * g + k], cD = sc[3 * g + k];
      const float mck = mc[moff + k];
      const float x1 = (bV * cD + bD * cV) * invB, x2 = (bH * cD + bD * cH) * invB, x3 = (bH * cV + bV * cH) * invB;
      const float yH = bH * mck + cH * mbk, yV = bV * mck + cV * mbk, yD = bD * mck + cD * mbk;
      const float bc = bH * cH + bV * cV + bD * cD;
      const float4* P = a.pk + (long long)(moff + k) * C;
#pragma unroll
      for (int ch = 0; ch < C; ++ch) {
        const float4 L4 = __ldg(P + ch);
        acc[ch] += L4.x * (x1 + yH) + L4.y * (x2 + yV) + L4.z * (x3 + yD) + bc * L4.w;
      }
      if (l == a.n) {                                  // three scaling functions
        const float s3 = A * sc[k] * invH;
#pragma unroll
        for (int ch = 0; ch < C; ++ch) acc[ch] += __ldg(a.light + (long long)ch * a.N + k) * s3;
      }
      sa[moff + k] = A;
    }
    __syncthreads();
  }
  const int lane = t & 31, warp = t >> 5;
#pragma unroll
  for (int ch = 0; ch < C; ++ch) {
    float x = acc[ch];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) red[warp][ch] = x;
  }
  __syncthreads();
  if (t < C) {
    float x = 0.0f;
#pragma unroll
    for (int w = 0; w < T / 32; ++w) x += red[w][t];
    a.out[(long long)v * C + t] = x;
  }
}

static long long round4(long long x) { return (x + 3) & ~3LL; }

long long shade_triple_work_floats(int H, int W, int C) {
  const long long N = (long long)H * W, q = W / H, Nm = (N - q) / 3;
  return 4 + round4((long long)C * Nm) + 4LL * C * Nm + round4(N) + 4LL * H + 4LL * W;
}

template <int C>
static haar_status_t launch_shade_triple_c(const ShadeTripleArgs& s, const float* brdf_local, float* F,
                                           float4* tab_t, float4* tab_p, cudaStream_t st) {
  const TripleArgs& a = s.t;
  const size_t setup_smem = 2 * (size_t)a.N * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(k_shade_triple_setup, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)setup_smem);
  if (e != cudaSuccess) return cuda_check(e, "k_shade_triple_setup attribute");
  k_shade_triple_setup<<<C + 1, 256, setup_smem, st>>>(s, brdf_local, F, tab_t, tab_p);
  haar_status_t r = cuda_check(cudaGetLastError(), "k_shade_triple_setup launch");
  if (r != HAAR_OK) return r;
  const size_t smem = ((((size_t)a.N + 2 * (size_t)a.Nm + 3) & ~(size_t)3) + 8 * ((size_t)a.W + a.H)) * sizeof(float);
  if (a.N <= 2048) {
    e = cudaFuncSetAttribute(k_shade_triple<C, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_check(e, "k_shade_triple attribute");
    k_shade_triple<C, 128><<<a.V, 128, smem, st>>>(s);
  } else {
    e = cudaFuncSetAttribute(k_shade_triple<C, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_check(e, "k_shade_triple attribute");
    k_shade_triple<C, 256><<<a.V, 256, smem, st>>>(s);
  }
  return cuda_check(cudaGetLastError(), "k_shade_triple launch");
}

static void triple_geometry(TripleArgs& a, int H, int W, int V) {
  a.H = H;
  a.W = W;
  a.n = 0;
  while ((1 << a.n) < H) ++a.n;
  a.q = W / H;
  a.N = H * W;
  a.Nm = (a.N - a.q) / 3;
  a.V = V;
}

haar_status_t launch_shade_triple(int H, int W, int C, int V, const float* light, const float* brdf_local,
                                  const double* params, const float* vis, long long sv, float* out, float* work,
                                  cudaStream_t st) {
  ShadeTripleArgs s;
  TripleArgs& a = s.t;
  triple_geometry(a, H, W, V);
  a.light = light;
  a.brdf = nullptr;
  a.sb = 0;
  a.vis = vis;
  a.sv = sv;
  a.out = out;
  a.status = reinterpret_cast<int*>(work);
  a.C = C;
  float* ma = work + 4;
  a.ma = ma;
  float4* pk = reinterpret_cast<float4*>(ma + round4((long long)C * a.Nm));
  a.pk = pk;
  float* F = reinterpret_cast<float*>(pk + (long long)C * a.Nm);
  float4* tab_t = reinterpret_cast<float4*>(F + round4(a.N));
  float4* tab_p = tab_t + H;
  s.F = F;
  s.tab_t = tab_t;
  s.tab_p = tab_p;
  s.params = params;
  switch (C) {
    case 1: return launch_shade_triple_c<1>(s, brdf_local, F, tab_t, tab_p, st);
    case 2: return launch_shade_triple_c<2>(s, brdf_local, F, tab_t, tab_p, st);
    case 3: return launch_shade_triple_c<3>(s, brdf_local, F, tab_t, tab_p, st);
    default: return launch_shade_triple_c<4>(s, brdf_local, F, tab_t, tab_p, st);
  }
}

long long triple_work_floats(int H, int W, int C) {
  const long long N = (long long)H * W, q = W / H, Nm = (N - q) / 3;
  return 4 + round4((long long)C * Nm) + 4LL * C * Nm;
}

size_t triple_smem_bytes(int H, int W) {
  const long long N = (long long)H * W, q = W / H;
  return (size_t)(2 * N + 2 * ((N - q) / 3)) * sizeof(float);
}

template <int C>
static haar_status_t launch_triple_c(const TripleArgs& a, float* ma, cudaStream_t st) {
  const size_t smem = triple_smem_bytes(a.H, a.W);
  k_triple_means<<<C, 256, 0, st>>>(a, ma, const_cast<float4*>(a.pk));
  haar_status_t r = cuda_check(cudaGetLastError(), "k_triple_means launch");
  if (r != HAAR_OK) return r;
  // up to 2048 coefficients both rows are staged by bulk copies; above, the
  // staged rows would leave 2 CTAs per SM, so the details stream from memory
  cudaError_t e;
  if (a.N <= 2048) {
    e = cudaFuncSetAttribute(k_triple<C, 128, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_check(e, "k_triple attribute");
    k_triple<C, 128, true><<<a.V, 128, smem, st>>>(a);
  } else {
    // (4 vertices per CTA sharing each square's lighting loads measured
    // slower, 1.56 against 1.27 ms: the kernel is latency-bound, not bound by
    // the lighting's L2 traffic)
    const size_t smem_m = 2 * (size_t)a.Nm * sizeof(float);
    e = cudaFuncSetAttribute(k_triple<C, 128, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_m);
    if (e != cudaSuccess) return cuda_check(e, "k_triple attribute");
    k_triple<C, 128, false><<<a.V, 128, smem_m, st>>>(a);
  }
  return cuda_check(cudaGetLastError(), "k_triple launch");
}

haar_status_t launch_triple(int H, int W, int C, int V, const float* light, const float* brdf, long long sb,
                            const float* vis, long long sv, float* out, float* work, cudaStream_t st) {
  TripleArgs a;
  triple_geometry(a, H, W, V);
  a.light = light;
  a.brdf = brdf;
  a.vis = vis;
  a.sb = sb;
  a.sv = sv;
  a.out = out;
  a.C = C;
  a.status = reinterpret_cast<int*>(work);
  float* ma = work + 4;
  a.ma = ma;
  a.pk = reinterpret_cast<float4*>(ma + round4((long long)C * a.Nm));
  switch (C) {
    case 1: return launch_triple_c<1>(a, ma, st);
    case 2: return launch_triple_c<2>(a, ma, st);
    case 3: return launch_triple_c<3>(a, ma, st);
    default: return launch_triple_c<4>(a, ma, st);
  }
}

}  // namespace hs
