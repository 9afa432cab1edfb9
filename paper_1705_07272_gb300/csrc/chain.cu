// The paper's own rotation route (an approximation of the exact shift):
// the rotated map's finest derivative fields by the chain rule (Sec.
// "Rotating Haar", Eq. pde1-pde3, with the mixed term's second-order chain
// rule completed), then its detail coefficients by the derivative-to-
// coefficient filters of Sec. "Mathematical description" (Eq. conv: a
// triangle of B - 1 taps, peak B / 2, along the derivative's direction
// (Eq. tker), a box of B taps, 1 / B, across it (Eq. sker), decimated by B;
// the diagonal band the triangle in both directions, divided by B).
//
// Fields on the output grid, in pixel-index units (source position u =
// Theta / dtheta - 1/2, v = Phi / dphi - 1/2):
//   g_theta(i, j)    at (i + 1/2, j):       F_u u_i + F_v v_i
//   g_phi(i, j)      at (i, j + 1/2):       F_u u_j + F_v v_j
//   g_thetaphi(i, j) at (i + 1/2, j + 1/2): F_uu u_i u_j + F_uv (u_i v_j + u_j v_i)
//                                           + F_vv v_i v_j + F_u u_ij + F_v v_ij
// with the source derivatives from the pixel map's finite differences,
// sampled bilinearly where each difference is centred, and the scaling
// coefficients from block sums of the bilinearly resampled map.
#include <math.h>

#include "common.cuh"

namespace hs {

struct ChainArgs {
  Geometry g;
  int K;
  long long st_s, st_c, st_k;
  float* out;
  const float* pix;       // [C][H][W] synthesised source map
  float* ws;              // [S][C][4][N]: g, g_theta, g_phi, g_thetaphi
  float* rot;             // [S][32]: R rounded to float (9), then R - that (9)
  float4* tab_t;          // [2H + 1]: sin, its residual, cos, its residual of t pi / (2H)
  float4* tab_p;          // [2W + 1]: the same for t pi / W
};

// Floats of the workspace: the fields, then the rotations and the tables
// (each part a multiple of 4 floats, so the tables stay 16-byte aligned).
size_t chain_ws_floats(const Geometry& g, int S) {
  return (size_t)S * g.C * 4 * (size_t)g.N + (size_t)S * 32 + 4 * (size_t)(2 * g.H + 1) + 4 * (size_t)(2 * g.W + 1);
}

// Per launch, in FP64: each rotation R = Rz(gamma) Ry(beta) Rx(alpha) (Eq. tRot)
// as a pair of floats (hi, lo) with hi + lo = R to about 2^-48, and the sines
// and cosines of the half-pixel polar and azimuth angles the same way.
__global__ void k_chain_setup(ChainArgs a, const double* params, int S) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int nt = 2 * a.g.H + 1, np = 2 * a.g.W + 1;
  if (e < S) {
    double ca, sa, cb, sb, cg, sg;
    sincos(params[3 * e], &sa, &ca);
    sincos(params[3 * e + 1], &sb, &cb);
    sincos(params[3 * e + 2], &sg, &cg);
    const double R[9] = {cg * cb, cg * sb * sa - sg * ca, cg * sb * ca + sg * sa,
                         sg * cb, sg * sb * sa + cg * ca, sg * sb * ca - cg * sa,
                         -sb,     cb * sa,                cb * ca};
    float* o = a.rot + 32 * e;
    for (int k = 0; k < 9; ++k) {
      const float hi = (float)R[k];
      o[k] = hi;
      o[9 + k] = (float)(R[k] - (double)hi);
    }
  } else if (e < S + nt + np) {
    const int t = e - S;
    double sv, cv;
    if (t < nt) sincospi((double)t / (2.0 * a.g.H), &sv, &cv);
    else sincospi((double)(t - nt) / (double)a.g.W, &sv, &cv);
    const float sh = (float)sv, ch = (float)cv;
    const float4 v = make_float4(sh, (float)(sv - (double)sh), ch, (float)(cv - (double)ch));
    if (t < nt) a.tab_t[t] = v;
    else a.tab_p[t - nt] = v;
  }
}

__device__ __forceinline__ void ch_ext(int& i, int& j, int H, int W, int boundary) {
  if (boundary == HAAR_BOUNDARY_TORUS) {
    i %= H;
    if (i < 0) i += H;
  } else {
#pragma unroll 1
    for (int it = 0; it < 8 && (i < 0 || i >= H); ++it) {
      i = (i < 0) ? -1 - i : 2 * H - 1 - i;
      j += W >> 1;
    }
  }
  j %= W;
  if (j < 0) j += W;
}

// bilinear value of the extended map at (row bu + du, column bv + dv): the
// position as an integer base plus a small float offset, so that its fraction
// keeps float precision whatever the index
__device__ __forceinline__ float ch_bil(const float* F, int bu, float du, int bv, float dv, const Geometry& g) {
  const float fi = floorf(du), fj = floorf(dv);
  const float fu = du - fi, fv = dv - fj;
  const int i0 = bu + (int)fi, j0 = bv + (int)fj;
  float t[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    int i = i0 + (k >> 1), j = j0 + (k & 1);
    ch_ext(i, j, g.H, g.W, g.boundary);
    t[k] = __ldg(F + (long long)i * g.W + j);
  }
  return (1.0f - fu) * ((1.0f - fv) * t[0] + fv * t[1]) + fu * ((1.0f - fv) * t[2] + fv * t[3]);
}

// Unevaluated float pairs (hi + lo) with Dekker's error-free product (via FMA)
// and Knuth's error-free sum; the _rn intrinsics keep the compiler from
// contracting or reordering them.
struct DF {
  float h, l;
};

__device__ __forceinline__ DF df_norm(float s, float e) {       // |e| <= ulp(s) afterwards
  const float h = __fadd_rn(s, e);
  return {h, __fsub_rn(e, __fsub_rn(h, s))};
}

__device__ __forceinline__ DF df_mul(DF a, DF b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  return df_norm(p, e);
}

__device__ __forceinline__ DF df_add(DF a, DF b) {
  const float s = __fadd_rn(a.h, b.h);
  const float bb = __fsub_rn(s, a.h);
  const float e = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bb)), __fsub_rn(b.h, bb));
  return df_norm(s, __fadd_rn(e, __fadd_rn(a.l, b.l)));
}

struct ChJac {
  int iu, iv;             // source position u = iu + fu, v = iv + fv
  float fu, fv;
  float ui, uj, vi, vj, uij, vij;
};

// Below this q_x^2 + q_z^2 the rotated position is recomputed with float
// pairs.  There q = R p is a small difference of O(1) terms, and the
// azimuth atan2(q_x, q_z) with the 1 / rho factors of the Jacobian would turn
// float rounding of p and R (~1e-7 absolute) into errors of 1e-7 / rho.  The
// azimuth is then taken relative to the nearest source column centre psi, as
// atan2 of (q_x, q_z) turned by -psi, so that the column offset does not carry
// the rounding of a float angle either (the route's second-order term
// multiplies it by v_theta v_phi ~ 1 / rho^2).
constexpr float kPoleRefine = 0.1f;

// source position and its derivatives (index units) at the output position
// with polar angle table entry T and azimuth entry P: Theta = acos(q_y),
// Phi = atan2(q_x, q_z), q = R p(theta, phi); where q_x^2 + q_z^2 < 1e-8
// (a pole) the derivatives are 0
__device__ ChJac ch_jac(const float (&Rh)[9], const float (&Rl)[9], float4 T, float4 P, const float4* tab_p,
                        const Geometry& g) {
  const float dth = 3.14159265358979f / (float)g.H, dph = 6.28318530717959f / (float)g.W;
  const float st = T.x, ct = T.z, sp = P.x, cp = P.z;
  const float p[3] = {st * sp, ct, st * cp};
  const float pt[3] = {ct * sp, -st, ct * cp};
  const float pp[3] = {st * cp, 0.0f, -st * sp};
  const float ptp[3] = {ct * cp, 0.0f, -ct * sp};
  float q[3], qt[3], qp[3], qtp[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    q[r] = Rh[3 * r] * p[0] + Rh[3 * r + 1] * p[1] + Rh[3 * r + 2] * p[2];
    qt[r] = Rh[3 * r] * pt[0] + Rh[3 * r + 1] * pt[1] + Rh[3 * r + 2] * pt[2];
    qp[r] = Rh[3 * r] * pp[0] + Rh[3 * r + 1] * pp[1] + Rh[3 * r + 2] * pp[2];
    qtp[r] = Rh[3 * r] * ptp[0] + Rh[3 * r + 1] * ptp[1] + Rh[3 * r + 2] * ptp[2];
  }
  ChJac J;
  if (q[0] * q[0] + q[2] * q[2] < kPoleRefine) {
    const DF STh = {T.x, T.y}, CTh = {T.z, T.w}, SPh = {P.x, P.y}, CPh = {P.z, P.w};
    const DF pd[3] = {df_mul(STh, SPh), CTh, df_mul(STh, CPh)};
    DF qd[3];
#pragma unroll
    for (int r = 0; r < 3; r += 2) {                    // q_x and q_z
      DF acc = df_mul({Rh[3 * r], Rl[3 * r]}, pd[0]);
      acc = df_add(acc, df_mul({Rh[3 * r + 1], Rl[3 * r + 1]}, pd[1]));
      acc = df_add(acc, df_mul({Rh[3 * r + 2], Rl[3 * r + 2]}, pd[2]));
      qd[r] = acc;
      q[r] = acc.h;
    }
    // azimuth: nearest column c0 (centre psi = (c0 + 1/2) dphi), then the
    // small angle from psi
    int c0 = (int)rintf(atan2f(q[0], q[2]) / dph - 0.5f);
    c0 = (c0 % g.W + g.W) % g.W;
    const float4 Ps = tab_p[2 * c0 + 1];
    const DF Sps = {Ps.x, Ps.y}, Cps = {Ps.z, Ps.w};
    const DF cr = df_add(df_mul(qd[0], Cps), df_mul({-qd[2].h, -qd[2].l}, Sps));   // rho sin(Phi - psi)
    const DF dt = df_add(df_mul(qd[2], Cps), df_mul(qd[0], Sps));                 // rho cos(Phi - psi)
    J.iv = c0;
    J.fv = atan2f(cr.h, dt.h) / dph;
    // polar: from the nearer pole
    const float rho_ = sqrtf(q[0] * q[0] + q[2] * q[2]);
    if (q[1] >= 0.0f) {
      J.iu = 0;
      J.fu = atan2f(rho_, q[1]) / dth - 0.5f;
    } else {
      J.iu = g.H - 1;
      J.fu = 0.5f - atan2f(rho_, -q[1]) / dth;
    }
  } else {
    const float u = atan2f(sqrtf(q[0] * q[0] + q[2] * q[2]), q[1]) / dth - 0.5f;
    const float v = atan2f(q[0], q[2]) / dph - 0.5f;
    const float bu = floorf(u), bv = floorf(v);
    J.iu = (int)bu;
    J.fu = u - bu;
    J.iv = (int)bv;
    J.fv = v - bv;
  }
  const float rho2 = q[0] * q[0] + q[2] * q[2];
  const float rho = sqrtf(rho2);
  if (rho2 < 1e-8f) {
    J.ui = J.uj = J.vi = J.vj = J.uij = J.vij = 0.0f;
    return J;
  }
  const float Th_t = -qt[1] / rho, Th_p = -qp[1] / rho;
  const float rho_p = (q[0] * qp[0] + q[2] * qp[2]) / rho;
  const float Th_tp = -qtp[1] / rho + qt[1] * rho_p / rho2;
  const float N_t = q[2] * qt[0] - q[0] * qt[2];
  const float N_p = q[2] * qp[0] - q[0] * qp[2];
  const float N_tp = qp[2] * qt[0] + q[2] * qtp[0] - qp[0] * qt[2] - q[0] * qtp[2];
  const float r2_p = 2.0f * (q[0] * qp[0] + q[2] * qp[2]);
  const float Ph_t = N_t / rho2, Ph_p = N_p / rho2;
  const float Ph_tp = (N_tp * rho2 - N_t * r2_p) / (rho2 * rho2);
  J.ui = Th_t;
  J.uj = Th_p * dph / dth;
  J.vi = Ph_t * dth / dph;
  J.vj = Ph_p;
  J.uij = Th_tp * dph;
  J.vij = Ph_tp * dth;
  return J;
}

// one thread per output pixel and shift: the coordinates and Jacobians at the
// pixel and the three difference midpoints once, then every channel's fields
__global__ void __launch_bounds__(256) k_chain_fields(ChainArgs a) {
  pdl_wait();
  const Geometry& g = a.g;
  const int s = blockIdx.y;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= g.N) return;
  const int i = (int)(e / g.W), j = (int)(e - (long long)i * g.W);
  float Rh[9], Rl[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    Rh[k] = a.rot[32 * s + k];
    Rl[k] = a.rot[32 * s + 9 + k];
  }
  // angle tables at (i + 1/2) dtheta, (i + 1) dtheta and (j + 1/2) dphi, (j + 1) dphi
  const float4 T0 = a.tab_t[2 * i + 1], T1 = a.tab_t[2 * i + 2];
  const float4 P0 = a.tab_p[2 * j + 1], P1 = a.tab_p[2 * j + 2];
  const ChJac J0 = ch_jac(Rh, Rl, T0, P0, a.tab_p, g);
  const ChJac Ja = ch_jac(Rh, Rl, T1, P0, a.tab_p, g);
  const ChJac Jb = ch_jac(Rh, Rl, T0, P1, a.tab_p, g);
  const ChJac Jc = ch_jac(Rh, Rl, T1, P1, a.tab_p, g);
  for (int c = 0; c < g.C; ++c) {
    const float* F = a.pix + (long long)c * g.N;
    // the map sampled at a Jacobian's position plus (du, dv)
    auto at = [&](const ChJac& J, float du, float dv) { return ch_bil(F, J.iu, J.fu + du, J.iv, J.fv + dv, g); };
    const float gv = at(J0, 0.0f, 0.0f);
    const float fu_a = at(Ja, 0.5f, 0.0f) - at(Ja, -0.5f, 0.0f);
    const float fv_a = at(Ja, 0.0f, 0.5f) - at(Ja, 0.0f, -0.5f);
    const float fu_b = at(Jb, 0.5f, 0.0f) - at(Jb, -0.5f, 0.0f);
    const float fv_b = at(Jb, 0.0f, 0.5f) - at(Jb, 0.0f, -0.5f);
    const float f0 = at(Jc, 0.0f, 0.0f);
    const float fuu = at(Jc, 1.0f, 0.0f) - 2.0f * f0 + at(Jc, -1.0f, 0.0f);
    const float fvv = at(Jc, 0.0f, 1.0f) - 2.0f * f0 + at(Jc, 0.0f, -1.0f);
    const float fuv = at(Jc, 0.5f, 0.5f) - at(Jc, 0.5f, -0.5f) - at(Jc, -0.5f, 0.5f) + at(Jc, -0.5f, -0.5f);
    const float fu = at(Jc, 0.5f, 0.0f) - at(Jc, -0.5f, 0.0f);
    const float fv = at(Jc, 0.0f, 0.5f) - at(Jc, 0.0f, -0.5f);
    float* w = a.ws + ((long long)(s * g.C + c) * 4) * g.N + e;
    w[0] = gv;
    w[g.N] = fu_a * Ja.ui + fv_a * Ja.vi;
    w[2 * g.N] = fu_b * Jb.uj + fv_b * Jb.vj;
    w[3 * g.N] = fuu * Jc.ui * Jc.uj + fuv * (Jc.ui * Jc.vj + Jc.uj * Jc.vi) + fvv * Jc.vi * Jc.vj +
                 fu * Jc.uij + fv * Jc.vij;
  }
}

__device__ __forceinline__ void ch_put(const ChainArgs& a, int s, int c, int k, float v) {
  if (k < a.K) a.out[(long long)s * a.st_s + (long long)c * a.st_c + (long long)k * a.st_k] = v;
}

// block (r, col) of level lvl from the fields of plane (s, c): the sums of
// Eq. conv over positions p0 .. p0 + step ... (lanes / threads share them)
struct ChSums {
  float h, v, d;
};

__device__ __forceinline__ ChSums ch_block_sums(const float* gt, const float* gp, const float* gtp, int W, int r0,
                                                int c0, int B, int first, int step) {
  ChSums t = {0.0f, 0.0f, 0.0f};
  for (int p = first; p < B * B; p += step) {
    const int di = p / B, dj = p - di * B;
    const long long o = (long long)(r0 + di) * W + c0 + dj;
    const float ti = (float)min(di + 1, B - 1 - di), tj = (float)min(dj + 1, B - 1 - dj);
    if (dj < B - 1) t.h = fmaf(tj, __ldg(gp + o), t.h);
    if (di < B - 1) t.v = fmaf(ti, __ldg(gt + o), t.v);
    if (di < B - 1 && dj < B - 1) t.d = fmaf(ti * tj, __ldg(gtp + o), t.d);
  }
  return t;
}

// levels 1..3 (blocks of side <= 8): one thread per (plane, block)
__global__ void __launch_bounds__(256) k_chain_fine(ChainArgs a, long long per_plane) {
  const Geometry& g = a.g;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int plane = blockIdx.y;                   // s * C + c
  if (e >= per_plane) return;
  const int s = plane / g.C, c = plane - s * g.C;
  long long k = e;
  int lvl = 1;
  while (lvl < 3 && k >= (g.N >> (2 * lvl))) {
    k -= g.N >> (2 * lvl);
    ++lvl;
  }
  const int B = 1 << lvl, cols = g.W >> lvl;
  const int r = (int)(k / cols), col = (int)(k - (long long)r * cols);
  const float* base = a.ws + (long long)plane * 4 * g.N;
  const ChSums t = ch_block_sums(base + g.N, base + 2 * g.N, base + 3 * g.N, g.W, r * B, col * B, B, 0, 1);
  const int gl = g.q << (2 * (g.n - lvl));
  const int k0 = r * cols + col;
  const float inv = 1.0f / (float)B;
  ch_put(a, s, c, gl + k0, t.h * inv);
  ch_put(a, s, c, 2 * gl + k0, t.v * inv);
  ch_put(a, s, c, 3 * gl + k0, t.d * inv);
}

// levels 4..n and the scaling coefficients: one warp per (plane, block)
__global__ void __launch_bounds__(256) k_chain_coarse(ChainArgs a, long long per_plane) {
  const Geometry& g = a.g;
  const long long wi = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int plane = blockIdx.y;
  if (wi >= per_plane) return;
  const int s = plane / g.C, c = plane - s * g.C;
  const float* base = a.ws + (long long)plane * 4 * g.N;
  long long k = wi;
  if (k < g.q) {                                  // scaling block k: (sum of g over H x H) / H
    float t = 0.0f;
    for (long long p = lane; p < (long long)g.H * g.H; p += 32) {
      const long long di = p / g.H, dj = p - di * g.H;
      t += __ldg(base + di * g.W + k * g.H + dj);
    }
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) ch_put(a, s, c, (int)k, t / (float)g.H);
    return;
  }
  k -= g.q;
  int lvl = 4;
  while (lvl < g.n && k >= (g.N >> (2 * lvl))) {
    k -= g.N >> (2 * lvl);
    ++lvl;
  }
  const int B = 1 << lvl, cols = g.W >> lvl;
  const int r = (int)(k / cols), col = (int)(k - (long long)r * cols);
  ChSums t = ch_block_sums(base + g.N, base + 2 * g.N, base + 3 * g.N, g.W, r * B, col * B, B, lane, 32);
  for (int o = 16; o > 0; o >>= 1) {
    t.h += __shfl_xor_sync(0xffffffffu, t.h, o);
    t.v += __shfl_xor_sync(0xffffffffu, t.v, o);
    t.d += __shfl_xor_sync(0xffffffffu, t.d, o);
  }
  if (lane == 0) {
    const int gl = g.q << (2 * (g.n - lvl));
    const int k0 = r * cols + col;
    const float inv = 1.0f / (float)B;
    ch_put(a, s, c, gl + k0, t.h * inv);
    ch_put(a, s, c, 2 * gl + k0, t.v * inv);
    ch_put(a, s, c, 3 * gl + k0, t.d * inv);
  }
}

haar_status_t launch_chain(haar_shift_plan_s* p, const double* params, int S, void* out, cudaStream_t st) {
  ChainArgs a;
  const Geometry& g = p->geo;
  a.g = g;
  a.K = p->K;
  const long long K = p->K, C = g.C;
  switch (p->desc.out_layout) {
    case HAAR_LAYOUT_SCK: a.st_s = C * K; a.st_c = K; a.st_k = 1; break;
    case HAAR_LAYOUT_SKC: a.st_s = K * C; a.st_c = 1; a.st_k = C; break;
    case HAAR_LAYOUT_SKC4: a.st_s = K * 4; a.st_c = 1; a.st_k = 4; break;
    default: a.st_s = C; a.st_c = 1; a.st_k = (long long)S * C; break;
  }
  a.out = static_cast<float*>(out);
  a.pix = p->pix;
  a.ws = p->chain_ws;
  a.rot = p->chain_ws + (size_t)p->desc.max_shifts * g.C * 4 * (size_t)g.N;
  a.tab_t = reinterpret_cast<float4*>(a.rot + (size_t)p->desc.max_shifts * 32);
  a.tab_p = a.tab_t + 2 * g.H + 1;
  const int ns = S + 2 * g.H + 1 + 2 * g.W + 1;
  k_chain_setup<<<(ns + 255) / 256, 256, 0, st>>>(a, params, S);
  haar_status_t r = cuda_check(cudaGetLastError(), "k_chain_setup launch");
  if (r != HAAR_OK) return r;
  const unsigned nb = (unsigned)((g.N + 255) / 256);
  r = cuda_check(launch_pdl(k_chain_fields, dim3(nb, S), dim3(256), 0, st, a), "k_chain_fields launch");
  if (r != HAAR_OK) return r;
  // levels 1..min(3, n): N/4 + N/16 + N/64 blocks per plane
  long long fine = 0;
  for (int l = 1; l <= 3 && l <= g.n; ++l) fine += g.N >> (2 * l);
  const int planes = S * g.C;
  k_chain_fine<<<dim3((unsigned)((fine + 255) / 256), planes), 256, 0, st>>>(a, fine);
  r = cuda_check(cudaGetLastError(), "k_chain_fine launch");
  if (r != HAAR_OK) return r;
  long long coarse = g.q;
  for (int l = 4; l <= g.n; ++l) coarse += g.N >> (2 * l);
  k_chain_coarse<<<dim3((unsigned)((coarse * 32 + 255) / 256), planes), 256, 0, st>>>(a, coarse);
  return cuda_check(cudaGetLastError(), "k_chain_coarse launch");
}

}  // namespace hs
