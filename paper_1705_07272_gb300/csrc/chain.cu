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
  float* mom;             // [S][C][tiles][9]: per 16 x 16 tile moments of the fields
  float* rot;             // [S][32]: R rounded to float (9), then R - that (9)
  float4* tab_t;          // [2H + 1]: sin, its residual, cos, its residual of t pi / (2H)
  float4* tab_p;          // [2W + 1]: the same for t pi / W
};

// Floats of the workspace: the tile moments, then the rotations and the
// tables (each part a multiple of 4 floats, so the tables stay 16-byte aligned).
static size_t chain_mom_floats(const Geometry& g, int S) {
  return ((size_t)S * g.C * (size_t)((g.H >> 4) * (g.W >> 4)) * 9 + 3) & ~(size_t)3;
}

size_t chain_ws_floats(const Geometry& g, int S) {
  return chain_mom_floats(g, S) + (size_t)S * 32 + 4 * (size_t)(2 * g.H + 1) + 4 * (size_t)(2 * g.W + 1);
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
    i &= H - 1;                                  // H, W are powers of two
  } else {
#pragma unroll 1
    for (int it = 0; it < 8 && (i < 0 || i >= H); ++it) {
      i = (i < 0) ? -1 - i : 2 * H - 1 - i;
      j += W >> 1;
    }
    if (i < 0 || i >= H) i = min(max(i, 0), H - 1);   // only a non-finite position gets here
  }
  j &= W - 1;
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

// What an evaluation needs besides the source position: the theta row of the
// Jacobian (u_i, v_i), the phi row (u_j, v_j), the mixed terms (u_ij, v_ij).
enum : int { kNeedTheta = 1, kNeedPhi = 2, kNeedMixed = 4 };

// source position and the derivatives NEED asks for (index units) at the
// output position with polar angle table entry T and azimuth entry P:
// Theta = acos(q_y), Phi = atan2(q_x, q_z), q = R p(theta, phi); where
// q_x^2 + q_z^2 < 1e-8 (a pole) the derivatives are 0
template <int NEED>
__device__ ChJac ch_jac(const float (&Rh)[9], const float (&Rl)[9], float4 T, float4 P, const float4* tab_p,
                        const Geometry& g) {
  const float dth = 3.14159265358979f / (float)g.H, dph = 6.28318530717959f / (float)g.W;
  const float inv_dth = (float)g.H * 0.318309886183791f, inv_dph = (float)g.W * 0.159154943091895f;
  const float st = T.x, ct = T.z, sp = P.x, cp = P.z;
  const float p[3] = {st * sp, ct, st * cp};
  float q[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) q[r] = Rh[3 * r] * p[0] + Rh[3 * r + 1] * p[1] + Rh[3 * r + 2] * p[2];
  ChJac J;
  J.ui = J.uj = J.vi = J.vj = J.uij = J.vij = 0.0f;
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
    int c0 = (int)rintf(atan2f(q[0], q[2]) * inv_dph - 0.5f);
    c0 &= g.W - 1;
    const float4 Ps = tab_p[2 * c0 + 1];
    const DF Sps = {Ps.x, Ps.y}, Cps = {Ps.z, Ps.w};
    const DF cr = df_add(df_mul(qd[0], Cps), df_mul({-qd[2].h, -qd[2].l}, Sps));   // rho sin(Phi - psi)
    const DF dt = df_add(df_mul(qd[2], Cps), df_mul(qd[0], Sps));                 // rho cos(Phi - psi)
    J.iv = c0;
    J.fv = atan2f(cr.h, dt.h) * inv_dph;
    // polar: from the nearer pole
    const float rho_ = sqrtf(q[0] * q[0] + q[2] * q[2]);
    if (q[1] >= 0.0f) {
      J.iu = 0;
      J.fu = atan2f(rho_, q[1]) * inv_dth - 0.5f;
    } else {
      J.iu = g.H - 1;
      J.fu = 0.5f - atan2f(rho_, -q[1]) * inv_dth;
    }
  } else {
    const float u = atan2f(sqrtf(q[0] * q[0] + q[2] * q[2]), q[1]) * inv_dth - 0.5f;
    const float v = atan2f(q[0], q[2]) * inv_dph - 0.5f;
    const float bu = floorf(u), bv = floorf(v);
    J.iu = (int)bu;
    J.fu = u - bu;
    J.iv = (int)bv;
    J.fv = v - bv;
  }
  if (NEED == 0) return J;
  const float rho2 = q[0] * q[0] + q[2] * q[2];
  if (rho2 < 1e-8f) return J;
  const float ir = rsqrtf(rho2), ir2 = ir * ir;
  // d/dtheta and d/dphi of q (row-major R times dp)
  float qt[3], qp[3];
  const float pt[3] = {ct * sp, -st, ct * cp};
  const float pp[3] = {st * cp, 0.0f, -st * sp};
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    qt[r] = Rh[3 * r] * pt[0] + Rh[3 * r + 1] * pt[1] + Rh[3 * r + 2] * pt[2];
    qp[r] = Rh[3 * r] * pp[0] + Rh[3 * r + 2] * pp[2];
  }
  const float rv = (float)(2 * g.H) / (float)g.W;   // dphi / dtheta
  if (NEED & kNeedTheta) {
    J.ui = -qt[1] * ir;
    J.vi = (q[2] * qt[0] - q[0] * qt[2]) * ir2 / rv;
  }
  if (NEED & kNeedPhi) {
    J.uj = -qp[1] * ir * rv;
    J.vj = (q[2] * qp[0] - q[0] * qp[2]) * ir2;
  }
  if (NEED & kNeedMixed) {
    const float ptp[3] = {ct * cp, 0.0f, -ct * sp};
    float qtp[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) qtp[r] = Rh[3 * r] * ptp[0] + Rh[3 * r + 2] * ptp[2];
    const float rho_p = (q[0] * qp[0] + q[2] * qp[2]) * ir;
    const float Th_tp = -qtp[1] * ir + qt[1] * rho_p * ir2;
    const float N_t = q[2] * qt[0] - q[0] * qt[2];
    const float N_tp = qp[2] * qt[0] + q[2] * qtp[0] - qp[0] * qt[2] - q[0] * qtp[2];
    const float r2_p = 2.0f * (q[0] * qp[0] + q[2] * qp[2]);
    const float Ph_tp = (N_tp * rho2 - N_t * r2_p) * ir2 * ir2;
    J.uij = Th_tp * dph;
    J.vij = Ph_tp * dth;
  }
  return J;
}

// ---------------------------------------------------------------------------
// Sampling windows.  A window holds NR x NC taps of one channel plane at rows
// r0 .. r0 + NR - 1 and columns c0 .. c0 + NC - 1 of the extended map; bilinear
// samples at the offsets the route needs are lerps of its rows, then columns.

template <int NR, int NC>
__device__ __forceinline__ void ch_offsets(int r0, int c0, const Geometry& g, int (&off)[NR][NC]) {
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    int i = r0 + r, j = c0;
    ch_ext(i, j, g.H, g.W, g.boundary);          // j carries the half-turn of a pole crossing
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      int jc = j + c;
      if (jc >= g.W) jc -= g.W;
      off[r][c] = i * g.W + jc;
    }
  }
}

template <int NR, int NC>
__device__ __forceinline__ void ch_load(const float* F, const int (&off)[NR][NC], float (&T)[NR][NC]) {
#pragma unroll
  for (int r = 0; r < NR; ++r)
#pragma unroll
    for (int c = 0; c < NC; ++c) T[r][c] = __ldg(F + off[r][c]);
}

__device__ __forceinline__ float ch_lerp(float a, float b, float w) { return fmaf(w, b - a, a); }

// element k (k in 0..N-2, chosen at run time) and k + 1 of a register row, by selects
template <int N>
__device__ __forceinline__ float ch_pick_lerp(const float (&A)[N], int k, float w) {
  float a = A[0], b = A[1];
#pragma unroll
  for (int m = 1; m < N - 1; ++m)
    if (k == m) {
      a = A[m];
      b = A[m + 1];
    }
  return ch_lerp(a, b, w);
}

// (window index, weight) of the sample at offset +-1/2 around a position whose
// window starts one below floor(position) and whose fraction is f
struct ChSpec {
  int k;
  float w;
};
__device__ __forceinline__ ChSpec ch_minus_half(float f) { return f >= 0.5f ? ChSpec{1, f - 0.5f} : ChSpec{0, f + 0.5f}; }

// floor of the position iu + fu and its fraction
__device__ __forceinline__ void ch_split(int ib, float fb, int& i0, float& fr) {
  const float fl = floorf(fb);
  i0 = ib + (int)fl;
  fr = fb - fl;
}

// ---------------------------------------------------------------------------
// One CTA per 16 x 16 output tile and shift, one thread per pixel (Morton
// order, so the 2^l x 2^l blocks of levels 1..4 are runs of 4^l threads).  The
// four fields of each channel stay in registers: levels 1..4 are reduced
// inside the tile, and each tile leaves the moments from which the coarser
// levels' sums follow (the filter weights are linear on each tile there):
//   g:          S0                       (scaling coefficients)
//   g_theta:    S0, Sx                   (V: triangle along rows, box across)
//   g_phi:      S0, Sy                   (H: triangle along columns)
//   g_thetaphi: S0, Sx, Sy, Sxy          (D: triangle both ways)
// with x, y the row and column inside the tile.
constexpr int kMoments = 9;

__device__ __forceinline__ void ch_put(const ChainArgs& a, int s, int c, int k, float v) {
  if (k < a.K) a.out[(long long)s * a.st_s + (long long)c * a.st_c + (long long)k * a.st_k] = v;
}

__device__ __forceinline__ float tent(int d, int B) { return (float)min(d + 1, B - 1 - d); }

__device__ __forceinline__ float xor_sum(float v, int m) { return v + __shfl_xor_sync(0xffffffffu, v, m); }

// Sum over the warp of 16 values at once: at each butterfly step a lane keeps
// one half of its values (by its lane bit), sends the other half to its
// partner and adds what it receives, so the values per lane halve; after the
// steps on lane bits 4..1 and a last one on bit 0, lane L holds the warp sum
// of value (L >> 1) & 15 (16 shuffles instead of 80).
__device__ __forceinline__ float warp_sum16(float (&v)[16], int lane) {
#pragma unroll
  for (int half = 8, m = 16; half >= 1; half >>= 1, m >>= 1) {
    const bool up = (lane & m) != 0;
#pragma unroll
    for (int k = 0; k < half; ++k) {
      const float keep = up ? v[k + half] : v[k];
      const float send = up ? v[k] : v[k + half];
      v[k] = keep + __shfl_xor_sync(0xffffffffu, send, m);
    }
  }
  return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

__global__ void __launch_bounds__(256, 2) k_chain_tile(ChainArgs a) {
  pdl_wait();
  const Geometry& g = a.g;
  const int s = blockIdx.y, tile = blockIdx.x;
  const int tcs = g.W >> 4;
  const int tr = tile / tcs, tc = tile - tr * tcs;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int x = ((t >> 1) & 1) | ((t >> 2) & 2) | ((t >> 3) & 4) | ((t >> 4) & 8);
  const int y = (t & 1) | ((t >> 1) & 2) | ((t >> 2) & 4) | ((t >> 3) & 8);
  const int i = tr * 16 + x, j = tc * 16 + y;
  __shared__ float red[8][3 + 3 + kMoments];

  float Rh[9], Rl[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    Rh[k] = a.rot[32 * s + k];
    Rl[k] = a.rot[32 * s + 9 + k];
  }
  // angle tables at (i + 1/2) dtheta, (i + 1) dtheta and (j + 1/2) dphi, (j + 1) dphi
  const float4 T0 = a.tab_t[2 * i + 1], T1 = a.tab_t[2 * i + 2];
  const float4 P0 = a.tab_p[2 * j + 1], P1 = a.tab_p[2 * j + 2];
  const ChJac J0 = ch_jac<0>(Rh, Rl, T0, P0, a.tab_p, g);
  const ChJac Ja = ch_jac<kNeedTheta>(Rh, Rl, T1, P0, a.tab_p, g);
  const ChJac Jb = ch_jac<kNeedPhi>(Rh, Rl, T0, P1, a.tab_p, g);
  const ChJac Jc = ch_jac<kNeedTheta | kNeedPhi | kNeedMixed>(Rh, Rl, T1, P1, a.tab_p, g);

  // window geometry (channel independent)
  int r0, c0, ra, ca, rb, cb, rc, cc;
  float f0u, f0v, eau, eav, ebu, ebv, fcu, fcv;
  ch_split(J0.iu, J0.fu, r0, f0u);
  ch_split(J0.iv, J0.fv, c0, f0v);
  ch_split(Ja.iu, Ja.fu + 0.5f, ra, eau);       // Ja, Jb: origin floor(u + 1/2) - 1
  ch_split(Ja.iv, Ja.fv + 0.5f, ca, eav);
  ch_split(Jb.iu, Jb.fu + 0.5f, rb, ebu);
  ch_split(Jb.iv, Jb.fv + 0.5f, cb, ebv);
  ch_split(Jc.iu, Jc.fu, rc, fcu);              // Jc: origin floor(u) - 1
  ch_split(Jc.iv, Jc.fv, cc, fcv);
  int o0[2][2], oa[3][3], ob[3][3], oc[4][4];
  ch_offsets<2, 2>(r0, c0, g, o0);
  ch_offsets<3, 3>(ra - 1, ca - 1, g, oa);
  ch_offsets<3, 3>(rb - 1, cb - 1, g, ob);
  ch_offsets<4, 4>(rc - 1, cc - 1, g, oc);

  for (int ch = 0; ch < g.C; ++ch) {
    const float* F = a.pix + (long long)ch * g.N;
    float gv, gt, gp, gtp;
    {  // g at the pixel
      float T[2][2];
      ch_load<2, 2>(F, o0, T);
      gv = ch_lerp(ch_lerp(T[0][0], T[0][1], f0v), ch_lerp(T[1][0], T[1][1], f0v), f0u);
    }
    // The source derivatives are differences of bilinear samples.  Since
    // bilinear sampling is linear, each one is taken as the same interpolation
    // of the taps' own differences (rows: dR[k] = T[k + 1] - T[k]; columns
    // likewise).  On a smooth map neighbouring taps are close, so these
    // differences are exact in float32, and the cancellation that differencing
    // interpolated values would leave (amplified near a pole by the 1 / rho
    // Jacobian factors) never happens.
    //
    // g_theta at (i + 1/2, j) and g_phi at (i, j + 1/2): F(u +- 1/2, v) and
    // F(u, v +- 1/2) on a 3 x 3 window whose origin is floor(u + 1/2) - 1
    // (fraction e); the position itself sits at e + 1/2 from row / column 0.
    auto first = [&](const int (&o)[3][3], float eu, float ev, const ChJac& J, bool theta) {
      float T[3][3];
      ch_load<3, 3>(F, o, T);
      const int ku = eu >= 0.5f ? 1 : 0, kv = ev >= 0.5f ? 1 : 0;
      const float wu = eu >= 0.5f ? eu - 0.5f : eu + 0.5f, wv = ev >= 0.5f ? ev - 0.5f : ev + 0.5f;
      float du[3], dv[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) du[c] = ch_lerp(T[1][c] - T[0][c], T[2][c] - T[1][c], eu);   // column c
#pragma unroll
      for (int r = 0; r < 3; ++r) dv[r] = ch_lerp(T[r][1] - T[r][0], T[r][2] - T[r][1], ev);   // row r
      const float fu = ch_pick_lerp<3>(du, kv, wv);
      const float fv = ch_pick_lerp<3>(dv, ku, wu);
      return theta ? fu * J.ui + fv * J.vi : fu * J.uj + fv * J.vj;
    };
    gt = first(oa, eau, eav, Ja, true);
    gp = first(ob, ebu, ebv, Jb, false);
    {  // g_thetaphi at (i + 1/2, j + 1/2): second-order chain rule on a 4 x 4
       // window with origin floor(u) - 1, so u sits at fcu from row 1
      float T[4][4];
      ch_load<4, 4>(F, oc, T);
      const ChSpec um = ch_minus_half(fcu), vm = ch_minus_half(fcv);
      float R[3][4], Cd[4][3];                        // row and column differences of the taps
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int c = 0; c < 4; ++c) R[k][c] = T[k + 1][c] - T[k][c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int l = 0; l < 3; ++l) Cd[r][l] = T[r][l + 1] - T[r][l];
      // F(u + 1/2) - F(u - 1/2) at every column, F(v + 1/2) - F(v - 1/2) at every row
      float dU[4], dV[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const float col[3] = {R[0][c], R[1][c], R[2][c]};
        dU[c] = ch_pick_lerp<3>(col, um.k, um.w);
      }
#pragma unroll
      for (int r = 0; r < 4; ++r) dV[r] = ch_pick_lerp<3>(Cd[r], vm.k, vm.w);
      const float fu = ch_lerp(dU[1], dU[2], fcv);
      const float fv = ch_lerp(dV[1], dV[2], fcu);
      const float dUc[3] = {dU[1] - dU[0], dU[2] - dU[1], dU[3] - dU[2]};
      const float fuv = ch_pick_lerp<3>(dUc, vm.k, vm.w);
      const float fuu = ch_lerp(ch_lerp(R[1][1] - R[0][1], R[2][1] - R[1][1], fcu),
                                ch_lerp(R[1][2] - R[0][2], R[2][2] - R[1][2], fcu), fcv);
      const float fvv = ch_lerp(ch_lerp(Cd[1][1] - Cd[1][0], Cd[1][2] - Cd[1][1], fcv),
                                ch_lerp(Cd[2][1] - Cd[2][0], Cd[2][2] - Cd[2][1], fcv), fcu);
      gtp = fuu * Jc.ui * Jc.uj + fuv * (Jc.ui * Jc.vj + Jc.uj * Jc.vi) + fvv * Jc.vi * Jc.vj + fu * Jc.uij +
            fv * Jc.vij;
    }

    // levels 1..4 (Eq. conv: triangle along the derivative, box across, / B)
    const int plane = s * g.C + ch;
    // the full-warp sums (level 3, level 4, tile moments) reduce together:
    // 16 values, each lane ends with the sum of value (lane >> 1) & 15
    float w16[16];
#pragma unroll
    for (int l = 1; l <= 4; ++l) {
      const int B = 1 << l;
      const float ti = tent(x & (B - 1), B), tj = tent(y & (B - 1), B);
      float h = tj * gp, v = ti * gt, d = ti * tj * gtp;
      if (l <= 2) {
#pragma unroll
        for (int o = 1; o < (l == 1 ? 4 : 16); o <<= 1) {
          h = xor_sum(h, o);
          v = xor_sum(v, o);
          d = xor_sum(d, o);
        }
        if ((t & ((1 << (2 * l)) - 1)) == 0) {
          const int gl = g.q << (2 * (g.n - l));
          const int cols = g.W >> l;
          const int k0 = ((tr * 16 + x) >> l) * cols + ((tc * 16 + y) >> l);
          const float inv = 1.0f / (float)B;
          ch_put(a, s, ch, gl + k0, h * inv);
          ch_put(a, s, ch, 2 * gl + k0, v * inv);
          ch_put(a, s, ch, 3 * gl + k0, d * inv);
        }
      } else {
        w16[3 * (l - 3)] = h;
        w16[3 * (l - 3) + 1] = v;
        w16[3 * (l - 3) + 2] = d;
      }
    }
    {
      const float fx = (float)x, fy = (float)y;
      w16[6] = gv;
      w16[7] = gt;      w16[8] = fx * gt;
      w16[9] = gp;      w16[10] = fy * gp;
      w16[11] = gtp;    w16[12] = fx * gtp;    w16[13] = fy * gtp;    w16[14] = fx * fy * gtp;
      w16[15] = 0.0f;
    }
    const float wsum = warp_sum16(w16, lane);
    __syncthreads();                                  // red[] of the previous channel is consumed
    if ((lane & 1) == 0 && lane < 30) red[warp][lane >> 1] = wsum;
    __syncthreads();
    if (t < 4) {                                      // level 3: warps 2t, 2t + 1 form block t
      const int bx = (t >> 1) & 1, by = t & 1;        // Morton: bit 0 -> column, bit 1 -> row
      const int gl = g.q << (2 * (g.n - 3));
      const int cols = g.W >> 3;
      const int k0 = (tr * 2 + bx) * cols + (tc * 2 + by);
      ch_put(a, s, ch, gl + k0, (red[2 * t][0] + red[2 * t + 1][0]) * 0.125f);
      ch_put(a, s, ch, 2 * gl + k0, (red[2 * t][1] + red[2 * t + 1][1]) * 0.125f);
      ch_put(a, s, ch, 3 * gl + k0, (red[2 * t][2] + red[2 * t + 1][2]) * 0.125f);
    } else if (t >= 32 && t < 32 + 3 + kMoments) {    // level 4 and the tile moments
      const int k = t - 32;
      float v = 0.0f;
#pragma unroll
      for (int w = 0; w < 8; ++w) v += red[w][3 + k];
      if (k < 3) {
        const int gl = g.q << (2 * (g.n - 4));
        const int k0 = tr * (g.W >> 4) + tc;
        ch_put(a, s, ch, (k + 1) * gl + k0, v * 0.0625f);
      } else {
        a.mom[((long long)plane * g.n_tiles + tile) * kMoments + (k - 3)] = v;
      }
    }
  }
}

// levels 5..n and the scaling coefficients from the tile moments: one warp per
// (plane, block).  In a block of side B >= 32 the weights are linear on each
// 16 x 16 tile: w = (o + 1) + x on the rising half (tile offset o < B / 2) and
// (B - 1 - o) - x on the falling half.
__global__ void __launch_bounds__(256) k_chain_coarse(ChainArgs a, long long per_plane) {
  pdl_wait();
  const Geometry& g = a.g;
  const long long wi = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int plane = blockIdx.y;
  if (wi >= per_plane) return;
  const int s = plane / g.C, c = plane - s * g.C;
  const float* M = a.mom + (long long)plane * g.n_tiles * kMoments;
  const int tcs = g.W >> 4;
  long long k = wi;
  if (k < g.q) {                                  // scaling block k: (sum of g over H x H) / H
    const int side = g.H >> 4;
    float t = 0.0f;
    for (int p = lane; p < side * side; p += 32) {
      const int di = p / side, dj = p - di * side;
      t += M[(long long)(di * tcs + k * side + dj) * kMoments];
    }
    for (int o = 16; o > 0; o >>= 1) t = xor_sum(t, o);
    if (lane == 0) ch_put(a, s, c, (int)k, t / (float)g.H);
    return;
  }
  k -= g.q;
  int lvl = 5;
  while (lvl < g.n && k >= (g.N >> (2 * lvl))) {
    k -= g.N >> (2 * lvl);
    ++lvl;
  }
  const int B = 1 << lvl, cols = g.W >> lvl, side = B >> 4;
  const int r = (int)(k / cols), col = (int)(k - (long long)r * cols);
  float h = 0.0f, v = 0.0f, d = 0.0f;
  for (int p = lane; p < side * side; p += 32) {
    const int di = p / side, dj = p - di * side;
    const float* m = M + (long long)((r * side + di) * tcs + col * side + dj) * kMoments;
    const int oi = di * 16, oj = dj * 16;
    const float ax = oi < B / 2 ? (float)(oi + 1) : (float)(B - 1 - oi), bx = oi < B / 2 ? 1.0f : -1.0f;
    const float ay = oj < B / 2 ? (float)(oj + 1) : (float)(B - 1 - oj), by = oj < B / 2 ? 1.0f : -1.0f;
    v += ax * m[1] + bx * m[2];
    h += ay * m[3] + by * m[4];
    d += ax * ay * m[5] + bx * ay * m[6] + ax * by * m[7] + bx * by * m[8];
  }
  for (int o = 16; o > 0; o >>= 1) {
    h = xor_sum(h, o);
    v = xor_sum(v, o);
    d = xor_sum(d, o);
  }
  if (lane == 0) {
    const int gl = g.q << (2 * (g.n - lvl));
    const int k0 = r * cols + col;
    const float inv = 1.0f / (float)B;
    ch_put(a, s, c, gl + k0, h * inv);
    ch_put(a, s, c, 2 * gl + k0, v * inv);
    ch_put(a, s, c, 3 * gl + k0, d * inv);
  }
}

haar_status_t launch_chain(haar_shift_plan_s* p, const double* params, int S, void* out, cudaStream_t st) {
  ChainArgs a;
  const Geometry& g = p->geo;
  a.g = g;
  a.g.n_tiles = (g.H >> 4) * (g.W >> 4);
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
  a.mom = p->chain_ws;
  a.rot = p->chain_ws + chain_mom_floats(g, p->desc.max_shifts);
  a.tab_t = reinterpret_cast<float4*>(a.rot + (size_t)p->desc.max_shifts * 32);
  a.tab_p = a.tab_t + 2 * g.H + 1;
  const int ns = S + 2 * g.H + 1 + 2 * g.W + 1;
  k_chain_setup<<<(ns + 255) / 256, 256, 0, st>>>(a, params, S);
  haar_status_t r = cuda_check(cudaGetLastError(), "k_chain_setup launch");
  if (r != HAAR_OK) return r;
  r = cuda_check(launch_pdl(k_chain_tile, dim3((unsigned)a.g.n_tiles, S), dim3(256), 0, st, a),
                 "k_chain_tile launch");
  if (r != HAAR_OK) return r;
  long long coarse = g.q;
  for (int l = 5; l <= g.n; ++l) coarse += g.N >> (2 * l);
  return cuda_check(launch_pdl(k_chain_coarse, dim3((unsigned)((coarse * 32 + 255) / 256), S * g.C), dim3(256), 0,
                               st, a, coarse),
                    "k_chain_coarse launch");
}

}  // namespace hs
