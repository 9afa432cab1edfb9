// Source coordinates of a rotated lat-long map (Sec. "Rotating Haar",
// Eq. tRot/theta/phi), accurate to ~1e-9 rad in FP32 arithmetic.
//
// The output pixel (i, j) looks up the source map at
//   theta' = atan2(sqrt(q_x^2 + q_z^2), q_y),  phi' = atan2(q_x, q_z),
//   q = R d(theta_i, phi_j),
// i.e. at fractional source row u = theta'/dtheta - 1/2 and column
// v = phi'/dphi - 1/2.  Plain FP32 evaluation carries ~1e-7 rad of rounding
// (3e-5 px at 512 columns, half of it the final rounding of u, v themselves),
// which the per-pixel lognormal maps turn into ~3e-5 relative error.  Here:
//
//  * R = Ry(a) Rx(b) Ry(c) (proper Euler angles about y, x, y), built once
//    per rotation in FP64.  Ry(c) only moves phi_j to psi_j = phi_j + c, so
//    with per-rotation FP64-built tables of sin/cos psi_j (columns) and of
//    sin b cos theta_i, cos b sin theta_i, cos b cos theta_i, sin b sin
//    theta_i (rows), the direction after Rx(b) Ry(c) is
//      x2 = sin theta sin psi,  y2 = C - D cos psi,  z2 = A + B cos psi,
//    evaluated in float pairs (unevaluated sums hi + lo, error-free products
//    and sums), and Ry(a) adds a to its azimuth.
//  * The source column nearest phi' is picked with a cheap arctangent; the
//    offset from that column's centre alpha_m (a per-rotation table of
//    sin/cos(phi_m - a)) is the small angle atan(cross / dot) of the float
//    pair cross and dot products of (x2, z2) with (sin, cos) alpha_m.
//  * Likewise for the row: the nearest row centre beta_k, and the small angle
//    between (rho, y2) and (sin, cos) beta_k, where rho = dot / cos(offset).
//  * The coordinates leave as integer anchors plus small fractions, so no
//    large FP32 number is ever rounded.
#pragma once

#include "common.cuh"

namespace hs {

// float pair: the unevaluated sum h + l (|l| <= a few ulp of h)
struct fpair {
  float h, l;
};

// Error-free transformations use the _rn intrinsics so that the compiler
// never contracts them into FMAs.
__device__ __forceinline__ fpair pmul(fpair a, fpair b) {
  const float p = __fmul_rn(a.h, b.h);
  const float e = __fmaf_rn(a.h, b.h, -p);                 // exact: a.h b.h - p
  return {p, __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, e))};
}

__device__ __forceinline__ fpair padd(fpair a, fpair b) {
  const float s = __fadd_rn(a.h, b.h);
  const float bb = __fsub_rn(s, a.h);
  const float e = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bb)), __fsub_rn(b.h, bb));   // Knuth's two-sum
  return {s, __fadd_rn(e, __fadd_rn(a.l, b.l))};
}

__device__ __forceinline__ fpair pneg(fpair a) { return {-a.h, -a.l}; }

// a b - c d rounded to float, for a result much smaller than either product:
// the difference of the rounded products is exact or rounded relative to the
// result, and the products' rounding errors and low parts are added to it.
__device__ __forceinline__ float pdiff(fpair a, fpair b, fpair c, fpair d) {
  const float p1 = __fmul_rn(a.h, b.h);
  const float e1 = __fmaf_rn(a.h, b.h, -p1);
  const float p2 = __fmul_rn(c.h, d.h);
  const float e2 = __fmaf_rn(c.h, d.h, -p2);
  const float lo = __fsub_rn(__fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, e1)), __fmaf_rn(c.h, d.l, __fmaf_rn(c.l, d.h, e2)));
  return __fadd_rn(__fsub_rn(p1, p2), lo);
}

// atan2(y, x) within 3.4e-3 rad (atan(t) ~ t (c0 + c1 t) on [0, 1], fitted
// by Lawson's algorithm; tests/atan_fit.py): only picks the nearest pixel
// centre.
__device__ __forceinline__ float anchor_atan2(float y, float x) {
  const float ax = fabsf(x), ay = fabsf(y);
  const float mx = fmaxf(ax, ay), mn = fminf(ax, ay);
  const float t = (mx > 0.0f) ? __fdividef(mn, mx) : 0.0f;
  float r = t * fmaf(-2.659289583e-01f, t, 1.054678131e+00f);
  if (ay > ax) r = 1.57079632679f - r;
  if (x < 0.0f) r = 3.14159265359f - r;
  return copysignf(r, y);
}

// The series of atan(t) to t^5 (error below 6e-10 rad for |t| <= 1/16).
__device__ __forceinline__ float small_atan(float t) {
  const float tt = t * t;
  return t * fmaf(tt, fmaf(tt, 0.2f, -0.333333343f), 1.0f);
}

// Per-map and per-rotation tables (float4 each):
//   rows   [H]    (sin theta_i hi, lo, cos theta_i hi, lo)        (map)
//   colpsi [W]    (sin psi_j hi, lo, cos psi_j hi, lo)            (rotation)
//   colal  [W]    (sin alpha_m hi, lo, cos alpha_m hi, lo)        (rotation)
//   rowab  [2H]   (A hi, lo, B hi, lo), (C hi, lo, D hi, lo)      (rotation)
// a_px = a / dphi - 1/2 (float; only used to pick the anchor column).
struct RotSrc {
  int r, c;        // source row r in [-1, H - 1] and column c (any integer) of the top-left tap
  float fu, fv;    // fractions in [0, 1): the sample is at (r + fu, c + fv)
};

// GLOBAL_TABLES: colal and rows are read through the read-only data path
// (global memory); otherwise by plain loads (e.g. tables in shared memory).
template <bool GLOBAL_TABLES = true>
__device__ __forceinline__ RotSrc rot_source(float4 th, float4 ab, float4 cd, float4 ps,
                                             const float4* __restrict__ colal, const float4* __restrict__ rows,
                                             float a_px, float u_scale, float v_scale, int H, int W) {
  const fpair cpsi{ps.z, ps.w};
  const fpair x2 = pmul(fpair{th.x, th.y}, fpair{ps.x, ps.y});
  const fpair y2 = padd(fpair{cd.x, cd.y}, pneg(pmul(fpair{cd.z, cd.w}, cpsi)));
  const fpair z2 = padd(fpair{ab.x, ab.y}, pmul(fpair{ab.z, ab.w}, cpsi));
  // azimuth: anchor column m, offset from its centre
  const int m = __float2int_rn(fmaf(anchor_atan2(x2.h, z2.h), v_scale, a_px)) & (W - 1);
  const float4 al = GLOBAL_TABLES ? __ldg(colal + m) : colal[m];
  const float cr = pdiff(x2, fpair{al.z, al.w}, z2, fpair{al.x, al.y});           // rho sin(offset)
  const fpair dt = padd(pmul(x2, fpair{al.x, al.y}), pmul(z2, fpair{al.z, al.w}));  // rho cos(offset)
  float dphi;
  fpair rho;
  if (fabsf(cr) <= 0.0625f * dt.h && dt.h > 1e-30f) {
    const float t = __fdividef(cr, dt.h);
    dphi = small_atan(t);
    rho = fpair{dt.h, fmaf(dt.h, 0.5f * t * t, dt.l)};                                // dot sqrt(1 + t^2)
  } else {  // the anchor was not near (small maps, or a direction within ~1e-7 of a source pole)
    dphi = rot_atan2(cr, dt.h);
    rho = fpair{sqrtf(fmaf(cr, cr, dt.h * dt.h)), 0.0f};
  }
  // elevation: anchor row k, offset from its centre
  int k = __float2int_rn(fmaf(anchor_atan2(rho.h, y2.h), u_scale, -0.5f));
  k = min(max(k, 0), H - 1);
  const float4 be = GLOBAL_TABLES ? __ldg(rows + k) : rows[k];
  const float sn = pdiff(rho, fpair{be.z, be.w}, y2, fpair{be.x, be.y});          // rho cos b - y2 sin b
  const float cs = fmaf(rho.h + rho.l, be.x, y2.h * be.z);                          // rho sin b + y2 cos b
  const float dth = (fabsf(sn) <= 0.0625f * cs) ? small_atan(__fdividef(sn, cs)) : rot_atan2(sn, cs);
  RotSrc o;
  const float uf = dth * u_scale, vf = dphi * v_scale;
  const float fl = floorf(uf), fk = floorf(vf);
  o.r = min(max(k + (int)fl, -1), H - 1);         // in range by construction; clamped for memory safety
  o.c = m + (int)fk;
  o.fu = uf - fl;
  o.fv = vf - fk;
  return o;
}

__device__ __forceinline__ fpair fp_split(double x) {
  const float h = (float)x;
  return fpair{h, (float)(x - (double)h)};
}

// Angles of R = Ry(a) Rx(b) Ry(c) as float pairs (from yxy_angles' output).
struct RotAngles {
  fpair sa, ca, sb, cb, sc, cc;
};

__device__ __forceinline__ RotAngles rot_angles(const double ang[6]) {
  return RotAngles{fp_split(ang[0]), fp_split(ang[1]), fp_split(ang[2]),
                   fp_split(ang[3]), fp_split(ang[4]), fp_split(ang[5])};
}

// One column's per-rotation entries from the map's pair table entry
// (sin phi_j hi, lo, cos phi_j hi, lo): sin/cos(phi_j + c) and
// sin/cos(phi_j - a), by error-free products and sums.
__device__ __forceinline__ void rot_col_entries(float4 p, const RotAngles& g, float4& psi, float4& al) {
  const fpair sp{p.x, p.y}, cp{p.z, p.w};
  const fpair s1 = padd(pmul(sp, g.cc), pmul(cp, g.sc)), c1 = padd(pmul(cp, g.cc), pneg(pmul(sp, g.sc)));
  const fpair s2 = padd(pmul(sp, g.ca), pneg(pmul(cp, g.sa))), c2 = padd(pmul(cp, g.ca), pmul(sp, g.sa));
  psi = make_float4(s1.h, s1.l, c1.h, c1.l);
  al = make_float4(s2.h, s2.l, c2.h, c2.l);
}

// One row's per-rotation entries from (sin theta_i hi, lo, cos theta_i hi,
// lo): (A, B) = (sin b cos theta_i, cos b sin theta_i), (C, D) = (cos b cos
// theta_i, sin b sin theta_i).
__device__ __forceinline__ void rot_row_entries(float4 q, const RotAngles& g, float4& ab, float4& cd) {
  const fpair st{q.x, q.y}, ct{q.z, q.w};
  const fpair A = pmul(g.sb, ct), B = pmul(g.cb, st), C = pmul(g.cb, ct), D = pmul(g.sb, st);
  ab = make_float4(A.h, A.l, B.h, B.l);
  cd = make_float4(C.h, C.l, D.h, D.l);
}

// R = Ry(a) Rx(b) Ry(c) for a rotation matrix R (row-major, FP64), without
// trigonometry: (sin a, cos a) from R's middle column, then M = Ry(-a) R =
// Rx(b) Ry(c) gives (cos c, sin c) from its first row and (sin b, cos b) from
// its middle column.  A positive multiple of a rotation gives the same
// angles.  out = {sin a, cos a, sin b, cos b, sin c, cos c}.
__device__ __forceinline__ void yxy_angles(const double R[9], double out[6]) {
  const double na = hypot(R[1], R[7]);
  const double sa = na > 0.0 ? R[1] / na : 0.0, ca = na > 0.0 ? R[7] / na : 1.0;
  const double m00 = ca * R[0] - sa * R[6], m02 = ca * R[2] - sa * R[8];
  const double m11 = R[4], m21 = sa * R[1] + ca * R[7];
  const double nc = hypot(m00, m02), nb = hypot(m21, m11);
  out[0] = sa;
  out[1] = ca;
  out[2] = nb > 0.0 ? m21 / nb : 0.0;
  out[3] = nb > 0.0 ? m11 / nb : 1.0;
  out[4] = nc > 0.0 ? m02 / nc : 0.0;
  out[5] = nc > 0.0 ? m00 / nc : 1.0;
}

}  // namespace hs
