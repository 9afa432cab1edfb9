"""The paper's own rotation route: the chain rule on the finest derivative
fields, then the derivative-to-coefficient filters (oracle, FP64).

Sec. "Rotating Haar" writes the rotated map as g(theta, phi) =
f(Theta(theta, phi), Phi(theta, phi)) and differentiates it (Eq. pde1-pde3);
Sec. "Mathematical description" turns the derivative fields of g into its
detail coefficients with the triangle / box filters of Eq. conv, tker, sker
(implemented in ``oracle.paper_route``).  This module restates that route
for rotations, an approximation of the exact operator of ``oracle.shift``.

Readings (where the text is garbled or silent):

* units: pixel indices; the source position of output pixel (i, j) is
  u = Theta / dtheta - 1/2, v = Phi / dphi - 1/2 with theta = (i + 1/2)
  dtheta, phi = (j + 1/2) dphi, so u_i = Theta_theta, u_j = Theta_phi
  dphi / dtheta, v_i = Phi_theta dtheta / dphi, v_j = Phi_phi,
  u_ij = Theta_thetaphi dphi, v_ij = Phi_thetaphi dtheta;
* the output fields are the forward differences of g, each approximated by
  the chain rule at the midpoint of its two samples: g_theta(i, j) at
  (i + 1/2, j) = F_u u_i + F_v v_i; g_phi(i, j) at (i, j + 1/2) = F_u u_j +
  F_v v_j; g_thetaphi(i, j) at (i + 1/2, j + 1/2) by the complete second-
  order chain rule (Eq. pde3 is garbled):
  F_uu u_i u_j + F_uv (u_i v_j + u_j v_i) + F_vv v_i v_j + F_u u_ij + F_v v_ij;
* the derivatives of the source map at a fractional position come from its
  finite-difference fields, sampled bilinearly where each difference is
  centred: F_u from F(a + 1, b) - F(a, b) at (u - 1/2, v), F_v from
  F(a, b + 1) - F(a, b) at (u, v - 1/2), F_uv from the mixed difference at
  (u - 1/2, v - 1/2), F_uu and F_vv from the central second differences at
  (u, v);
* Theta = acos(q_y) and Phi = atan2(q_x, q_z) for q = R p(theta, phi), so
  Theta_a = -q_y,a / rho and Phi_a = (q_z q_x,a - q_x q_z,a) / rho^2 with
  rho^2 = q_x^2 + q_z^2; where rho^2 < 1e-8 (a rotated pixel centre on a
  pole) the Phi derivatives are taken as 0;
* the scaling coefficient (no derivative carries it) is the block sum of
  the bilinearly resampled map over the block side, as on the exact route.

For a rotation about Y (a pure azimuth shift) the Jacobian is the identity
and the route equals ``oracle.paper_route`` for the translation, i.e. the
exact operator.  Test infrastructure only.
"""
from __future__ import annotations

import math

import numpy as np

from . import paper_route
from .resample import bilinear

RHO2_MIN = 1e-8


def coords_and_jacobian(R: np.ndarray, H: int, W: int, ii: np.ndarray, jj: np.ndarray) -> dict:
    """u, v and their first / mixed derivatives in index units at the
    (fractional) output positions (ii, jj)."""
    dth, dph = math.pi / H, 2.0 * math.pi / W
    th = (np.asarray(ii, dtype=np.float64) + 0.5) * dth
    ph = (np.asarray(jj, dtype=np.float64) + 0.5) * dph
    st, ct, sp, cp = np.sin(th), np.cos(th), np.sin(ph), np.cos(ph)
    p = np.stack([st * sp, ct, st * cp], axis=-1)
    p_t = np.stack([ct * sp, -st, ct * cp], axis=-1)
    p_p = np.stack([st * cp, np.zeros_like(st), -st * sp], axis=-1)
    p_tp = np.stack([ct * cp, np.zeros_like(st), -ct * sp], axis=-1)
    R = np.asarray(R, dtype=np.float64)
    q, q_t, q_p, q_tp = (x @ R.T for x in (p, p_t, p_p, p_tp))
    qx, qy, qz = q[..., 0], q[..., 1], q[..., 2]
    rho2 = qx * qx + qz * qz
    rho = np.sqrt(rho2)
    theta2 = np.arctan2(rho, qy)
    phi2 = np.mod(np.arctan2(qx, qz), 2.0 * math.pi)
    ok = rho2 >= RHO2_MIN
    srho = np.where(ok, rho, 1.0)
    srho2 = np.where(ok, rho2, 1.0)
    # Theta = acos(q_y)
    Th_t = -q_t[..., 1] / srho
    Th_p = -q_p[..., 1] / srho
    rho_p = (qx * q_p[..., 0] + qz * q_p[..., 2]) / srho
    Th_tp = -q_tp[..., 1] / srho + q_t[..., 1] * rho_p / srho2
    # Phi = atan2(q_x, q_z)
    N_t = qz * q_t[..., 0] - qx * q_t[..., 2]
    N_p = qz * q_p[..., 0] - qx * q_p[..., 2]
    N_tp = q_p[..., 2] * q_t[..., 0] + qz * q_tp[..., 0] - q_p[..., 0] * q_t[..., 2] - qx * q_tp[..., 2]
    r2_p = 2.0 * (qx * q_p[..., 0] + qz * q_p[..., 2])
    Ph_t = np.where(ok, N_t / srho2, 0.0)
    Ph_p = np.where(ok, N_p / srho2, 0.0)
    Ph_tp = np.where(ok, (N_tp * srho2 - N_t * r2_p) / (srho2 * srho2), 0.0)
    Th_t, Th_p, Th_tp = (np.where(ok, x, 0.0) for x in (Th_t, Th_p, Th_tp))
    return {
        "u": theta2 / dth - 0.5, "v": phi2 / dph - 0.5,
        "u_i": Th_t, "u_j": Th_p * dph / dth, "v_i": Ph_t * dth / dph, "v_j": Ph_p,
        "u_ij": Th_tp * dph, "v_ij": Ph_tp * dth,
        "Theta_t": Th_t, "Theta_p": Th_p, "Phi_t": Ph_t, "Phi_p": Ph_p,
    }


def _diff_fields(P: np.ndarray, boundary: int) -> dict:
    """Finite-difference fields of the extended map, as functions sampled
    bilinearly at fractional (u, v) with their centring offsets."""
    def shifted(di, dj):
        return lambda u, v: bilinear(P, u + di, v + dj, boundary)

    def f_u(u, v):   # F(a + 1, b) - F(a, b) at a = u - 1/2
        return shifted(0.5, 0.0)(u, v) - shifted(-0.5, 0.0)(u, v)

    def f_v(u, v):
        return shifted(0.0, 0.5)(u, v) - shifted(0.0, -0.5)(u, v)

    def f_uv(u, v):
        return (shifted(0.5, 0.5)(u, v) - shifted(0.5, -0.5)(u, v)
                - shifted(-0.5, 0.5)(u, v) + shifted(-0.5, -0.5)(u, v))

    def f_uu(u, v):
        return shifted(1.0, 0.0)(u, v) - 2.0 * shifted(0.0, 0.0)(u, v) + shifted(-1.0, 0.0)(u, v)

    def f_vv(u, v):
        return shifted(0.0, 1.0)(u, v) - 2.0 * shifted(0.0, 0.0)(u, v) + shifted(0.0, -1.0)(u, v)

    return {"u": f_u, "v": f_v, "uv": f_uv, "uu": f_uu, "vv": f_vv}


def rotated_fields(P: np.ndarray, R: np.ndarray, boundary: int):
    """(g, g_theta, g_phi, g_thetaphi) of the rotated map on the output grid:
    g by bilinear resampling, the differences by the chain rule."""
    H, W = P.shape
    I, J = np.meshgrid(np.arange(H, dtype=np.float64), np.arange(W, dtype=np.float64), indexing="ij")
    D = _diff_fields(P, boundary)
    c0 = coords_and_jacobian(R, H, W, I, J)
    g = bilinear(P, c0["u"], c0["v"], boundary)
    a = coords_and_jacobian(R, H, W, I + 0.5, J)                 # g_theta at (i + 1/2, j)
    g_t = D["u"](a["u"], a["v"]) * a["u_i"] + D["v"](a["u"], a["v"]) * a["v_i"]
    b = coords_and_jacobian(R, H, W, I, J + 0.5)                 # g_phi at (i, j + 1/2)
    g_p = D["u"](b["u"], b["v"]) * b["u_j"] + D["v"](b["u"], b["v"]) * b["v_j"]
    c = coords_and_jacobian(R, H, W, I + 0.5, J + 0.5)           # g_thetaphi at (i + 1/2, j + 1/2)
    u, v = c["u"], c["v"]
    g_tp = (D["uu"](u, v) * c["u_i"] * c["u_j"]
            + D["uv"](u, v) * (c["u_i"] * c["v_j"] + c["u_j"] * c["v_i"])
            + D["vv"](u, v) * c["v_i"] * c["v_j"]
            + D["u"](u, v) * c["u_ij"] + D["v"](u, v) * c["v_ij"])
    return g, g_t, g_p, g_tp


def details_from_fields(g_t: np.ndarray, g_p: np.ndarray, g_tp: np.ndarray) -> dict:
    """{level: (H_l, V_l, D_l)} by Eq. conv / tker / sker (the filters and the
    recursion of ``oracle.paper_route``)."""
    H, W = g_t.shape
    n = int(H).bit_length() - 1
    out = {}
    for lvl in range(1, n + 1):
        B = 1 << lvl
        Vf = paper_route._atrous_box(paper_route._atrous_triangle(g_t, 0, B), 1, B)
        Hf = paper_route._atrous_box(paper_route._atrous_triangle(g_p, 1, B), 0, B)
        Df = paper_route._atrous_triangle(paper_route._atrous_triangle(g_tp, 0, B), 1, B) / B
        out[lvl] = (Hf[::B, ::B], Vf[::B, ::B], Df[::B, ::B])
    return out


def rotate_coeffs(P: np.ndarray, R: np.ndarray, boundary: int = 0) -> np.ndarray:
    """Canonical coefficient vector of the rotated map by the chain-rule route."""
    H, W = P.shape
    n = int(H).bit_length() - 1
    q = W // H
    g, g_t, g_p, g_tp = rotated_fields(P, R, boundary)
    det = details_from_fields(g_t, g_p, g_tp)
    parts = [np.array([g[:, k * H:(k + 1) * H].sum() / H for k in range(q)])]
    for lvl in range(n, 0, -1):
        for band in det[lvl]:
            parts.append(band.reshape(-1))
    return np.concatenate(parts)
