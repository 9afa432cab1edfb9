"""The paper's derivative route to the shifted coefficients (oracle pin).

Sec. "Mathematical description" computes the detail coefficients of the
shifted map from its finest-scale derivative fields:

* the derivative fields g_theta, g_phi, g_theta_phi of the shifted map come
  from those of the original map by the chain rule (Eq. pde1-pde3); for a
  translation the Jacobian is the identity, so each field is the original
  field sampled at the shifted position;
* vertical details at block side B = 2^(l+2) are g_theta filtered by a
  triangle kernel along theta (Eq. tker: peak B/2, B-1 taps) and a box along
  phi (Eq. sker, 1/B), then decimated by B (Eq. conv); horizontal details
  swap the two directions; diagonal details filter the mixed difference with
  the triangle in both directions;
* Sec. "Algorithmic optimization": the triangle for side 2B is the triangle
  for side B convolved with the 3-tap kernel (1, 2, 1) upsampled by B/2, and
  the box for 2B is the box for B convolved with the 2-tap (1, 1)/2 upsampled
  by B, so every level follows from the previous one with 3 (or 2) taps.

Readings taken where the text is garbled or silent: the derivative fields
are the undecimated forward differences F(i+1, j) - F(i, j), F(i, j+1) - F(i, j)
and the mixed difference at every pixel; the box has B taps; the scaling
coefficient (which no derivative carries) is the block sum of the shifted
map divided by the block side.

This module is independent of ``oracle.haar.forward``: it pins that
transform (and ``oracle.shift``) for translations.  Test infrastructure only.
"""
from __future__ import annotations

import numpy as np

from .resample import extend_index


def _ext(P, i, j, boundary):
    H, W = P.shape
    ii, jj = extend_index(i, j, H, W, boundary)
    return P[ii, jj]


def _shifted_field(P, dx, dy, boundary, di, dj, mixed=False):
    """Field of forward differences of the extended map along (di, dj) (or the
    mixed difference), bilinearly sampled at (i - dy, j - dx)."""
    H, W = P.shape
    I, J = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    u = I - dy
    v = J - dx
    i0 = np.floor(u).astype(np.int64)
    j0 = np.floor(v).astype(np.int64)
    fu = u - i0
    fv = v - j0

    def diff(a, b):
        if mixed:
            return (_ext(P, a + 1, b + 1, boundary) - _ext(P, a + 1, b, boundary)
                    - _ext(P, a, b + 1, boundary) + _ext(P, a, b, boundary))
        return _ext(P, a + di, b + dj, boundary) - _ext(P, a, b, boundary)

    return ((1 - fu) * (1 - fv) * diff(i0, j0) + (1 - fu) * fv * diff(i0, j0 + 1)
            + fu * (1 - fv) * diff(i0 + 1, j0) + fu * fv * diff(i0 + 1, j0 + 1))


def _atrous_triangle(field, axis, B):
    """Correlate ``field`` with the triangle of side B along ``axis`` by the
    recursion tri_2 = (1), tri_2b = tri_b * up_{b/2}(1, 2, 1)."""
    Y = field.copy()
    b = 2
    while b < B:
        h = b // 2
        n = Y.shape[axis]
        Yn = np.zeros_like(Y)
        idx = np.arange(n)
        for off, wgt in ((0, 1.0), (h, 2.0), (b, 1.0)):
            ok = idx + off < n
            src = np.take(Y, (idx + off)[ok], axis=axis)
            sl = [slice(None)] * Y.ndim
            sl[axis] = idx[ok]
            Yn[tuple(sl)] += wgt * src
        Y = Yn
        b *= 2
    return Y


def _atrous_box(field, axis, B):
    """Correlate with the box of B taps, 1/B each, by the recursion
    box_1 = (1), box_2b = (box_b + box_b shifted by b) / 2."""
    Y = field.copy()
    b = 1
    while b < B:
        n = Y.shape[axis]
        idx = np.arange(n)
        ok = idx + b < n
        Yn = np.zeros_like(Y)
        sl = [slice(None)] * Y.ndim
        sl[axis] = idx[ok]
        Yn[tuple(sl)] = (np.take(Y, idx[ok], axis=axis) + np.take(Y, (idx + b)[ok], axis=axis)) / 2
        Y = Yn
        b *= 2
    return Y


def translate_details(P: np.ndarray, dx: float, dy: float, boundary: int):
    """{level: (H_l, V_l, D_l)} of the translated map, by the derivative route."""
    H, W = P.shape
    n = int(H).bit_length() - 1
    g_th = _shifted_field(P, dx, dy, boundary, 1, 0)
    g_ph = _shifted_field(P, dx, dy, boundary, 0, 1)
    g_tp = _shifted_field(P, dx, dy, boundary, 0, 0, mixed=True)
    out = {}
    for lvl in range(1, n + 1):
        B = 1 << lvl
        Vf = _atrous_box(_atrous_triangle(g_th, 0, B), 1, B)
        Hf = _atrous_box(_atrous_triangle(g_ph, 1, B), 0, B)
        Df = _atrous_triangle(_atrous_triangle(g_tp, 0, B), 1, B) / B
        out[lvl] = (Hf[::B, ::B], Vf[::B, ::B], Df[::B, ::B])
    return out


def translate_coeffs(P: np.ndarray, dx: float, dy: float, boundary: int) -> np.ndarray:
    """Canonical coefficient vector of the translated map (derivative route for
    the details, block sums of the shifted map for the scaling coefficients)."""
    H, W = P.shape
    n = int(H).bit_length() - 1
    q = W // H
    det = translate_details(P, dx, dy, boundary)
    I, J = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    u, v = I - dy, J - dx
    i0, j0 = np.floor(u).astype(np.int64), np.floor(v).astype(np.int64)
    fu, fv = u - i0, v - j0
    g = ((1 - fu) * (1 - fv) * _ext(P, i0, j0, boundary) + (1 - fu) * fv * _ext(P, i0, j0 + 1, boundary)
         + fu * (1 - fv) * _ext(P, i0 + 1, j0, boundary) + fu * fv * _ext(P, i0 + 1, j0 + 1, boundary))
    parts = [np.array([g[:, k * H:(k + 1) * H].sum() / H for k in range(q)])]
    for lvl in range(n, 0, -1):
        for band in det[lvl]:
            parts.append(band.reshape(-1))
    return np.concatenate(parts)
