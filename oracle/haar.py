"""Orthonormal 2-D non-standard Haar transform of an H x W lat-long map.

The paper works with the standard non-separable 2-D Haar basis (Sec. "Our
contributions"; Sec. "Haar-domain methods", Eq. 2-5) whose horizontal,
vertical and diagonal coefficients are first differences along phi, along
theta and mixed (Sec. "Mathematical description").  Convention used here:

* A_0 = P.  For level l = 1..n (n = log2 H), on every 2x2 block of A_{l-1}
  with a = top-left, b = top-right, c = bottom-left, d = bottom-right
  (rows grow with theta, columns with phi):
      A_l = (a + b + c + d) / 2
      H_l = (b + d - a - c) / 2      (difference along phi)
      V_l = (c + d - a - b) / 2      (difference along theta)
      D_l = (a + d - b - c) / 2      (mixed difference)
* after n levels A_n is 1 x (W/H) (W = H or W = 2H);
* canonical order: A_n row-major, then for l = n down to 1 the bands H_l,
  V_l, D_l, each row-major.  With q = W/H and g_l = q 4^(n-l) (the number of
  blocks at level l) band b of level l occupies [g_l (1+b), g_l (2+b)).

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import numpy as np

BAND_H, BAND_V, BAND_D = 0, 1, 2


def dims(H: int, W: int):
    n = int(H).bit_length() - 1
    if H < 1 or (1 << n) != H or W not in (H, 2 * H):
        raise ValueError(f"unsupported map {H}x{W}")
    return n, W // H


def level_count(H: int, W: int) -> int:
    return dims(H, W)[0]


def block_count(H: int, W: int, level: int) -> int:
    n, q = dims(H, W)
    return q * 4 ** (n - level)


def band_range(H: int, W: int, level: int, band: int):
    g = block_count(H, W, level)
    return g * (1 + band), g * (2 + band)


def forward(P: np.ndarray) -> np.ndarray:
    """Haar coefficients [..., N] of maps P [..., H, W] (float64)."""
    P = np.asarray(P, dtype=np.float64)
    H, W = P.shape[-2:]
    n, q = dims(H, W)
    lead = P.shape[:-2]
    A = P
    details = []
    for _ in range(n):
        a = A[..., 0::2, 0::2]
        b = A[..., 0::2, 1::2]
        c = A[..., 1::2, 0::2]
        d = A[..., 1::2, 1::2]
        details.append(((b + d - a - c) / 2, (c + d - a - b) / 2, (a + d - b - c) / 2))
        A = (a + b + c + d) / 2
    parts = [A.reshape(lead + (q,))]
    for lvl in range(n, 0, -1):
        for band in details[lvl - 1]:
            parts.append(band.reshape(lead + (-1,)))
    return np.concatenate(parts, axis=-1)


def inverse(coeffs: np.ndarray, H: int, W: int) -> np.ndarray:
    """Maps [..., H, W] from Haar coefficients [..., N] (float64)."""
    c = np.asarray(coeffs, dtype=np.float64)
    n, q = dims(H, W)
    lead = c.shape[:-1]
    A = c[..., :q].reshape(lead + (1, q))
    for lvl in range(n, 0, -1):
        rows, cols = H >> lvl, W >> lvl
        g = q * 4 ** (n - lvl)
        Hb = c[..., g:2 * g].reshape(lead + (rows, cols))
        Vb = c[..., 2 * g:3 * g].reshape(lead + (rows, cols))
        Db = c[..., 3 * g:4 * g].reshape(lead + (rows, cols))
        out = np.empty(lead + (2 * rows, 2 * cols))
        out[..., 0::2, 0::2] = (A - Hb - Vb + Db) / 2
        out[..., 0::2, 1::2] = (A + Hb - Vb - Db) / 2
        out[..., 1::2, 0::2] = (A - Hb + Vb - Db) / 2
        out[..., 1::2, 1::2] = (A + Hb + Vb + Db) / 2
        A = out
    return A


def index(H: int, W: int, level: int, band: int, r: int, col: int) -> int:
    """Canonical index of detail (level, band) at block (r, col)."""
    n, q = dims(H, W)
    g = q * 4 ** (n - level)
    return g * (1 + band) + r * (W >> level) + col


def decode(H: int, W: int, k: int):
    """(level, band, r, col) of canonical index k; level 0 / band -1 is A_n."""
    n, q = dims(H, W)
    if k < q:
        return 0, -1, 0, k
    for lvl in range(n, 0, -1):
        g = q * 4 ** (n - lvl)
        if k < 4 * g:
            band = k // g - 1
            off = k - g * (1 + band)
            cols = W >> lvl
            return lvl, band, off // cols, off % cols
    raise ValueError(k)


def basis_matrix(H: int, W: int) -> np.ndarray:
    """N x N matrix whose row k is basis function k as a flattened map."""
    N = H * W
    return np.stack([inverse(np.eye(N)[k], H, W).reshape(-1) for k in range(N)])
