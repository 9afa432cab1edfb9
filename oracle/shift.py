"""The phase shift of a lighting map's Haar coefficients (oracle).

The paper's goal (Sec. "Rotating Haar" and "Mathematical description") is
the Haar coefficients of the rotated map g(theta, phi) = f(Theta, Phi) given
the coefficients of f.  The oracle computes that plain definition:

    c' = Haar( resample( Haar^-1 c ) )

with the resampling of ``oracle.resample``.  A translation (dx, dy) in pixels
is the linear phase shift; a rotation R is the non-linear one (Eq. theta,
Eq. phi); a rotation about Y is a shift along phi (Sec. "Algorithmic
optimization").

``dyadic_permutation`` restates, independently of the resampler, what an
integer shift does to the levels whose block side divides it: it moves whole
blocks, so those coefficients are a signed permutation of the input.

``start_level`` k > 0 is the paper's start-level approximation (Sec.
"Algorithmic optimization": the shift can begin at a coarser level, with
O(N / 4^k) work): the coarsest N / 4^k coefficients of the map are those of
its level-k scaling image (an (H / 2^k) x (W / 2^k) map whose pixels are
2^k x the 2^k x 2^k block means), so the shift is taken of that image -- a
translation by (dx, dy) / 2^k, a rotation unchanged -- and gives the N / 4^k
coarsest coefficients; the finer ones are not produced.

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import numpy as np

from . import haar, resample
from .resample import SPHERE, TORUS

TRANSLATE = 0
ROTATE = 1          # params: 3x3 matrix, row-major (9 numbers)
ROTATE_EULER = 2    # params: (alpha, beta, gamma), R = Rz(gamma) Ry(beta) Rx(alpha)


def shifted_maps(P: np.ndarray, kind: int, params: np.ndarray, boundary: int) -> np.ndarray:
    """Resampled maps [S, ..., H, W] for every parameter row."""
    out = []
    for prm in np.asarray(params, dtype=np.float64):
        if kind == TRANSLATE:
            out.append(resample.translate(P, prm[0], prm[1], boundary))
        elif kind == ROTATE:
            out.append(resample.rotate(P, prm.reshape(3, 3), boundary))
        elif kind == ROTATE_EULER:
            out.append(resample.rotate(P, resample.euler_matrix(*prm), boundary))
        else:
            raise ValueError(kind)
    return np.stack(out)


def haar_shift(coeffs: np.ndarray, H: int, W: int, kind: int, params: np.ndarray,
               boundary: int = SPHERE, out_coeffs: int | None = None, start_level: int = 0) -> np.ndarray:
    """Shifted coefficients [S, C, K] of coefficients [C, N] (float64).

    start_level k: the shift of the level-k scaling image (see the module
    docstring); K <= N / 4^k."""
    c = np.asarray(coeffs, dtype=np.float64)
    k = int(start_level)
    if k:
        H, W = H >> k, W >> k
        c = c[..., :H * W]                      # the scaling image's own coefficients
        params = np.asarray(params, dtype=np.float64)
        if kind == TRANSLATE:
            params = params / float(1 << k)
    P = haar.inverse(c, H, W)
    G = shifted_maps(P, kind, params, boundary)
    out = haar.forward(G)
    if out_coeffs is not None:
        out = out[..., :out_coeffs]
    return out


def _source_block(r: int, col: int, ky_b: int, kx_b: int, rows: int, cols: int,
                  half_turn_b, boundary: int):
    """Source block of output block (r, col) under a block-aligned shift,
    and whether it arrives mirrored in theta."""
    rs = r - ky_b
    cs = col - kx_b
    flip = False
    if boundary == TORUS:
        return rs % rows, cs % cols, False
    while rs < 0 or rs >= rows:
        rs = -1 - rs if rs < 0 else 2 * rows - 1 - rs
        cs += half_turn_b
        flip = not flip
    return rs, cs % cols, flip


def permutation_levels(H: int, W: int, kx: int, ky: int, boundary: int):
    """Levels (1..n, and n+1 standing for the scaling block) whose coefficients
    an integer shift (kx, ky) only permutes (with signs)."""
    n, _ = haar.dims(H, W)
    out = []
    for lvl in range(1, n + 2):
        B = 1 << min(lvl, n)
        if kx % B or ky % B:
            continue
        period = 2 * H if boundary == SPHERE else H
        crosses = boundary == SPHERE and (ky % period) != 0
        if crosses and (W // 2) % B:
            continue
        out.append(lvl)
    return out


def dyadic_permutation(coeffs: np.ndarray, H: int, W: int, kx: int, ky: int,
                       boundary: int = SPHERE) -> dict:
    """Closed-form coefficients of the permuted levels: {canonical index: value}.

    For level l with block side B = 2^l dividing kx and ky, output block
    (r, col) takes the coefficients of source block (r - ky/B, col - kx/B);
    a block mirrored across a pole (SPHERE) moves half a turn in azimuth and
    its V and D coefficients change sign (mirroring in theta swaps the top and
    bottom halves of the block)."""
    n, q = haar.dims(H, W)
    c = np.asarray(coeffs, dtype=np.float64)
    res = {}
    for lvl in permutation_levels(H, W, kx, ky, boundary):
        if lvl == n + 1:       # scaling coefficients: 1 x q blocks of side H
            B, rows, cols = H, 1, q
            for col in range(cols):
                rs, cs, _ = _source_block(0, col, ky // B, kx // B, rows, cols,
                                          (W // 2) // B if (W // 2) % B == 0 else 0, boundary)
                res[col] = c[..., cs]
            continue
        B = 1 << lvl
        rows, cols = H >> lvl, W >> lvl
        half = (W // 2) // B if (W // 2) % B == 0 else 0
        for r in range(rows):
            for col in range(cols):
                rs, cs, flip = _source_block(r, col, ky // B, kx // B, rows, cols, half, boundary)
                for band in (haar.BAND_H, haar.BAND_V, haar.BAND_D):
                    sgn = -1.0 if (flip and band != haar.BAND_H) else 1.0
                    res[haar.index(H, W, lvl, band, r, col)] = \
                        sgn * c[..., haar.index(H, W, lvl, band, rs, cs)]
    return res
