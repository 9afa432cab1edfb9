"""The paper's shading loop: per-vertex BRDF rotation and the Haar triple
product (oracle, FP64).

Outgoing radiance with lighting L, the cosine-weighted BRDF f~ and visibility
V (Sec. "Related work", the triple-product form of the rendering equation):
L_o(p) = int_S L(w) f~(p, w) V(p, w) dw.  With each factor expanded in the
2-D Haar basis, this is sum_ijk C_ijk a_i b_j c_k with tripling coefficients
C_ijk = int Psi_i Psi_j Psi_k.  The Tripling Coefficient Theorem (Ng et al.
2004, restated in that section) says C_ijk is non-zero only when
- all three are scaling functions;
- all three are distinct wavelet types on one square;
- two are the same wavelet and the third is the scaling function or a
  wavelet on a strictly coarser square that contains it.

On the lat-long pixel grid, with unit pixel measure and the solid-angle
weight sin(theta) dtheta dphi folded into the visibility factor, the integral
is the plain sum over pixels of the three reconstructed maps.  That
definition is ``triple_product``.  ``tripling_coefficients`` builds C_ijk by
brute force (small maps).  ``triple_product_by_theorem`` sums the theorem's
three cases, with the third factor's mean over the square for the
"coarser" case; it is pinned equal to the definition.

Each vertex's BRDF map is given in the local frame, with the normal at
theta = 0 (the +y pole).  It is rotated to the vertex's normal N (Sec.
"Algorithmic optimization": a rotation about the x axis by the normal's polar
angle and a shift along phi by its azimuth).  With the shift convention
g(w) = f(R w) this is R = Rx(-theta_N) Ry(-phi_N), which takes N to +y
(``normal_rotation``).  The rotation itself is the exact operator of
``oracle.shift``.

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import math

import numpy as np

from . import haar, shift
from .resample import rot_x, rot_y


def triple_product(a: np.ndarray, b: np.ndarray, c: np.ndarray, H: int, W: int) -> np.ndarray:
    """sum over pixels of the three reconstructed maps; coefficient vectors
    [..., N] broadcast against each other."""
    A, B, C = (haar.inverse(np.asarray(x, dtype=np.float64), H, W) for x in (a, b, c))
    return (A * B * C).sum(axis=(-2, -1))


def tripling_coefficients(H: int, W: int) -> np.ndarray:
    """C[i, j, k] = sum over pixels of basis functions i, j, k (N^3 entries)."""
    Bm = haar.basis_matrix(H, W)
    return np.einsum("ip,jp,kp->ijk", Bm, Bm, Bm)


def _means(x: np.ndarray, H: int, W: int) -> dict:
    """{level: [rows, cols] mean of the map over each square of that level},
    top down from the scaling blocks (the finer details average to zero over
    a square, so its mean follows from the coarser coefficients alone)."""
    n, q = haar.dims(H, W)
    out = {n: (x[:q] / H).reshape(1, q)}
    for lvl in range(n, 1, -1):
        B = 1 << lvl
        rows, cols = H >> lvl, W >> lvl
        g = q * 4 ** (n - lvl)
        h = x[g:2 * g].reshape(rows, cols)
        v = x[2 * g:3 * g].reshape(rows, cols)
        d = x[3 * g:4 * g].reshape(rows, cols)
        m = out[lvl]
        child = np.empty((2 * rows, 2 * cols))
        # quadrant values of the H, V, D wavelets of side B are +-1/B
        child[0::2, 0::2] = m + (-h - v + d) / B
        child[0::2, 1::2] = m + (h - v - d) / B
        child[1::2, 0::2] = m + (-h + v - d) / B
        child[1::2, 1::2] = m + (h + v + d) / B
        out[lvl - 1] = child
    return out


def triple_product_by_theorem(a: np.ndarray, b: np.ndarray, c: np.ndarray, H: int, W: int) -> float:
    """The three cases of the Tripling Coefficient Theorem, summed square by
    square (unit pixel measure: C = 1/H for three scaling functions, 1/B for
    three distinct types on a square of side B, the third factor's value on
    the square for a repeated wavelet)."""
    n, q = haar.dims(H, W)
    a, b, c = (np.asarray(x, dtype=np.float64) for x in (a, b, c))
    total = float((a[:q] * b[:q] * c[:q]).sum()) / H
    ma, mb, mc = _means(a, H, W), _means(b, H, W), _means(c, H, W)
    for lvl in range(n, 0, -1):
        B = 1 << lvl
        g = q * 4 ** (n - lvl)
        rows, cols = H >> lvl, W >> lvl
        A = [a[g * (1 + t):g * (2 + t)].reshape(rows, cols) for t in range(3)]
        Bc = [b[g * (1 + t):g * (2 + t)].reshape(rows, cols) for t in range(3)]
        Cc = [c[g * (1 + t):g * (2 + t)].reshape(rows, cols) for t in range(3)]
        distinct = sum(A[i] * Bc[j] * Cc[k] for i, j, k in
                       ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)))
        pairs = sum(A[t] * Bc[t] * mc[lvl] + A[t] * Cc[t] * mb[lvl] + Bc[t] * Cc[t] * ma[lvl] for t in range(3))
        total += float((distinct / B + pairs).sum())
    return total


def normal_rotation(nrm: np.ndarray) -> np.ndarray:
    """R = Rx(-theta_N) Ry(-phi_N) for a unit normal (theta_N = acos(n_y),
    phi_N = atan2(n_x, n_z)): R N = +y, so g(w) = f(R w) carries a map whose
    normal is at the +y pole onto N."""
    n = np.asarray(nrm, dtype=np.float64)
    th = math.acos(max(-1.0, min(1.0, n[1])))
    ph = math.atan2(n[0], n[2])
    return rot_x(-th) @ rot_y(-ph)


def shade_triple(light: np.ndarray, brdf_local: np.ndarray, normals: np.ndarray, vis: np.ndarray,
                 H: int, W: int, boundary: int = shift.SPHERE) -> np.ndarray:
    """Radiance [V, C]: lighting coefficients [C, N], one local-frame BRDF map's
    coefficients [N], normals [V, 3], visibility coefficients [V, N] (with the
    solid-angle weight folded in)."""
    light = np.asarray(light, dtype=np.float64)
    out = np.zeros((len(normals), light.shape[0]))
    for v, nrm in enumerate(normals):
        R = normal_rotation(nrm)
        b = shift.haar_shift(np.asarray(brdf_local, dtype=np.float64)[None], H, W, shift.ROTATE,
                             R.reshape(1, 9), boundary)[0, 0]
        out[v] = triple_product(light, b[None], np.asarray(vis[v], dtype=np.float64)[None], H, W)
    return out
