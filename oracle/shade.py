"""The double product: outgoing radiance of every vertex (oracle).

Eq. (1)-(3) with the BRDF, cosine and visibility folded into one transfer
function: L_o(v) = sum over directions of L_in(w) * t_v(w) dw.  With the
lighting map g and the transport weights w_v both sampled on the lat-long
grid this is r_v = sum_p g[p] w_v[p]; for orthonormal Haar bases it equals
sum_k G_k T_k (Parseval), which is the form the fast path evaluates.

The brute-force form below reconstructs both factors in pixel space from the
stored coefficient vectors, so truncation and storage rounding are included.

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import numpy as np

from . import haar


def radiance_pixels(lighting_maps: np.ndarray, weight_maps: np.ndarray) -> np.ndarray:
    """r[v, s, c] = sum_p g[s, c, p] w[v, p] for maps g [S, C, H, W], w [V, H, W]."""
    g = np.asarray(lighting_maps, dtype=np.float64)
    w = np.asarray(weight_maps, dtype=np.float64)
    S, C = g.shape[:2]
    V = w.shape[0]
    out = np.zeros((V, S, C))
    for v in range(V):
        out[v] = (g * w[v][None, None]).sum(axis=(-2, -1))
    return out


def radiance(lighting_coeffs: np.ndarray, transport: np.ndarray, H: int, W: int) -> np.ndarray:
    """Brute force through pixel space: lighting [S, C, N'] and stored
    transport [V, N''] (zero-padded to N = H W) -> r [V, S, C]."""
    N = H * W
    L = np.zeros(lighting_coeffs.shape[:-1] + (N,))
    L[..., :lighting_coeffs.shape[-1]] = lighting_coeffs
    T = np.zeros(transport.shape[:-1] + (N,))
    T[..., :transport.shape[-1]] = transport
    g = haar.inverse(L, H, W)
    w = haar.inverse(T, H, W)
    return radiance_pixels(g, w)
