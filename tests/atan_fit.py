"""Derivation of the kernels' arctangent polynomials.

Both are fitted to atan on [0, 1] in float64 by Lawson's algorithm
(C. L. Lawson, 1961: iteratively reweighted least squares whose weights grow
where the error is largest, converging to the minimax fit):

* ``fit_atan_precise()``: atan(t) = t P(t^2), P of degree 7 (8 coefficients),
  the rotation kernels' full-range atan2 (used where a source offset is not
  small and for the chain-rule and shading-loop coordinates);
* ``fit_atan_anchor()``: atan(t) = t (c0 + c1 t), |error| < 3.4e-3 rad, only
  used to pick the pixel centre nearest a rotated direction, from which the
  exact offset is then computed (so its error never reaches a result).

``python tests/atan_fit.py`` prints both sets in the form the CUDA sources
hold; ``tests/test_atan_polynomial.py`` checks that the committed constants
are these.
"""
from __future__ import annotations

import numpy as np


def _lawson(A: np.ndarray, y: np.ndarray, iters: int) -> np.ndarray:
    w = np.ones_like(y)
    c = None
    for _ in range(iters):
        c = np.linalg.lstsq(A * w[:, None], y * w, rcond=None)[0]
        e = np.abs(A @ c - y)
        w = w * np.sqrt(e / e.max() + 1e-3)
        w /= w.max()
    return c


def fit_atan_precise(iters: int = 400) -> np.ndarray:
    """Coefficients P[0..7] of atan(t) ~ t * sum_k P[k] t^(2k), t in [0, 1]."""
    t = np.linspace(0.0, 1.0, 40001)
    A = np.stack([t ** (2 * k + 1) for k in range(8)], axis=1)
    return _lawson(A, np.arctan(t), iters)


def fit_atan_anchor(iters: int = 400) -> np.ndarray:
    """Coefficients (c0, c1) of atan(t) ~ t (c0 + c1 t), t in [0, 1]."""
    t = np.linspace(0.0, 1.0, 20001)
    A = np.stack([t, t * t], axis=1)
    return _lawson(A, np.arctan(t), iters)


def as_cuda(c) -> str:
    return ", ".join(f"{x:.9e}f" for x in c)


if __name__ == "__main__":
    print("precise:", as_cuda(fit_atan_precise()))
    print("anchor: ", as_cuda(fit_atan_anchor()))
