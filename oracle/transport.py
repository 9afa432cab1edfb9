"""Transport vectors: Haar projection, truncation, CSR packing and the
storage roundings (oracle).

The transport vector of a vertex is the Haar projection of its transfer
function (BRDF x cosine x visibility, Eq. 2-3 with the visibility folded into
the transfer function) weighted by the solid angle of each pixel.  Storage
forms:

* lowest-K: the first K canonical coefficients (coarse levels first);
* top-K: the K largest |T_k| (non-linear wavelet approximation, cited in
  Sec. "Haar-domain methods"), ties to the lower index, rows sorted by index;
* BF16 / FP16 values rounded to nearest-even.

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import numpy as np

from . import haar


def project(w: np.ndarray, H: int | None = None, W: int | None = None) -> np.ndarray:
    """Haar transport vectors [..., N] of pixel weights [..., h, w].

    If (H, W) is larger than the weight grid, every weight is spread
    uniformly over the pixels of its block before the transform."""
    w = np.asarray(w, dtype=np.float64)
    h, ww = w.shape[-2:]
    if H is not None and (H, W) != (h, ww):
        b = H // h
        w = np.repeat(np.repeat(w, b, axis=-2), b, axis=-1) / float(b * b)
    return haar.forward(w)


def lowest(T: np.ndarray, K: int) -> np.ndarray:
    return np.ascontiguousarray(T[..., :K])


def topk_csr(T: np.ndarray, K: int):
    """CSR (vals [V*K], idx [V*K], rowptr [V+1]) of the K largest |T| per row;
    equal magnitudes keep the lower index; every row sorted by index."""
    T = np.asarray(T)
    V, N = T.shape
    # stable sort on -|T| keeps the lower index first among equal magnitudes
    order = np.argsort(-np.abs(T), axis=1, kind="stable")[:, :K]
    idx = np.sort(order, axis=1)
    vals = np.take_along_axis(T, idx, axis=1)
    rowptr = np.arange(V + 1, dtype=np.int64) * K
    return vals.reshape(-1), idx.reshape(-1), rowptr


def csr_dense(vals, idx, rowptr, N: int) -> np.ndarray:
    V = len(rowptr) - 1
    out = np.zeros((V, N))
    for v in range(V):
        a, b = rowptr[v], rowptr[v + 1]
        out[v, idx[a:b]] = vals[a:b]
    return out


def to_bf16_bits(x) -> np.ndarray:
    """Round to bfloat16 (nearest-even on the float32 value); uint16 bit patterns.

    bfloat16 is the upper half of an IEEE binary32 word; rounding adds
    0x7FFF plus the lowest kept bit before truncation (ties to even)."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    r = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
    nan = np.isnan(f)
    r = np.where(nan, 0x7FC0, r)
    return r.astype(np.uint16)


def bf16_bits_to_f64(b) -> np.ndarray:
    u = np.asarray(b, dtype=np.uint16).astype(np.uint32) << 16
    return u.view(np.float32).astype(np.float64)


def to_bf16(x) -> np.ndarray:
    return bf16_bits_to_f64(to_bf16_bits(x))


def split_hilo(x):
    """(hi, lo) bfloat16 pair of float32 values: hi = bf16(x), lo = bf16(x - hi)."""
    f = np.asarray(x, dtype=np.float32)
    hi_b = to_bf16_bits(f)
    hi = bf16_bits_to_f64(hi_b).astype(np.float32)
    lo_b = to_bf16_bits(f - hi)
    return hi_b, lo_b


def to_f16(x) -> np.ndarray:
    """IEEE binary16, nearest-even (numpy's conversion), as float64."""
    return np.asarray(np.asarray(x, dtype=np.float64).astype(np.float16), dtype=np.float64)
