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
    among equal magnitudes the lower index is kept; every row sorted by index."""
    T = np.asarray(T)
    V, N = T.shape
    a = np.abs(T)
    kth = np.partition(a, N - K, axis=1)[:, N - K]          # K-th largest magnitude
    gt = a > kth[:, None]
    eq = a == kth[:, None]
    need = K - gt.sum(axis=1)
    sel = gt | (eq & (np.cumsum(eq, axis=1) <= need[:, None]))
    rows, cols = np.nonzero(sel)                              # row-major: indices ascend
    vals = T[rows, cols]
    rowptr = np.arange(V + 1, dtype=np.int64) * K
    return vals, cols.astype(np.int64), rowptr


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


def frame(n: np.ndarray):
    """Orthonormal tangent frame (b1, b2) around unit normals n [V, 3]: the
    branchless construction of Duff et al., 'Building an Orthonormal Basis,
    Revisited' (2017)."""
    n = np.asarray(n, dtype=np.float64)
    sign = np.where(n[:, 2] >= 0.0, 1.0, -1.0)
    a = -1.0 / (sign + n[:, 2])
    b = n[:, 0] * n[:, 1] * a
    b1 = np.stack([1.0 + sign * n[:, 0] * n[:, 0] * a, sign * b, -sign * n[:, 0]], axis=1)
    b2 = np.stack([b, sign + n[:, 1] * n[:, 1] * a, -n[:, 1]], axis=1)
    return b1, b2


def view_bins(pos, nrm, cams, bin_dirs):
    """(bin_of [S, V], margin [S, V]): for every camera s and vertex v the bin
    whose local direction has the largest dot product with the local view
    direction normalize(cam - pos) (lower bin on ties), and the gap between
    the best and the second-best dot product."""
    pos = np.asarray(pos, dtype=np.float64)
    b1, b2 = frame(nrm)
    n = np.asarray(nrm, dtype=np.float64)
    out = np.zeros((len(cams), len(pos)), dtype=np.int64)
    margin = np.zeros((len(cams), len(pos)))
    for s, cam in enumerate(np.asarray(cams, dtype=np.float64)):
        w = cam[None, :] - pos
        w /= np.linalg.norm(w, axis=1, keepdims=True)
        loc = np.stack([(w * b1).sum(1), (w * b2).sum(1), (w * n).sum(1)], axis=1)
        d = loc @ np.asarray(bin_dirs, dtype=np.float64).T
        out[s] = np.argmax(d, axis=1)
        srt = np.sort(d, axis=1)
        margin[s] = srt[:, -1] - srt[:, -2] if d.shape[1] > 1 else np.inf
    return out, margin
