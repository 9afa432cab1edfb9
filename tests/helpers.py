"""Shared helpers of the test-suite (input marshalling and error metrics)."""
import numpy as np


def rel_l2(a, b, axis=None):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    num = np.sqrt(((a - b) ** 2).sum(axis=axis))
    den = np.sqrt((b ** 2).sum(axis=axis))
    return num / np.maximum(den, 1e-300)


def f32(x):
    """float32 rounding, returned as float64 (what both sides consume)."""
    return np.asarray(x, dtype=np.float32).astype(np.float64)
