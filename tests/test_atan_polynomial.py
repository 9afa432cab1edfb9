"""The rotation kernels' atan2 (octant reduction + a degree-7 polynomial in
t^2, coefficients fitted for that kernel) evaluated step by step in float32
on the CPU against numpy's float64 atan2: the coordinate error it adds is
bounded here, independently of the GPU."""
import os
import re

import numpy as np

SRC = os.path.join(os.path.dirname(__file__), "..", "paper_1705_07272_gb300", "csrc", "common.cuh")


def _coeffs(dtype=np.float32):
    src = open(SRC).read()
    body = src[src.index("float rot_atan2("):]
    m = re.search(r"constexpr float P\[8\] = \{([^}]*)\}", body)
    return np.array([float(x.strip().rstrip("f")) for x in m.group(1).split(",")], dtype=dtype)


def _atan2_f32(y, x, P):
    f = np.float32
    y = y.astype(f)
    x = x.astype(f)
    ax, ay = np.abs(x), np.abs(y)
    mx, mn = np.maximum(ax, ay), np.minimum(ax, ay)
    with np.errstate(divide="ignore", invalid="ignore"):
        t = np.where(mx > 0, (mn / mx).astype(f), f(0))
    u = (t * t).astype(f)
    p = np.full_like(u, P[7])
    for i in range(6, -1, -1):
        p = (p * u + P[i]).astype(f)                 # fmaf rounds once; this rounds twice (pessimistic)
    r = (t * p).astype(f)
    r = np.where(ay > ax, (f(1.57079632679) - r).astype(f), r)
    r = np.where(x < 0, (f(3.14159265359) - r).astype(f), r)
    return np.copysign(r, y)


def test_rotation_atan2_error_bound():
    P = _coeffs()
    rng = np.random.default_rng(0)
    ang = rng.uniform(-np.pi, np.pi, 400000)
    rad = rng.uniform(1e-3, 1.0, ang.size)
    y, x = rad * np.sin(ang), rad * np.cos(ang)
    y32, x32 = y.astype(np.float32), x.astype(np.float32)
    got = _atan2_f32(y32, x32, P).astype(np.float64)
    ref = np.arctan2(y32.astype(np.float64), x32.astype(np.float64))
    err = np.abs(got - ref)
    err = np.minimum(err, 2 * np.pi - err)        # +-pi wrap
    assert err.max() < 4e-7, err.max()


def test_rotation_atan2_axes_and_origin():
    P = _coeffs()
    y = np.array([0.0, 1.0, 0.0, -1.0, 0.0, 1.0, -1.0], dtype=np.float32)
    x = np.array([1.0, 0.0, -1.0, 0.0, 0.0, 1.0, -1.0], dtype=np.float32)
    got = _atan2_f32(y, x, P)
    want = np.array([0.0, np.pi / 2, np.pi, -np.pi / 2, 0.0, np.pi / 4, -3 * np.pi / 4])
    assert np.allclose(got, want, atol=4e-7)


def test_committed_constants_are_the_lawson_fits():
    # the kernels' polynomials are exactly what tests/atan_fit.py derives
    from tests.atan_fit import fit_atan_anchor, fit_atan_precise
    assert np.allclose(_coeffs(np.float64), fit_atan_precise(), rtol=2e-9, atol=0)
    src = open(os.path.join(os.path.dirname(SRC), "rotcoord.cuh")).read()
    body = src[src.index("float anchor_atan2("):]
    m = re.search(r"t \* fmaf\(([-0-9.e+]+)f, t, ([-0-9.e+]+)f\)", body)
    got = np.array([float(m.group(2)), float(m.group(1))])
    assert np.allclose(got, fit_atan_anchor(), rtol=2e-9, atol=0)


def test_anchor_atan2_error_bound():
    # the anchor arctangent only picks a pixel centre: 3.4e-3 rad is < 0.3 px at 512 columns
    from tests.atan_fit import fit_atan_anchor
    c0, c1 = fit_atan_anchor()
    t = np.linspace(0.0, 1.0, 100001)
    assert np.abs(t * (c0 + c1 * t) - np.arctan(t)).max() < 3.4e-3
