"""Pins of the oracle's chain-rule rotation route (Sec. "Rotating Haar",
Eq. pde1-pde3, and Sec. "Mathematical description", Eq. conv/tker/sker)."""
import math

import numpy as np
import pytest

from oracle import chain_rule, haar, resample, shift
from oracle.resample import SPHERE, TORUS


def _map(H, W, seed, smooth=False):
    rng = np.random.default_rng(seed)
    if not smooth:
        return rng.lognormal(0.0, 1.0, (H, W))
    th = (np.arange(H) + 0.5) * math.pi / H
    ph = (np.arange(W) + 0.5) * 2 * math.pi / W
    T, F = np.meshgrid(th, ph, indexing="ij")
    d = np.stack([np.sin(T) * np.sin(F), np.cos(T), np.sin(T) * np.cos(F)], -1)
    out = np.full((H, W), 1.0)
    for _ in range(3):
        c = rng.standard_normal(3)
        c /= np.linalg.norm(c)
        out += 2.0 * np.exp(4.0 * (d @ c - 1.0))
    return out


@pytest.mark.parametrize("beta", [0.0, 0.3, -1.234, 2 * math.pi / 64 * 5])
def test_rotation_about_y_is_the_exact_shift(beta):
    # Jacobian = identity: the route equals the exact operator (a column shift)
    H, W = 16, 32
    P = _map(H, W, 1)
    R = resample.rot_y(beta)
    got = chain_rule.rotate_coeffs(P, R, SPHERE)
    ref = shift.haar_shift(haar.forward(P)[None], H, W, shift.ROTATE, R.reshape(1, 9))[0, 0]
    assert np.allclose(got, ref, rtol=0, atol=1e-10)


def test_identity_rotation_returns_the_coefficients():
    H, W = 16, 32
    P = _map(H, W, 2)
    got = chain_rule.rotate_coeffs(P, np.eye(3), SPHERE)
    assert np.allclose(got, haar.forward(P), rtol=0, atol=1e-10)


def test_jacobian_matches_finite_differences():
    H, W = 32, 64
    R = resample.euler_matrix(0.4, -1.1, 2.3)
    rng = np.random.default_rng(3)
    ii = rng.uniform(4, H - 5, 200)
    jj = rng.uniform(0, W, 200)
    c = chain_rule.coords_and_jacobian(R, H, W, ii, jj)
    h = 1e-5

    def uv(a, b):
        d = chain_rule.coords_and_jacobian(R, H, W, a, b)
        return d["u"], d["v"]

    def wrap(x):                       # v lives on a circle of W columns
        return (x + W / 2) % W - W / 2

    up, vp = uv(ii + h, jj)
    um, vm = uv(ii - h, jj)
    u_i, v_i = (up - um) / (2 * h), wrap(vp - vm) / (2 * h)
    up, vp = uv(ii, jj + h)
    um, vm = uv(ii, jj - h)
    u_j, v_j = (up - um) / (2 * h), wrap(vp - vm) / (2 * h)
    upp, vpp = uv(ii + h, jj + h)
    upm, vpm = uv(ii + h, jj - h)
    ump, vmp = uv(ii - h, jj + h)
    umm, vmm = uv(ii - h, jj - h)
    u_ij = (upp - upm - ump + umm) / (4 * h * h)
    v_ij = wrap(vpp - vpm - vmp + vmm) / (4 * h * h)
    ok = np.hypot(np.sin(c["u"] * math.pi / H), 0) > 0.05          # away from the poles
    for name, fd, tol in (("u_i", u_i, 1e-6), ("u_j", u_j, 1e-6), ("v_i", v_i, 1e-6), ("v_j", v_j, 1e-6),
                          ("u_ij", u_ij, 1e-3), ("v_ij", v_ij, 1e-3)):
        err = np.abs(c[name][ok] - fd[ok]).max() / max(1.0, np.abs(fd[ok]).max())
        assert err < tol, (name, err)


def test_small_tilt_of_a_smooth_map_is_close_to_the_exact_operator():
    # the route is a first-order approximation: on a smooth map and a small tilt
    # it is near the exact result, and a sign error in any Jacobian term breaks it
    H, W = 32, 64
    P = _map(H, W, 4, smooth=True)
    R = resample.rot_x(0.08)
    got = chain_rule.rotate_coeffs(P, R, SPHERE)
    ref = shift.haar_shift(haar.forward(P)[None], H, W, shift.ROTATE, R.reshape(1, 9))[0, 0]
    n0 = 2                                                   # the scaling block is exact by construction
    err = np.linalg.norm(got[n0:] - ref[n0:]) / np.linalg.norm(ref[n0:])
    assert err < 0.01, err
    assert np.allclose(got[:n0], ref[:n0], rtol=1e-12, atol=1e-12)


def test_linearity():
    H, W = 16, 32
    P1, P2 = _map(H, W, 5), _map(H, W, 6)
    R = resample.euler_matrix(0.7, 0.2, -0.4)
    a = chain_rule.rotate_coeffs(2.0 * P1 - 0.5 * P2, R, TORUS)
    b = 2.0 * chain_rule.rotate_coeffs(P1, R, TORUS) - 0.5 * chain_rule.rotate_coeffs(P2, R, TORUS)
    assert np.allclose(a, b, rtol=1e-10, atol=1e-10)
