"""Pins of the oracle's phase shift: closed forms and invariants that the
paper and the mathematics fix (Sec. "Rotating Haar", "Mathematical
description", "Algorithmic optimization")."""
import math

import numpy as np
import pytest

from oracle import haar, paper_route, resample, shift
from oracle.resample import SPHERE, TORUS

TR, ROT = shift.TRANSLATE, shift.ROTATE


def _coeffs(H, W, C=1, seed=0):
    rng = np.random.default_rng(seed)
    return haar.forward(rng.lognormal(0.0, 1.5, (C, H, W)))


@pytest.mark.parametrize("boundary", [SPHERE, TORUS])
@pytest.mark.parametrize("H,W", [(4, 8), (8, 8), (16, 32)])
def test_identity_shifts(H, W, boundary):
    # P4: zero shift, full azimuth period and full elevation period are the identity
    c = _coeffs(H, W, 2)
    period_y = 2 * H if boundary == SPHERE else H
    for dx, dy in ((0, 0), (W, 0), (0, period_y), (2 * W, -period_y)):
        out = shift.haar_shift(c, H, W, TR, np.array([[dx, dy]]), boundary)[0]
        assert np.abs(out - c).max() < 1e-12


@pytest.mark.parametrize("boundary", [SPHERE, TORUS])
@pytest.mark.parametrize("H,W,dx,dy", [(8, 16, 0.3, 0.7), (16, 16, 5.25, 3.5),
                                       (8, 16, 11.9, -2.2), (16, 32, 30.0, 20.5)])
def test_derivative_route_equals_definition(H, W, dx, dy, boundary):
    # P15: the paper's derivative route (difference fields + triangle/box kernels,
    # a-trous recursion) equals Haar(resample(Haar^-1 c)) for translations
    c = _coeffs(H, W)[0]
    P = haar.inverse(c, H, W)
    a = shift.haar_shift(c[None], H, W, TR, np.array([[dx, dy]]), boundary)[0, 0]
    b = paper_route.translate_coeffs(P, dx, dy, boundary)
    assert np.abs(a - b).max() < 1e-12 * np.abs(c).max()


def test_triangle_kernel_recursion():
    # Eq. tker: side B = 2^(l+2) has peak B/2 and B-1 taps; the recursion reproduces it
    for B in (2, 4, 8, 16, 32):
        imp = np.zeros((1, 64))
        imp[0, 0] = 1.0
        tri = paper_route._atrous_triangle(imp.T, 0, B)[:, 0]
        # correlation of an impulse at 0 gives the kernel reversed at negative lags;
        # use a shifted impulse instead
        imp = np.zeros(64)
        imp[B] = 1.0
        got = paper_route._atrous_triangle(imp[:, None], 0, B)[:, 0]
        want = np.zeros(64)
        for t in range(B - 1):
            want[B - t] = min(t + 1, B - 1 - t)
        assert np.allclose(got, want), B
        assert got.max() == B // 2 and (got > 0).sum() == B - 1
        del tri


@pytest.mark.parametrize("boundary", [SPHERE, TORUS])
@pytest.mark.parametrize("H,W", [(8, 16), (16, 16), (32, 32)])
def test_dyadic_shifts_are_signed_permutations(H, W, boundary):
    # P5: an integer shift that is a multiple of the block side 2^l moves whole
    # blocks, so those levels are a signed permutation of the input
    c = _coeffs(H, W, 2, seed=3)
    cases = [(2, 0), (4, 4), (8, 2), (W // 2, H), (0, 2 * H - 4), (6, 10)]
    seen_flip = False
    for kx, ky in cases:
        out = shift.haar_shift(c, H, W, TR, np.array([[kx, ky]]), boundary)[0]
        res = shift.dyadic_permutation(c, H, W, kx, ky, boundary)
        assert res, (kx, ky)
        for k, val in res.items():
            assert np.abs(out[:, k] - val).max() < 1e-12 * np.abs(c).max()
        seen_flip |= boundary == SPHERE and ky % (2 * H) != 0
    assert boundary == TORUS or seen_flip


def test_pole_crossing_flips_vertical_and_diagonal_signs():
    # a shift by H rows mirrors the whole map across a pole: V and D change sign
    H, W = 8, 16
    c = _coeffs(H, W)[0]
    out = shift.haar_shift(c[None], H, W, TR, np.array([[0.0, H]]), SPHERE)[0, 0]
    for lvl in range(1, 4):
        for band, sgn in ((haar.BAND_H, 1), (haar.BAND_V, -1), (haar.BAND_D, -1)):
            r, cc = 0, 0
            k_out = haar.index(H, W, lvl, band, r, cc)
            rows, cols = H >> lvl, W >> lvl
            k_in = haar.index(H, W, lvl, band, rows - 1, (cc + cols // 2) % cols)
            assert out[k_out] == pytest.approx(sgn * c[k_in], rel=1e-12, abs=1e-12)


def test_shift_composition():
    # P6: S_a S_b = S_(a+b) when at most one of the two is fractional (azimuth always;
    # elevation in TORUS mode)
    H, W = 8, 16
    c = _coeffs(H, W, 1, seed=5)
    for boundary, (a, b) in ((SPHERE, ((3.0, 0.0), (4.6, 0.0))), (TORUS, ((2.0, 3.0), (1.3, 0.45)))):
        one = shift.haar_shift(c, H, W, TR, np.array([a]), boundary)[0]
        two = shift.haar_shift(one, H, W, TR, np.array([b]), boundary)[0]
        both = shift.haar_shift(c, H, W, TR, np.array([[a[0] + b[0], a[1] + b[1]]]), boundary)[0]
        assert np.abs(two - both).max() < 1e-12 * np.abs(c).max()


def test_sphere_elevation_shifts_do_not_compose():
    # documented non-invariant: two fractional elevation shifts differ from their sum
    H, W = 8, 16
    c = _coeffs(H, W, 1, seed=6)
    one = shift.haar_shift(c, H, W, TR, np.array([[0.0, 0.5]]), SPHERE)[0]
    two = shift.haar_shift(one, H, W, TR, np.array([[0.0, 0.5]]), SPHERE)[0]
    both = shift.haar_shift(c, H, W, TR, np.array([[0.0, 1.0]]), SPHERE)[0]
    assert np.abs(two - both).max() > 1e-3


def test_dc_preserved_and_constants_invariant():
    H, W = 16, 32
    c = _coeffs(H, W, 2, seed=7)
    prm = np.array([[3.3, 0.0], [7.1, 5.6], [0.4, 31.2]])
    out = shift.haar_shift(c, H, W, TR, prm, TORUS)
    # P7: the sum (scaling coefficients' total) survives any TORUS translation
    assert np.allclose(out[..., :2].sum(-1), c[None, :, :2].sum(-1), rtol=1e-13)
    out_s = shift.haar_shift(c, H, W, TR, prm[:1] * [1, 0], SPHERE)
    assert np.allclose(out_s[..., :2].sum(-1), c[None, :, :2].sum(-1), rtol=1e-13)
    # P8: a constant map is invariant under every shift and rotation
    const = haar.forward(np.full((1, H, W), 2.5))
    for kind, p in ((TR, prm), (ROT, np.stack([resample.euler_matrix(0.3, 1.1, 2.0).ravel(),
                                               resample.euler_matrix(2.9, 0.2, 4.4).ravel()]))):
        for boundary in (SPHERE, TORUS):
            o = shift.haar_shift(const, H, W, kind, p, boundary)
            assert np.abs(o - const[None]).max() < 1e-12


def test_rotation_about_y_is_azimuth_shift():
    # P9 / Sec. "Algorithmic optimization": R_y(beta) maps phi -> phi + beta, so
    # R_y(-dx dphi) is the translation by dx columns (integer or fractional)
    H, W = 16, 32
    c = _coeffs(H, W, 2, seed=8)
    dph = 2 * math.pi / W
    for dx in (3.0, 5.37, 30.5):
        a = shift.haar_shift(c, H, W, ROT, resample.rot_y(-dx * dph).reshape(1, 9), SPHERE)[0]
        b = shift.haar_shift(c, H, W, TR, np.array([[dx, 0.0]]), SPHERE)[0]
        assert np.abs(a - b).max() < 1e-11 * np.abs(c).max()


def test_identity_rotation():
    # P10
    H, W = 16, 32
    c = _coeffs(H, W, 1, seed=9)
    o = shift.haar_shift(c, H, W, shift.ROTATE_EULER, np.zeros((1, 3)), SPHERE)[0]
    assert np.abs(o - c).max() < 1e-12 * np.abs(c).max()


def test_half_turns_are_pixel_permutations():
    # R_x(pi): (x, y, z) -> (x, -y, -z): theta' = pi - theta, phi' = pi - phi
    # R_z(pi): (x, y, z) -> (-x, -y, z): theta' = pi - theta, phi' = -phi
    H, W = 8, 16
    rng = np.random.default_rng(10)
    P = rng.standard_normal((H, W))
    i = np.arange(H)[:, None]
    j = np.arange(W)[None, :]
    gx = P[H - 1 - i, (W // 2 - 1 - j) % W]
    gz = P[H - 1 - i, (W - 1 - j) % W]
    assert np.abs(resample.rotate(P, resample.rot_x(math.pi)) - gx).max() < 1e-9
    assert np.abs(resample.rotate(P, resample.rot_z(math.pi)) - gz).max() < 1e-9


def test_rotation_coordinates_match_acos_atan_form():
    # Eq. theta / Eq. phi: theta' = acos(R_2 p), phi' = atan(R_1 p / R_3 p) with the
    # quadrant taken from the signs, against the atan2 form the oracle uses
    H, W = 16, 32
    R = resample.euler_matrix(0.7, 2.1, 4.0)
    u, v = resample.rotation_coords(R, H, W)
    rng = np.random.default_rng(11)
    for _ in range(50):
        i, j = rng.integers(0, H), rng.integers(0, W)
        th, ph = (i + 0.5) * math.pi / H, (j + 0.5) * 2 * math.pi / W
        p = np.array([math.sin(th) * math.sin(ph), math.cos(th), math.sin(th) * math.cos(ph)])
        q = R @ p
        th2 = math.acos(max(-1.0, min(1.0, q[1])))
        ph2 = math.atan(q[0] / q[2]) if q[2] != 0 else math.copysign(math.pi / 2, q[0])
        if q[2] < 0:
            ph2 += math.pi
        ph2 %= 2 * math.pi
        assert u[i, j] == pytest.approx(th2 / (math.pi / H) - 0.5, abs=1e-9)
        dv = (v[i, j] - (ph2 / (2 * math.pi / W) - 0.5) + W / 2) % W - W / 2
        assert abs(dv) < 1e-9


def test_linearity():
    # P14
    H, W = 8, 16
    a, b = _coeffs(H, W, 1, 12), _coeffs(H, W, 1, 13)
    prm = np.array([[2.7, 5.1]])
    lhs = shift.haar_shift(2.0 * a - 3.0 * b, H, W, TR, prm, SPHERE)
    rhs = 2.0 * shift.haar_shift(a, H, W, TR, prm, SPHERE) - 3.0 * shift.haar_shift(b, H, W, TR, prm, SPHERE)
    assert np.abs(lhs - rhs).max() < 1e-12 * np.abs(lhs).max()


def test_translation_by_bilinear_equals_area_projection():
    # for a translation, bilinear sampling at centres equals the exact area
    # average of the shifted piecewise-constant map (TORUS, away from poles)
    H, W = 8, 16
    rng = np.random.default_rng(14)
    P = rng.standard_normal((H, W))
    dx, dy = 0.25, 0.6
    g = resample.translate(P, dx, dy, TORUS)
    # area average: pixel [i, i+1) x [j, j+1) of the map shifted by (dy, dx)
    ref = np.zeros_like(P)
    for i in range(H):
        for j in range(W):
            acc = 0.0
            for (a0, a1, si) in ((i - dy, math.floor(i - dy) + 1, math.floor(i - dy)),
                                 (math.floor(i - dy) + 1, i + 1 - dy, math.floor(i - dy) + 1)):
                for (b0, b1, sj) in ((j - dx, math.floor(j - dx) + 1, math.floor(j - dx)),
                                     (math.floor(j - dx) + 1, j + 1 - dx, math.floor(j - dx) + 1)):
                    acc += (a1 - a0) * (b1 - b0) * P[si % H, sj % W]
            ref[i, j] = acc
    assert np.abs(g - ref).max() < 1e-12


# ---------------------------------------------------------------- start level

def _block_image(P, k):
    """2^k x (mean over each 2^k x 2^k block): the level-k scaling image in pixel form."""
    H, W = P.shape[-2:]
    b = 1 << k
    return P.reshape(P.shape[:-2] + (H // b, b, W // b, b)).mean(axis=(-3, -1)) * b


@pytest.mark.parametrize("k", [1, 2, 3])
def test_start_level_is_the_shift_of_the_block_mean_image(k):
    # the N / 4^k coarsest coefficients are those of the 2^k-scaled block-mean
    # image, built here from pixels, not from coefficients
    H, W = 32, 64
    rng = np.random.default_rng(k)
    P = rng.lognormal(0.0, 1.0, (2, H, W))
    c = haar.forward(P)
    assert np.allclose(c[:, :(H * W) >> (2 * k)], haar.forward(_block_image(P, k)), rtol=0, atol=1e-12)
    prm = np.array([[3.25, 1.5], [100.7, -40.2]])
    got = shift.haar_shift(c, H, W, TR, prm, start_level=k)
    Pb = _block_image(P, k)
    ref = np.stack([haar.forward(resample.translate(Pb, dx / (1 << k), dy / (1 << k), SPHERE)) for dx, dy in prm])
    assert got.shape == (2, 2, (H * W) >> (2 * k))
    assert np.allclose(got, ref, rtol=0, atol=1e-10)


@pytest.mark.parametrize("boundary", [SPHERE, TORUS])
@pytest.mark.parametrize("k", [1, 2])
def test_start_level_exact_for_block_aligned_shifts(k, boundary):
    # whole-block moves commute with block averaging: the start-level result is
    # then the exact shift's coarsest N / 4^k coefficients
    H, W = 32, 64
    rng = np.random.default_rng(10 + k)
    c = haar.forward(rng.lognormal(0.0, 1.0, (3, H, W)))
    b = 1 << k
    prm = np.array([[b, 0], [3 * b, 5 * b], [W - b, 2 * H - 2 * b], [0, 7 * b]], dtype=np.float64)
    exact = shift.haar_shift(c, H, W, TR, prm, boundary)
    got = shift.haar_shift(c, H, W, TR, prm, boundary, start_level=k)
    n = (H * W) >> (2 * k)
    assert np.allclose(got, exact[..., :n], rtol=0, atol=1e-10)
    # a fractional shift is only approximated at the start level
    frac = shift.haar_shift(c, H, W, TR, np.array([[0.5 * b, 0.25 * b]]), boundary, start_level=k)
    full = shift.haar_shift(c, H, W, TR, np.array([[0.5 * b, 0.25 * b]]), boundary)[..., :n]
    assert not np.allclose(frac, full, atol=1e-6)


def test_start_level_rotation_identity_and_constants():
    H, W = 32, 64
    rng = np.random.default_rng(5)
    c = haar.forward(rng.lognormal(0.0, 1.0, (1, H, W)))
    for k in (1, 2):
        n = (H * W) >> (2 * k)
        got = shift.haar_shift(c, H, W, shift.ROTATE_EULER, np.zeros((1, 3)), start_level=k)
        assert np.allclose(got[0], c[:, :n], rtol=0, atol=1e-10)
        const = haar.forward(np.full((1, H, W), 2.5))
        rot = shift.haar_shift(const, H, W, shift.ROTATE_EULER, np.array([[0.3, 1.1, -2.0]]), start_level=k)
        assert np.allclose(rot[0], const[:, :n], rtol=0, atol=1e-10)
