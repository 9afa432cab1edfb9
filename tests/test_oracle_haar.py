"""Pins of the oracle's Haar transform (orthonormal non-standard 2-D Haar,
Sec. "Our contributions" / "Mathematical description")."""
import numpy as np
import pytest

from oracle import haar

SHAPES = [(2, 2), (2, 4), (4, 4), (4, 8), (8, 16), (32, 32), (16, 32)]


@pytest.mark.parametrize("H,W", SHAPES)
def test_parseval_and_reconstruction(H, W):
    rng = np.random.default_rng(H * 100 + W)
    P = rng.lognormal(0.0, 1.5, (3, H, W))
    c = haar.forward(P)
    assert c.shape == (3, H * W)
    # P1: energy preserved
    assert np.allclose((c ** 2).sum(-1), (P ** 2).sum((-2, -1)), rtol=1e-13)
    # P2: perfect reconstruction
    assert np.abs(haar.inverse(c, H, W) - P).max() < 1e-12 * np.abs(P).max()


@pytest.mark.parametrize("H,W", [(2, 2), (2, 4), (4, 4), (4, 8)])
def test_basis_orthonormal(H, W):
    # P3: basis matrix built from the definition is orthonormal
    B = haar.basis_matrix(H, W)
    assert np.abs(B @ B.T - np.eye(H * W)).max() < 1e-14


def test_2x2_block_by_hand():
    # a=1 b=2 / c=3 d=5: A=(11)/2, H=(b+d-a-c)/2=1.5, V=(c+d-a-b)/2=2.5, D=(a+d-b-c)/2=0.5
    P = np.array([[1.0, 2.0], [3.0, 5.0]])
    assert np.allclose(haar.forward(P), [5.5, 1.5, 2.5, 0.5])


def test_basis_functions_are_differences():
    # H band of the finest level is a difference along phi (columns), V along theta (rows)
    H, W = 4, 8
    k_h = haar.index(H, W, 1, haar.BAND_H, 1, 2)
    k_v = haar.index(H, W, 1, haar.BAND_V, 1, 2)
    k_d = haar.index(H, W, 1, haar.BAND_D, 1, 2)
    e = np.zeros(H * W)
    for k, expect in ((k_h, [[-1, 1], [-1, 1]]), (k_v, [[-1, -1], [1, 1]]), (k_d, [[1, -1], [-1, 1]])):
        e[:] = 0
        e[k] = 1.0
        m = haar.inverse(e, H, W)
        assert np.allclose(m[2:4, 4:6], 0.5 * np.array(expect))
        assert np.abs(m).sum() == pytest.approx(2.0)


@pytest.mark.parametrize("H,W", [(32, 32), (128, 256), (256, 512)])
def test_canonical_layout(H, W):
    n, q = haar.dims(H, W)
    total = q
    for lvl in range(n, 0, -1):
        g = haar.block_count(H, W, lvl)
        assert g == (H >> lvl) * (W >> lvl)
        for band in range(3):
            assert haar.band_range(H, W, lvl, band) == (total, total + g)
            total += g
    assert total == H * W
    for k in [0, q - 1, q, 4 * q - 1, H * W // 4, H * W - 1]:
        lvl, band, r, c = haar.decode(H, W, k)
        if lvl:
            assert haar.index(H, W, lvl, band, r, c) == k


def test_lowest_4096_of_256x512_is_H_band_of_level_3():
    # c2 keeps the first 4096 coefficients: A, levels 8..4, and the H band of level 3
    assert haar.band_range(256, 512, 3, haar.BAND_H) == (2048, 4096)
    assert haar.band_range(256, 512, 4, haar.BAND_D) == (1536, 2048)


def test_scaling_is_block_mean_times_side():
    rng = np.random.default_rng(1)
    P = rng.standard_normal((16, 32))
    c = haar.forward(P)
    assert np.allclose(c[:2], [P[:, :16].sum() / 16, P[:, 16:].sum() / 16])
