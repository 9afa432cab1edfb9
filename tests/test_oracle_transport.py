"""Pins of the transport side: the integrand's closed forms, Parseval for the
double product (Eq. 2-5 reduced to two factors), top-K packing and the
storage roundings."""
import math

import numpy as np
import pytest

import synth
from oracle import haar, shade, shift, transport


def _weights(pos, nrm, occ_c, occ_r, Ht, Wt, **kw):
    return synth.transport_weights(pos, nrm, occ_c, occ_r, Ht, Wt, **kw).numpy()


def test_unoccluded_diffuse_integrates_to_pi():
    # P12: integral of max(0, n.w) over the sphere is pi
    rng = synth.rng_for(99)
    pos, nrm = synth.sphere_vertices(rng, 8)
    w = _weights(pos, nrm, np.zeros((0, 3)), np.zeros(0), 128, 256)
    assert np.allclose(w.sum((1, 2)), math.pi, rtol=2e-3)


def test_unoccluded_phong_mirror_view_integrates_to_one():
    # P12: with v = n the lobe is (s+2)/(2 pi) cos^(s+1), whose integral is 1
    rng = synth.rng_for(98)
    pos, nrm = synth.sphere_vertices(rng, 6)
    expo = np.array([8.0, 32.0, 8.0, 32.0, 8.0, 32.0])
    w = _weights(pos, nrm, np.zeros((0, 3)), np.zeros(0), 256, 512, view=nrm, expo=expo)
    assert np.allclose(w.sum((1, 2)), 1.0, rtol=3e-3)


def test_visibility_blocks_the_occluder_disc():
    # a sphere of radius r at distance D blocks the cone of half-angle asin(r/D)
    pos = np.array([[0.0, 0.0, 0.0]])
    axis = np.array([0.6, 0.3, -0.5])
    axis /= np.linalg.norm(axis)
    nrm = axis[None]
    D, r = 2.0, 0.5
    w_open = _weights(pos, nrm, np.zeros((0, 3)), np.zeros(0), 256, 512)
    w_occ = _weights(pos, nrm, (D * axis)[None], np.array([r]), 256, 512)
    lost = (w_open - w_occ).sum()
    a = math.asin(r / D)
    assert lost == pytest.approx(math.pi * math.sin(a) ** 2, rel=2e-2)   # int cos over cap


def test_occluders_keep_clear_of_surfaces():
    for surface, cid in (("sphere", 0), ("torus", 1)):
        c, r = synth.occluders(synth.rng_for(cid, 2), 8, surface)
        for ci, ri in zip(c, r):
            gap = (np.linalg.norm(ci) - 1.0) if surface == "sphere" else synth._torus_surface_distance(ci)
            assert gap - ri > 0.05


def test_double_product_parseval():
    # P11: sum_k G'_k T_k = sum_p g_p w_p for dense untruncated storage
    sc = synth.scene(0, V=12, S=2)
    H, W = sc["H"], sc["W"]
    w = _weights(sc["pos"], sc["nrm"], sc["occ_c"], sc["occ_r"], H, W)
    T = transport.project(w)
    L = haar.forward(sc["light"])
    Ls = shift.haar_shift(L, H, W, shift.TRANSLATE, sc["params"])
    coef = np.einsum("vk,sck->vsc", T, Ls)
    g = haar.inverse(Ls, H, W)
    pix = shade.radiance_pixels(g, w)
    assert np.abs(coef - pix).max() < 1e-11 * np.abs(pix).max()
    assert np.abs(shade.radiance(Ls, T, H, W) - pix).max() < 1e-11 * np.abs(pix).max()


def test_truncated_storage_equals_truncated_sum():
    sc = synth.scene(1, V=6, S=2, H=16, W=32)
    H, W = 16, 32
    w = _weights(sc["pos"], sc["nrm"], sc["occ_c"], sc["occ_r"], H, W)
    T = transport.project(w)
    L = shift.haar_shift(haar.forward(sc["light"]), H, W, shift.TRANSLATE, sc["params"])
    low = transport.lowest(T, 100)
    r = shade.radiance(L, low, H, W)
    assert np.allclose(r, np.einsum("vk,sck->vsc", low, L[..., :100]), rtol=1e-11, atol=1e-13)
    vals, idx, rp = transport.topk_csr(T, 40)
    dense = transport.csr_dense(vals, idx, rp, H * W)
    assert np.allclose(shade.radiance(L, dense, H, W), np.einsum("vk,sck->vsc", dense, L),
                       rtol=1e-11, atol=1e-13)


def test_coarse_quadrature_projection():
    # spreading a block's weight over its pixels leaves levels 1..log2(b) empty and
    # the coarser coefficients equal the coarse map's transform divided by b
    rng = np.random.default_rng(3)
    w = rng.random((2, 8, 16))
    T = transport.project(w, 32, 64)
    assert np.abs(T[:, 8 * 16:]).max() < 1e-14
    assert np.allclose(T[:, :8 * 16], haar.forward(w) / 4.0)


def test_topk_ties_and_order():
    T = np.array([[0.0, 3.0, -3.0, 1.0, 3.0, -0.5]])
    vals, idx, rp = transport.topk_csr(T, 3)
    assert idx.tolist() == [1, 2, 4]
    assert vals.tolist() == [3.0, -3.0, 3.0]
    assert rp.tolist() == [0, 3]
    vals, idx, _ = transport.topk_csr(T, 2)
    assert idx.tolist() == [1, 2]          # equal magnitudes: lower index first


def test_bf16_rounding():
    x = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -8 + 2.0 ** -20,
                  -2.5, 3.0e38, 1e-40])
    got = transport.to_bf16(x)
    want = [1.0, 1.0, 1.0 + 4 * 2.0 ** -8, 1.0 + 2.0 ** -7, -2.5]
    assert got[:5].tolist() == want
    assert np.isfinite(got[5])
    hi, lo = transport.split_hilo(np.array([math.pi, -1e-3, 123.456]))
    s = transport.bf16_bits_to_f64(hi) + transport.bf16_bits_to_f64(lo)
    assert np.all(np.abs(s - np.array([math.pi, -1e-3, 123.456], dtype=np.float32)) <=
                  2.0 ** -16 * np.abs(s))


def test_f16_rounding():
    x = np.array([1.0 + 2.0 ** -11, 1.0 + 3 * 2.0 ** -11, 65504.0, 1e-8])
    assert transport.to_f16(x).tolist() == [1.0, 1.0 + 2.0 ** -9, 65504.0, 0.0]
