"""GPU parity of the tcgen05 tensor-core double product (BF16 transport x
BF16 hi + lo lighting, FP32 accumulation) through the C ABI."""
import numpy as np
import pytest

import synth
from oracle import haar as oh
from oracle import shade as osd
from oracle import shift as osh
from oracle import transport as otr
from tests.helpers import f32, rel_l2

pytestmark = pytest.mark.gpu


def _t(x, dtype=None):
    import torch
    return torch.tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


def _bf16_tensor(bits):
    import torch
    return _t(bits.astype(np.int16), torch.int16).view(torch.bfloat16)


def _contract(hs, V, K, S, C, seed):
    """Random bf16 transport against hi/lo lighting produced by haar_shift."""
    import torch
    rng = np.random.default_rng(seed)
    H, W = 64, 128
    L = f32(oh.forward(synth.lighting_pixels(rng, C, H, W)))
    prm = rng.uniform(0, 100, (S, 2))
    plan = hs.Plan(H, W, C, max_shifts=S, out_coeffs=K, out_type=hs.HAAR_OUT_BF16_HILO)
    Ls = hs.haar_shift(plan, _t(L, torch.float32), _t(prm, torch.float64))      # [2, S, C, K] bf16
    Tb = otr.to_bf16_bits(rng.standard_normal((V, K)) * np.exp(-np.arange(K) / 800.0))
    tr = hs.Transport(hs.HAAR_T_DENSE_BF16, V, K, _bf16_tensor(Tb))
    R = hs.shade_vertices(plan, tr, Ls, S)
    torch.cuda.synchronize()
    lh = Ls.float().cpu().numpy().astype(np.float64)
    Tf = otr.bf16_bits_to_f64(Tb)
    ref = np.einsum("vk,sck->vsc", Tf, lh[0] + lh[1])
    plan.close()
    return R.cpu().numpy(), ref


def _acc_tol(K):
    """The tensor core adds each K=16 MMA's products into the FP32 accumulator
    with truncation (measured as a systematic shrink), at most ~1 ulp
    (2^-23 relative) per update; hi and lo make 2 K/16 updates."""
    return max(1e-5, 2 * (K // 16) * 2.0 ** -23)


@pytest.mark.parametrize("V,K,S,C", [(300, 128, 16, 3), (128, 64, 1, 16), (1000, 4096, 64, 3),
                                     (4099, 1024, 32, 8), (77, 256, 16, 16),
                                     # more 128-row tiles than the GB300's 152 SMs with a
                                     # remainder: the leftover tiles run as column slices
                                     (128 * 160 + 40, 256, 16, 3), (128 * 162, 128, 64, 3)])
def test_tensor_core_contraction_matches_fp64(hs, V, K, S, C):
    got, ref = _contract(hs, V, K, S, C, V + K)
    assert got.shape == ref.shape
    assert rel_l2(got, ref) <= _acc_tol(K)


def test_rejects_unsupported_shapes(hs):
    import torch
    plan = hs.Plan(16, 32, 3, max_shifts=5, out_coeffs=128, out_type=hs.HAAR_OUT_BF16_HILO)
    Ls = torch.zeros((2, 5, 3, 128), dtype=torch.bfloat16, device="cuda")
    tr = hs.Transport(hs.HAAR_T_DENSE_BF16, 10, 128, torch.zeros((10, 128), dtype=torch.bfloat16, device="cuda"))
    with pytest.raises(hs.HaarError):
        hs.shade_vertices(plan, tr, Ls, 5)          # S*C = 15 is not a multiple of 16
    plan2 = hs.Plan(16, 32, 3, max_shifts=16, out_coeffs=100, out_type=hs.HAAR_OUT_BF16_HILO)
    tr2 = hs.Transport(hs.HAAR_T_DENSE_BF16, 10, 100, torch.zeros((10, 100), dtype=torch.bfloat16, device="cuda"))
    with pytest.raises(hs.HaarError):
        hs.shade_vertices(plan2, tr2, torch.zeros((2, 16, 3, 100), dtype=torch.bfloat16, device="cuda"), 16)


def _c2_transport(sc, chunk=20000):
    """Lowest-4096 bf16 transport of the c2 scene: diffuse integrand on the
    64x128 quadrature grid, projected by the oracle."""
    H, W = sc["H"], sc["W"]
    out = []
    for v0 in range(0, sc["V"], chunk):
        w = synth.transport_weights(sc["pos"][v0:v0 + chunk], sc["nrm"][v0:v0 + chunk], sc["occ_c"],
                                    sc["occ_r"], 64, 128, device="cuda").double().cpu().numpy()
        T = oh.forward(w)[:, :4096] / 4.0        # coefficients of the 256x512 map (blocks of 4x4 pixels)
        out.append(otr.to_bf16_bits(T))
    return np.concatenate(out)


def test_full_size_c2_sampled(hs):
    # 200 000 vertices x 64 rotations x RGB: shade_batch (rotation -> bf16 hi/lo lowest
    # 4096 -> tcgen05 contraction); the oracle checks sampled (vertex, rotation) pairs
    # through pixel space against its own FP64 rotation of the lighting
    import torch
    sc = synth.scene(2)
    H, W, S, V = sc["H"], sc["W"], sc["S"], sc["V"]
    Tb = _c2_transport(sc)
    L = f32(oh.forward(sc["light"]))
    plan = hs.Plan(H, W, 3, kind=hs.HAAR_SHIFT_ROTATE_EULER, max_shifts=S, out_coeffs=4096,
                   out_type=hs.HAAR_OUT_BF16_HILO)
    tr = hs.Transport(hs.HAAR_T_DENSE_BF16, V, 4096, _bf16_tensor(Tb))
    R = hs.shade_batch(plan, _t(L, torch.float32), _t(sc["params"], torch.float64), tr)
    torch.cuda.synchronize()
    got = R.cpu().numpy()
    assert np.isfinite(got).all()
    rng = np.random.default_rng(1)
    pick = np.sort(rng.choice(V, 200, replace=False))
    Tf = otr.bf16_bits_to_f64(Tb[pick])
    for s in (0, 31, 63):
        Ls = osh.haar_shift(L, H, W, osh.ROTATE_EULER, sc["params"][s:s + 1])
        ref = osd.radiance(Ls, Tf, H, W)[:, 0]
        err = rel_l2(got[pick, s], ref)
        assert err <= 2e-3, err
        # hi + lo keeps the lighting to ~2^-17; the rotation's FP32 coordinates and
        # the accumulator truncation add ~3e-5 and ~6e-5
        assert err <= 2e-4, err
