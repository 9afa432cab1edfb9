"""GPU parity of the paper's shading loop through the C ABI:
- the rotation input pass (haar_normal_rotations);
- the triple integral pass (haar_triple_product, by the Tripling Coefficient
  Theorem);
- the whole loop: normals -> haar_shift -> triple product.
Each is checked against the FP64 oracle (oracle.triple)."""
import numpy as np
import pytest

import synth
from oracle import haar as oh, triple as otr
from tests.helpers import f32

pytestmark = pytest.mark.gpu


def _positive_coeffs(rng, rows, H, W):
    # non-negative maps (lighting, BRDF and visibility are): no cancellation,
    # so a relative bound applies to every vertex
    return f32(oh.forward(rng.lognormal(0.0, 1.0, (rows, H, W))))


def test_normal_rotations_match_the_oracle(hs):
    import torch
    rng = np.random.default_rng(1)
    n = rng.standard_normal((257, 3))
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    n[0] = [0.0, 1.0, 0.0]
    n[1] = [0.0, -1.0, 0.0]
    n[2] = [1.0, 0.0, 0.0]
    n = f32(n)
    got = hs.haar_normal_rotations(torch.tensor(n, dtype=torch.float32, device="cuda")).cpu().numpy()
    for v in range(len(n)):
        nv = n[v] / np.linalg.norm(n[v])
        assert np.allclose(got[v].reshape(3, 3), otr.normal_rotation(nv), atol=1e-12), v


@pytest.mark.parametrize("H,W,C,V", [(2, 4, 1, 3), (4, 4, 3, 5), (16, 32, 3, 37), (32, 64, 3, 64),
                                     (32, 64, 4, 9), (64, 128, 2, 11), (64, 64, 1, 7)])
def test_triple_product_matches_the_definition(hs, H, W, C, V):
    import torch
    rng = np.random.default_rng(H * 7 + C)
    N = H * W
    light = _positive_coeffs(rng, C, H, W)
    brdf = _positive_coeffs(rng, V, H, W)
    vis = _positive_coeffs(rng, V, H, W)
    # rows padded to a stride that is not N (a multiple of 4 floats)
    pad = 8
    bt = torch.zeros((V, N + pad), dtype=torch.float32, device="cuda")
    vt = torch.zeros((V, N + pad), dtype=torch.float32, device="cuda")
    bt[:, :N] = torch.tensor(brdf, dtype=torch.float32)
    vt[:, :N] = torch.tensor(vis, dtype=torch.float32)
    got = hs.haar_triple_product(H, W, torch.tensor(light, dtype=torch.float32, device="cuda"), bt, vt)
    ref = np.stack([otr.triple_product(light, brdf[v][None], vis[v][None], H, W) for v in range(V)])
    rel = np.abs(got.cpu().numpy() - ref) / np.abs(ref)
    # FP32 sums over N/3 squares of non-negative-dominated terms
    assert rel.max() <= 1e-5, rel.max()


def test_triple_product_signed_inputs(hs):
    # signed coefficients: bounded against the pixel sum of |A B C|
    import torch
    H, W, C, V = 32, 64, 3, 16
    rng = np.random.default_rng(3)
    light, brdf, vis = (f32(rng.standard_normal((r, H * W))) for r in (C, V, V))
    dev = dict(dtype=torch.float32, device="cuda")
    got = hs.haar_triple_product(H, W, torch.tensor(light, **dev), torch.tensor(brdf, **dev),
                                 torch.tensor(vis, **dev)).cpu().numpy()
    A, B, Cm = (oh.inverse(x, H, W) for x in (light, brdf, vis))
    for v in range(V):
        ref = (A * B[v] * Cm[v]).sum(axis=(-2, -1))
        scale = (np.abs(A) * np.abs(B[v]) * np.abs(Cm[v])).sum(axis=(-2, -1))
        assert (np.abs(got[v] - ref) / scale).max() <= 1e-5


def test_empty_vertex_set_is_a_no_op(hs):
    import torch
    out = torch.full((0, 3), 7.0, device="cuda")
    hs.haar_triple_product(16, 32, torch.ones((3, 512), device="cuda"), torch.zeros((0, 512), device="cuda"),
                           torch.zeros((0, 512), device="cuda"), out=out)
    assert out.numel() == 0


def test_work_status_is_clear(hs):
    import torch
    H, W = 16, 32
    work = torch.full((hs.haar_triple_work_floats(H, W, 3),), 3.0, device="cuda")
    hs.haar_triple_product(H, W, torch.ones((3, 512), device="cuda"), torch.ones((4, 512), device="cuda"),
                           torch.ones((4, 512), device="cuda"), work=work)
    torch.cuda.synchronize()
    assert int(work[:1].view(torch.int32).item()) == 0


@pytest.mark.parametrize("expo", [0.0, 32.0])
def test_shading_loop_matches_the_oracle(hs, expo):
    # normals -> rotation records -> BRDF rotation per vertex (haar_shift,
    # HAAR_SHIFT_ROTATE) -> triple product; against rotating and integrating
    # in FP64 on the CPU
    import torch
    H, W, V = 32, 64, 24
    sc = synth.scene(1, V=V, H=H, W=W)
    light = f32(oh.forward(sc["light"]))
    brdf = f32(oh.forward(synth.local_brdf_map(H, W, expo, 0.4)))
    w = synth.transport_weights(sc["pos"], sc["nrm"], sc["occ_c"], sc["occ_r"], H, W, cosine=False).numpy()
    vis = f32(oh.forward(w))
    nrm = torch.tensor(f32(sc["nrm"]), dtype=torch.float32, device="cuda")
    prm = hs.haar_normal_rotations(nrm)
    plan = hs.Plan(H, W, 1, kind=hs.HAAR_SHIFT_ROTATE, max_shifts=V)
    rot = hs.haar_shift(plan, torch.tensor(brdf[None], dtype=torch.float32, device="cuda"), prm)   # [V, 1, N]
    got = hs.haar_triple_product(H, W, torch.tensor(light, dtype=torch.float32, device="cuda"), rot[:, 0, :],
                                 torch.tensor(vis, dtype=torch.float32, device="cuda")).cpu().numpy()
    plan.close()
    ref = otr.shade_triple(light, brdf, f32(sc["nrm"]), vis, H, W)
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    # the FP32 bar of the rotation and of the triple product alike
    assert rel <= 1e-5, rel
    assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max() * 4


@pytest.mark.parametrize("H,W,C,expo", [(32, 64, 3, 0.0), (32, 64, 3, 32.0), (64, 128, 3, 8.0), (16, 16, 1, 0.0),
                                        (4, 8, 4, 0.0)])
def test_fused_shading_loop_matches_the_oracle(hs, H, W, C, expo):
    # haar_shade_triple (rotation pass + triple product in one kernel) against
    # the FP64 oracle, and against the unfused haar_shift + haar_triple_product
    import torch
    V = 21
    sc = synth.scene(1, V=V, H=H, W=W)
    light = f32(oh.forward(synth.lighting_pixels(np.random.default_rng(H + C), C, H, W)))
    brdf = f32(oh.forward(synth.local_brdf_map(H, W, expo, 0.4)))
    w = synth.transport_weights(sc["pos"], sc["nrm"], sc["occ_c"], sc["occ_r"], H, W, cosine=False).numpy()
    vis = f32(oh.forward(w))
    dev = dict(dtype=torch.float32, device="cuda")
    lt, bt = torch.tensor(light, **dev), torch.tensor(brdf, **dev)
    vt = torch.zeros((V, H * W + 4), **dev)
    vt[:, :H * W] = torch.tensor(vis, **dev)
    prm = hs.haar_normal_rotations(torch.tensor(f32(sc["nrm"]), **dev))
    got = hs.haar_shade_triple(H, W, lt, bt, prm, vt).cpu().numpy()
    ref = otr.shade_triple(light, brdf, f32(sc["nrm"]), vis, H, W)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-5
    plan = hs.Plan(H, W, 1, kind=hs.HAAR_SHIFT_ROTATE, max_shifts=V)
    rot = hs.haar_shift(plan, bt[None], prm)
    unfused = hs.haar_triple_product(H, W, lt, rot[:, 0, :], vt).cpu().numpy()
    plan.close()
    assert np.linalg.norm(got - unfused) / np.linalg.norm(unfused) <= 2e-6


def test_full_size_fused_loop_sampled(hs):
    # the bench's level-6 launch: 50 000 c1 torus vertices, RGB 64x128; the
    # oracle shades 12 sampled vertices one by one (their visibility rows come
    # from the oracle, the others' only give the launch its size)
    import torch
    H, W = 64, 128
    sc = synth.scene(1)
    V = sc["V"]
    dev = dict(dtype=torch.float32, device="cuda")
    light = f32(oh.forward(synth.lighting_pixels(np.random.default_rng(46), 3, H, W)))
    brdf = f32(oh.forward(synth.local_brdf_map(H, W)))
    vis = torch.empty((V, H * W), **dev)
    for v0 in range(0, V, 8192):
        v1 = min(V, v0 + 8192)
        w = synth.transport_weights(sc["pos"][v0:v1], sc["nrm"][v0:v1], sc["occ_c"], sc["occ_r"], H, W,
                                    device="cuda", dtype=torch.float32, chunk=4096, cosine=False).contiguous()
        vis[v0:v1] = hs.haar_forward(w)
    pick = np.sort(np.random.default_rng(5).choice(V, 12, replace=False))
    wp = synth.transport_weights(sc["pos"][pick], sc["nrm"][pick], sc["occ_c"], sc["occ_r"], H, W,
                                 cosine=False).numpy()
    vis_np = f32(oh.forward(wp))
    vis[torch.tensor(pick, device="cuda")] = torch.tensor(vis_np, **dev)
    prm = hs.haar_normal_rotations(torch.tensor(f32(sc["nrm"]), **dev))
    got = hs.haar_shade_triple(H, W, torch.tensor(light, **dev), torch.tensor(brdf, **dev), prm, vis).cpu().numpy()
    assert np.isfinite(got).all()
    ref = otr.shade_triple(light, brdf, f32(sc["nrm"])[pick], vis_np, H, W)
    assert np.linalg.norm(got[pick] - ref) / np.linalg.norm(ref) <= 1e-5
