"""GPU parity of the phase shift (translation and rotation) against the FP64
oracle, through the C ABI."""
import math

import numpy as np
import pytest

import synth
from oracle import haar as oh
from oracle import resample as ors
from oracle import shift as osh
from oracle import transport as otr
from tests.helpers import f32, rel_l2

pytestmark = pytest.mark.gpu

SPH, TOR = 0, 1


def _lighting(C, H, W, seed):
    rng = np.random.default_rng(seed)
    return f32(oh.forward(synth.lighting_pixels(rng, C, H, W)))


def _run(hs, coeffs, H, W, kind, params, boundary=SPH, out_type=0, layout=0, K=0, start_level=0):
    import torch
    C = coeffs.shape[0]
    S = params.shape[0]
    plan = hs.Plan(H, W, C, kind=kind, boundary=boundary, max_shifts=S, out_coeffs=K,
                   out_type=out_type, out_layout=layout, start_level=start_level)
    cin = torch.tensor(coeffs, dtype=torch.float32, device="cuda")
    prm = torch.tensor(np.asarray(params, dtype=np.float64), device="cuda")
    out = hs.haar_shift(plan, cin, prm)
    torch.cuda.synchronize()
    o = out.float().cpu().numpy().astype(np.float64)
    if out_type == hs.HAAR_OUT_BF16_HILO:
        raw = out.cpu()
        o = o[0] + o[1]
    else:
        raw = out.cpu()
    if layout == hs.HAAR_LAYOUT_SKC4:
        o = o[..., :C].transpose(0, 2, 1)
    elif layout == hs.HAAR_LAYOUT_SKC:
        o = o.transpose(0, 2, 1)
    elif layout == hs.HAAR_LAYOUT_KSC:
        o = o.transpose(1, 2, 0)
    plan.close()
    return np.ascontiguousarray(o), raw


@pytest.mark.parametrize("H,W", [(8, 16), (32, 32), (64, 128), (128, 256)])
@pytest.mark.parametrize("boundary", [SPH, TOR])
def test_translation_matches_oracle(hs, H, W, boundary):
    c = _lighting(3, H, W, H + W + boundary)
    rng = np.random.default_rng(7)
    prm = np.stack([rng.uniform(-3 * W, 3 * W, 6), rng.uniform(-3 * H, 3 * H, 6)], axis=1)
    prm[0] = [0.25, 0.5]
    got, _ = _run(hs, c, H, W, 0, prm, boundary)
    ref = osh.haar_shift(c, H, W, osh.TRANSLATE, prm, boundary)
    for s in range(len(prm)):
        assert rel_l2(got[s], ref[s]) <= 1e-5, (s, rel_l2(got[s], ref[s]))


@pytest.mark.parametrize("C,S", [(3, 3), (3, 17), (4, 13), (1, 50)])
def test_layouts_and_truncation_agree(hs, C, S):
    # every layout (and the coefficient-major kernel, with full and partial
    # plane groups) gives the same bits as the shift-major one
    H, W = 64, 128
    c = _lighting(C, H, W, 11)
    rng = np.random.default_rng(S)
    prm = np.stack([rng.uniform(-W, W, S), rng.uniform(-H, H, S)], axis=1)
    prm[:3] = [[3.3, 1.7], [100.25, 40.5], [7.0, 0.0]][:S]
    base, _ = _run(hs, c, H, W, 0, prm, SPH, 0, hs.HAAR_LAYOUT_SCK)
    for lay in (hs.HAAR_LAYOUT_SKC, hs.HAAR_LAYOUT_KSC, hs.HAAR_LAYOUT_SKC4):
        o, _ = _run(hs, c, H, W, 0, prm, SPH, 0, lay)
        assert np.array_equal(o, base)
    for K in (1000, 7):
        o, _ = _run(hs, c, H, W, 0, prm, SPH, 0, hs.HAAR_LAYOUT_SCK, K=K)
        assert np.array_equal(o, base[..., :K])
        o, _ = _run(hs, c, H, W, 0, prm, SPH, 0, hs.HAAR_LAYOUT_KSC, K=K)
        assert np.array_equal(o, base[..., :K])


def test_bf16_hilo_and_f16_outputs(hs):
    H, W = 64, 128
    c = _lighting(3, H, W, 12)
    prm = np.array([[3.3, 1.7], [50.6, 90.1]])
    base, _ = _run(hs, c, H, W, 0, prm)
    hilo, raw = _run(hs, c, H, W, 0, prm, out_type=hs.HAAR_OUT_BF16_HILO)
    # hi / lo are the bfloat16 split of the float32 result, bit for bit
    hi_b, lo_b = otr.split_hilo(base.astype(np.float32))
    raw_bits = raw.view(__import__("torch").int16).numpy().astype(np.uint16)
    assert np.array_equal(raw_bits[0], hi_b)
    assert np.array_equal(raw_bits[1], lo_b)
    ref = osh.haar_shift(c, H, W, osh.TRANSLATE, prm)
    assert rel_l2(hilo, ref) <= 1e-5
    h16, _ = _run(hs, c, H, W, 0, prm, out_type=hs.HAAR_OUT_F16)
    assert np.array_equal(h16, otr.to_f16(base.astype(np.float32)))


@pytest.mark.parametrize("boundary", [SPH, TOR])
@pytest.mark.parametrize("H,W", [(16, 32), (32, 32), (128, 256)])
@pytest.mark.parametrize("layout", [0, 2])
def test_dyadic_shifts_bit_exact(hs, H, W, boundary, layout):
    # layout 2 (KSC) runs the coefficient-major kernel
    c = _lighting(2, H, W, 13)
    cases = np.array([[0, 0], [W, 0], [2, 0], [4, 4], [8, 2], [W // 2, H], [16, 2 * H - 16], [6, 10],
                      [64, 32], [-4, -8]], dtype=np.float64)
    got, _ = _run(hs, c, H, W, 0, cases, boundary, 0, layout)
    for s, (kx, ky) in enumerate(cases.astype(int)):
        per = 2 * H if boundary == SPH else H
        res = osh.dyadic_permutation(c, H, W, int(kx) % W, int(ky) % per, boundary)
        idx = np.array(sorted(res))
        want = np.stack([res[k] for k in idx], axis=-1)
        assert np.array_equal(got[s][:, idx], want), (kx, ky)


@pytest.mark.parametrize("boundary", [SPH, TOR])
@pytest.mark.parametrize("H,W", [(64, 128), (128, 256), (256, 512)])
def test_dyadic_shifts_bit_exact_batch(hs, H, W, boundary):
    # enough shifts for the 8 x 8-block batch kernel (>= 2432 tile-shifts):
    # integer shifts that are multiples of 2^l give signed permutations of
    # levels <= l, bit-exact, and the other coefficients stay within FP32
    # rounding of the oracle
    c = _lighting(2, H, W, 17)
    base = np.array([[0, 0], [W, 0], [2, 0], [4, 4], [8, 2], [W // 2, H], [16, 2 * H - 16], [6, 10],
                     [64, 32], [-4, -8], [W - 8, 3 * H // 2 + 8], [32, -64]], dtype=np.float64)
    S = -(-2432 // ((H // 64) * (W // 64)))
    cases = np.concatenate([base, np.tile(base, (S // len(base) + 1, 1))])[:max(S, len(base))]
    got, _ = _run(hs, c, H, W, 0, cases, boundary, 0, 0)
    per = 2 * H if boundary == SPH else H
    for s in range(len(base)):
        kx, ky = cases[s].astype(int)
        res = osh.dyadic_permutation(c, H, W, int(kx) % W, int(ky) % per, boundary)
        idx = np.array(sorted(res))
        want = np.stack([res[k] for k in idx], axis=-1)
        assert np.array_equal(got[s][:, idx], want), (kx, ky)
    # repeated shifts give the same bits wherever they sit in the batch
    for s in range(len(base), len(cases), 37):
        assert np.array_equal(got[s], got[s % len(base)])
    ref = osh.haar_shift(c, H, W, osh.TRANSLATE, cases[:len(base)], boundary)
    assert rel_l2(got[:len(base)], ref, axis=(1, 2)).max() <= 1e-5


@pytest.mark.parametrize("H,W", [(2, 2), (2, 4), (4, 4), (4, 8), (8, 16)])
def test_exhaustive_operator_matrices(hs, H, W):
    # P13: M = Haar . S . Haar^-1 for all integer shifts and a 1/8 grid
    N = H * W
    rng = np.random.default_rng(N)
    per = 2 * H
    ints = np.array([[x, y] for x in range(W) for y in range(per)], dtype=np.float64)
    grid = np.array([[x / 8, y / 8] for x in range(8 * W) for y in range(8 * per)], dtype=np.float64)
    if len(grid) > 512:
        grid = grid[rng.choice(len(grid), 512, replace=False)]
    prm = np.concatenate([ints, grid])
    eye = np.eye(N)
    for boundary in (SPH, TOR):
        for c0 in range(0, N, 64):
            basis = eye[c0:c0 + 64]
            got, _ = _run(hs, basis, H, W, 0, prm, boundary)
            ref = osh.haar_shift(basis, H, W, osh.TRANSLATE, prm, boundary)
            assert np.abs(got - ref).max() < 2e-6


@pytest.mark.parametrize("H,W", [(4, 8), (32, 32), (64, 128), (256, 512)])
def test_forward_inverse(hs, H, W):
    import torch
    rng = np.random.default_rng(H)
    P = f32(synth.lighting_pixels(rng, 5, H, W))
    t = torch.tensor(P, dtype=torch.float32, device="cuda")
    c = hs.haar_forward(t).cpu().numpy()
    ref = oh.forward(P)
    assert rel_l2(c, ref) <= 1e-6
    c2 = hs.haar_forward(t, scale=0.25).cpu().numpy()
    assert np.allclose(c2, 0.25 * c, rtol=1e-6, atol=0)
    back = hs.haar_inverse(torch.tensor(f32(ref), dtype=torch.float32, device="cuda"), H, W).cpu().numpy()
    assert rel_l2(back, P) <= 1e-6


# Rotations are held to the FP32 bar.  Plain FP32 source coordinates (up to
# 512 px, ~2^-24 * 512 = 3e-5 px of rounding) would give ~3e-5 relative error
# on the i.i.d. lognormal maps (pixel-to-pixel contrast ~1.3x their RMS); the
# kernels take each coordinate as an integer anchor plus a float-pair offset
# (~1e-9 rad), which leaves the error at ~1e-7.
ROT_TOL = 1e-5


@pytest.mark.parametrize("H,W", [(16, 32), (64, 128), (256, 512)])
def test_rotation_matches_oracle(hs, H, W):
    c = _lighting(3, H, W, 21 + H)
    eul = synth.euler_angles(np.random.default_rng(H), 4)
    got, _ = _run(hs, c, H, W, hs.HAAR_SHIFT_ROTATE_EULER, eul)
    ref = osh.haar_shift(c, H, W, osh.ROTATE_EULER, eul)
    for s in range(4):
        assert rel_l2(got[s], ref[s]) <= ROT_TOL, (s, rel_l2(got[s], ref[s]))
    # same rotations given as matrices
    mats = np.stack([ors.euler_matrix(*e).ravel() for e in eul])
    got2, _ = _run(hs, c, H, W, hs.HAAR_SHIFT_ROTATE, mats)
    assert rel_l2(got2, got) <= 1e-5


def test_rotation_smooth_map_fp32_tolerance(hs):
    # a map of hot spots only (no per-pixel noise)
    H, W = 128, 256
    rng = np.random.default_rng(5)
    P = synth.lighting_pixels(rng, 1, H, W, sigma=0.0) - 1.0    # hot spots only
    c = f32(oh.forward(P))
    eul = synth.euler_angles(rng, 3)
    got, _ = _run(hs, c, H, W, hs.HAAR_SHIFT_ROTATE_EULER, eul)
    ref = osh.haar_shift(c, H, W, osh.ROTATE_EULER, eul)
    assert rel_l2(got, ref) <= 1e-5


@pytest.mark.parametrize("boundary", [SPH, TOR])
def test_rotation_near_source_poles(hs, boundary):
    # rotations that send output pixel centres onto or next to the source
    # poles (the azimuth there is decided by float-pair products near zero):
    # quarter and half turns about x and z, and tiny tilts
    H, W = 64, 128
    c = _lighting(3, H, W, 41)
    mats = [ors.rot_x(math.pi / 2), ors.rot_z(math.pi / 2), ors.rot_x(math.pi), ors.rot_x(1e-7),
            ors.rot_z(-1e-9) @ ors.rot_x(math.pi / 2), ors.rot_x(0.5 * math.pi / H)]
    prm = np.stack([m.ravel() for m in mats])
    got, _ = _run(hs, c, H, W, hs.HAAR_SHIFT_ROTATE, prm, boundary)
    ref = osh.haar_shift(c, H, W, osh.ROTATE, prm, boundary)
    for s in range(len(mats)):
        assert rel_l2(got[s], ref[s]) <= ROT_TOL, (s, rel_l2(got[s], ref[s]))


def test_rotation_about_y_equals_translation(hs):
    # P9: R_y(-dx dphi) is the azimuth translation by dx
    H, W = 64, 128
    c = _lighting(3, H, W, 31)
    dxs = np.array([5.0, 17.37, 100.5])
    mats = np.stack([ors.rot_y(-dx * 2 * math.pi / W).ravel() for dx in dxs])
    rot, _ = _run(hs, c, H, W, hs.HAAR_SHIFT_ROTATE, mats)
    tr, _ = _run(hs, c, H, W, 0, np.stack([dxs, np.zeros(3)], axis=1))
    assert rel_l2(rot, tr) <= ROT_TOL


def test_rotation_constant_and_identity(hs):
    H, W = 32, 64
    const = f32(oh.forward(np.full((1, H, W), 3.0)))
    eul = synth.euler_angles(np.random.default_rng(3), 5)
    got, _ = _run(hs, const, H, W, hs.HAAR_SHIFT_ROTATE_EULER, eul)
    assert np.abs(got - const[None]).max() <= 1e-5 * np.abs(const).max()
    c = _lighting(1, H, W, 4)
    ident, _ = _run(hs, c, H, W, hs.HAAR_SHIFT_ROTATE_EULER, np.zeros((1, 3)))
    assert rel_l2(ident[0], c) <= ROT_TOL


def test_full_size_translation_c1(hs):
    # the 16-shift RGB 128x256 frame in the coefficient-major layout shading uses
    sc = synth.scene(1, V=1)
    H, W = sc["H"], sc["W"]
    c = f32(oh.forward(sc["light"]))
    got, _ = _run(hs, c, H, W, 0, sc["params"], SPH, 0, hs.HAAR_LAYOUT_KSC)
    ref = osh.haar_shift(c, H, W, osh.TRANSLATE, sc["params"])
    assert rel_l2(got, ref, axis=(1, 2)).max() <= 1e-5


def test_full_size_rotation_c2_hilo(hs):
    # 64 rotations of the RGB 256x512 map, lowest 4096 as bf16 hi + lo; the oracle
    # checks a sample of the rotations one by one
    sc = synth.scene(2, V=1)
    H, W = sc["H"], sc["W"]
    c = f32(oh.forward(sc["light"]))
    got, _ = _run(hs, c, H, W, hs.HAAR_SHIFT_ROTATE_EULER, sc["params"], SPH, hs.HAAR_OUT_BF16_HILO,
                  hs.HAAR_LAYOUT_SCK, K=4096)
    for s in (0, 17, 63):
        ref = osh.haar_shift(c, H, W, osh.ROTATE_EULER, sc["params"][s:s + 1], out_coeffs=4096)[0]
        assert rel_l2(got[s], ref) <= ROT_TOL


def _run_sampled(hs, coeffs, H, W, kind, params, sample, boundary=SPH):
    """Full launch of len(params) shifts (FP32, SCK); only the sampled shifts
    come back to the host."""
    import torch
    C = coeffs.shape[0]
    S = params.shape[0]
    plan = hs.Plan(H, W, C, kind=kind, boundary=boundary, max_shifts=S)
    cin = torch.tensor(coeffs, dtype=torch.float32, device="cuda")
    prm = torch.tensor(np.asarray(params, dtype=np.float64), device="cuda")
    out = hs.haar_shift(plan, cin, prm)
    got = out[torch.tensor(sample, device="cuda")].double().cpu().numpy()
    plan.close()
    del out
    return got


def test_full_size_translation_batch(hs):
    # the bench's translation row: 4096 fractional shifts of the RGB 128x256 map in
    # one launch (three channels per thread); sampled shifts against the oracle
    sc = synth.scene(1, V=1)
    H, W = sc["H"], sc["W"]
    c = f32(oh.forward(sc["light"]))
    prm = synth.translations(synth.rng_for(1, 7), 4096, 256.0, 256.0)
    sample = [0, 1, 777, 2048, 4095]
    got = _run_sampled(hs, c, H, W, 0, prm, sample)
    ref = osh.haar_shift(c, H, W, osh.TRANSLATE, prm[sample])
    assert rel_l2(got, ref, axis=(1, 2)).max() <= 1e-5


@pytest.mark.parametrize("C,boundary", [(4, SPH), (1, TOR), (24, SPH)])
def test_translation_many_shifts_channel_groups(hs, C, boundary):
    # enough shifts for the batch kernel, with a partial channel group (C =
    # 4), a single channel, and 24 channels (the batch kernel's per-channel
    # level means then no longer fit the slack of a fixed shared-memory tail)
    H, W = 128, 256
    c = _lighting(C, H, W, 31 + C)
    rng = np.random.default_rng(C)
    prm = np.stack([rng.uniform(-2 * W, 2 * W, 320), rng.uniform(-2 * H, 2 * H, 320)], axis=1)
    prm[5] = [64.0, 32.0]                                     # dyadic: permuted levels
    sample = [0, 5, 161, 319]
    got = _run_sampled(hs, c, H, W, 0, prm, sample, boundary)
    ref = osh.haar_shift(c, H, W, osh.TRANSLATE, prm[sample], boundary)
    assert rel_l2(got, ref, axis=(1, 2)).max() <= 1e-5


def test_maximum_map_size_translation(hs):
    # the largest map a plan accepts: 4096 x 8192 (12 levels, 8192 tiles of
    # 64 x 64), one channel, every coefficient of two fractional shifts against
    # the oracle.  Two shifts already take the TMA-fed batch kernel, whose
    # level means and coarse images (8192 tile means) then sit after the
    # window in shared memory, not in it.
    H, W = 4096, 8192
    c = _lighting(1, H, W, 4096)
    prm = np.array([[1234.37, -517.81], [-3000.5, 2222.25]])
    got, _ = _run(hs, c, H, W, 0, prm)
    ref = osh.haar_shift(c, H, W, osh.TRANSLATE, prm)
    assert rel_l2(got, ref, axis=(1, 2)).max() <= 1e-5


def test_full_size_rotation_batch(hs):
    # the bench's rotation row: 512 rotations of the RGB 256x512 map in one launch
    sc = synth.scene(2, V=1)
    H, W = sc["H"], sc["W"]
    c = f32(oh.forward(sc["light"]))
    eul = synth.euler_angles(synth.rng_for(2, 7), 512)
    sample = [0, 300, 511]
    got = _run_sampled(hs, c, H, W, hs.HAAR_SHIFT_ROTATE_EULER, eul, sample)
    ref = osh.haar_shift(c, H, W, osh.ROTATE_EULER, eul[sample])
    assert rel_l2(got, ref, axis=(1, 2)).max() <= ROT_TOL


@pytest.mark.parametrize("k,layout", [(1, 0), (2, 0), (1, 2), (3, 2)])
def test_start_level_translation_matches_oracle(hs, k, layout):
    # the shift of the level-k scaling image of the RGB 128x256 map (Sec.
    # "Algorithmic optimization"); layout 2 (KSC) runs the coefficient-major kernel
    sc = synth.scene(1, V=1)
    H, W = sc["H"], sc["W"]
    c = f32(oh.forward(sc["light"]))
    prm = np.asarray(sc["params"], dtype=np.float64)
    prm[1] = [64.0, 32.0]                                     # block-aligned at every k used here
    import torch
    plan = hs.Plan(H, W, 3, max_shifts=len(prm), out_layout=layout, start_level=k)
    out = hs.haar_shift(plan, torch.tensor(c, dtype=torch.float32, device="cuda"),
                        torch.tensor(prm, dtype=torch.float64, device="cuda"))
    got = out.double().cpu().numpy()
    if layout == hs.HAAR_LAYOUT_KSC:
        got = got.transpose(1, 2, 0)
    plan.close()
    n = (H * W) >> (2 * k)
    assert got.shape == (len(prm), 3, n)
    ref = osh.haar_shift(c, H, W, osh.TRANSLATE, prm, start_level=k)
    assert rel_l2(got, ref, axis=(1, 2)).max() <= 1e-5
    # block-aligned shifts: the start level is exact, against the full-map shift
    full = osh.haar_shift(c, H, W, osh.TRANSLATE, prm[1:2])[0, :, :n]
    assert rel_l2(got[1], full) <= 1e-5


def test_start_level_rotation_matches_oracle(hs):
    sc = synth.scene(2, V=1)
    H, W = sc["H"], sc["W"]
    c = f32(oh.forward(sc["light"]))
    eul = np.asarray(sc["params"][:8], dtype=np.float64)
    got, _ = _run(hs, c, H, W, hs.HAAR_SHIFT_ROTATE_EULER, eul, SPH, 0, 0, K=0, start_level=1)
    ref = osh.haar_shift(c, H, W, osh.ROTATE_EULER, eul, start_level=1)
    assert got.shape == ref.shape == (8, 3, (H * W) >> 2)
    assert rel_l2(got, ref, axis=(1, 2)).max() <= ROT_TOL


def test_whole_map_kernel_layouts_and_truncation(hs):
    # enough (channel, shift) items for the whole-map kernel (map held in shared
    # memory): every layout and a truncated K give the bits of the full SCK result
    H, W = 128, 256
    c = _lighting(3, H, W, 77)
    rng = np.random.default_rng(77)
    prm = np.stack([rng.uniform(-W, W, 110), rng.uniform(-2 * H, 2 * H, 110)], axis=1)
    prm[3] = [128.0, 64.0]                                    # dyadic: permuted levels
    base, _ = _run(hs, c, H, W, 0, prm, SPH, 0, hs.HAAR_LAYOUT_SCK)
    sample = [0, 3, 57, 109]
    ref = osh.haar_shift(c, H, W, osh.TRANSLATE, prm[sample])
    assert rel_l2(base[sample], ref, axis=(1, 2)).max() <= 1e-5
    for lay in (hs.HAAR_LAYOUT_SKC, hs.HAAR_LAYOUT_KSC):
        o, _ = _run(hs, c, H, W, 0, prm, SPH, 0, lay)
        assert np.array_equal(o, base)
    o, _ = _run(hs, c, H, W, 0, prm, SPH, 0, hs.HAAR_LAYOUT_SKC, K=1000)
    assert np.array_equal(o, base[..., :1000])


def test_output_not_16_byte_aligned(hs):
    # an output one float past a 16-byte boundary takes the scalar store path:
    # the same values as an aligned output
    import torch
    H, W = 64, 128
    c = _lighting(3, H, W, 5)
    prm = np.asarray(synth.translations(np.random.default_rng(5), 6, 128.0, 64.0), dtype=np.float64)
    plan = hs.Plan(H, W, 3, max_shifts=6)
    cin = torch.tensor(c, dtype=torch.float32, device="cuda")
    pt = torch.tensor(prm, device="cuda")
    ref = hs.haar_shift(plan, cin, pt)
    buf = torch.zeros(ref.numel() + 1, dtype=torch.float32, device="cuda")
    out = buf[1:].view(ref.shape)
    hs.haar_shift(plan, cin, pt, out)
    assert torch.equal(out, ref)
    plan.close()
