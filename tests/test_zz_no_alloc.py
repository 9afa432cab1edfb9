"""haar_shift_noalloc: the phase shift for callers that cannot allocate
device memory (its scratch is a fixed array inside the library), checked
through the C ABI against haar_shift, which runs on a plan's allocated
workspace.  Collected last on purpose."""
import ctypes

import numpy as np
import pytest

import synth
from oracle import haar as oh
from tests.helpers import f32

pytestmark = pytest.mark.gpu


def _noalloc(hs, desc, cin, params, out):
    import torch
    st = hs.lib().haar_shift_noalloc(ctypes.byref(desc), cin.data_ptr(), params.data_ptr(), params.shape[0],
                                     out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    return st


def test_noalloc_matches_plan_shift_twice(hs):
    import torch
    # two calls in a row per case (each must start from cleared counters and
    # overwrite what the previous call left in the shared scratch); the cases
    # cover every output type and layout, the coefficient-major kernel, start
    # levels of a translation and a rotation, and the small-map kernel
    eul = synth.euler_angles(np.random.default_rng(1), 4)
    tr = np.array([[3.3, 1.7], [100.25, 40.5], [8.0, 4.0]])
    T, RE = hs.HAAR_SHIFT_TRANSLATE, hs.HAAR_SHIFT_ROTATE_EULER
    F32, HILO, F16 = hs.HAAR_OUT_F32, hs.HAAR_OUT_BF16_HILO, hs.HAAR_OUT_F16
    SCK, SKC, KSC, SKC4 = hs.HAAR_LAYOUT_SCK, hs.HAAR_LAYOUT_SKC, hs.HAAR_LAYOUT_KSC, hs.HAAR_LAYOUT_SKC4
    # (H, W, C, kind, out_type, layout, params, start_level, out_coeffs)
    cases = [
        (64, 128, 3, T, F32, KSC, tr, 0, 0),
        (32, 64, 3, RE, F32, SCK, eul, 0, 0),
        (128, 256, 3, T, F32, KSC, np.array([[5.5, 2.25], [40.0, 16.0]]), 2, 0),
        (64, 128, 3, RE, F32, SCK, eul, 1, 0),
        (64, 128, 3, T, F16, SKC, tr, 0, 0),
        (64, 128, 3, RE, HILO, SCK, eul, 0, 1000),
        (64, 128, 3, RE, F32, SKC4, eul, 0, 0),
        (64, 128, 2, RE, F16, SKC, eul, 0, 0),
        (16, 32, 1, RE, F32, SCK, eul, 0, 0),
    ]
    for H, W, C, kind, ot, layout, prm, k, K in cases:
        rng = np.random.default_rng(H + C)
        c = f32(oh.forward(synth.lighting_pixels(rng, C, H, W)))
        cin = torch.tensor(c, dtype=torch.float32, device="cuda")
        params = torch.tensor(prm, dtype=torch.float64, device="cuda")
        plan = hs.Plan(H, W, C, kind=kind, max_shifts=len(prm), out_coeffs=K, out_type=ot, out_layout=layout,
                       start_level=k)
        ref = hs.haar_shift(plan, cin, params)
        desc = hs.HaarShiftDesc(H, W, C, kind, 0, len(prm), K, ot, layout, k)
        for _ in range(2):
            out = torch.full_like(ref, float("nan"))
            assert _noalloc(hs, desc, cin, params, out) == hs.HAAR_OK, hs.lib().haar_last_error()
            assert hs.lib().haar_last_error() == b""
            torch.cuda.synchronize()
            if layout == SKC4:                         # the pad lane is not written
                assert torch.equal(out[..., :C], ref[..., :C])
            else:
                assert torch.equal(out, ref), (H, W, C, kind, ot, layout, k)
        plan.close()


def test_noalloc_rejects_oversized_calls(hs):
    import torch
    desc = hs.HaarShiftDesc(1024, 2048, 3, hs.HAAR_SHIFT_TRANSLATE, 0, 1, 0, 0, 0)
    cin = torch.zeros(3 * 1024 * 2048, dtype=torch.float32, device="cuda")
    params = torch.zeros((1, 2), dtype=torch.float64, device="cuda")
    out = torch.zeros(16, dtype=torch.float32, device="cuda")
    assert _noalloc(hs, desc, cin, params, out) == hs.HAAR_ERR_INVALID_ARG
    assert b"maximum" in hs.lib().haar_last_error()
    # a start level past the plan path's limit is rejected the same way
    bad = hs.HaarShiftDesc(64, 128, 3, hs.HAAR_SHIFT_TRANSLATE, 0, 1, 0, 0, 0, 13)
    assert _noalloc(hs, bad, cin, params, out) == hs.HAAR_ERR_INVALID_ARG
    # 167 rotations of RGB 256x512 no longer fit (166 do)
    big = hs.HaarShiftDesc(256, 512, 3, hs.HAAR_SHIFT_ROTATE_EULER, 0, 167, 0, 0, 0, 0)
    eul = torch.zeros((167, 3), dtype=torch.float64, device="cuda")
    assert _noalloc(hs, big, cin, eul, out) == hs.HAAR_ERR_INVALID_ARG
