"""haar_shift_noalloc: the phase shift for callers that cannot allocate
device memory (its scratch is a fixed array inside the library), checked
through the C ABI against haar_shift, which runs on a plan's allocated
workspace.  Collected last on purpose."""
import ctypes

import numpy as np
import pytest

import synth
from oracle import haar as oh
from tests.helpers import f32, rel_l2

pytestmark = pytest.mark.gpu


def _noalloc(hs, desc, cin, params, out):
    import torch
    st = hs.lib().haar_shift_noalloc(ctypes.byref(desc), cin.data_ptr(), params.data_ptr(), params.shape[0],
                                     out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    return st


def test_noalloc_matches_plan_shift_twice(hs):
    import torch
    # two different calls in a row (each must start from cleared counters and
    # overwrite what the previous call left in the shared scratch)
    cases = [
        (64, 128, 3, hs.HAAR_SHIFT_TRANSLATE, hs.HAAR_LAYOUT_KSC, np.array([[3.3, 1.7], [100.25, 40.5], [8.0, 4.0]])),
        (32, 64, 3, hs.HAAR_SHIFT_ROTATE_EULER, hs.HAAR_LAYOUT_SCK, synth.euler_angles(np.random.default_rng(1), 4)),
    ]
    cases.append((128, 256, 3, hs.HAAR_SHIFT_TRANSLATE, hs.HAAR_LAYOUT_KSC, np.array([[5.5, 2.25], [40.0, 16.0]]), 2))
    for case in cases:
        H, W, C, kind, layout, prm = case[:6]
        k = case[6] if len(case) > 6 else 0
        rng = np.random.default_rng(H)
        c = f32(oh.forward(synth.lighting_pixels(rng, C, H, W)))
        cin = torch.tensor(c, dtype=torch.float32, device="cuda")
        params = torch.tensor(prm, dtype=torch.float64, device="cuda")
        plan = hs.Plan(H, W, C, kind=kind, max_shifts=len(prm), out_layout=layout, start_level=k)
        ref = hs.haar_shift(plan, cin, params)
        desc = hs.HaarShiftDesc(H, W, C, kind, 0, len(prm), 0, 0, layout, k)
        for _ in range(2):
            out = torch.full_like(ref, float("nan"))
            assert _noalloc(hs, desc, cin, params, out) == hs.HAAR_OK, hs.lib().haar_last_error()
            torch.cuda.synchronize()
            assert torch.isfinite(out).all()
            assert rel_l2(out.cpu().numpy(), ref.cpu().numpy()) <= 1e-6
        plan.close()


def test_noalloc_rejects_oversized_calls(hs):
    import torch
    desc = hs.HaarShiftDesc(1024, 2048, 3, hs.HAAR_SHIFT_TRANSLATE, 0, 1, 0, 0, 0)
    cin = torch.zeros(3 * 1024 * 2048, dtype=torch.float32, device="cuda")
    params = torch.zeros((1, 2), dtype=torch.float64, device="cuda")
    out = torch.zeros(16, dtype=torch.float32, device="cuda")
    assert _noalloc(hs, desc, cin, params, out) == hs.HAAR_ERR_INVALID_ARG
    assert b"maximum" in hs.lib().haar_last_error()
