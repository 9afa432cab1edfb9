"""GPU parity of the headless rasteriser and per-pixel shading through the
C ABI, against the oracle (oracle.raster): triangle ids bit-exact (both
sides take every coverage and depth decision in float32 with one operation
order), barycentrics and shaded pixels within float32 rounding."""
import numpy as np
import pytest

import synth
from oracle import raster as ora

pytestmark = pytest.mark.gpu


def _run(hs, pos, tris, M, W, H):
    import torch
    dev = "cuda"
    r = hs.Raster(W, H, len(pos))
    tid, bary = r.rasterize(torch.tensor(pos, dtype=torch.float32, device=dev),
                            torch.tensor(np.asarray(tris).reshape(-1, 3), dtype=torch.int32, device=dev),
                            torch.tensor(np.asarray(M, dtype=np.float32).reshape(-1), device=dev))
    return r, tid.cpu().numpy(), bary.cpu().numpy()


@pytest.mark.parametrize("W,H,nu,nv", [(96, 64, 24, 12), (160, 90, 64, 24), (33, 17, 12, 6)])
def test_torus_fragments_match_the_oracle(hs, W, H, nu, nv):
    pos, nrm, tris = synth.torus_mesh(nu, nv)
    M = synth.view_projection((0.4, 1.6, 2.6), (0.0, 0.0, 0.0), aspect=W / H)
    _, tid, bary = _run(hs, pos, tris, M, W, H)
    ref_tid, ref_bary, _ = ora.rasterize(pos, tris, M, W, H)
    assert (tid >= 0).sum() > 0.2 * W * H
    assert np.array_equal(tid, ref_tid)
    hit = tid >= 0
    assert np.abs(bary[hit] - ref_bary[hit]).max() <= 2e-5


def test_shaded_image_matches_the_oracle(hs):
    import torch
    W, H = 96, 64
    pos, nrm, tris = synth.torus_mesh(32, 16)
    M = synth.view_projection((0.0, 2.0, 2.2), (0.0, 0.0, 0.0), aspect=W / H)
    r, tid, bary = _run(hs, pos, tris, M, W, H)
    rad = np.random.default_rng(1).uniform(0.0, 2.0, (len(pos), 3)).astype(np.float32)
    bg = np.array([0.1, 0.2, 0.3], np.float32)
    img = r.shade(torch.tensor(tris, device="cuda"), torch.tensor(rad, device="cuda"),
                  torch.tensor(bg, device="cuda")).cpu().numpy()
    ref = ora.shade_pixels(tid, bary.astype(np.float64), tris, rad, bg)
    assert np.abs(img - ref).max() <= 1e-5 * np.abs(ref).max()
    assert np.allclose(img[tid < 0], bg)


def test_full_screen_quad_at_odd_sizes(hs):
    pos = np.array([[-1, -1, 0], [1, -1, 0], [1, 1, 0], [-1, 1, 0]], np.float32)
    tris = [[0, 1, 2], [0, 2, 3]]
    for W, H in ((1, 1), (7, 3), (129, 65)):
        _, tid, _ = _run(hs, pos, tris, np.eye(4), W, H)
        ref, _, _ = ora.rasterize(pos, tris, np.eye(4), W, H)
        assert (tid >= 0).all() and np.array_equal(tid, ref)


def test_dropped_triangles(hs):
    # an index out of range, a vertex behind the eye, a degenerate triangle,
    # and no triangles at all
    pos = np.array([[-0.5, -0.5, 0], [0.5, -0.5, 0], [0, 0.5, 0], [0, 0, 0]], np.float32)
    M = synth.view_projection((0, 0, 2), (0, 0, 0), aspect=1.0)
    _, tid, _ = _run(hs, pos, [[0, 1, 9], [0, 1, 1]], M, 16, 16)
    assert (tid == -1).all()
    behind = np.array([[-0.5, -0.5, 0], [0.5, -0.5, 0], [0, 0.5, 3.0]], np.float32)
    _, tid, _ = _run(hs, behind, [[0, 1, 2]], M, 16, 16)
    assert (tid == -1).all()
    _, tid, _ = _run(hs, pos, np.zeros((0, 3), np.int32), M, 16, 16)
    assert (tid == -1).all()


def test_full_size_frame_matches_the_oracle(hs):
    # the bench's frame: the 50 176-vertex / 100 352-triangle torus at 1920x1080
    W, H = 1920, 1080
    pos, nrm, tris = synth.torus_mesh(256, 196)
    M = synth.view_projection((0.4, 1.6, 2.6), (0.0, 0.0, 0.0), aspect=W / H)
    _, tid, bary = _run(hs, pos, tris, M, W, H)
    ref_tid, ref_bary, _ = ora.rasterize(pos, tris, M, W, H)
    assert np.array_equal(tid, ref_tid)
    hit = tid >= 0
    assert hit.sum() > 500_000
    assert np.abs(bary[hit] - ref_bary[hit]).max() <= 1e-4
