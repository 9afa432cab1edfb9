"""Pins of the rasterisation oracle (the fragment-buffer pass of Sec.
"Experimental results", restated without a graphics API): exact single
coverage of shared edges, closed-form coverage areas, depth order,
perspective-correct interpolation against ray casting, near-plane drops."""
import math

import numpy as np

from oracle import raster

I4 = np.eye(4)


def _perspective(fov_y, aspect, near, far):
    f = 1.0 / math.tan(fov_y / 2)
    return np.array([[f / aspect, 0, 0, 0], [0, f, 0, 0],
                     [0, 0, (far + near) / (near - far), 2 * far * near / (near - far)], [0, 0, -1, 0]])


def _coverage(pos, tris, M, W, H):
    cnt = np.zeros((H, W), int)
    for t in tris:
        tid, _, _ = raster.rasterize(pos, [t], M, W, H)
        cnt += tid >= 0
    return cnt


def test_full_screen_quad_covers_every_pixel_once():
    pos = np.array([[-1, -1, 0], [1, -1, 0], [1, 1, 0], [-1, 1, 0]], float)
    tris = [[0, 1, 2], [0, 2, 3]]
    for W, H in ((16, 16), (37, 23)):
        assert (_coverage(pos, tris, I4, W, H) == 1).all()
        tid, _, _ = raster.rasterize(pos, tris, I4, W, H)
        assert (tid >= 0).all()


def test_fan_with_shared_edges_through_pixel_centres_covers_once():
    # a fan whose spokes run through pixel centres and along rows / columns /
    # diagonals: every covered pixel belongs to exactly one triangle
    W = H = 16
    c = np.array([0.0625, -0.0625, 0.0])             # a pixel centre in ndc
    ring = [(-0.75, -0.75), (0.0625, -0.75), (0.75, -0.75), (0.75, -0.0625), (0.75, 0.75),
            (0.0625, 0.75), (-0.75, 0.75), (-0.75, -0.0625)]
    pos = np.array([c] + [[x, y, 0.0] for x, y in ring])
    tris = [[0, 1 + k, 1 + (k + 1) % 8] for k in range(8)]
    cnt = _coverage(pos, tris, I4, W, H)
    assert cnt.max() == 1
    tid, _, _ = raster.rasterize(pos, tris, I4, W, H)
    assert ((tid >= 0) == (cnt == 1)).all()


def test_coverage_count_matches_area():
    rng = np.random.default_rng(1)
    W, H = 64, 48
    for _ in range(10):
        p = np.c_[rng.uniform(-0.9, 0.9, (3, 2)), np.zeros(3)]
        tid, _, _ = raster.rasterize(p, [[0, 1, 2]], I4, W, H)
        sx = (p[:, 0] + 1) / 2 * W
        sy = (1 - p[:, 1]) / 2 * H
        area = abs((sx[1] - sx[0]) * (sy[2] - sy[0]) - (sy[1] - sy[0]) * (sx[2] - sx[0])) / 2
        per = sum(math.hypot(sx[i] - sx[(i + 1) % 3], sy[i] - sy[(i + 1) % 3]) for i in range(3))
        assert abs((tid >= 0).sum() - area) <= per + 4


def test_nearer_triangle_wins_and_ties_keep_the_lower_id():
    W = H = 16
    far = [[-0.8, -0.8, 0.5], [0.8, -0.8, 0.5], [0.0, 0.8, 0.5]]
    near = [[-0.8, -0.8, -0.5], [0.8, -0.8, -0.5], [0.0, 0.8, -0.5]]
    for order, want in (((far, near), 1), ((near, far), 0)):
        pos = np.array(order[0] + order[1])
        tid, _, depth = raster.rasterize(pos, [[0, 1, 2], [3, 4, 5]], I4, W, H)
        hit = tid >= 0
        assert hit.any() and (tid[hit] == want).all()
        assert np.allclose(depth[hit], 0.25)
    pos = np.array(far + far)
    tid, _, _ = raster.rasterize(pos, [[3, 4, 5], [0, 1, 2]], I4, W, H)
    assert (tid[tid >= 0] == 0).all()


def test_perspective_correct_interpolation_matches_ray_casting():
    W, H = 40, 30
    M = _perspective(1.0, W / H, 0.1, 10.0)
    pos = np.array([[-1.0, -0.8, -2.0], [1.5, -0.5, -4.0], [0.2, 1.0, -3.0]])
    tid, bary, _ = raster.rasterize(pos, [[0, 1, 2]], M, W, H)
    f = 1.0 / math.tan(0.5)
    n = np.cross(pos[1] - pos[0], pos[2] - pos[0])
    checked = 0
    for py, px in zip(*np.nonzero(tid >= 0)):
        # the eye ray through the pixel centre, intersected with the plane
        ndx = (px + 0.5) / W * 2 - 1
        ndy = 1 - (py + 0.5) / H * 2
        d = np.array([ndx * (W / H) / f, ndy / f, -1.0])
        P = d * (n @ pos[0]) / (n @ d)
        b1, b2 = bary[py, px]
        Q = (1 - b1 - b2) * pos[0] + b1 * pos[1] + b2 * pos[2]
        assert np.allclose(Q, P, atol=1e-5)
        checked += 1
    assert checked > 50


def test_vertices_behind_the_eye_drop_the_triangle():
    M = _perspective(1.0, 1.0, 0.1, 10.0)
    pos = np.array([[-1.0, -1.0, -2.0], [1.0, -1.0, -2.0], [0.0, 1.0, 1.0]])
    tid, _, _ = raster.rasterize(pos, [[0, 1, 2]], M, 16, 16)
    assert (tid == raster.EMPTY).all()


def test_shade_pixels_interpolates_and_fills_the_background():
    pos = np.array([[-1, -1, 0], [1, -1, 0], [1, 1, 0], [-1, 1, 0]], float) * 0.5
    tris = [[0, 1, 2], [0, 2, 3]]
    tid, bary, _ = raster.rasterize(pos, tris, I4, 20, 20)
    rad = np.array([[1.0, 2.0], [1.0, 2.0], [1.0, 2.0], [1.0, 2.0]])
    img = raster.shade_pixels(tid, bary, tris, rad, [7.0, 8.0])
    assert np.allclose(img[tid >= 0], [1.0, 2.0])
    assert np.allclose(img[tid < 0], [7.0, 8.0])
    # a radiance linear in x is reproduced at pixel centres (orthographic)
    rad = np.c_[pos[:, 0], pos[:, 1]]
    img = raster.shade_pixels(tid, bary, tris, rad, [0.0, 0.0])
    for py, px in zip(*np.nonzero(tid >= 0)):
        assert np.allclose(img[py, px], [(px + 0.5) / 10 - 1, 1 - (py + 0.5) / 10], atol=1e-6)
