"""Pins of the oracle's view-bin choice (which of a vertex's 16 stored
view-dependent transports a camera uses, in the glossy workload): the Duff
et al. (2017) tangent frame at hand-derived cases, its orthonormality and
handedness, and the bin choice against closed forms that do not go through
the oracle's frame."""
import numpy as np

import synth
from oracle import transport as otr


def _unit(v):
    v = np.asarray(v, dtype=np.float64)
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def test_frame_at_the_axes():
    # the construction's values at the coordinate axes, worked out by hand from
    # its definition (n = +z gives the identity basis)
    n = np.array([[0, 0, 1], [0, 0, -1], [1, 0, 0], [0, 1, 0]], dtype=np.float64)
    b1, b2 = otr.frame(n)
    want_b1 = np.array([[1, 0, 0], [1, 0, 0], [0, 0, -1], [1, 0, 0]], dtype=np.float64)
    want_b2 = np.array([[0, 1, 0], [0, -1, 0], [0, 1, 0], [0, 0, -1]], dtype=np.float64)
    assert np.array_equal(b1, want_b1) and np.array_equal(b2, want_b2)
    # the scene generator's own copy of the construction agrees
    s1, s2 = synth.onb(n)
    assert np.array_equal(s1, want_b1) and np.array_equal(s2, want_b2)


def test_frame_orthonormal_and_right_handed():
    rng = np.random.default_rng(0)
    n = _unit(rng.standard_normal((2000, 3)))
    # the region where earlier constructions break down: n_z -> -1
    n[:4] = _unit(np.array([[1e-4, 0, -1], [0, 1e-7, -1], [-1e-8, 1e-8, -1], [0.3, -0.2, -0.9]]))
    b1, b2 = otr.frame(n)
    for x, y in ((b1, b1), (b2, b2), (n, n)):
        assert np.allclose((x * y).sum(1), 1.0, atol=1e-12)
    for x, y in ((b1, b2), (b1, n), (b2, n)):
        assert np.abs((x * y).sum(1)).max() < 1e-12
    assert np.allclose(np.cross(b1, b2), n, atol=1e-12)     # (b1, b2, n) right-handed


def _scene(V=400, P=6, seed=3):
    rng = np.random.default_rng(seed)
    pos, nrm = synth.torus_vertices(rng, V)
    cams = synth.cameras(rng, P)
    return pos, nrm, cams


def test_view_along_the_normal_picks_the_top_bin():
    # a camera straight above the vertex sees it along n: the local view is
    # (0, 0, 1) whatever the tangent frame, so the bin with the largest z wins
    pos, nrm, _ = _scene()
    dirs = synth.view_bin_dirs(16)
    top = int(np.argmax(dirs[:, 2]))
    for dist in (0.5, 3.0):
        cams = pos[:1] + dist * nrm[:1]
        b, _ = otr.view_bins(pos[:1], nrm[:1], cams, dirs)
        assert b[0, 0] == top


def test_view_along_each_bin_direction_picks_that_bin():
    # cameras placed along each bin's world direction (built by the scene
    # generator, which is what the stored transport was computed for)
    pos, nrm, _ = _scene(V=30)
    dirs = synth.view_bin_dirs(16)
    world = synth.bin_view_world(nrm, 16)                    # [V, bins, 3]
    for v in range(len(pos)):
        cams = pos[v][None, :] + 4.0 * world[v]
        b, _ = otr.view_bins(pos[v:v + 1], nrm[v:v + 1], cams, dirs)
        assert np.array_equal(b[:, 0], np.arange(16))


def test_bin_choice_equals_nearest_world_bin_direction():
    # argmax over local coordinates = argmax of the world view direction's dot
    # product with each bin's world direction (the frame is orthonormal)
    pos, nrm, cams = _scene()
    dirs = synth.view_bin_dirs(16)
    world = synth.bin_view_world(nrm, 16)
    b, margin = otr.view_bins(pos, nrm, cams, dirs)
    for s, cam in enumerate(cams):
        w = _unit(cam[None, :] - pos)
        d = np.einsum("vk,vbk->vb", w, world)
        want = np.argmax(d, axis=1)
        ok = margin[s] > 1e-9
        assert np.array_equal(b[s][ok], want[ok])
        assert ok.mean() > 0.99


def test_bin_choice_invariances():
    # moving vertex and camera together, or the camera along its ray from the
    # vertex, leaves the view direction and hence the bin unchanged; a half
    # turn of the camera about the normal maps the local view (x, y, z) to
    # (-x, -y, z), so bins turned the same way are chosen with the same index
    pos, nrm, cams = _scene(V=200, P=4, seed=9)
    dirs = synth.view_bin_dirs(16)
    b0, m0 = otr.view_bins(pos, nrm, cams, dirs)
    off = np.array([0.7, -1.3, 2.1])
    b1, _ = otr.view_bins(pos + off, nrm, cams + off, dirs)
    assert np.array_equal(b0, b1)
    far = [pos + 2.5 * (c[None, :] - pos) for c in cams]
    for s in range(len(cams)):
        b2, _ = otr.view_bins(pos, nrm, far[s], dirs)      # one camera per vertex, same rays
        ok = m0[s] > 1e-9
        assert np.array_equal(np.diag(b2)[ok], b0[s][ok])
    # half turn about the normal: local (x, y, z) -> (-x, -y, z); with bin
    # directions turned the same way the choice is the same bin index
    turned = dirs * np.array([-1.0, -1.0, 1.0])
    for s, cam in enumerate(cams):
        w = cam[None, :] - pos
        wn = (w * nrm).sum(1, keepdims=True) * nrm
        cam_t = pos + 2 * wn - w                                # w rotated by pi about n
        b3, _ = otr.view_bins(pos, nrm, cam_t, turned)
        ok = m0[s] > 1e-9
        assert np.array_equal(np.diag(b3)[ok], b0[s][ok])
