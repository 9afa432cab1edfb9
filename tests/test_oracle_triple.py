"""Pins of the triple-product oracle: the Tripling Coefficient Theorem
(Sec. "Related work", after Ng et al. 2004) against brute-force C_ijk, the
theorem's case sum against the pixel-space definition, closed forms, and the
normal rotation of Sec. "Algorithmic optimization"."""
import math

import numpy as np
import pytest

from oracle import haar, shift, triple
from oracle.resample import rot_x, rot_y


def _case(H, W, i, j, k):
    """The theorem's value for (i, j, k) in unit pixel measure, or 0."""
    n, q = haar.dims(H, W)
    di, dj, dk = (haar.decode(H, W, x) for x in (i, j, k))
    scal = [d[1] == -1 for d in (di, dj, dk)]
    if all(scal):                                            # (a) three scaling functions
        return 1.0 / H if i == j == k else 0.0
    trip = [(i, di), (j, dj), (k, dk)]
    wav = [t for t in trip if t[1][1] != -1]
    if len(wav) == 3 and len({(d[0], d[2], d[3]) for _, d in wav}) == 1 \
            and len({d[1] for _, d in wav}) == 3:            # (b) one square, three types
        return 1.0 / (1 << di[0])
    for x, y, z in ((0, 1, 2), (0, 2, 1), (1, 2, 0)):        # (c) a repeated wavelet
        (ix, dx), (iy, dy), (iz, dz) = trip[x], trip[y], trip[z]
        if ix == iy and dx[1] != -1 and ix != iz:
            lvl, _, r, cidx = dx
            if dz[1] == -1:                                  # third: a scaling block
                inside = (cidx << lvl) // H == dz[3]
                return 1.0 / H if inside else 0.0
            l3, b3, r3, c3 = dz
            if l3 <= lvl or (r >> (l3 - lvl)) != r3 or (cidx >> (l3 - lvl)) != c3:
                return 0.0
            # quadrant of the coarser square that holds the finer one
            sub = 1 << (l3 - lvl - 1)
            top, left = (r // sub) % 2 == 0, (cidx // sub) % 2 == 0
            sign = {0: (-1 if left else 1), 1: (-1 if top else 1),
                    2: (1 if top == left else -1)}[b3]
            return sign / (1 << l3)
    return 0.0


@pytest.mark.parametrize("H,W", [(2, 4), (4, 4), (4, 8)])
def test_tripling_coefficients_follow_the_theorem(H, W):
    C = triple.tripling_coefficients(H, W)
    N = H * W
    for i in range(N):
        for j in range(N):
            for k in range(N):
                assert abs(C[i, j, k] - _case(H, W, i, j, k)) < 1e-12, (i, j, k, C[i, j, k])


def test_tripling_coefficients_are_mostly_zero():
    # the theorem's point: the nonzero count grows like N log N, not N^3
    C = triple.tripling_coefficients(8, 16)
    nz = int((np.abs(C) > 1e-12).sum())
    assert nz < 0.02 * C.size


@pytest.mark.parametrize("H,W", [(2, 4), (4, 4), (8, 16), (32, 64)])
def test_theorem_sum_equals_the_definition(H, W):
    rng = np.random.default_rng(H + W)
    a, b, c = (rng.standard_normal(H * W) for _ in range(3))
    ref = triple.triple_product(a, b, c, H, W)
    got = triple.triple_product_by_theorem(a, b, c, H, W)
    assert abs(got - ref) <= 1e-12 * max(1.0, abs(ref)) * H


def test_brute_force_triple_sum_equals_the_definition():
    H, W = 4, 8
    rng = np.random.default_rng(5)
    a, b, c = (rng.standard_normal(H * W) for _ in range(3))
    C = triple.tripling_coefficients(H, W)
    assert np.isclose(np.einsum("ijk,i,j,k->", C, a, b, c), triple.triple_product(a, b, c, H, W), atol=1e-12)


def test_constant_factor_reduces_to_the_double_product():
    # a constant map 1 makes the triple product the inner product (Parseval)
    H, W = 16, 32
    rng = np.random.default_rng(6)
    a, b = rng.standard_normal(H * W), rng.standard_normal(H * W)
    one = haar.forward(np.ones((H, W)))
    assert np.isclose(triple.triple_product_by_theorem(a, b, one, H, W), a @ b, rtol=1e-12)
    assert np.isclose(triple.triple_product_by_theorem(one, a, b, H, W), a @ b, rtol=1e-12)


def test_triple_product_is_symmetric():
    H, W = 8, 16
    rng = np.random.default_rng(7)
    a, b, c = (rng.standard_normal(H * W) for _ in range(3))
    v = triple.triple_product_by_theorem(a, b, c, H, W)
    for p in ((b, a, c), (c, b, a), (a, c, b)):
        assert np.isclose(triple.triple_product_by_theorem(*p, H, W), v, rtol=1e-12)


def test_normal_rotation_takes_the_normal_to_the_pole():
    rng = np.random.default_rng(8)
    for _ in range(50):
        n = rng.standard_normal(3)
        n /= np.linalg.norm(n)
        R = triple.normal_rotation(n)
        assert np.allclose(R @ n, [0, 1, 0], atol=1e-12)
        assert np.allclose(R @ R.T, np.eye(3), atol=1e-12) and np.isclose(np.linalg.det(R), 1.0)
    assert np.allclose(triple.normal_rotation(np.array([0.0, 1.0, 0.0])), np.eye(3))
    # the decomposition: a tilt about x after an azimuth turn
    n = np.array([math.sin(0.7) * math.sin(2.1), math.cos(0.7), math.sin(0.7) * math.cos(2.1)])
    assert np.allclose(triple.normal_rotation(n), rot_x(-0.7) @ rot_y(-2.1))


def test_white_furnace():
    # constant unit lighting, no occluder, Lambertian BRDF (cos / pi): the
    # radiance is the hemisphere integral of cos / pi = 1, up to the midpoint
    # rule and the resampling of the rotated lobe
    H, W = 32, 64
    th = (np.arange(H) + 0.5) * math.pi / H
    ph = (np.arange(W) + 0.5) * 2 * math.pi / W
    T, _ = np.meshgrid(th, ph, indexing="ij")
    brdf = haar.forward(np.maximum(np.cos(T), 0.0) / math.pi)
    vis = haar.forward(np.sin(T) * (math.pi / H) * (2 * math.pi / W))
    light = haar.forward(np.ones((1, H, W)))
    normals = np.array([[0.0, 1.0, 0.0], [0.0, -1.0, 0.0], [0.6, 0.0, 0.8]])
    r = triple.shade_triple(light, brdf, normals, np.repeat(vis[None], 3, 0), H, W)
    assert np.allclose(r, 1.0, atol=5e-3), r
    # the unrotated normal is exact up to the midpoint rule alone
    assert abs(r[0, 0] - 1.0) < 2e-3


def test_shade_triple_matches_rotating_in_pixel_space():
    H, W = 8, 16
    rng = np.random.default_rng(9)
    light = rng.standard_normal((2, H * W))
    brdf = rng.standard_normal(H * W)
    n = rng.standard_normal((3, 3))
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    vis = rng.standard_normal((3, H * W))
    got = triple.shade_triple(light, brdf, n, vis, H, W)
    from oracle.resample import rotate
    for v in range(3):
        Bm = rotate(haar.inverse(brdf, H, W), triple.normal_rotation(n[v]), shift.SPHERE)
        for ch in range(2):
            ref = (haar.inverse(light[ch], H, W) * Bm * haar.inverse(vis[v], H, W)).sum()
            assert np.isclose(got[v, ch], ref, rtol=1e-12, atol=1e-12)


def _golden_cases():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "tripling_coefficients.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    return {case: value for case, value in rows}


def test_tripling_values_match_the_papers_statement():
    # the paper's values are for the unit square; on an H x H pixel map the
    # oracle's unit-pixel measure gives C_pixel = C_paper / H, and a square of
    # side B pixels is the paper's level l = log2(H / B)
    golden = _golden_cases()
    assert golden == {"a": "1", "b": "2^l", "c": "+-2^l"}
    H = W = 8
    C = triple.tripling_coefficients(H, W) * H
    N = H * W
    seen = set()
    for i in range(N):
        for j in range(N):
            for k in range(N):
                v = C[i, j, k]
                if abs(v) < 1e-12:
                    continue
                d = [haar.decode(H, W, x) for x in (i, j, k)]
                if all(x[1] == -1 for x in d):                             # case a
                    assert abs(v - 1.0) < 1e-12
                    seen.add("a")
                elif i != j and j != k and i != k and len({(x[0], x[2], x[3]) for x in d}) == 1:   # case b
                    lvl = int(round(math.log2(H / (1 << d[0][0]))))
                    assert abs(v - 2.0 ** lvl) < 1e-12
                    seen.add("b")
                else:                                                        # case c
                    # the third function is the one that differs from the repeated pair
                    third = d[2] if i == j else (d[1] if i == k else d[0])
                    lvl = 0 if third[1] == -1 else int(round(math.log2(H / (1 << third[0]))))
                    assert abs(abs(v) - 2.0 ** lvl) < 1e-12, (i, j, k, v)
                    seen.add("c")
    assert seen == {"a", "b", "c"}
