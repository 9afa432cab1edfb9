"""Headless rasterisation of a triangle mesh into a fragment buffer, and
per-pixel shading from per-vertex radiance (oracle).

The paper's renderer has a rasterisation pass (Sec. "Experimental results",
the Cg pass) that writes, for every pixel, the interpolation data and the id
of the surface it sees.  Shading follows from those.  This module restates
that pass without a graphics API.

Definition:
- Project each vertex: clip = M [x, y, z, 1] (M row-major 4 x 4).
  ndc = clip.xyz / clip.w, screen x = (ndc_x + 1) / 2 * width,
  y = (1 - ndc_y) / 2 * height (rows grow downwards).
- A triangle is dropped if any vertex has w <= 1e-6 (no near-plane
  clipping) or its screen area is 0.
- Pixel (px, py) samples its centre (px + 1/2, py + 1/2).  It is covered
  when the three edge functions, in the orientation that makes the area
  positive, are all > 0, or = 0 on an "owning" edge: the edge direction
  (dx, dy) has dy > 0, or dy = 0 and dx < 0.  Two triangles that share an
  edge see it in opposite directions, so it is covered exactly once.
- Depth = (z + 1) / 2 with z the screen-linear interpolation of ndc z.
  Samples outside [0, 1] are dropped.  The nearest fragment wins, and on
  equal depth the lower triangle id.
- Barycentrics of the winner are perspective-correct: the screen-space
  weights divided by each vertex's w, renormalised.

Every value that decides an integer (coverage, the depth order) is computed
in float32 with the operations in one fixed order: products, then sums left
to right, no fused multiply-add.  The GPU kernels do the same, so both sides
make the same decisions.  Radiance interpolation is plain float64.

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import numpy as np

F = np.float32
EMPTY = -1


def project(pos: np.ndarray, M: np.ndarray, width: int, height: int):
    """Screen (x, y), depth-space z (ndc) and w of every vertex, float32."""
    p = np.asarray(pos, dtype=F)
    M = np.asarray(M, dtype=F).reshape(4, 4)
    x, y, z = p[:, 0], p[:, 1], p[:, 2]

    def row(r):
        return ((M[r, 0] * x + M[r, 1] * y) + M[r, 2] * z) + M[r, 3]

    cx, cy, cz, cw = row(0), row(1), row(2), row(3)
    with np.errstate(divide="ignore", invalid="ignore"):
        nx, ny, nz = cx / cw, cy / cw, cz / cw
    sx = ((nx + F(1)) * F(0.5)) * F(width)
    sy = ((F(1) - ny) * F(0.5)) * F(height)
    return sx.astype(F), sy.astype(F), nz.astype(F), cw.astype(F)


def _edge(ax, ay, bx, by, px, py):
    # (b - a) x (p - a), products first, then the difference
    return (bx - ax) * (py - ay) - (by - ay) * (px - ax)


def rasterize(pos, tris, M, width: int, height: int):
    """tri_id [H, W] int32 (EMPTY where nothing is hit), bary [H, W, 2]
    (weights of vertices 1 and 2; vertex 0 gets 1 - b1 - b2), depth [H, W]."""
    sx, sy, sz, sw = project(pos, M, width, height)
    tris = np.asarray(tris, dtype=np.int64)
    best = np.full((height, width), np.inf, dtype=np.float64)
    tid = np.full((height, width), EMPTY, dtype=np.int64)
    PX, PY = np.meshgrid(np.arange(width, dtype=F) + F(0.5), np.arange(height, dtype=F) + F(0.5))
    for t, (i0, i1, i2) in enumerate(tris):
        if not (sw[i0] > F(1e-6) and sw[i1] > F(1e-6) and sw[i2] > F(1e-6)):
            continue
        x = [sx[i0], sx[i1], sx[i2]]
        y = [sy[i0], sy[i1], sy[i2]]
        z = [sz[i0], sz[i1], sz[i2]]
        area = _edge(x[0], y[0], x[1], y[1], x[2], y[2])
        if not np.isfinite(area) or area == 0:
            continue
        if area < 0:                                      # orientation with positive area
            x[1], x[2] = x[2], x[1]
            y[1], y[2] = y[2], y[1]
            z[1], z[2] = z[2], z[1]
            area = -area
        x0 = max(int(np.floor(min(x))), 0)
        x1 = min(int(np.ceil(max(x))), width - 1)
        y0 = max(int(np.floor(min(y))), 0)
        y1 = min(int(np.ceil(max(y))), height - 1)
        if x0 > x1 or y0 > y1:
            continue
        px, py = PX[y0:y1 + 1, x0:x1 + 1], PY[y0:y1 + 1, x0:x1 + 1]
        inside = np.ones(px.shape, bool)
        e = []
        for a, b in ((1, 2), (2, 0), (0, 1)):
            w = _edge(x[a], y[a], x[b], y[b], px, py).astype(F)
            dx, dy = x[b] - x[a], y[b] - y[a]
            owns = (dy > 0) or (dy == 0 and dx < 0)
            inside &= (w > 0) | ((w == 0) & owns)
            e.append(w)
        zi = ((e[0] * z[0] + e[1] * z[1]) + e[2] * z[2]) / area
        depth = ((zi + F(1)) * F(0.5)).astype(F)
        ok = inside & (depth >= 0) & (depth <= 1)
        cur = best[y0:y1 + 1, x0:x1 + 1]
        ct = tid[y0:y1 + 1, x0:x1 + 1]
        win = ok & ((depth < cur) | ((depth == cur) & (t < ct)))
        cur[win] = depth[win]
        ct[win] = t
    bary = np.zeros((height, width, 2))
    for (py_, px_) in zip(*np.nonzero(tid >= 0)):
        i0, i1, i2 = tris[tid[py_, px_]]
        pxc, pyc = F(px_) + F(0.5), F(py_) + F(0.5)
        # screen weights of the original vertex order, then perspective
        w0 = float(_edge(sx[i1], sy[i1], sx[i2], sy[i2], pxc, pyc))
        w1 = float(_edge(sx[i2], sy[i2], sx[i0], sy[i0], pxc, pyc))
        w2 = float(_edge(sx[i0], sy[i0], sx[i1], sy[i1], pxc, pyc))
        a0, a1, a2 = w0 / float(sw[i0]), w1 / float(sw[i1]), w2 / float(sw[i2])
        s = a0 + a1 + a2
        bary[py_, px_] = (a1 / s, a2 / s)
    return tid.astype(np.int32), bary, np.where(tid >= 0, best, np.nan)


def shade_pixels(tid, bary, tris, vert_rad, background):
    """image [H, W, C]: barycentric interpolation of per-vertex radiance
    [V, C], background where nothing is hit."""
    tid = np.asarray(tid)
    vr = np.asarray(vert_rad, dtype=np.float64)
    tris = np.asarray(tris, dtype=np.int64)
    img = np.empty(tid.shape + (vr.shape[1],))
    img[:] = np.asarray(background, dtype=np.float64)
    hit = tid >= 0
    t = tris[tid[hit]]
    b1, b2 = bary[hit][:, 0:1], bary[hit][:, 1:2]
    img[hit] = (1 - b1 - b2) * vr[t[:, 0]] + b1 * vr[t[:, 1]] + b2 * vr[t[:, 2]]
    return img
