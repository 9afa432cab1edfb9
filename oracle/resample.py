"""Resampling of a lat-long map under a translation or a rotation.

The paper defines the rotated map by g(theta, phi) = f(theta', phi') with
p = d(theta, phi) = (sin t sin p, cos t, sin t cos p) (Y up), p' = R p,
R = R_z R_y R_x (Sec. "Rotating Haar", Eq. tRot), theta' = acos(R_2 p)
(Eq. theta) and phi' = atan(R_1 p / R_3 p) (Eq. phi).  A rotation about the
Y axis is a pure shift along phi (Sec. "Algorithmic optimization").  The
paper does not say how f is sampled between pixel centres; the reading used
here (and by the CUDA path) is bilinear interpolation between pixel centres
of the map extended across its borders:

* columns are cyclic (phi has period 2 pi);
* SPHERE boundary: a row above the north pole or below the south pole is the
  row mirrored across that pole, half a turn away in azimuth:
  F(i, j) = F(-1 - i, j + W/2) for i < 0 and F(2H - 1 - i, j + W/2) for i >= H;
* TORUS boundary: rows are cyclic too.

Translation by (dx, dy) pixels: g[i, j] = F~(i - dy, j - dx).
Rotation: u = theta'/dtheta - 1/2, v = phi'/dphi - 1/2 with
theta' = atan2(sqrt(p'x^2 + p'z^2), p'y) (equal to acos(p'y) for unit p') and
phi' = atan2(p'x, p'z) taken in [0, 2 pi) (the quadrant-correct reading of
Eq. phi).

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import math

import numpy as np

SPHERE = 0
TORUS = 1


def extend_index(i, j, H: int, W: int, boundary: int):
    """Map integer sample coordinates onto the map (arrays, any range)."""
    i = np.asarray(i, dtype=np.int64).copy()
    j = np.asarray(j, dtype=np.int64).copy()
    if boundary == TORUS:
        return np.mod(i, H), np.mod(j, W)
    for _ in range(64):
        lo = i < 0
        hi = i >= H
        if not (lo.any() or hi.any()):
            break
        i = np.where(lo, -1 - i, np.where(hi, 2 * H - 1 - i, i))
        j = np.where(lo | hi, j + W // 2, j)
    return i, np.mod(j, W)


def sample(P: np.ndarray, i, j, boundary: int):
    H, W = P.shape[-2:]
    ii, jj = extend_index(i, j, H, W, boundary)
    return P[..., ii, jj]


def bilinear(P: np.ndarray, u, v, boundary: int):
    """Bilinear value of the extended map at fractional (row u, column v)."""
    u = np.asarray(u, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    i0 = np.floor(u)
    j0 = np.floor(v)
    fu = u - i0
    fv = v - j0
    i0 = i0.astype(np.int64)
    j0 = j0.astype(np.int64)
    f00 = sample(P, i0, j0, boundary)
    f01 = sample(P, i0, j0 + 1, boundary)
    f10 = sample(P, i0 + 1, j0, boundary)
    f11 = sample(P, i0 + 1, j0 + 1, boundary)
    return ((1 - fu) * ((1 - fv) * f00 + fv * f01)
            + fu * ((1 - fv) * f10 + fv * f11))


def translate(P: np.ndarray, dx: float, dy: float, boundary: int) -> np.ndarray:
    """g[i, j] = F~(i - dy, j - dx) for maps P [..., H, W]."""
    H, W = P.shape[-2:]
    ii, jj = np.meshgrid(np.arange(H, dtype=np.float64), np.arange(W, dtype=np.float64),
                         indexing="ij")
    return bilinear(P, ii - dy, jj - dx, boundary)


def rot_x(a):
    c, s = math.cos(a), math.sin(a)
    return np.array([[1, 0, 0], [0, c, -s], [0, s, c]], dtype=np.float64)


def rot_y(b):
    c, s = math.cos(b), math.sin(b)
    return np.array([[c, 0, s], [0, 1, 0], [-s, 0, c]], dtype=np.float64)


def rot_z(g):
    c, s = math.cos(g), math.sin(g)
    return np.array([[c, -s, 0], [s, c, 0], [0, 0, 1]], dtype=np.float64)


def euler_matrix(alpha, beta, gamma) -> np.ndarray:
    """R = R_z(gamma) R_y(beta) R_x(alpha) (Sec. "Rotating Haar")."""
    return rot_z(gamma) @ rot_y(beta) @ rot_x(alpha)


def rotation_coords(R: np.ndarray, H: int, W: int):
    """Fractional source coordinates (u, v) of every output pixel."""
    dth = math.pi / H
    dph = 2.0 * math.pi / W
    theta = (np.arange(H) + 0.5) * dth
    phi = (np.arange(W) + 0.5) * dph
    T, F = np.meshgrid(theta, phi, indexing="ij")
    p = np.stack([np.sin(T) * np.sin(F), np.cos(T), np.sin(T) * np.cos(F)], axis=-1)
    q = p @ np.asarray(R, dtype=np.float64).T
    th2 = np.arctan2(np.hypot(q[..., 0], q[..., 2]), q[..., 1])
    ph2 = np.mod(np.arctan2(q[..., 0], q[..., 2]), 2.0 * math.pi)
    return th2 / dth - 0.5, ph2 / dph - 0.5


def rotate(P: np.ndarray, R: np.ndarray, boundary: int = SPHERE) -> np.ndarray:
    """g(theta, phi) = f(Theta, Phi) sampled bilinearly, for maps [..., H, W]."""
    H, W = P.shape[-2:]
    u, v = rotation_coords(R, H, W)
    return bilinear(P, u, v, boundary)
