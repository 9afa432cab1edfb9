"""Seeded synthetic scenes for the Haar-domain phase-shift and shading path.

This module only *describes* scenes: lighting maps in pixel space, vertex
positions and normals, occluder spheres, shift/rotation parameters, cameras,
Phong exponents, view-bin directions and the per-vertex light-transport
integrand sampled on a lat-long grid.  It contains none of the method's own
arithmetic (no Haar transform, no resampling, no double product): both the
CPU oracle and the CUDA path consume what it produces.

Scene recipe (stand-ins for the paper's light probes, meshes and measured
BRDFs, Sec. "Experimental results", none of which are available):

* lat-long map, rows = elevation theta in [0, pi], columns = azimuth phi in
  [0, 2 pi), pixel centres theta_i = (i + 1/2) pi / H, phi_j = (j + 1/2) 2 pi / W,
  direction d(theta, phi) = (sin t sin p, cos t, sin t cos p), Y up (Sec.
  "Rotating Haar", the spherical-to-Cartesian map);
* lighting: every pixel and channel i.i.d. lognormal(mu=0, sigma=1.5), plus
  three Gaussian hot spots 50 exp(-gamma^2 / (2 sigma_h^2)), sigma_h = 3 dtheta,
  centres uniform on the sphere, shared by all channels;
* occluders: spheres with centre direction uniform, centre distance
  U[1.6, 3.0], radius U[0.2, 0.6], rejected when closer than 0.05 to the
  object's surface;
* transport integrand (rendering equation, Eq. 1, with BRDF x cosine x
  visibility folded into one transfer function): diffuse t = max(0, n.w) V(w),
  Phong t = V max(0, n.w) (s+2)/(2 pi) max(0, r.w)^s with r = 2 (n.v) n - v;
  V(w) = 0 iff the ray x + tau w, tau > 1e-6, meets an occluder;
  midpoint-rule weight w_p = t(d_p) sin(theta_i) dtheta dphi.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 1705072720

SPHERE = 0
TORUS = 1


def rng_for(config_id: int, stream: int = 0) -> np.random.Generator:
    """PCG64 generator seeded with SEED_BASE + config id (+ 1000 * stream)."""
    return np.random.Generator(np.random.PCG64(SEED_BASE + config_id + 1000 * stream))


# ---------------------------------------------------------------- geometry

def pixel_angles(H: int, W: int):
    """Pixel-centre elevation (H,) and azimuth (W,) in float64."""
    theta = (np.arange(H, dtype=np.float64) + 0.5) * (math.pi / H)
    phi = (np.arange(W, dtype=np.float64) + 0.5) * (2.0 * math.pi / W)
    return theta, phi


def pixel_directions(H: int, W: int) -> np.ndarray:
    """Unit directions [H, W, 3] of the lat-long pixel centres (Y up)."""
    theta, phi = pixel_angles(H, W)
    st, ct = np.sin(theta)[:, None], np.cos(theta)[:, None]
    sp, cp = np.sin(phi)[None, :], np.cos(phi)[None, :]
    d = np.empty((H, W, 3), dtype=np.float64)
    d[..., 0] = st * sp
    d[..., 1] = np.broadcast_to(ct, (H, W))
    d[..., 2] = st * cp
    return d


def uniform_sphere(rng: np.random.Generator, n: int) -> np.ndarray:
    z = rng.uniform(-1.0, 1.0, n)
    a = rng.uniform(0.0, 2.0 * math.pi, n)
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([r * np.cos(a), z, r * np.sin(a)], axis=1)


def lighting_pixels(rng: np.random.Generator, C: int, H: int, W: int,
                    sigma: float = 1.5, spots: int = 3, amp: float = 50.0) -> np.ndarray:
    """HDR lat-long lighting map [C, H, W] (float64)."""
    base = rng.lognormal(mean=0.0, sigma=sigma, size=(C, H, W))
    centres = uniform_sphere(rng, spots)
    d = pixel_directions(H, W)
    sig_h = 3.0 * math.pi / H
    add = np.zeros((H, W))
    for c in centres:
        cosg = np.clip(d @ c, -1.0, 1.0)
        g = np.arccos(cosg)
        add += amp * np.exp(-(g * g) / (2.0 * sig_h * sig_h))
    return base + add[None]


def smooth_lighting(rng: np.random.Generator, C: int, H: int, W: int, lobes: int = 4,
                    kappa: float = 6.0, amp: float = 4.0) -> np.ndarray:
    """Band-limited lat-long lighting map [C, H, W] (float64): 1 plus a few
    broad lobes amp * exp(kappa (d . c - 1)) around random directions c, smooth
    everywhere on the sphere, the poles included (a stand-in for a measured
    environment map's low-frequency content)."""
    d = pixel_directions(H, W)
    out = np.ones((C, H, W))
    for ch in range(C):
        for c in uniform_sphere(rng, lobes):
            out[ch] += amp * rng.uniform(0.5, 1.0) * np.exp(kappa * (d @ c - 1.0))
    return out


def local_brdf_map(H: int, W: int, expo: float = 0.0, view_theta: float = 0.0) -> np.ndarray:
    """A cosine-weighted BRDF map [H, W] in the local frame (normal at the +y
    pole): Lambertian cos / pi for expo = 0, else a normalised Phong lobe
    (expo + 2) / (2 pi) max(0, r . w)^expo cos about the mirror direction r of
    a view at polar angle view_theta in the phi = 0 half-plane."""
    d = pixel_directions(H, W)
    cos = np.maximum(d[..., 1], 0.0)
    if expo <= 0.0:
        return cos / math.pi
    r = np.array([0.0, math.cos(view_theta), -math.sin(view_theta)])
    return (expo + 2.0) / (2.0 * math.pi) * np.maximum(d @ r, 0.0) ** expo * cos


def torus_mesh(nu: int, nv: int, R: float = 1.0, r: float = 0.4):
    """A closed triangle mesh of the torus (axis Y, core radius R, tube radius
    r) on an nu x nv parameter grid: positions and normals [nu nv, 3] float32,
    triangles [2 nu nv, 3] int32, consistently wound."""
    u = np.arange(nu) * 2.0 * math.pi / nu
    v = np.arange(nv) * 2.0 * math.pi / nv
    U, Vv = np.meshgrid(u, v, indexing="ij")
    ring = R + r * np.cos(Vv)
    pos = np.stack([ring * np.sin(U), r * np.sin(Vv), ring * np.cos(U)], -1).reshape(-1, 3)
    nrm = np.stack([np.cos(Vv) * np.sin(U), np.sin(Vv), np.cos(Vv) * np.cos(U)], -1).reshape(-1, 3)
    i, j = np.meshgrid(np.arange(nu), np.arange(nv), indexing="ij")
    a = i * nv + j
    b = ((i + 1) % nu) * nv + j
    c = ((i + 1) % nu) * nv + (j + 1) % nv
    d = i * nv + (j + 1) % nv
    tris = np.concatenate([np.stack([a, b, c], -1).reshape(-1, 3), np.stack([a, c, d], -1).reshape(-1, 3)])
    return pos.astype(np.float32), nrm.astype(np.float32), tris.astype(np.int32)


def view_projection(eye, target, up=(0.0, 1.0, 0.0), fov_y: float = 0.8, aspect: float = 16 / 9,
                    near: float = 0.1, far: float = 20.0) -> np.ndarray:
    """Row-major 4 x 4 float32 perspective x look-at matrix (OpenGL clip
    conventions: the camera looks down -z of its frame, ndc z in [-1, 1])."""
    eye, target, up = (np.asarray(x, dtype=np.float64) for x in (eye, target, up))
    f = target - eye
    f /= np.linalg.norm(f)
    s_ = np.cross(f, up)
    s_ /= np.linalg.norm(s_)
    u_ = np.cross(s_, f)
    view = np.eye(4)
    view[0, :3], view[1, :3], view[2, :3] = s_, u_, -f
    view[:3, 3] = -view[:3, :3] @ eye
    t = 1.0 / math.tan(fov_y / 2)
    proj = np.array([[t / aspect, 0, 0, 0], [0, t, 0, 0],
                     [0, 0, (far + near) / (near - far), 2 * far * near / (near - far)], [0, 0, -1, 0]])
    return (proj @ view).astype(np.float32)


def sphere_vertices(rng: np.random.Generator, V: int):
    """Vertices uniform on the unit sphere; normal = position."""
    p = uniform_sphere(rng, V)
    return p.copy(), p.copy()


def torus_vertices(rng: np.random.Generator, V: int, R: float = 1.0, r: float = 0.4):
    """Vertices on a torus (axis Y, core radius R, tube radius r), uniform by
    area; ordered by a coarse (u, v) raster so neighbouring vertices are close."""
    u = rng.uniform(0.0, 2.0 * math.pi, V)
    v = np.empty(V)
    filled = 0
    while filled < V:           # rejection: density of v proportional to R + r cos v
        m = 2 * (V - filled) + 16
        cand = rng.uniform(0.0, 2.0 * math.pi, m)
        acc = rng.uniform(0.0, R + r, m) < (R + r * np.cos(cand))
        take = cand[acc][: V - filled]
        v[filled: filled + take.size] = take
        filled += take.size
    ub = np.floor(u / (2.0 * math.pi) * 256).astype(np.int64)
    order = np.lexsort((v, ub))
    u, v = u[order], v[order]
    cu, su, cv, sv = np.cos(u), np.sin(u), np.cos(v), np.sin(v)
    pos = np.stack([(R + r * cv) * cu, r * sv, (R + r * cv) * su], axis=1)
    nrm = np.stack([cv * cu, sv, cv * su], axis=1)
    return pos, nrm


def _torus_surface_distance(c: np.ndarray, R: float = 1.0, r: float = 0.4) -> float:
    rho = math.hypot(c[0], c[2])
    return math.hypot(rho - R, c[1]) - r


def occluders(rng: np.random.Generator, count: int, surface: str):
    """Occluder spheres (centres [count, 3], radii [count])."""
    cs, rs = [], []
    while len(cs) < count:
        dirn = uniform_sphere(rng, 1)[0]
        dist = rng.uniform(1.6, 3.0)
        rad = rng.uniform(0.2, 0.6)
        c = dirn * dist
        gap = (dist - 1.0) if surface == "sphere" else _torus_surface_distance(c)
        if gap - rad > 0.05:
            cs.append(c)
            rs.append(rad)
    return np.array(cs), np.array(rs)


def translations(rng: np.random.Generator, S: int, xmax: float, ymax: float) -> np.ndarray:
    """[S, 2] fractional (dx, dy) pixel shifts, dx ~ U[0, xmax), dy ~ U[0, ymax)."""
    out = np.empty((S, 2))
    out[:, 0] = rng.uniform(0.0, xmax, S)
    out[:, 1] = rng.uniform(0.0, ymax, S)
    return out


def euler_angles(rng: np.random.Generator, S: int) -> np.ndarray:
    """[S, 3] Euler angles (alpha about X, beta about Y, gamma about Z) ~ U[0, 2 pi)."""
    return rng.uniform(0.0, 2.0 * math.pi, (S, 3))


def cameras(rng: np.random.Generator, P: int, radius: float = 5.0) -> np.ndarray:
    return uniform_sphere(rng, P) * radius


def phong_exponents(rng: np.random.Generator, V: int) -> np.ndarray:
    return rng.choice(np.array([8.0, 32.0, 128.0]), size=V)


def view_bin_dirs(nbins: int = 16) -> np.ndarray:
    """Fibonacci points on the local upper hemisphere (z up), area-uniform."""
    i = np.arange(nbins, dtype=np.float64)
    z = 1.0 - (i + 0.5) / nbins
    ga = math.pi * (3.0 - math.sqrt(5.0))
    a = i * ga
    s = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([s * np.cos(a), s * np.sin(a), z], axis=1)


def onb(n: np.ndarray):
    """Branchless orthonormal basis (b1, b2) around unit normals n [V, 3]
    (Duff et al., 'Building an Orthonormal Basis, Revisited', 2017)."""
    sign = np.where(n[:, 2] >= 0.0, 1.0, -1.0)
    a = -1.0 / (sign + n[:, 2])
    b = n[:, 0] * n[:, 1] * a
    b1 = np.stack([1.0 + sign * n[:, 0] ** 2 * a, sign * b, -sign * n[:, 0]], axis=1)
    b2 = np.stack([b, sign + n[:, 1] ** 2 * a, -n[:, 1]], axis=1)
    return b1, b2


def bin_view_world(nrm: np.ndarray, nbins: int = 16) -> np.ndarray:
    """World-space view direction of every (vertex, bin): [V, nbins, 3]."""
    b1, b2 = onb(nrm)
    L = view_bin_dirs(nbins)
    return (L[None, :, 0:1] * b1[:, None, :] + L[None, :, 1:2] * b2[:, None, :]
            + L[None, :, 2:3] * nrm[:, None, :])


# ---------------------------------------------------------------- transport integrand

def transport_weights(pos, nrm, occ_c, occ_r, Ht: int, Wt: int, *, view=None, expo=None,
                      device="cpu", dtype=None, chunk: int = 256, cosine: bool = True):
    """Midpoint-rule transport weights w[v, i, j] = t_v(d_ij) sin(theta_i) dtheta dphi
    on an Ht x Wt lat-long quadrature grid, as a torch tensor [V, Ht, Wt].

    ``view`` [V, 3] and ``expo`` [V] select the Phong integrand; otherwise the
    diffuse one; ``cosine=False`` (no view) leaves the visibility alone, for
    the triple product's visibility factor.  Evaluated in chunks of vertices
    with torch on ``device``."""
    import torch
    if dtype is None:
        dtype = torch.float64 if str(device) == "cpu" else torch.float32
    d = torch.as_tensor(pixel_directions(Ht, Wt).reshape(-1, 3), dtype=dtype, device=device)
    theta, _ = pixel_angles(Ht, Wt)
    sa = torch.as_tensor(np.repeat(np.sin(theta) * (math.pi / Ht) * (2.0 * math.pi / Wt), Wt),
                         dtype=dtype, device=device)
    P = d.shape[0]
    pos_t = torch.as_tensor(pos, dtype=dtype, device=device)
    nrm_t = torch.as_tensor(nrm, dtype=dtype, device=device)
    oc_t = torch.as_tensor(occ_c, dtype=dtype, device=device)
    orr = torch.as_tensor(occ_r, dtype=dtype, device=device)
    view_t = None if view is None else torch.as_tensor(view, dtype=dtype, device=device)
    expo_t = None if expo is None else torch.as_tensor(expo, dtype=dtype, device=device)
    V = pos_t.shape[0]
    out = torch.empty((V, P), dtype=dtype, device=device)
    dx, dy, dz = d[:, 0], d[:, 1], d[:, 2]
    for v0 in range(0, V, chunk):
        v1 = min(V, v0 + chunk)
        n = nrm_t[v0:v1]
        cosn = n[:, 0:1] * dx + n[:, 1:2] * dy + n[:, 2:3] * dz
        t = torch.clamp(cosn, min=0.0) if cosine else torch.ones_like(cosn)
        if view_t is not None:
            vv = view_t[v0:v1]
            ndv = (n * vv).sum(1, keepdim=True)
            r = 2.0 * ndv * n - vv
            cr = torch.clamp(r[:, 0:1] * dx + r[:, 1:2] * dy + r[:, 2:3] * dz, min=0.0)
            s = expo_t[v0:v1, None]
            t = t * ((s + 2.0) / (2.0 * math.pi)) * torch.pow(cr, s)
        x = pos_t[v0:v1]
        vis = torch.ones_like(t, dtype=torch.bool)
        for o in range(oc_t.shape[0]):
            oc = x - oc_t[o]
            b = oc[:, 0:1] * dx + oc[:, 1:2] * dy + oc[:, 2:3] * dz
            cc = (oc * oc).sum(1, keepdim=True) - orr[o] * orr[o]
            disc = b * b - cc
            far = -b + torch.sqrt(torch.clamp(disc, min=0.0))
            vis &= ~((disc >= 0.0) & (far > 1e-6))
        out[v0:v1] = t * vis.to(dtype) * sa
    return out.reshape(V, Ht, Wt)


def spread(w: np.ndarray, H: int, W: int) -> np.ndarray:
    """Spread coarse quadrature weights [..., Ht, Wt] uniformly over the
    H x W pixels of each block (the weight of a block is shared by its pixels)."""
    Ht, Wt = w.shape[-2:]
    b = H // Ht
    assert b * Ht == H and b * Wt == W
    return np.repeat(np.repeat(w, b, axis=-2), b, axis=-1) / float(b * b)


# ---------------------------------------------------------------- workload configs

@dataclass
class Workload:
    """Sizes and seed of one synthetic workload."""
    cid: int
    name: str
    C: int
    H: int
    W: int
    S: int
    V: int
    kind: str             # "translate" or "rotate"
    surface: str          # "sphere" or "torus"
    n_occ: int
    storage: str          # dense_f32 | csr_f32 | dense_bf16 | bincsr_f16 | mlp
    K: int                # coefficients kept per vertex (dense: lowest K; csr: top-K)
    tgrid: tuple = None   # transport quadrature grid (Ht, Wt); None = lighting grid
    bins: int = 0
    extra: dict = field(default_factory=dict)


WORKLOADS = {
    0: Workload(0, "c0: 1ch 32x32 lat-long, 1 fractional shift, 1000 sphere vertices, dense 1024 FP32",
                C=1, H=32, W=32, S=1, V=1000, kind="translate", surface="sphere", n_occ=4,
                storage="dense_f32", K=1024, extra={"xmax": 32.0, "ymax": 32.0}),
    1: Workload(1, "c1: RGB 128x256, 16 fractional shifts, 50000 torus vertices, top-256 CSR FP32",
                C=3, H=128, W=256, S=16, V=50000, kind="translate", surface="torus", n_occ=8,
                storage="csr_f32", K=256, extra={"xmax": 256.0, "ymax": 256.0}),
    2: Workload(2, "c2: RGB 256x512, 64 rotations, 200000 torus vertices, lowest-4096 BF16 dense",
                C=3, H=256, W=512, S=64, V=200000, kind="rotate", surface="torus", n_occ=8,
                storage="dense_bf16", K=4096, tgrid=(64, 128)),
    3: Workload(3, "c3: RGB 256x512, 32 (rotation, view) pairs, 100000 torus vertices, Phong, "
                   "16 view bins x top-512 FP16",
                C=3, H=256, W=512, S=32, V=100000, kind="rotate", surface="torus", n_occ=8,
                storage="bincsr_f16", K=512, tgrid=(64, 128), bins=16),
    4: Workload(4, "c4: c3 scene, MLP surrogate (4x256 GELU, 512 outputs) fused with shift+shade",
                C=3, H=256, W=512, S=32, V=100000, kind="rotate", surface="torus", n_occ=8,
                storage="mlp", K=512, tgrid=(64, 128), bins=16),
}


def scene(cid: int, *, V: int = None, S: int = None, H: int = None, W: int = None):
    """Geometry, lighting pixels and shift parameters of workload ``cid``
    (optionally with overridden sizes for small test cases)."""
    wl = WORKLOADS[cid]
    V = wl.V if V is None else V
    S = wl.S if S is None else S
    H = wl.H if H is None else H
    W = wl.W if W is None else W
    rl = rng_for(cid, 0)
    light = lighting_pixels(rl, wl.C, H, W)
    rg = rng_for(cid, 1)
    if wl.surface == "sphere":
        pos, nrm = sphere_vertices(rg, V)
    else:
        pos, nrm = torus_vertices(rg, V)
    occ_c, occ_r = occluders(rng_for(cid, 2), wl.n_occ, wl.surface)
    rp = rng_for(cid, 3)
    if wl.kind == "translate":
        params = translations(rp, S, wl.extra["xmax"] * W / wl.W, wl.extra["ymax"] * H / wl.H)
    else:
        params = euler_angles(rp, S)
    out = dict(wl=wl, H=H, W=W, C=wl.C, S=S, V=V, light=light, pos=pos, nrm=nrm,
               occ_c=occ_c, occ_r=occ_r, params=params)
    if wl.storage in ("bincsr_f16", "mlp"):
        out["cams"] = cameras(rng_for(cid, 4), S)
        out["expo"] = phong_exponents(rng_for(cid, 5), V)
    return out
