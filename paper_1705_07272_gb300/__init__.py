"""Python binding of libhaarshift.so: the Haar-domain phase shift of a
lat-long lighting map and the per-vertex double product on sm_103a.

The functions here only marshal arguments (torch tensors -> device pointers,
the current CUDA stream) into the C ABI declared in include/haarshift.h;
every step of the computation runs in the library's CUDA kernels.  The
library must have been built (``paper_1705_07272_gb300.build.build()``);
importing the binding does not build it and there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libhaarshift.so")

# haar_status_t
HAAR_OK = 0
HAAR_ERR_INVALID_ARG = 1
HAAR_ERR_UNSUPPORTED = 2
HAAR_ERR_CUDA = 3
HAAR_ERR_TIMEOUT = 4
HAAR_ERR_INJECTED = 5
HAAR_ERR_NOMEM = 6
# haar_shift_kind_t
HAAR_SHIFT_TRANSLATE = 0
HAAR_SHIFT_ROTATE = 1
HAAR_SHIFT_ROTATE_EULER = 2
HAAR_SHIFT_ROTATE_CHAIN = 3
# haar_boundary_t
HAAR_BOUNDARY_SPHERE = 0
HAAR_BOUNDARY_TORUS = 1
# haar_out_t
HAAR_OUT_F32 = 0
HAAR_OUT_BF16_HILO = 1
HAAR_OUT_F16 = 2
# haar_layout_t
HAAR_LAYOUT_SCK = 0
HAAR_LAYOUT_SKC = 1
HAAR_LAYOUT_KSC = 2
HAAR_LAYOUT_SKC4 = 3
# haar_transport_kind_t
HAAR_T_DENSE_F32 = 0
HAAR_T_DENSE_BF16 = 1
HAAR_T_CSR_F32_U16 = 2
HAAR_T_BINCSR_F16_U32 = 3
HAAR_T_GCSR_F32_U16 = 4
GROUP = 4            # vertices per group of HAAR_T_GCSR_F32_U16 (HAAR_GCSR_GROUP)

EXPORTS = ("haar_shift_plan", "haar_shift_plan_destroy", "haar_shift", "haar_forward",
           "haar_inverse", "shade_vertices", "shade_batch", "haar_view_bins",
           "haar_last_error", "haar_version", "haar_mlp_param_count", "haar_mlp_create",
           "haar_mlp_destroy", "haar_mlp_set_params", "haar_mlp_get_params", "haar_mlp_forward",
           "haar_mlp_grads", "haar_mlp_train_step", "haar_mlp_shade", "haar_mlp_status",
           "haar_shift_noalloc", "haar_transport_group", "haar_shift_plan_status", "haar_normal_rotations",
           "haar_triple_work_floats", "haar_triple_product", "haar_shade_triple_work_floats", "haar_shade_triple",
           "haar_rasterize", "haar_shade_pixels")


class HaarShiftDesc(ctypes.Structure):
    _fields_ = [("height", ctypes.c_int), ("width", ctypes.c_int), ("channels", ctypes.c_int),
                ("kind", ctypes.c_int), ("boundary", ctypes.c_int), ("max_shifts", ctypes.c_int),
                ("out_coeffs", ctypes.c_int), ("out_type", ctypes.c_int), ("out_layout", ctypes.c_int),
                ("start_level", ctypes.c_int)]


class HaarTransportDesc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("V", ctypes.c_int), ("K", ctypes.c_int), ("bins", ctypes.c_int),
                ("vals", ctypes.c_void_p), ("idx", ctypes.c_void_p), ("rowptr", ctypes.c_void_p),
                ("bin_of", ctypes.c_void_p)]


class HaarError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"haarshift status {status}: {message}")
        self.status = status


_lib = None


def lib() -> ctypes.CDLL:
    """The loaded library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1705_07272_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp, i, st = ctypes.c_void_p, ctypes.c_int, ctypes.c_int
    L.haar_shift_plan.argtypes = [ctypes.POINTER(HaarShiftDesc), ctypes.POINTER(vp)]
    L.haar_shift_plan_destroy.argtypes = [vp]
    L.haar_shift.argtypes = [vp, vp, vp, i, vp, vp]
    L.haar_shift_noalloc.argtypes = [ctypes.POINTER(HaarShiftDesc), vp, vp, i, vp, vp]
    L.haar_forward.argtypes = [i, i, i, vp, vp, ctypes.c_float, vp]
    L.haar_inverse.argtypes = [i, i, i, vp, vp, vp]
    L.shade_vertices.argtypes = [vp, ctypes.POINTER(HaarTransportDesc), vp, i, vp, vp]
    L.shade_batch.argtypes = [vp, vp, vp, i, ctypes.POINTER(HaarTransportDesc), vp, vp]
    L.haar_view_bins.argtypes = [i, i, i, vp, vp, vp, vp, vp, vp]
    L.haar_transport_group.argtypes = [i, i, vp, vp, vp, vp, vp, vp, vp]
    L.haar_transport_group.restype = st
    L.haar_shift_plan_status.argtypes = [vp, ctypes.POINTER(ctypes.c_int), i]
    L.haar_shift_plan_status.restype = st
    L.haar_normal_rotations.argtypes = [i, vp, vp, vp]
    L.haar_normal_rotations.restype = st
    L.haar_triple_work_floats.argtypes = [i, i, i]
    L.haar_triple_work_floats.restype = ctypes.c_longlong
    L.haar_triple_product.argtypes = [i, i, i, i, vp, vp, ctypes.c_longlong, vp, ctypes.c_longlong, vp, vp, vp]
    L.haar_triple_product.restype = st
    L.haar_shade_triple_work_floats.argtypes = [i, i, i]
    L.haar_shade_triple_work_floats.restype = ctypes.c_longlong
    L.haar_shade_triple.argtypes = [i, i, i, i, vp, vp, vp, vp, ctypes.c_longlong, vp, vp, vp]
    L.haar_shade_triple.restype = st
    L.haar_rasterize.argtypes = [i, vp, i, vp, vp, i, i, vp, vp, vp, vp, vp]
    L.haar_rasterize.restype = st
    L.haar_shade_pixels.argtypes = [i, i, i, i, i, vp, vp, vp, vp, vp, vp, vp]
    L.haar_shade_pixels.restype = st
    for name in ("haar_shift_plan", "haar_shift_plan_destroy", "haar_shift", "haar_shift_noalloc", "haar_forward", "haar_inverse",
                 "shade_vertices", "shade_batch", "haar_view_bins"):
        getattr(L, name).restype = st
    ll = ctypes.c_longlong
    L.haar_mlp_param_count.restype = ll
    L.haar_mlp_param_count.argtypes = []
    L.haar_mlp_create.argtypes = [i, i, i, ctypes.POINTER(vp)]
    L.haar_mlp_destroy.argtypes = [vp]
    L.haar_mlp_set_params.argtypes = [vp, vp, vp]
    L.haar_mlp_get_params.argtypes = [vp, vp, vp]
    L.haar_mlp_forward.argtypes = [vp, vp, i, vp, vp]
    L.haar_mlp_grads.argtypes = [vp, vp, vp, i, vp, vp, vp]
    L.haar_mlp_train_step.argtypes = [vp, vp, vp, i, ctypes.c_float, vp, vp]
    L.haar_mlp_shade.argtypes = [vp, i, i, vp, vp, vp, vp, vp, vp, vp, i, ll, ll, ll, vp, vp]
    L.haar_mlp_status.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
    for name in ("haar_mlp_create", "haar_mlp_destroy", "haar_mlp_set_params", "haar_mlp_get_params",
                 "haar_mlp_forward", "haar_mlp_grads", "haar_mlp_train_step", "haar_mlp_shade", "haar_mlp_status",
           "haar_shift_noalloc", "haar_transport_group"):
        getattr(L, name).restype = st
    L.haar_last_error.restype = ctypes.c_char_p
    L.haar_last_error.argtypes = []
    L.haar_version.restype = ctypes.c_char_p
    L.haar_version.argtypes = []
    _lib = L
    return L


def _check(status: int):
    if status != HAAR_OK:
        raise HaarError(status, lib().haar_last_error().decode(errors="replace"))


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _dev(t, dtype=None, name="tensor"):
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must be on a CUDA device")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    return t.data_ptr()


def _out(t, dtype, name):
    """An output buffer: a CUDA tensor, or a pinned (page-locked) host tensor,
    which the kernels write straight over the host link."""
    import torch
    if isinstance(t, torch.Tensor) and not t.is_cuda and t.is_pinned():
        if not t.is_contiguous() or t.dtype != dtype:
            raise TypeError(f"{name} must be a contiguous {dtype} tensor")
        return t.data_ptr()
    return _dev(t, dtype, name)


def _stream(stream):
    import torch
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Plan:
    """A haar_shift_plan_t and its descriptor."""

    def __init__(self, height, width, channels, kind=HAAR_SHIFT_TRANSLATE, boundary=HAAR_BOUNDARY_SPHERE,
                 max_shifts=1, out_coeffs=0, out_type=HAAR_OUT_F32, out_layout=HAAR_LAYOUT_SCK, start_level=0):
        self.desc = HaarShiftDesc(height, width, channels, kind, boundary, max_shifts, out_coeffs,
                                  out_type, out_layout, start_level)
        h = ctypes.c_void_p()
        _check(lib().haar_shift_plan(ctypes.byref(self.desc), ctypes.byref(h)))
        self.handle = h.value
        self.H, self.W, self.C = height, width, channels
        self.N = height * width
        self.start_level = start_level
        self.K = out_coeffs or (self.N >> (2 * start_level))
        self.kind, self.out_type, self.out_layout = kind, out_type, out_layout

    def close(self):
        if getattr(self, "handle", None):
            lib().haar_shift_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def status(self, reset=False):
        """Device status bits of the plan's kernels (0 = fine; bit 1 << 4: a
        bounded wait gave up).  Synchronises the device."""
        v = ctypes.c_int(0)
        _check(lib().haar_shift_plan_status(self.handle, ctypes.byref(v), 1 if reset else 0))
        return v.value

    def out_shape(self, S):
        """Shape of haar_shift's output tensor for S shifts."""
        planes = 2 if self.out_type == HAAR_OUT_BF16_HILO else 1
        if self.out_layout == HAAR_LAYOUT_SCK:
            shp = (S, self.C, self.K)
        elif self.out_layout == HAAR_LAYOUT_SKC4:
            shp = (S, self.K, 4)
        elif self.out_layout == HAAR_LAYOUT_SKC:
            shp = (S, self.K, self.C)
        else:
            shp = (self.K, S, self.C)
        return ((planes,) + shp) if planes == 2 else shp

    def out_dtype(self):
        import torch
        return {HAAR_OUT_F32: torch.float32, HAAR_OUT_BF16_HILO: torch.bfloat16,
                HAAR_OUT_F16: torch.float16}[self.out_type]


def haar_shift_plan(height, width, channels, **kw) -> Plan:
    return Plan(height, width, channels, **kw)


def haar_shift_plan_destroy(plan: Plan):
    plan.close()


def haar_shift(plan: Plan, coeffs_in, params, coeffs_out=None, stream=None):
    """Shifted coefficients of coeffs_in [C][N] for params [S][2|9|3] (float64)."""
    import torch
    S = params.shape[0]
    if coeffs_out is None:
        coeffs_out = torch.empty(plan.out_shape(S), dtype=plan.out_dtype(), device=coeffs_in.device)
    _check(lib().haar_shift(plan.handle, _dev(coeffs_in, torch.float32, "coeffs_in"),
                            _dev(params, torch.float64, "params"), S, _dev(coeffs_out, None, "coeffs_out"),
                            _stream(stream)))
    return coeffs_out


def haar_forward(maps, out=None, scale=1.0, stream=None):
    """Haar coefficients [B][N] of maps [B][H][W] (float32)."""
    import torch
    B, H, W = maps.shape
    if out is None:
        out = torch.empty((B, H * W), dtype=torch.float32, device=maps.device)
    _check(lib().haar_forward(H, W, B, _dev(maps, torch.float32, "maps"), _dev(out, torch.float32, "out"),
                              float(scale), _stream(stream)))
    return out


def haar_inverse(coeffs, H, W, out=None, stream=None):
    import torch
    B = coeffs.shape[0]
    if out is None:
        out = torch.empty((B, H, W), dtype=torch.float32, device=coeffs.device)
    _check(lib().haar_inverse(H, W, B, _dev(coeffs, torch.float32, "coeffs"), _dev(out, torch.float32, "out"),
                              _stream(stream)))
    return out


class Transport:
    """Device transport storage and its haar_transport_desc_t."""

    def __init__(self, kind, V, K, vals, idx=None, rowptr=None, bins=0, bin_of=None):
        self.kind, self.V, self.K, self.bins = kind, V, K, bins
        self.vals, self.idx, self.rowptr, self.bin_of = vals, idx, rowptr, bin_of
        for name in ("vals", "idx", "rowptr", "bin_of"):
            t = getattr(self, name)
            if t is not None:
                _dev(t, None, name)

    def desc(self) -> HaarTransportDesc:
        return HaarTransportDesc(self.kind, self.V, self.K, self.bins, _ptr(self.vals), _ptr(self.idx),
                                 _ptr(self.rowptr), _ptr(self.bin_of))


def shade_vertices(plan: Plan, transport: Transport, lighting, S, radiance=None, stream=None):
    """radiance [V][S][C] = sum_k T[v][k] L'[s][c][k]; radiance may be a
    pinned host tensor (written by the kernel over the host link)."""
    import torch
    if radiance is None:
        radiance = torch.empty((transport.V, S, plan.C), dtype=torch.float32, device=lighting.device)
    d = transport.desc()
    _check(lib().shade_vertices(plan.handle, ctypes.byref(d), _dev(lighting, None, "lighting"), S,
                                _out(radiance, torch.float32, "radiance"), _stream(stream)))
    return radiance


def shade_batch(plan: Plan, coeffs_in, params, transport: Transport, radiance=None, stream=None):
    """haar_shift then shade_vertices, the shifted lighting kept in the plan."""
    import torch
    S = params.shape[0]
    if radiance is None:
        radiance = torch.empty((transport.V, S, plan.C), dtype=torch.float32, device=coeffs_in.device)
    d = transport.desc()
    _check(lib().shade_batch(plan.handle, _dev(coeffs_in, torch.float32, "coeffs_in"),
                             _dev(params, torch.float64, "params"), S, ctypes.byref(d),
                             _out(radiance, torch.float32, "radiance"), _stream(stream)))
    return radiance


def haar_transport_group(V, N, rowptr, idx, vals, stream=None):
    """Vertex-group CSR (Transport of kind HAAR_T_GCSR_F32_U16) from top-K CSR."""
    import torch
    G = (V + GROUP - 1) // GROUP
    gptr = torch.empty(G + 1, dtype=torch.int32, device=rowptr.device)
    st = _stream(stream)
    _check(lib().haar_transport_group(V, N, _dev(rowptr, torch.int32, "rowptr"), _dev(idx, None, "idx"),
                                      _dev(vals, torch.float32, "vals"), gptr.data_ptr(), None, None, st))
    total = int(gptr[-1].item())
    gidx = torch.empty(max(total, 1), dtype=torch.int16, device=rowptr.device)
    gvals = torch.empty((max(total, 1), GROUP), dtype=torch.float32, device=rowptr.device)
    _check(lib().haar_transport_group(V, N, rowptr.data_ptr(), idx.data_ptr(), vals.data_ptr(), gptr.data_ptr(),
                                      gidx.data_ptr(), gvals.data_ptr(), st))
    return Transport(HAAR_T_GCSR_F32_U16, V, 0, gvals, gidx, gptr)


def haar_view_bins(pos, nrm, cams, bin_dirs, out=None, stream=None):
    """bin_of [S][V] uint8: the view bin of every (s, v)."""
    import torch
    V, S, bins = pos.shape[0], cams.shape[0], bin_dirs.shape[0]
    if out is None:
        out = torch.empty((S, V), dtype=torch.uint8, device=pos.device)
    _check(lib().haar_view_bins(V, S, bins, _dev(pos, torch.float32, "pos"), _dev(nrm, torch.float32, "nrm"),
                                _dev(cams, torch.float32, "cams"), _dev(bin_dirs, torch.float32, "bin_dirs"),
                                _dev(out, torch.uint8, "bin_of"), _stream(stream)))
    return out


def haar_normal_rotations(normals, out=None, stream=None):
    """Rotation records [V][9] float64 (HAAR_SHIFT_ROTATE parameters) that
    carry a local-frame map (normal at the +y pole) onto each normal."""
    import torch
    V = normals.shape[0]
    if out is None:
        out = torch.empty((V, 9), dtype=torch.float64, device=normals.device)
    _check(lib().haar_normal_rotations(V, _dev(normals, torch.float32, "normals"), _dev(out, torch.float64, "params"),
                                       _stream(stream)))
    return out


def haar_triple_work_floats(H, W, C):
    n = lib().haar_triple_work_floats(H, W, C)
    if n < 0:
        raise HaarError(HAAR_ERR_INVALID_ARG, f"no triple-product workspace for {H}x{W}, C={C}")
    return n


def haar_triple_product(H, W, light, brdf, vis, out=None, work=None, stream=None):
    """out [V][C]: the Haar triple product of lighting [C][N] with each
    vertex's BRDF row and visibility row ([V][>=N] float32, rows 16-byte aligned)."""
    import torch
    C, V = light.shape[0], brdf.shape[0]
    if vis.shape[0] != V:
        raise ValueError("brdf and vis need the same number of rows")
    for name, t in (("brdf", brdf), ("vis", vis)):
        if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32:
            raise TypeError(f"{name} must be a float32 CUDA tensor")
        if t.dim() != 2 or t.stride(1) != 1:
            raise ValueError(f"{name} must be [V][>=N] with unit column stride")
    if out is None:
        out = torch.empty((V, C), dtype=torch.float32, device=light.device)
    if work is None:
        work = torch.empty(haar_triple_work_floats(H, W, C), dtype=torch.float32, device=light.device)
    _check(lib().haar_triple_product(H, W, C, V, _dev(light, torch.float32, "light"), brdf.data_ptr(),
                                     brdf.stride(0), vis.data_ptr(), vis.stride(0), _dev(out, torch.float32, "out"),
                                     _dev(work, torch.float32, "work"), _stream(stream)))
    return out


def haar_shade_triple_work_floats(H, W, C):
    n = lib().haar_shade_triple_work_floats(H, W, C)
    if n < 0:
        raise HaarError(HAAR_ERR_INVALID_ARG, f"no shading-loop workspace for {H}x{W}, C={C}")
    return n


def haar_shade_triple(H, W, light, brdf_local, params, vis, out=None, work=None, stream=None):
    """out [V][C]: the rotation pass and the triple product fused; light [C][N],
    brdf_local [N] (local frame), params [V][9] float64 rotation records,
    vis [V][>=N] float32 rows (16-byte aligned)."""
    import torch
    C, V = light.shape[0], params.shape[0]
    if vis.shape[0] != V:
        raise ValueError("params and vis need the same number of rows")
    if not isinstance(vis, torch.Tensor) or not vis.is_cuda or vis.dtype != torch.float32:
        raise TypeError("vis must be a float32 CUDA tensor")
    if vis.dim() != 2 or vis.stride(1) != 1:
        raise ValueError("vis must be [V][>=N] with unit column stride")
    if out is None:
        out = torch.empty((V, C), dtype=torch.float32, device=light.device)
    if work is None:
        work = torch.empty(haar_shade_triple_work_floats(H, W, C), dtype=torch.float32, device=light.device)
    _check(lib().haar_shade_triple(H, W, C, V, _dev(light, torch.float32, "light"),
                                   _dev(brdf_local, torch.float32, "brdf_local"), _dev(params, torch.float64, "params"),
                                   vis.data_ptr(), vis.stride(0), _dev(out, torch.float32, "out"),
                                   _dev(work, torch.float32, "work"), _stream(stream)))
    return out


class Raster:
    """Device buffers of a headless rasteriser for a width x height image and
    V vertices; rasterize() fills tri_id [H][W] and bary [H][W][2]."""

    def __init__(self, width, height, V, device="cuda"):
        import torch
        self.width, self.height, self.V = width, height, V
        self.screen = torch.empty((max(V, 1), 4), dtype=torch.float32, device=device)
        self.zbuf = torch.empty((height, width), dtype=torch.int64, device=device)
        self.tri_id = torch.empty((height, width), dtype=torch.int32, device=device)
        self.bary = torch.empty((height, width, 2), dtype=torch.float32, device=device)

    def rasterize(self, pos, tris, view_proj, stream=None):
        import torch
        V, T = pos.shape[0], tris.shape[0]
        if V > self.V:
            raise ValueError(f"{V} vertices > {self.V}")
        _check(lib().haar_rasterize(V, _dev(pos, torch.float32, "pos"), T, _dev(tris, torch.int32, "tris"),
                                    _dev(view_proj, torch.float32, "view_proj"), self.width, self.height,
                                    self.screen.data_ptr(), self.zbuf.data_ptr(), self.tri_id.data_ptr(),
                                    self.bary.data_ptr(), _stream(stream)))
        return self.tri_id, self.bary

    def shade(self, tris, vert_rad, background, image=None, stream=None):
        """image [H][W][C]: per-vertex radiance [V][C] interpolated per pixel."""
        import torch
        C = vert_rad.shape[1]
        if image is None:
            image = torch.empty((self.height, self.width, C), dtype=torch.float32, device=vert_rad.device)
        _check(lib().haar_shade_pixels(self.width, self.height, C, vert_rad.shape[0], tris.shape[0],
                                       self.tri_id.data_ptr(), self.bary.data_ptr(), _dev(tris, torch.int32, "tris"),
                                       _dev(vert_rad, torch.float32, "vert_rad"),
                                       _dev(background, torch.float32, "background"),
                                       _dev(image, torch.float32, "image"), _stream(stream)))
        return image


class Surrogate:
    """haar_mlp_t: the transport-surrogate MLP (training and fused shading)."""

    N_IN, WIDTH, N_OUT, N_RAW = 320, 256, 512, 9

    def __init__(self, max_batch=8192, max_rows=262144, max_groups=64):
        h = ctypes.c_void_p()
        _check(lib().haar_mlp_create(max_batch, max_rows, max_groups, ctypes.byref(h)))
        self.handle = h.value
        self.n_params = int(lib().haar_mlp_param_count())

    def close(self):
        if getattr(self, "handle", None):
            lib().haar_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, flat, stream=None):
        _check(lib().haar_mlp_set_params(self.handle, _dev(flat, None, "params"), _stream(stream)))

    def get_params(self, stream=None):
        import torch
        out = torch.empty(self.n_params, dtype=torch.float32, device="cuda")
        _check(lib().haar_mlp_get_params(self.handle, out.data_ptr(), _stream(stream)))
        return out

    def forward(self, raw, out=None, stream=None):
        import torch
        B = raw.shape[0]
        if out is None:
            out = torch.empty((B, self.N_OUT), dtype=torch.float32, device=raw.device)
        _check(lib().haar_mlp_forward(self.handle, _dev(raw, torch.float32, "raw"), B,
                                      _dev(out, torch.float32, "out"), _stream(stream)))
        return out

    def grads(self, raw, target, stream=None):
        import torch
        g = torch.empty(self.n_params, dtype=torch.float32, device=raw.device)
        loss = torch.zeros(1, dtype=torch.float32, device=raw.device)
        _check(lib().haar_mlp_grads(self.handle, _dev(raw, torch.float32, "raw"), _dev(target, torch.float32, "target"),
                                    raw.shape[0], g.data_ptr(), loss.data_ptr(), _stream(stream)))
        return g, loss

    def train_step(self, raw, target, lr, loss=None, stream=None):
        import torch
        if loss is None:
            loss = torch.zeros(1, dtype=torch.float32, device=raw.device)
        _check(lib().haar_mlp_train_step(self.handle, _dev(raw, torch.float32, "raw"),
                                         _dev(target, torch.float32, "target"), raw.shape[0], float(lr),
                                         loss.data_ptr(), _stream(stream)))
        return loss

    def capture_train_step(self, raw, target, lr):
        """A CUDA graph of one training step on the fixed buffers raw / target
        (copy each new batch into them, then replay()); returns (graph, loss)."""
        import torch
        loss = torch.zeros(1, dtype=torch.float32, device=raw.device)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            self.train_step(raw, target, lr, loss)
        return graph, loss

    def shade(self, pos, nrm, cams, mu, sigma, idx, lighting, C, strides, radiance=None, stream=None):
        """radiance [V][S][C]; strides = (st_s, st_c, st_k) of the float32 lighting."""
        import torch
        V, S = pos.shape[0], cams.shape[0]
        if radiance is None:
            radiance = torch.empty((V, S, C), dtype=torch.float32, device=pos.device)
        _check(lib().haar_mlp_shade(self.handle, V, S, _dev(pos, torch.float32, "pos"), _dev(nrm, torch.float32, "nrm"),
                                    _dev(cams, torch.float32, "cams"), _dev(mu, torch.float32, "mu"),
                                    _dev(sigma, torch.float32, "sigma"), _dev(idx, torch.int32, "idx"),
                                    _dev(lighting, torch.float32, "lighting"), C, int(strides[0]), int(strides[1]),
                                    int(strides[2]), _dev(radiance, torch.float32, "radiance"), _stream(stream)))
        return radiance

    def status(self) -> int:
        v = ctypes.c_int(0)
        _check(lib().haar_mlp_status(self.handle, ctypes.byref(v)))
        return v.value


def version() -> str:
    return lib().haar_version().decode()
