"""The C ABI without a GPU: the library builds, loads, exports every entry
point the headers declare, and rejects bad arguments before any launch."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1705_07272_gb300 import build
    build.build()
    import paper_1705_07272_gb300 as hs
    return hs


def _declared():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        names += [n for n in re.findall(r"^HAAR_API\s+[\w\s\*]*?\b(\w+)\s*\(", txt, re.M)]
    return names


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 10
    L = lib.lib()
    for n in names:
        assert hasattr(L, n), n
        assert n in lib.EXPORTS, n


def test_version(lib):
    assert "sm_103a" in lib.version()


def _desc(lib, **kw):
    d = dict(height=32, width=64, channels=3, kind=0, boundary=0, max_shifts=4, out_coeffs=0,
             out_type=0, out_layout=0, start_level=0)
    d.update(kw)
    return lib.HaarShiftDesc(**d)


@pytest.mark.parametrize("bad", [dict(height=48), dict(height=1), dict(width=128), dict(width=16),
                                 dict(channels=0), dict(channels=65), dict(kind=7), dict(boundary=2),
                                 dict(max_shifts=0), dict(out_coeffs=-1), dict(out_coeffs=32 * 64 + 1),
                                 dict(out_type=3), dict(out_layout=5), dict(height=8192, width=8192),
                                 dict(start_level=-1), dict(start_level=5), dict(start_level=40),
                                 dict(start_level=2, out_coeffs=(32 * 64 >> 4) + 1)])
def test_plan_rejects_bad_descriptors(lib, bad):
    h = ctypes.c_void_p()
    st = lib.lib().haar_shift_plan(ctypes.byref(_desc(lib, **bad)), ctypes.byref(h))
    assert st == lib.HAAR_ERR_INVALID_ARG
    assert h.value is None
    assert lib.lib().haar_last_error()


@pytest.mark.parametrize("bad", [dict(out_type=1), dict(height=8, width=16), dict(start_level=2)])
def test_chain_route_rejects_what_it_does_not_support(lib, bad):
    # float32 output only; the tile kernel needs a map of at least 16 rows
    h = ctypes.c_void_p()
    st = lib.lib().haar_shift_plan(ctypes.byref(_desc(lib, kind=lib.HAAR_SHIFT_ROTATE_CHAIN, **bad)), ctypes.byref(h))
    assert st == lib.HAAR_ERR_UNSUPPORTED
    assert h.value is None


def test_null_arguments(lib):
    L = lib.lib()
    assert L.haar_shift_plan(None, None) == lib.HAAR_ERR_INVALID_ARG
    assert L.haar_shift(None, None, None, 1, None, None) == lib.HAAR_ERR_INVALID_ARG
    assert L.shade_vertices(None, None, None, 1, None, None) == lib.HAAR_ERR_INVALID_ARG
    assert L.shade_batch(None, None, None, 1, None, None, None) == lib.HAAR_ERR_INVALID_ARG
    assert L.haar_forward(48, 48, 1, None, None, 1.0, None) == lib.HAAR_ERR_INVALID_ARG
    assert L.haar_forward(32, 32, 1, None, None, 1.0, None) == lib.HAAR_ERR_INVALID_ARG
    assert L.haar_forward(32, 32, 1, 8, 16, 1.0, None) == lib.HAAR_ERR_INVALID_ARG      # misaligned
    assert L.haar_forward(32, 32, 0, None, None, 1.0, None) == lib.HAAR_OK            # empty batch
    assert L.haar_inverse(32, 96, 1, None, None, None) == lib.HAAR_ERR_INVALID_ARG
    assert L.haar_view_bins(10, 1, 0, None, None, None, None, None, None) == lib.HAAR_ERR_INVALID_ARG
    assert L.haar_view_bins(0, 1, 16, None, None, None, None, None, None) == lib.HAAR_OK
    assert L.haar_shift_plan_destroy(None) == lib.HAAR_OK


def test_fault_injection(lib, monkeypatch):
    L = lib.lib()
    monkeypatch.setenv("HAAR_FAULT_INJECT", "haar_forward,shade_batch")
    assert L.haar_forward(32, 32, 1, None, None, 1.0, None) == lib.HAAR_ERR_INJECTED
    assert b"injected" in L.haar_last_error()
    assert L.shade_batch(None, None, None, 1, None, None, None) == lib.HAAR_ERR_INJECTED
    assert L.haar_inverse(32, 96, 1, None, None, None) == lib.HAAR_ERR_INVALID_ARG
    monkeypatch.setenv("HAAR_FAULT_INJECT", "*")
    h = ctypes.c_void_p()
    assert L.haar_shift_plan(ctypes.byref(_desc(lib)), ctypes.byref(h)) == lib.HAAR_ERR_INJECTED
    monkeypatch.delenv("HAAR_FAULT_INJECT")
    assert L.haar_forward(48, 48, 1, None, None, 1.0, None) == lib.HAAR_ERR_INVALID_ARG


def test_binding_rejects_host_tensors(lib):
    import torch
    with pytest.raises(ValueError):
        lib._dev(torch.zeros(4), torch.float32, "x")


@pytest.mark.parametrize("args,err", [
    (dict(H=128, W=128), "UNSUPPORTED"),          # N > 8192
    (dict(H=12, W=24), "INVALID_ARG"),
    (dict(H=16, W=64), "INVALID_ARG"),
    (dict(C=0), "INVALID_ARG"), (dict(C=5), "INVALID_ARG"), (dict(V=-1), "INVALID_ARG"),
    (dict(sb=100), "INVALID_ARG"),                # shorter than N
    (dict(sb=514), "INVALID_ARG"),                # not a multiple of 4
    (dict(brdf=0x1008), "INVALID_ARG"),           # not 16-byte aligned
    (dict(work=0x1004), "INVALID_ARG"),
    (dict(light=0), "INVALID_ARG"),
])
def test_triple_product_rejects_bad_arguments(lib, args, err):
    # validation happens before any launch, so fake device addresses suffice
    a = dict(H=16, W=32, C=3, V=4, light=0x1000, brdf=0x2000, sb=512, vis=0x3000, sv=512, out=0x4000, work=0x5000)
    a.update(args)
    st = lib.lib().haar_triple_product(a["H"], a["W"], a["C"], a["V"], a["light"], a["brdf"], a["sb"], a["vis"],
                                       a["sv"], a["out"], a["work"], None)
    assert st == getattr(lib, "HAAR_ERR_" + err)
    assert lib.lib().haar_last_error()


def test_triple_work_size(lib):
    # 4 status floats + C means over the (N - q) / 3 squares (rounded up to 4)
    # + one float4 per square and channel
    nm = (2048 - 2) // 3
    assert lib.lib().haar_triple_work_floats(32, 64, 3) == 4 + ((3 * nm + 3) & ~3) + 4 * 3 * nm
    assert lib.lib().haar_triple_work_floats(128, 128, 3) == -1
    assert lib.lib().haar_triple_work_floats(32, 64, 5) == -1


def test_normal_rotations_rejects_bad_arguments(lib):
    L = lib.lib()
    assert L.haar_normal_rotations(-1, 0x1000, 0x2000, None) == lib.HAAR_ERR_INVALID_ARG
    assert L.haar_normal_rotations(4, 0, 0x2000, None) == lib.HAAR_ERR_INVALID_ARG
    assert L.haar_normal_rotations(4, 0x1000, 0x2004, None) == lib.HAAR_ERR_INVALID_ARG
    assert L.haar_normal_rotations(0, 0, 0, None) == lib.HAAR_OK


@pytest.mark.parametrize("args,err", [
    (dict(H=128, W=128), "UNSUPPORTED"), (dict(H=16, W=64), "INVALID_ARG"), (dict(C=5), "INVALID_ARG"),
    (dict(sv=510), "INVALID_ARG"), (dict(vis=0x3004), "INVALID_ARG"), (dict(params=0x6004), "INVALID_ARG"),
    (dict(brdf=0), "INVALID_ARG"),
])
def test_shade_triple_rejects_bad_arguments(lib, args, err):
    a = dict(H=16, W=32, C=3, V=4, light=0x1000, brdf=0x2000, params=0x6000, vis=0x3000, sv=512, out=0x4000,
             work=0x5000)
    a.update(args)
    st = lib.lib().haar_shade_triple(a["H"], a["W"], a["C"], a["V"], a["light"], a["brdf"], a["params"], a["vis"],
                                     a["sv"], a["out"], a["work"], None)
    assert st == getattr(lib, "HAAR_ERR_" + err)
    assert lib.lib().haar_shade_triple_work_floats(16, 32, 3) > 0


def test_raster_rejects_bad_arguments(lib):
    L = lib.lib()
    ok = dict(V=3, pos=0x1000, T=1, tris=0x2000, M=0x3000, w=16, h=16, screen=0x4000, zbuf=0x5000, tid=0x6000,
              bary=0x7000)
    for bad in (dict(w=0), dict(h=20000), dict(V=-1), dict(T=-2), dict(pos=0), dict(M=0), dict(screen=0x4008),
                dict(zbuf=0x5004), dict(bary=0x7004)):
        a = dict(ok, **bad)
        st = L.haar_rasterize(a["V"], a["pos"], a["T"], a["tris"], a["M"], a["w"], a["h"], a["screen"], a["zbuf"],
                              a["tid"], a["bary"], None)
        assert st == lib.HAAR_ERR_INVALID_ARG, bad
    assert L.haar_shade_pixels(16, 16, 0, 3, 1, 0x1000, 0x2000, 0x3000, 0x4000, 0x5000, 0x6000, None) == \
        lib.HAAR_ERR_INVALID_ARG
    assert L.haar_shade_pixels(16, 16, 3, 3, 1, 0x1000, 0x2004, 0x3000, 0x4000, 0x5000, 0x6000, None) == \
        lib.HAAR_ERR_INVALID_ARG
