"""C-ABI checks that need no GPU: the library loads, exports every function
include/pyhst.h declares, sizes workspaces, and rejects bad arguments before
it touches the device (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_1306_1392_b300 import _lib
    return _lib


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(pyhst_\w+)\s*\(", src))
    return names


def test_exports_every_declared_symbol(L):
    declared = _declared()
    assert {"pyhst_fbp", "pyhst_backproject", "pyhst_project", "pyhst_tv_solve"} <= declared
    for name in sorted(declared):
        assert hasattr(L.lib, name), name
    bound = {n for n, _, _ in L.SIGNATURES}
    assert declared == bound, declared ^ bound


def test_library_is_built_for_sm103a(L):
    from paper_1306_1392_b300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert os.path.exists(L.LIB_PATH) and not build.stale()


def _geom(L, **kw):
    d = dict(n_angles=180, n_bins=256, nx=256, ny=256, n_slices=1, angles=8, axis=8, cx=127.5, cy=127.5,
             pixel_size=2 / 256)
    d.update(kw)
    return L.pyhst_geometry(**d)


def test_workspace_sizes(L):
    g = _geom(L)
    ws = lambda op: L.lib.pyhst_workspace_size(ctypes.byref(g), op)
    assert ws(L.PYHST_OP_BACKPROJECT) >= 180 * 32
    assert ws(L.PYHST_OP_PROJECT) >= 256 * 256 * 4
    assert ws(L.PYHST_OP_FBP) >= 180 * 256 * 4 + 512 * 8
    assert all(ws(op) % 256 == 0 for op in range(3))
    g4 = _geom(L, n_slices=16)
    assert L.lib.pyhst_workspace_size(ctypes.byref(g4), L.PYHST_OP_FBP) >= 4 * 180 * 256 * 4
    bad = _geom(L, n_angles=0)
    assert L.lib.pyhst_workspace_size(ctypes.byref(bad), L.PYHST_OP_FBP) == 0
    assert L.lib.pyhst_workspace_size(None, 0) == 0
    o = L.pyhst_tv_opts(0.1, 10, 20, 0.125, 1, 0, 0.0, 50)
    assert L.lib.pyhst_tv_workspace_size(ctypes.byref(g), ctypes.byref(o)) >= 6 * 256 * 256 * 4


@pytest.mark.parametrize("field,value,msg", [
    ("n_angles", 0, "n_angles"), ("n_bins", 0, "n_bins"), ("nx", 0, "image"), ("n_slices", 0, "n_slices"),
    ("angles", None, "angles"), ("pixel_size", 0.0, "pixel_size"), ("cx", float("nan"), "cx"),
])
def test_invalid_geometry_rejected_before_launch(L, field, value, msg):
    g = _geom(L, **{field: value})
    rc = L.lib.pyhst_backproject(ctypes.byref(g), 8, 8, 1.0, 256, 1 << 20, None)
    assert rc == L.PYHST_ERR_INVALID_ARG
    assert msg in L.lib.pyhst_last_error().decode()


def test_fbp_argument_checks(L):
    g = _geom(L)
    big = 1 << 30
    call = lambda **kw: L.lib.pyhst_fbp(ctypes.byref(g), kw.get("kind", 0), kw.get("data", 8), 256, 256,
                                        kw.get("flat", 8), kw.get("dark", 8), kw.get("filt", 0),
                                        kw.get("pad", 0), 8, kw.get("ws", 256), kw.get("wsb", big), None)
    assert call(kind=7) == L.PYHST_ERR_INVALID_ARG
    assert call(filt=3) == L.PYHST_ERR_INVALID_ARG
    assert call(data=None) == L.PYHST_ERR_INVALID_ARG
    assert call(flat=None) == L.PYHST_ERR_INVALID_ARG
    assert call(pad=500) == L.PYHST_ERR_INVALID_ARG          # not a power of two
    assert call(pad=256) == L.PYHST_ERR_INVALID_ARG          # < 2 n_bins
    assert call(pad=32768) == L.PYHST_ERR_INVALID_ARG        # > 16384
    assert call(ws=None) == L.PYHST_ERR_WORKSPACE
    assert call(ws=264) == L.PYHST_ERR_WORKSPACE             # misaligned
    assert call(wsb=1024) == L.PYHST_ERR_WORKSPACE
    assert "workspace" in L.lib.pyhst_last_error().decode()


def test_tv_argument_checks(L):
    g = _geom(L)
    ok = dict(beta=0.1, n_iter=5, n_inner=20, tau=0.125, use_fista=1, warm_start=0, lipschitz=0.0, n_power_iter=10)
    for k, v in [("beta", -1.0), ("n_iter", 0), ("n_inner", 0), ("tau", 0.0), ("tau", 0.3), ("lipschitz", -2.0),
                 ("n_power_iter", 0), ("warm_dual", 2), ("warm_dual", -1)]:
        o = L.pyhst_tv_opts(**{**ok, k: v})
        rc = L.lib.pyhst_tv_solve(ctypes.byref(g), 8, ctypes.byref(o), 8, None, None, None, 256, 1 << 30, None)
        assert rc == L.PYHST_ERR_INVALID_ARG, (k, v)
    o = L.pyhst_tv_opts(**ok)
    assert L.lib.pyhst_tv_solve(ctypes.byref(g), 8, ctypes.byref(o), 8, None, None, None, 256, 64, None) == \
        L.PYHST_ERR_WORKSPACE
