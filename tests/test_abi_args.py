"""Host-side argument checks of entry points beyond the FBP and the solver
(no GPU: every call here returns before any launch), and the binding's
refusal of host tensors (there is no CPU fallback)."""
import ctypes

import pytest
import torch

BIG = 1 << 30


@pytest.fixture(scope="module")
def L():
    from paper_1306_1392_b300 import _lib as L
    return L


def _prox(L, z=256, nx=64, ny=64, ns=1, lam=0.1, n_inner=20, tau=0.125, x=1 << 20, ws=1024, wsb=BIG):
    f = L.lib.pyhst_tv_prox
    f.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_float, ctypes.c_int32,
                  ctypes.c_float, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]
    return f(z, nx, ny, ns, lam, n_inner, tau, x, ws, wsb, None)


def test_tv_prox_argument_checks(L):
    E = L.PYHST_ERR_INVALID_ARG
    assert _prox(L, nx=0) == E
    assert _prox(L, ny=16385) == E
    assert _prox(L, z=None) == E
    assert _prox(L, n_inner=0) == E
    assert _prox(L, lam=-0.1) == E
    assert _prox(L, lam=float("nan")) == E
    assert _prox(L, tau=0.0) == E and _prox(L, tau=0.3) == E
    assert _prox(L, wsb=16) == L.PYHST_ERR_WORKSPACE


def test_tv_prox_rejects_overlapping_output(L):
    """x = z - lam div p is written while other tiles still read z."""
    n = 64 * 64 * 4
    assert _prox(L, z=1 << 20, x=1 << 20) == L.PYHST_ERR_INVALID_ARG
    assert "overlaps" in L.lib.pyhst_last_error().decode()
    assert _prox(L, z=1 << 20, x=(1 << 20) + n - 4) == L.PYHST_ERR_INVALID_ARG
    assert _prox(L, z=(1 << 20) + n - 4, x=1 << 20) == L.PYHST_ERR_INVALID_ARG


def test_cnn_forward_argument_checks(L):
    f = L.lib.pyhst_cnn_forward
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                  ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]
    E = L.PYHST_ERR_INVALID_ARG
    assert f(256, 512, 1024, 0, 64, 64, 2048, BIG, None) == E
    assert f(256, 512, 1024, 1, 16385, 64, 2048, BIG, None) == E
    assert f(None, 512, 1024, 1, 64, 64, 2048, BIG, None) == E
    assert f(256, 512, 1024, 1, 64, 64, 2048, 16, None) == L.PYHST_ERR_WORKSPACE


def test_patch_grid_counts_and_checks(L):
    """Patches per axis of the grid at step `stride` that covers the image
    (host arithmetic only): 2048^2 with 8 x 8 patches at stride 4 gives the
    511 x 511 = 261,121 patches of the patch study."""
    f = L.lib.pyhst_patch_grid
    f.argtypes = [ctypes.c_int32] * 4 + [ctypes.POINTER(ctypes.c_int32)] * 2
    kr, kc = ctypes.c_int32(), ctypes.c_int32()
    assert f(2048, 2048, 8, 4, ctypes.byref(kr), ctypes.byref(kc)) == 0
    assert (kr.value, kc.value) == (511, 511)
    assert f(8, 8, 8, 8, ctypes.byref(kr), ctypes.byref(kc)) == 0 and (kr.value, kc.value) == (1, 1)
    E = L.PYHST_ERR_INVALID_ARG
    assert f(4, 77, 8, 3, ctypes.byref(kr), ctypes.byref(kc)) == E      # patch larger than the image
    assert f(100, 77, 8, 0, ctypes.byref(kr), ctypes.byref(kc)) == E    # zero step
    assert f(100, 77, 8, 9, ctypes.byref(kr), ctypes.byref(kc)) == E    # step beyond the patch: gaps


def test_binding_refuses_host_tensors():
    import paper_1306_1392_b300 as P
    with pytest.raises(TypeError, match="CUDA tensor"):
        P.Geometry(torch.zeros(4), torch.zeros(4), 8, 8, 8, 0.1)
    with pytest.raises(TypeError, match="CUDA tensor"):
        P.pyhst_tv_prox(torch.zeros((8, 8)), 0.1)
    with pytest.raises(TypeError, match="CUDA tensor"):
        P.pyhst_cnn_forward(torch.zeros(P.pyhst_cnn_param_count()), torch.zeros((1, 8, 8)))
