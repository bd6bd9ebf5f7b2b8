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


def _prox(L, z=256, nx=64, ny=64, ns=1, lam=0.1, n_inner=20, tau=0.125, x=1 << 20, ws=1024, wsb=BIG, gap=None):
    return L.lib.pyhst_tv_prox(z, nx, ny, ns, lam, n_inner, tau, x, gap, ws, wsb, None)


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
    f = L.lib.pyhst_cnn_forward      # argument types as the binding declares them
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


def _geom(L, **kw):
    d = dict(n_angles=180, n_bins=256, nx=256, ny=256, n_slices=1, angles=8, axis=8, cx=127.5, cy=127.5,
             pixel_size=2 / 256)
    d.update(kw)
    return L.pyhst_geometry(**d)


def _opts(L, **kw):
    d = dict(beta=0.1, n_iter=5, n_inner=20, tau=0.125, use_fista=1, warm_start=0, lipschitz=0.0, n_power_iter=10)
    d.update(kw)
    return L.pyhst_tv_opts(**d)


def test_tv_batch_argument_checks(L):
    o = _opts(L)
    items = (L.pyhst_tv_item * 2)()
    for it in items:
        it.geom, it.sino, it.x, it.energy, it.beta = _geom(L), 1024, 2048, None, -1.0
    call = lambda n=2, wsb=BIG: L.lib.pyhst_tv_solve_batch(items, n, ctypes.byref(o), None, 256, wsb, None)
    E = L.PYHST_ERR_INVALID_ARG
    assert call(n=0) == E
    items[1].sino = None
    assert call() == E and L.lib.pyhst_last_error().decode().startswith("item 1:")
    items[1].sino = 1024
    items[1].beta = float("nan")
    assert call() == E
    items[1].beta = -1.0
    items[1].geom = _geom(L, nx=0)
    assert call() == E
    assert L.lib.pyhst_last_error().decode() == "item 1: image 0 x 256 outside [1, 16384]^2"
    items[1].geom = _geom(L)
    o.warm_dual = 2
    assert call() == E and "warm_dual" in L.lib.pyhst_last_error().decode()
    o.warm_dual = 0
    assert call(wsb=64) == L.PYHST_ERR_WORKSPACE


def test_beta_scan_argument_checks(L):
    g, o = _geom(L), _opts(L)
    betas = (ctypes.c_float * 3)(1e-5, 1e-3, 1e-2)
    call = lambda b=betas, n=3, held=5, cv=None: L.lib.pyhst_beta_scan(ctypes.byref(g), 1024, b, n, held,
                                                                       ctypes.byref(o), 2048, cv, None, 256, BIG,
                                                                       None)
    E = L.PYHST_ERR_INVALID_ARG
    assert call(n=0) == E
    assert call(held=180) == E and call(held=-2) == E       # an angle index of the 180, or -1
    assert call(held=-1, cv=4096) == E                      # cross-validation needs a held-out angle
    assert call(b=None) == E
    assert call(b=(ctypes.c_float * 3)(1e-5, -1e-3, 1e-2)) == E


def test_cnn_training_argument_checks(L):
    E = L.PYHST_ERR_INVALID_ARG
    assert L.lib.pyhst_cnn_grad(256, 512, 768, 0, 64, 64, 1024, None, 2048, BIG, None) == E
    assert L.lib.pyhst_cnn_grad(256, None, 768, 1, 64, 64, 1024, None, 2048, BIG, None) == E
    adam = lambda count=100, step=1, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8: L.lib.pyhst_cnn_adam(
        256, 512, 768, 1024, count, step, lr, b1, b2, eps, None)
    assert adam(step=0) == E and adam(count=0) == E
    assert adam(lr=0.0) == E and adam(b1=1.0) == E and adam(b2=1.0) == E and adam(eps=0.0) == E


def test_patch_argument_checks(L):
    E = L.PYHST_ERR_INVALID_ARG
    pp = lambda **kw: L.pyhst_patch_problem(**{**dict(ny=64, nx=64, m=8, stride=4, n_atoms=64, dict=4096,
                                                      rho=1.0), **kw})
    image = lambda p, wsb=BIG: L.lib.pyhst_patch_image(ctypes.byref(p) if p else None, 256, 512, 1024, wsb, None)
    assert image(None) == E
    assert image(pp(n_atoms=2048)) == E          # n_atoms x m^2 above 65536
    assert image(pp(m=32, stride=4)) == E        # patches above 16 x 16
    assert image(pp(rho=-1.0)) == E
    assert image(pp(dict=None)) == E
    assert image(pp(), wsb=16) == L.PYHST_ERR_WORKSPACE
    gp = _geom(L, nx=64, ny=64, n_bins=64)
    solve = lambda beta=0.1, n_iter=5: L.lib.pyhst_patch_solve(ctypes.byref(pp()), ctypes.byref(gp), 256, beta, 0.0,
                                                               10, n_iter, 1, 512, None, None, None, 1024, BIG, None)
    assert solve(n_iter=0) == E and solve(beta=-0.1) == E
    other = _geom(L, nx=128, ny=128, n_bins=64)
    assert L.lib.pyhst_patch_gradient(ctypes.byref(pp()), ctypes.byref(other), 256, 512, 768, None, 1024, BIG,
                                      None) == E


def test_capture_pnp_profile_and_tuning_checks(L):
    g, o = _geom(L), _opts(L)
    E = L.PYHST_ERR_INVALID_ARG
    iters = (ctypes.c_int32 * 2)(1, 9)                    # 9 > n_iter = 5
    assert L.lib.pyhst_tv_solve_capture(ctypes.byref(g), 1024, ctypes.byref(o), 2048, 2, iters, 4096, 256, BIG,
                                        None) == E
    assert L.lib.pyhst_pnp_solve(ctypes.byref(g), 1024, None, ctypes.byref(o), 2048, None, None, 256, BIG,
                                 None) == E
    d, n = ctypes.c_double(), ctypes.c_int64()
    assert L.lib.pyhst_profile_read(b"nonsense", ctypes.byref(d), ctypes.byref(n)) == E
    assert L.lib.pyhst_set_tv_prox_steps(64, 64, 7) == E   # supported: 2, 3, 4, 5, 6, 8


def test_fbp_pre_and_host_argument_checks(L):
    g = _geom(L, n_slices=2)
    E = L.PYHST_ERR_INVALID_ARG
    ok = dict(n_flats=2, flats=4096, flat_pos=8192, hotspot_threshold=0.0, ring_window=0)
    pre = lambda kind=0, wsb=BIG, **kw: L.lib.pyhst_fbp_pre(
        ctypes.byref(g), kind, 256, 256, 512, 8, ctypes.byref(L.pyhst_preproc(**{**ok, **kw})), 0, 0, 512, 1024,
        wsb, None)
    assert pre(kind=L.PYHST_F32_SINO) == E              # raw counts only
    assert pre(n_flats=0, flats=None, flat_pos=None) == E
    assert pre(flats=None) == E
    assert pre(hotspot_threshold=-1.0) == E
    assert pre(ring_window=2) == E                      # 0 or odd >= 3
    assert pre(wsb=16) == L.PYHST_ERR_WORKSPACE
    assert L.lib.pyhst_fbp_pre(ctypes.byref(g), 0, 256, 256, 512, 8, None, 0, 0, 512, 1024, BIG, None) == E
    host = lambda data=256, flat=8, spc=16, wsb=BIG: L.lib.pyhst_fbp_host(
        ctypes.byref(g), 0, data, 256, 512, flat, 8, 0, 0, 4096, spc, 1024, wsb, None)
    assert host(spc=0) == E and host(data=None) == E and host(flat=None) == E
    assert host(wsb=16) == L.PYHST_ERR_WORKSPACE


def test_microbench_argument_checks(L):
    """Invalid kinds, iteration counts and pointers are refused before any
    launch."""
    units = ctypes.c_double()
    E = L.PYHST_ERR_INVALID_ARG
    assert L.lib.pyhst_microbench(4, 10, 256, ctypes.byref(units), None) == E
    assert L.lib.pyhst_microbench(-1, 10, 256, ctypes.byref(units), None) == E
    assert L.lib.pyhst_microbench(0, 0, 256, ctypes.byref(units), None) == E
    assert L.lib.pyhst_microbench(1, 10, None, ctypes.byref(units), None) == E
    assert L.lib.pyhst_microbench(2, 10, 256, None, None) == E
