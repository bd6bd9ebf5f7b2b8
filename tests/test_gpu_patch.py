"""GPU parity of the overlapping-patch prior (Sec. 3.2.1, Eqs. 7-9,
Algorithm 1) against the FP64 oracle."""
import math

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / np.linalg.norm(b)


# (shape, m, stride, atoms): the dictionary products run on the tensor cores
# (split-bf16) when the padded B fits, else on the SIMT kernel (260 atoms:
# G = 2 P' D^T has N = 260 > 256); m = 3 with 10 atoms gives k = 9 and 10
# (scalar loads, one 16-k step in the last stage).
CASES = [((11, 9), 4, 3, 20), ((16, 16), 4, 2, 16), ((21, 34), 6, 4, 40), ((64, 64), 8, 4, 64),
         ((25, 19), 3, 2, 10), ((40, 36), 4, 2, 260), ((130, 70), 8, 4, 144)]


def _problem(orc, shape, m, stride, nc, tomo, seed, rho=0.8):
    import paper_1306_1392_b300 as P
    dev = torch.device("cuda:0")
    g = np.random.default_rng(seed)
    Dm = (orc.dct_dictionary(m) if nc == m * m and m == 8 else g.standard_normal((nc, m * m)) / m).astype(np.float32)
    ny, nx = shape
    geo = ogeo = None
    if tomo:
        na, nb = 13, max(shape) + 4
        ang = (np.arange(na) * math.pi / na + 0.05).astype(np.float32)
        ax = np.full(na, (nb - 1) / 2 - 0.3, np.float32)
        geo = P.Geometry(torch.from_numpy(ang).to(dev), torch.from_numpy(ax).to(dev), nb, nx, ny, 0.5)
        ogeo = orc.Geometry(ang.astype(np.float64), ax.astype(np.float64), nb, nx, ny, 0.5)
        y = g.standard_normal((na, nb)).astype(np.float32)
    else:
        y = g.standard_normal((ny, nx)).astype(np.float32)
    pp = P.PatchProblem(ny, nx, m, stride, torch.from_numpy(Dm).to(dev), rho)
    opp = orc.PatchProblem(ny, nx, m, stride, Dm.astype(np.float64), float(np.float32(rho)), g=ogeo)
    return pp, opp, geo, y, g


@pytest.mark.parametrize("shape,m,stride,nc", CASES)
def test_patch_image_matches_oracle(orc, shape, m, stride, nc):
    import paper_1306_1392_b300 as P
    pp, opp, _, _, g = _problem(orc, shape, m, stride, nc, False, 1)
    assert pp.grid() == (opp.kr, opp.kc)
    W = g.standard_normal(opp.shape_w).astype(np.float32)
    x = P.pyhst_patch_image(pp, torch.from_numpy(W).cuda()).cpu().numpy()
    ref = orc.patch_assemble(W.astype(np.float64) @ opp.Dm, *shape, m, stride)
    assert rel(x, ref) <= 1e-5


@pytest.mark.parametrize("tomo", [False, True])
@pytest.mark.parametrize("shape,m,stride,nc", CASES)
def test_patch_gradient_matches_oracle(orc, shape, m, stride, nc, tomo):
    """Algorithm 1 on the GPU (float32) against the oracle's: relative L2
    1e-5 on the gradient, 1e-5 on f (Eq. 8)."""
    import paper_1306_1392_b300 as P
    pp, opp, geo, y, g = _problem(orc, shape, m, stride, nc, tomo, 2 + nc)
    W = g.standard_normal(opp.shape_w).astype(np.float32)
    G, f = P.pyhst_patch_gradient(pp, geo, torch.from_numpy(W).cuda(), torch.from_numpy(y).cuda())
    Gr = opp.gradient(W.astype(np.float64), y.astype(np.float64))
    assert P.pyhst_device_status() == 0             # the tensor-core product's waits all completed
    assert rel(G.cpu().numpy(), Gr) <= 1e-5
    assert f.item() == pytest.approx(opp.f(W.astype(np.float64), y.astype(np.float64)), rel=1e-5)


@pytest.mark.parametrize("fista", [True, False])
@pytest.mark.parametrize("tomo", [False, True])
def test_patch_solve_matches_oracle(orc, fista, tomo):
    """20 ISTA/FISTA iterations with the same L (the oracle's power
    iteration on f's Hessian): coefficients and image within 1e-4 relative
    L2 (float32 rounding over the iterations), F history within 1e-5."""
    import paper_1306_1392_b300 as P
    shape, m, stride, nc = (24, 20), 4, 2, 20
    pp, opp, geo, y, g = _problem(orc, shape, m, stride, nc, tomo, 7)
    L = 1.01 * _power(opp, y.astype(np.float64))
    beta = 0.02
    W, x, e, lip = P.pyhst_patch_solve(pp, geo, torch.from_numpy(y).cuda(), beta, 20, lipschitz=L, use_fista=fista)
    Wr, er, Xr = opp.fista(y.astype(np.float64), beta, L, 20, use_fista=fista)
    assert lip.item() == L
    assert rel(W.cpu().numpy(), Wr) <= 1e-4
    assert rel(x.cpu().numpy(), Xr) <= 1e-4
    np.testing.assert_allclose(e.cpu().numpy(), er, rtol=1e-5)


def test_patch_gradient_full_size(orc):
    """The patch study's configuration: a 2048^2 image, 150 angles over
    180 degrees, 8 x 8 patches at stride 4 (261,121 patches), the 144-atom
    over-complete DCT: Algorithm 1's gradient and f (Eq. 8) for seeded
    coefficients against the oracle's, same bounds as the small cases (the
    oracle's gradient takes ~20-30 s here)."""
    import paper_1306_1392_b300 as P
    from synth.patches import overcomplete_dct
    n, na, m, stride = 2048, 150, 8, 4
    dev = torch.device("cuda:0")
    ang = (np.arange(na) * math.pi / na).astype(np.float32)
    ax = np.full(na, (n - 1) / 2.0, np.float32)
    geo = P.Geometry(torch.from_numpy(ang).to(dev), torch.from_numpy(ax).to(dev), n, n, n, 2.0 / n)
    ogeo = orc.Geometry(ang.astype(np.float64), ax.astype(np.float64), n, n, n, 2.0 / n)
    Dm = overcomplete_dct(m, 12).astype(np.float32)
    pp = P.PatchProblem(n, n, m, stride, torch.from_numpy(Dm).to(dev), 1.0)
    opp = orc.PatchProblem(n, n, m, stride, Dm.astype(np.float64), 1.0, g=ogeo)
    g = np.random.default_rng(31)
    W = g.standard_normal(opp.shape_w).astype(np.float32)
    y = g.standard_normal((na, n)).astype(np.float32)
    G, f = P.pyhst_patch_gradient(pp, geo, torch.from_numpy(W).to(dev), torch.from_numpy(y).to(dev))
    torch.cuda.synchronize()
    assert P.pyhst_device_status() == 0
    Wd, yd = W.astype(np.float64), y.astype(np.float64)
    assert rel(G.cpu().numpy(), opp.gradient(Wd, yd)) <= 1e-5
    assert f.item() == pytest.approx(opp.f(Wd, yd), rel=1e-5)


def _power(opp, y, iters=300):
    """Largest eigenvalue of f's constant Hessian (H v = grad f(v) - grad f(0))."""
    g0 = opp.gradient(np.zeros(opp.shape_w), y)
    v = np.ones(opp.shape_w)
    lam = 0.0
    for _ in range(iters):
        h = opp.gradient(v, y) - g0
        lam = np.vdot(v, h) / np.vdot(v, v)
        v = h / np.linalg.norm(h)
    return lam


def test_patch_step_size_estimate(orc):
    """The GPU's power iteration (from W = 1, 50 steps) approaches the top
    eigenvalue of f's Hessian from below."""
    import paper_1306_1392_b300 as P
    pp, opp, geo, y, _ = _problem(orc, (16, 16), 4, 2, 16, True, 9)
    lam = _power(opp, y.astype(np.float64), 2000)
    _, _, _, lip = P.pyhst_patch_solve(pp, geo, torch.from_numpy(y).cuda(), 0.0, 1, n_power_iter=50, energy=False)
    est = lip.item() / 1.01
    assert 0.95 * lam <= est <= lam * (1 + 1e-5)


def test_patch_rejects_bad_arguments():
    import paper_1306_1392_b300 as P
    from paper_1306_1392_b300 import _lib as L
    with pytest.raises(P.PyhstError):
        P.pyhst_patch_grid(8, 8, 4, 5)              # stride > m leaves gaps
    d = torch.zeros((4, 4), device="cuda")
    pp = P.PatchProblem(8, 8, 2, 2, d, 1.0)
    pc = pp.c()
    ws = torch.empty(16, dtype=torch.uint8, device="cuda")
    W = torch.zeros((16, 4), device="cuda")
    assert L.lib.pyhst_patch_image(ctypes_byref(pc), W.data_ptr(), d.data_ptr(), ws.data_ptr(), 16, None) == -3


def ctypes_byref(s):
    import ctypes
    return ctypes.byref(s)


def test_product_wait_give_up_is_reported_and_the_next_call_succeeds(orc):
    """As for the CNN: with pipeline waits that give up without polling the
    tensor-core patch product gives up, drains its issued operations, frees its tensor memory
    and records bit 1; with the default limit the next gradient matches the
    oracle and sets no bit."""
    import paper_1306_1392_b300 as P
    dev = torch.device("cuda:0")
    gen = np.random.default_rng(3)
    Dm = (gen.standard_normal((96, 64)) / 8).astype(np.float32)
    pp = P.PatchProblem(400, 400, 8, 4, torch.from_numpy(Dm).to(dev), 0.8)
    W = torch.from_numpy(gen.standard_normal(pp.coef_shape()).astype(np.float32)).to(dev)
    y = torch.from_numpy(gen.standard_normal((400, 400)).astype(np.float32)).to(dev)
    P.pyhst_device_status(clear=True)
    hit = 0
    try:
        P.pyhst_set_wait_limit(0)
        for _ in range(2):
            P.pyhst_patch_gradient(pp, None, W, y)
            torch.cuda.synchronize()
            hit |= P.pyhst_device_status(clear=True)
            if hit:
                break
    finally:
        P.pyhst_set_wait_limit(-1)
    assert hit & 1
    G, _ = P.pyhst_patch_gradient(pp, None, W, y)
    torch.cuda.synchronize()
    assert P.pyhst_device_status(clear=True) == 0
    opp = orc.PatchProblem(400, 400, 8, 4, Dm.astype(np.float64), float(np.float32(0.8)))
    Gr = opp.gradient(W.cpu().double().numpy(), y.cpu().double().numpy())
    assert np.linalg.norm(G.cpu().numpy() - Gr) / np.linalg.norm(Gr) <= 1e-5
