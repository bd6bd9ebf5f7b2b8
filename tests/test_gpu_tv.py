"""GPU parity of the TV prox, the power-iteration step size and the ISTA/FISTA
solve of Eq. 3 against the FP64 oracle, through the C ABI.

Tolerances.  The prox and single operator applications are held to the
float32 bar (relative L2 <= 1e-5).  An iterative solve compounds float32
rounding over its iterations, so its iterate is held to relative L2 <= 1e-4
after up to 50 outer iterations and its float64 energy history to relative
1e-5 (the energy is a sum of squares and is less sensitive than x).
"""
import math

import numpy as np
import pytest
import torch

from synth import acquisition as acq

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_1306_1392_b300 as P
    return P


# Batched and single-slice energies: the same float64 partials except that
# the batched TV term adds each warp's 32 terms in float32 first (a fixed
# tree, at most ~5 roundings of 2^-24 relative to that term, which is part
# of E), so they agree to ~1e-7; the iterates themselves are compared bit
# for bit.
ENERGY_BATCH_RTOL = 1e-6


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("shape,lam,n_inner", [((64, 64), 0.3, 20), ((77, 100), 0.05, 20), ((31, 9), 1.5, 7),
                                               ((1, 50), 0.2, 20)])
def test_tv_prox_parity(P, orc, cuda_device, shape, lam, n_inner):
    g = np.random.default_rng(sum(shape))
    z = g.standard_normal((2,) + shape).astype(np.float32)
    got = P.pyhst_tv_prox(torch.from_numpy(z).to(cuda_device), lam, n_inner).cpu().numpy()
    for k in range(2):
        ref, _, _ = orc.tv_prox(z[k].astype(np.float64), lam, n_inner)
        assert rel(got[k], ref) <= 1e-5


def test_tv_prox_full_size_sampled(P, orc, cuda_device):
    """The prox at the size its kernel benchmark runs (16 x 1024^2, 20
    steps, the autotuned steps per launch): sampled pixels against the
    oracle's prox of a crop around each.  A step reads neighbours at
    Chebyshev distance 1, so after n steps the crop's own borders have not
    reached a pixel n + 3 away from them, and the crop gives the full
    image's value there; pixels on the image border keep the true border."""
    n, ns, n_inner, lam = 1024, 16, 20, 0.05
    g = torch.Generator(device=cuda_device).manual_seed(11)
    z = torch.randn((ns, n, n), device=cuda_device, generator=g)
    P.pyhst_autotune_tv_prox(z, lam, n_inner)
    got = P.pyhst_tv_prox(z, lam, n_inner).cpu().numpy()
    zc = z.cpu().numpy()
    rng = np.random.default_rng(3)
    R = n_inner + 3
    pts = list(zip(rng.integers(0, ns, 40), rng.integers(0, n, 40), rng.integers(0, n, 40)))
    pts += [(0, 0, 0), (1, n - 1, n - 1), (2, 0, n - 1), (3, n - 1, 0), (4, n // 2, 0), (15, 0, n // 2),
            (7, 53, 54), (8, 54, 107)]      # on tile seams of the fused kernel's output tiles
    gv, rv = [], []
    for s_, i, j in pts:
        i0, i1, j0, j1 = max(0, i - R), min(n, i + R + 1), max(0, j - R), min(n, j + R + 1)
        ref, _, _ = orc.tv_prox(zc[s_, i0:i1, j0:j1].astype(np.float64), lam, n_inner)
        rv.append(ref[i - i0, j - j0])
        gv.append(got[s_, i, j])
    assert rel(gv, rv) <= 1e-5
    P.pyhst_set_tv_prox_steps(n, n, 0)


def test_tv_prox_zero_lambda_is_identity(P, cuda_device):
    z = torch.randn(1, 40, 30, device=cuda_device)
    torch.testing.assert_close(P.pyhst_tv_prox(z, 0.0), z, rtol=0, atol=0)


def _foam_problem(P, orc, dev, n=64, na=24, seed=7):
    fs = acq.foam_slice(n, na, seed=seed, truth=False)
    geo = P.Geometry(fs.angles.to(dev), fs.axis.to(dev), fs.n_bins, fs.nx, fs.ny, fs.pixel_size)
    og = orc.Geometry(fs.angles.double().numpy(), fs.axis.double().numpy(), fs.n_bins, fs.nx, fs.ny, fs.pixel_size)
    return fs, geo, og


def test_power_iteration_step_size(P, orc, cuda_device):
    """L = 1.01 ||P v||^2 after n power iterations from the all-ones image."""
    fs, geo, og = _foam_problem(P, orc, cuda_device)
    lam, _ = orc.power_iteration(og, np.ones((fs.ny, fs.nx)), 30)
    _, _, lip = P.pyhst_tv_solve(geo, fs.extra["sino"].to(cuda_device),
                                 P.TvOptions(beta=1e-3, n_iter=1, n_inner=1, n_power_iter=30), energy=False)
    assert abs(lip.item() - 1.01 * lam) <= 1e-5 * 1.01 * lam


@pytest.mark.parametrize("fista,beta,n_iter", [(True, 2e-3, 20), (False, 2e-3, 20), (True, 5e-3, 50),
                                               (True, 0.0, 30)])
def test_tv_solve_parity(P, orc, cuda_device, fista, beta, n_iter):
    fs, geo, og = _foam_problem(P, orc, cuda_device)
    L = 1.01 * orc.power_iteration(og, np.ones((fs.ny, fs.nx)), 30)[0]
    sino = fs.extra["sino"]
    opts = P.TvOptions(beta=beta, n_iter=n_iter, n_inner=20, lipschitz=L, use_fista=fista)
    x, e, lip = P.pyhst_tv_solve(geo, sino.to(cuda_device), opts)
    xr, er = orc.fista(og, sino.double().numpy(), beta, L, n_iter, n_inner=20, use_fista=fista)
    assert lip.item() == L
    assert rel(x[0].cpu().numpy(), xr) <= 1e-4
    np.testing.assert_allclose(e[0].cpu().numpy(), er, rtol=1e-5)


def test_tv_solve_warm_start(P, orc, cuda_device):
    fs, geo, og = _foam_problem(P, orc, cuda_device, n=48, na=16, seed=3)
    L = 1.01 * orc.power_iteration(og, np.ones((fs.ny, fs.nx)), 30)[0]
    x0 = np.random.default_rng(1).uniform(0, 1, (fs.ny, fs.nx)).astype(np.float32)
    sino = fs.extra["sino"]
    opts = P.TvOptions(beta=3e-3, n_iter=15, n_inner=10, lipschitz=L, warm_start=True)
    x, e, _ = P.pyhst_tv_solve(geo, sino.to(cuda_device), opts, x=torch.from_numpy(x0[None]).to(cuda_device))
    xr, er = orc.fista(og, sino.double().numpy(), 3e-3, L, 15, n_inner=10, x0=x0.astype(np.float64))
    assert rel(x[0].cpu().numpy(), xr) <= 1e-4
    np.testing.assert_allclose(e[0].cpu().numpy(), er, rtol=1e-5)


def test_tv_solve_slices_are_independent(P, orc, cuda_device):
    """A stack of slices gives bitwise the results of solving each alone."""
    fs, geo, og = _foam_problem(P, orc, cuda_device, n=40, na=20)
    g = np.random.default_rng(2)
    sinos = torch.stack([fs.extra["sino"], fs.extra["sino"] * 0.5,
                         torch.from_numpy(g.uniform(0, 1, fs.extra["sino"].shape).astype(np.float32))]).to(cuda_device)
    opts = P.TvOptions(beta=2e-3, n_iter=8, n_inner=5, n_power_iter=10)
    xs, es, ls = P.pyhst_tv_solve(geo, sinos, opts)
    for k in range(3):
        x1, e1, l1 = P.pyhst_tv_solve(geo, sinos[k:k + 1].contiguous(), opts)
        assert torch.equal(x1[0], xs[k]) and torch.equal(e1[0], es[k]) and torch.equal(l1[0], ls[k])


def test_tv_solve_energy_decreases_and_beats_fbp(P, cuda_device):
    """FISTA's energy drops over the run (Sec. 3.1) and, at one tenth of the
    angles with Poisson noise, TV beats unregularised reconstructions."""
    fs = acq.foam_slice(128, 26, seed=11)
    dev = cuda_device
    geo = P.Geometry(fs.angles.to(dev), fs.axis.to(dev), fs.n_bins, fs.nx, fs.ny, fs.pixel_size)
    sino = fs.extra["sino"].to(dev)
    x, e, _ = P.pyhst_tv_solve(geo, sino, P.TvOptions(beta=2e-3, n_iter=150))
    e = e[0].cpu().numpy()
    assert e[-1] < 0.5 * e[0] and e[-1] <= e[10:].min() * (1 + 1e-6)
    fbp = P.pyhst_fbp(geo, sino[None].contiguous(), "f32_sino")
    truth = fs.truth.numpy()
    err_tv = np.linalg.norm(x[0].cpu().numpy() - truth)
    err_fbp = np.linalg.norm(fbp[0].cpu().numpy() - truth)
    assert err_tv < 0.8 * err_fbp


# ------------------------------------------------------------------ mixed batch
def _mixed(P, orc, dev):
    """Five slices of three geometries: 48^2/40 angles, 64^2/24 angles and a
    non-square 40 x 32 grid with 30 angles and an off-centre axis."""
    out = []
    specs = [(48, 48, 40, 0.0, 1), (64, 64, 24, 0.0, 2), (48, 48, 40, 0.0, 3), (40, 32, 30, 2.5, 4),
             (64, 64, 24, 0.0, 5)]
    geos = {}
    for nx, ny, na, off, seed in specs:
        key = (nx, ny, na, off)
        if key not in geos:
            ang = acq.uniform_angles(na)
            nb = max(nx, ny) + 6
            axis = torch.full((na,), (nb - 1) / 2.0 + off)
            geos[key] = (P.Geometry(ang.to(dev), axis.to(dev), nb, nx, ny, 2.0 / max(nx, ny)), ang, axis, nb)
        geo, ang, axis, nb = geos[key]
        g = np.random.default_rng(seed)
        img = np.zeros((ny, nx))
        img[ny // 4: 3 * ny // 4, nx // 3: 2 * nx // 3] = 1.0
        # the oracle's projector makes the data (scaled like pyhst_project)
        sino = orc.project(img, ang.double().numpy(), axis.double().numpy(), nb, scale=2.0 / max(nx, ny))
        sino = (sino + 0.01 * g.standard_normal(sino.shape)).astype(np.float32)
        out.append((geo, torch.from_numpy(sino).to(dev).contiguous(), ang, axis, nb))
    return out


def test_batch_matches_single_slice_solves(P, orc, cuda_device):
    """With the same step size, every slice of a mixed batch equals its
    single-slice solve bit for bit (same kernels), its energies agree to
    ENERGY_BATCH_RTOL, and it matches the FP64 oracle like the single-slice
    solver."""
    items = _mixed(P, orc, cuda_device)
    L = 1.01 * max(orc.power_iteration(orc.Geometry(a.double().numpy(), ax.double().numpy(), nb, g.nx, g.ny,
                                                    g.pixel_size), np.ones((g.ny, g.nx)), 40)[0]
                   for g, _, a, ax, nb in items)
    opts = P.TvOptions(beta=3e-3, n_iter=12, n_inner=8, lipschitz=L)
    xs, es, lip = P.pyhst_tv_solve_batch([(g, s, None) for g, s, *_ in items], opts)
    torch.cuda.synchronize()
    for k, (g, s, a, ax, nb) in enumerate(items):
        x1, e1, _ = P.pyhst_tv_solve(g, s[None].contiguous(), opts)
        assert torch.equal(xs[k], x1[0]), k
        np.testing.assert_allclose(es[k].cpu().numpy(), e1[0].cpu().numpy(), rtol=ENERGY_BATCH_RTOL)
        og = orc.Geometry(a.double().numpy(), ax.double().numpy(), nb, g.nx, g.ny, g.pixel_size)
        xr, er = orc.fista(og, s.double().cpu().numpy(), 3e-3, L, 12, n_inner=8)
        assert rel(xs[k].cpu().numpy(), xr) <= 1e-4
        np.testing.assert_allclose(es[k].cpu().numpy(), er, rtol=1e-5)
    assert torch.all(lip == L)


def test_batch_at_benchmark_sizes(P, orc, cuda_device):
    """One slice of each reduced-dose size (256^2 / 50, 512^2 / 100 and
    1024^2 / 200 angles, bins = N, Poisson 1e4 foams) in one batched solve
    with the benchmark's 20 Chambolle steps and tuned fusion depth: every
    slice equals its single-slice solve bit for bit, and after 3 FISTA
    iterations matches the oracle's FISTA with the same step size."""
    items, ogs = [], []
    for k, (n, na) in enumerate([(256, 50), (512, 100), (1024, 200)]):
        fs = acq.foam_slice(n, na, seed=3000 + k, truth=False)
        geo = P.Geometry(fs.angles.to(cuda_device), fs.axis.to(cuda_device), n, n, n, fs.pixel_size)
        items.append((geo, fs.extra["sino"].to(cuda_device).contiguous(), fs.extra["sino"]))
        ogs.append(orc.Geometry(fs.angles.double().numpy(), fs.axis.double().numpy(), n, n, n, fs.pixel_size))
        z = torch.randn((2, n, n), device=cuda_device, generator=torch.Generator(device=cuda_device).manual_seed(n))
        P.pyhst_autotune_tv_prox(z, 0.01, 20)
    L = 1.01 * max(orc.power_iteration(og, np.ones((og.ny, og.nx)), 8)[0] for og in ogs)
    opts = P.TvOptions(beta=1e-3, n_iter=3, n_inner=20, lipschitz=L)
    xs, es, _ = P.pyhst_tv_solve_batch([(g, s, None) for g, s, _ in items], opts)
    torch.cuda.synchronize()
    for k, ((g, s, s_host), og) in enumerate(zip(items, ogs)):
        x1, e1, _ = P.pyhst_tv_solve(g, s[None].contiguous(), opts)
        assert torch.equal(xs[k], x1[0]), k
        xr, er = orc.fista(og, s_host.double().numpy(), 1e-3, L, 3, n_inner=20)
        assert rel(xs[k].cpu().numpy(), xr) <= 1e-4
        np.testing.assert_allclose(es[k].cpu().numpy(), er, rtol=1e-5)
    for n in (256, 512, 1024):
        P.pyhst_set_tv_prox_steps(n, n, 0)


def test_tv_solve_full_iteration_count(P, orc, cuda_device):
    """One reduced-dose slice (256^2 foam, 50 angles, Poisson 1e4) at the
    benchmark's full count, 200 FISTA iterations x 20 Chambolle steps with the
    benchmark's beta for that size, through the batched solver, against the
    oracle's FISTA with the same step size.  float32 rounding compounds over
    the iterations, but the drift measured at 200 iterations on a B300
    (iterate 4.9e-7 relative L2, energies 2.0e-7) is well inside the float32
    bar, which holds here: iterate relative L2 <= 1e-5, every energy of the
    history within 1e-5 relative."""
    n, na, beta = 256, 50, 1.7783e-3
    fs = acq.foam_slice(n, na, seed=3000, truth=False)
    geo = P.Geometry(fs.angles.to(cuda_device), fs.axis.to(cuda_device), n, n, n, fs.pixel_size)
    og = orc.Geometry(fs.angles.double().numpy(), fs.axis.double().numpy(), n, n, n, fs.pixel_size)
    L = 1.01 * orc.power_iteration(og, np.ones((n, n)), 50)[0]
    sino = fs.extra["sino"]
    opts = P.TvOptions(beta=beta, n_iter=200, n_inner=20, lipschitz=L)
    xs, es, _ = P.pyhst_tv_solve_batch([(geo, sino.to(cuda_device).contiguous(), None)], opts)
    torch.cuda.synchronize()
    xr, er = orc.fista(og, sino.double().numpy(), beta, L, 200, n_inner=20)
    rx = rel(xs[0].cpu().numpy(), xr)
    re = np.abs(es[0].cpu().numpy() - er) / np.abs(er)
    print(f"\n200 x 20 iterations at 256^2 / 50 angles: iterate rel L2 {rx:.3e}, "
          f"energy rel error max {re.max():.3e}, last {re[-1]:.3e}")
    assert rx <= 1e-5
    assert re.max() <= 1e-5


def test_batch_step_size_per_geometry(P, orc, cuda_device):
    """Estimated L: one power iteration per distinct geometry, equal (to
    float64 summation order) to the single-slice estimate."""
    items = _mixed(P, orc, cuda_device)
    opts = P.TvOptions(beta=2e-3, n_iter=3, n_inner=5, n_power_iter=25)
    _, _, lip = P.pyhst_tv_solve_batch([(g, s, None) for g, s, *_ in items], opts)
    for k, (g, s, *_r) in enumerate(items):
        _, _, l1 = P.pyhst_tv_solve(g, s[None].contiguous(), opts)
        assert abs(lip[k].item() - l1.item()) <= 1e-6 * l1.item()
    assert lip[0].item() == lip[2].item() and lip[1].item() == lip[4].item()


@pytest.mark.parametrize("fista,beta,warm", [(False, 2e-3, False), (True, 0.0, False), (True, 4e-3, True)])
def test_batch_variants(P, orc, cuda_device, fista, beta, warm):
    items = _mixed(P, orc, cuda_device)
    L = 5.0
    opts = P.TvOptions(beta=beta, n_iter=9, n_inner=6, lipschitz=L, use_fista=fista, warm_start=warm)
    x0s = [torch.rand((g.ny, g.nx), device=cuda_device) for g, *_ in items]
    xs, es, _ = P.pyhst_tv_solve_batch([(g, s, x0.clone()) for (g, s, *_), x0 in zip(items, x0s)], opts)
    for k, (g, s, *_r) in enumerate(items):
        x1, e1, _ = P.pyhst_tv_solve(g, s[None].contiguous(), opts, x=x0s[k][None].clone())
        assert torch.equal(xs[k], x1[0]), k
        np.testing.assert_allclose(es[k].cpu().numpy(), e1[0].cpu().numpy(), rtol=ENERGY_BATCH_RTOL)


def test_batch_per_item_beta(P, orc, cuda_device):
    """Each batch item may carry its own beta (0 included): every slice
    equals its single-slice solve with that beta, bit for bit."""
    items = _mixed(P, orc, cuda_device)
    betas = [1e-3, 0.0, 5e-3, 2e-3, None]
    opts = P.TvOptions(beta=3e-3, n_iter=7, n_inner=6, lipschitz=6.0)
    xs, es, _ = P.pyhst_tv_solve_batch([(g, s, None, b) for (g, s, *_), b in zip(items, betas)], opts)
    for k, ((g, s, *_r), b) in enumerate(zip(items, betas)):
        o1 = P.TvOptions(beta=3e-3 if b is None else b, n_iter=7, n_inner=6, lipschitz=6.0)
        x1, e1, _ = P.pyhst_tv_solve(g, s[None].contiguous(), o1)
        assert torch.equal(xs[k], x1[0]), k
        np.testing.assert_allclose(es[k].cpu().numpy(), e1[0].cpu().numpy(), rtol=ENERGY_BATCH_RTOL)


# ------------------------------------------------------------------ beta estimators (Sec. 4)
@pytest.mark.parametrize("held_out", [5, 0, -1])
def test_beta_scan_estimators_parity(P, orc, cuda_device, held_out):
    """Cross-validation error and E_cohe (Eq. 11) over a beta grid against
    the oracle's, with the same step size; the iterates as in the solver
    parity tests."""
    fs, geo, og = _foam_problem(P, orc, cuda_device, n=48, na=20, seed=13)
    sino = fs.extra["sino"]
    keep = [a for a in range(20) if a != held_out]
    ogk = orc.Geometry(og.angles[keep], og.axis[keep], og.n_bins, og.nx, og.ny, og.pixel_size)
    L = 1.01 * orc.power_iteration(ogk, np.ones((48, 48)), 30)[0]
    betas = [1e-5, 5e-4, 2e-3, 8e-3]
    opts = P.TvOptions(beta=0.0, n_iter=25, n_inner=10, lipschitz=L)
    x, cv, ec = P.pyhst_beta_scan(geo, sino.to(cuda_device), betas, opts, held_out=held_out)
    torch.cuda.synchronize()
    if held_out >= 0:
        cv_ref, imgs = orc.cross_validation(og, sino.double().numpy(), held_out, betas, L, 25, n_inner=10)
        np.testing.assert_allclose(cv.cpu().numpy(), cv_ref, rtol=1e-4)
    else:
        assert cv is None
        imgs = [orc.fista(og, sino.double().numpy(), b, L, 25, n_inner=10)[0] for b in betas]
    for k in range(len(betas)):
        assert rel(x[k].cpu().numpy(), imgs[k]) <= 1e-4
    ec_ref = [orc.ecohe(im, imgs[0]) for im in imgs]
    assert math.isnan(ec[0].item()) and math.isnan(ec_ref[0])
    np.testing.assert_allclose(ec.cpu().numpy()[1:], ec_ref[1:], atol=2e-4)


def test_beta_scan_full_size_properties(P, cuda_device):
    """The scan at the size of the Sec. 4 study (2048^2 foam, 150
    projections, angle 75 held out), a few iterations per beta.  Properties
    that hold at any size: each reconstruction equals, bit for bit, the
    single-slice solve of the 149 kept projections with its beta and the same
    step size; the cross-validation error is the squared distance between
    the held-out row and that reconstruction's projection at the held-out
    angle; E_cohe is Cos(x_b - x_0, x_b) of the returned reconstructions."""
    dev = cuda_device
    n, na, h = 2048, 150, 75
    fs = acq.foam_slice(n, na, seed=5150, device=dev, truth=False)
    sino = fs.extra["sino"].to(dev)
    ang, ax = fs.angles.to(dev), fs.axis.to(dev)
    keep = torch.tensor([a for a in range(na) if a != h], device=dev)
    geo = P.Geometry(ang, ax, n, n, n, fs.pixel_size)
    geo_k = P.Geometry(ang[keep].contiguous(), ax[keep].contiguous(), n, n, n, fs.pixel_size)
    geo_h = P.Geometry(ang[h:h + 1].contiguous(), ax[h:h + 1].contiguous(), n, n, n, fs.pixel_size)
    sino_k = sino[keep].contiguous()
    _, _, lip = P.pyhst_tv_solve(geo_k, sino_k[None], P.TvOptions(beta=1e-3, n_iter=1, n_inner=1, n_power_iter=30),
                                 energy=False)
    L = lip.item()
    betas = [1e-5, 1e-3, 1e-2]
    opts = P.TvOptions(beta=0.0, n_iter=4, n_inner=20, lipschitz=L)
    x, cv, ec = P.pyhst_beta_scan(geo, sino, betas, opts, held_out=h)
    torch.cuda.synchronize()
    for k, b in enumerate(betas):
        x1, _, _ = P.pyhst_tv_solve(geo_k, sino_k[None], P.TvOptions(beta=b, n_iter=4, n_inner=20, lipschitz=L),
                                    energy=False)
        assert torch.equal(x[k], x1[0]), k
    rows = P.pyhst_project(geo_h, x)[:, 0, :].double()
    cv_ref = ((rows - sino[h].double()[None]) ** 2).sum(dim=1).cpu().numpy()
    np.testing.assert_allclose(cv.cpu().numpy(), cv_ref, rtol=1e-9)
    xd = x.double()
    for k in range(1, len(betas)):
        d = xd[k] - xd[0]
        cos = (d * xd[k]).sum() / (d.norm() * xd[k].norm())
        assert abs(ec[k].item() - cos.item()) <= 1e-9
    assert math.isnan(ec[0].item())


def test_tv_solve_capture_matches_oracle_prox_inputs(P, orc, cuda_device):
    """The captured prox inputs z_k of iterations 1, 4 and 9 equal the
    oracle's (FISTA stopped after k iterations returns its last z), and the
    run's iterate equals the plain solve's bit for bit."""
    fs, geo, og = _foam_problem(P, orc, cuda_device, n=48, na=16, seed=5)
    L = 1.01 * orc.power_iteration(og, np.ones((fs.ny, fs.nx)), 30)[0]
    sino = fs.extra["sino"]
    opts = P.TvOptions(beta=2e-3, n_iter=9, n_inner=20, lipschitz=L)
    x, cap = P.pyhst_tv_solve_capture(geo, sino.to(cuda_device), opts, [1, 4, 9])
    x1, _, _ = P.pyhst_tv_solve(geo, sino.to(cuda_device), opts, energy=False)
    assert torch.equal(x, x1)
    for c, k in enumerate((1, 4, 9)):
        _, _, zr = orc.fista(og, sino.double().numpy(), 2e-3, L, k, n_inner=20, return_z=True)
        assert rel(cap[c, 0].cpu().numpy(), zr) <= 1e-4


def test_tv_prox_steps_per_launch_are_bit_identical(P, cuda_device):
    """Every choice of Chambolle steps fused per launch gives the same bits
    (the halo is recomputed with the same arithmetic); the autotuner picks one
    of them and the prox then uses it."""
    g = np.random.default_rng(3)
    z = torch.from_numpy(g.standard_normal((3, 150, 133)).astype(np.float32)).to(cuda_device)
    outs = {}
    try:
        for k in (2, 3, 4, 5, 6, 8):
            P.pyhst_set_tv_prox_steps(133, 150, k)
            outs[k] = P.pyhst_tv_prox(z, 0.4, 17)
        for k, o in outs.items():
            assert torch.equal(o, outs[5]), k
        best = P.pyhst_autotune_tv_prox(z, 0.4, 17)
        assert best in outs
        assert torch.equal(P.pyhst_tv_prox(z, 0.4, 17), outs[5])
        with pytest.raises(P.PyhstError):
            P.pyhst_set_tv_prox_steps(133, 150, 7)
    finally:
        P.pyhst_set_tv_prox_steps(133, 150, 0)


def test_batch_solve_with_tuned_steps_matches_default(P, orc, cuda_device):
    """The batched solver builds its Chambolle tiles for the tuned choice of
    its largest slice; the result is the same bits as with the default."""
    items = _mixed(P, orc, cuda_device)
    opts = P.TvOptions(beta=3e-3, n_iter=6, n_inner=7, lipschitz=50.0)
    xs0, _, _ = P.pyhst_tv_solve_batch([(g, s, None) for g, s, *_ in items], opts, energy=False)
    try:
        P.pyhst_set_tv_prox_steps(64, 64, 3)
        xs1, _, _ = P.pyhst_tv_solve_batch([(g, s, None) for g, s, *_ in items], opts, energy=False)
    finally:
        P.pyhst_set_tv_prox_steps(64, 64, 0)
    for a, b in zip(xs0, xs1):
        assert torch.equal(a, b)


# ------------------------------------------------------------------ ROF duality gap of the prox
# The gap is primal minus dual, two nearly equal quantities; float32 rounding
# of the dual field moves it by about 1e-7 of the TV term lam TV(x) that
# the reduction sums, so the gap is compared with the oracle's within
# GAP_TOL * lam TV(x) (and printed as a plain relative error as well).
GAP_TOL = 1e-5


@pytest.mark.parametrize("shape,lam,n_inner", [((64, 64), 0.3, 20), ((77, 100), 0.05, 20), ((31, 9), 1.5, 7),
                                               ((200, 160), 0.1, 60)])
def test_tv_prox_gap_parity(P, orc, cuda_device, shape, lam, n_inner):
    g = np.random.default_rng(sum(shape) + 1)
    z = g.standard_normal((2,) + shape).astype(np.float32)
    gap = torch.empty(2, dtype=torch.float64, device=cuda_device)
    x = P.pyhst_tv_prox(torch.from_numpy(z).to(cuda_device), lam, n_inner, gap=gap).cpu().numpy()
    gap = gap.cpu().numpy()
    for k in range(2):
        xr, p1, p2 = orc.tv_prox(z[k].astype(np.float64), lam, n_inner)
        gr = orc.rof_gap(z[k].astype(np.float64), lam, p1, p2)
        scale = lam * orc.tv(xr)
        print(f"\nprox gap {shape} lam {lam} n {n_inner}: gpu {gap[k]:.6e} oracle {gr:.6e} "
              f"rel {abs(gap[k] - gr) / gr:.2e} (of lam TV {abs(gap[k] - gr) / scale:.2e})")
        assert gap[k] >= 0
        assert abs(gap[k] - gr) <= GAP_TOL * scale
        assert rel(x[k], xr) <= 1e-5


def test_tv_prox_gap_decreases_with_inner_steps(P, cuda_device):
    g = torch.Generator(device=cuda_device).manual_seed(5)
    z = torch.randn((3, 96, 80), device=cuda_device, generator=g)
    gaps = []
    for n_inner in (5, 20, 80, 320):
        gp = torch.empty(3, dtype=torch.float64, device=cuda_device)
        P.pyhst_tv_prox(z, 0.2, n_inner, gap=gp)
        gaps.append(gp.cpu().numpy())
    gaps = np.array(gaps)
    assert np.all(gaps > 0)
    assert np.all(np.diff(gaps, axis=0) < 0), gaps
    gz = torch.empty(3, dtype=torch.float64, device=cuda_device)
    P.pyhst_tv_prox(z, 0.0, 5, gap=gz)
    assert torch.all(gz == 0)


@pytest.mark.parametrize("fista,beta", [(True, 2e-3), (False, 5e-3), (True, 0.0)])
def test_tv_solve_gap_history_parity(P, orc, cuda_device, fista, beta):
    """The gap of every iteration's prox in pyhst_tv_solve against the
    oracle FISTA's, and the batched solver's equal to the single-slice
    solver's (different reduction order: 1e-6 relative)."""
    fs, geo, og = _foam_problem(P, orc, cuda_device)
    L = 1.01 * orc.power_iteration(og, np.ones((fs.ny, fs.nx)), 30)[0]
    sino = fs.extra["sino"]
    n_iter = 15
    opts = P.TvOptions(beta=beta, n_iter=n_iter, n_inner=20, lipschitz=L, use_fista=fista)
    gap = torch.empty((1, n_iter), dtype=torch.float64, device=cuda_device)
    x, e, _ = P.pyhst_tv_solve(geo, sino.to(cuda_device), opts, gap=gap)
    xr, er, gr = orc.fista(og, sino.double().numpy(), beta, L, n_iter, n_inner=20, use_fista=fista, return_gap=True)
    gap = gap[0].cpu().numpy()
    gb = torch.empty(n_iter, dtype=torch.float64, device=cuda_device)
    xs, _, _ = P.pyhst_tv_solve_batch([(geo, sino.to(cuda_device).contiguous(), None)], opts, gaps=[gb])
    gb = gb.cpu().numpy()
    assert torch.equal(xs[0], x[0])
    if beta == 0.0:
        assert np.all(gap == 0) and np.all(gr == 0) and np.all(gb == 0)
        return
    # lam TV(x_k) of every iterate, from the oracle's energies: E - 1/2 ||P x - y||^2 is beta TV
    scale = np.array([(beta / L) * orc.tv(orc.fista(og, sino.double().numpy(), beta, L, k + 1, n_inner=20,
                                                    use_fista=fista)[0]) for k in (0, n_iter - 1)])
    err = np.abs(gap - gr)
    print(f"\nsolve gaps fista={fista}: rel max {np.max(err / gr):.2e}, of lam TV {err.max() / scale.min():.2e}; "
          f"batch vs single rel {np.max(np.abs(gb - gap) / gap):.2e}")
    assert np.all(gap >= 0)
    assert err.max() <= GAP_TOL * scale.min()
    np.testing.assert_allclose(gb, gap, rtol=1e-6)


# ------------------------------------------------------------------ dual warm start of the prox
@pytest.mark.parametrize("n_inner,fista", [(5, True), (7, True), (12, False)])
def test_tv_solve_warm_dual_parity(P, orc, cuda_device, n_inner, fista):
    """warm_dual = 1: each prox after the first starts Chambolle's steps from
    the previous prox's final dual field.  Against the oracle's FISTA/ISTA
    with the same warm start: the iterate, the energies and every prox's
    duality gap to the solver bars.  With 5 steps fused per launch, 5, 7 and
    12 inner steps take 1, 2 and 3 launches, so the kept field alternates
    between the two dual buffers or stays in one.  The batched solver gives
    the same iterate bit for bit."""
    fs, geo, og = _foam_problem(P, orc, cuda_device)
    L = 1.01 * orc.power_iteration(og, np.ones((fs.ny, fs.nx)), 30)[0]
    sino = fs.extra["sino"]
    beta, n_iter = 3e-3, 20
    opts = P.TvOptions(beta=beta, n_iter=n_iter, n_inner=n_inner, lipschitz=L, use_fista=fista, warm_dual=True)
    gap = torch.empty((1, n_iter), dtype=torch.float64, device=cuda_device)
    x, e, _ = P.pyhst_tv_solve(geo, sino.to(cuda_device), opts, gap=gap)
    xr, er, gr = orc.fista(og, sino.double().numpy(), beta, L, n_iter, n_inner=n_inner, use_fista=fista,
                           return_gap=True, warm_dual=True)
    assert rel(x[0].cpu().numpy(), xr) <= 1e-4
    np.testing.assert_allclose(e[0].cpu().numpy(), er, rtol=1e-5)
    gap = gap[0].cpu().numpy()
    scale = (beta / L) * orc.tv(xr)
    assert np.all(gap >= 0)
    assert np.abs(gap - gr).max() <= GAP_TOL * scale
    xs, _, _ = P.pyhst_tv_solve_batch([(geo, sino.to(cuda_device).contiguous(), None)], opts)
    assert torch.equal(xs[0], x[0])
    # the cold start differs once the second prox has run
    xc, _, _ = P.pyhst_tv_solve(geo, sino.to(cuda_device), P.TvOptions(beta=beta, n_iter=n_iter, n_inner=n_inner,
                                                                       lipschitz=L, use_fista=fista), energy=False)
    assert not torch.equal(xc[0], x[0])


def test_tv_solve_warm_dual_first_iteration_is_cold(P, cuda_device):
    """One outer iteration has no earlier field to start from: warm_dual
    changes no bit."""
    fs = acq.foam_slice(48, 16, seed=9, truth=False)
    geo = P.Geometry(fs.angles.to(cuda_device), fs.axis.to(cuda_device), fs.n_bins, fs.nx, fs.ny, fs.pixel_size)
    sino = fs.extra["sino"].to(cuda_device)
    out = [P.pyhst_tv_solve(geo, sino, P.TvOptions(beta=4e-3, n_iter=1, n_inner=9, lipschitz=3.0, warm_dual=w))
           for w in (False, True)]
    assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][1], out[1][1])


def test_batch_warm_dual_matches_single_slice(P, orc, cuda_device):
    """A mixed batch (three geometries, per-item beta with a zero) with the
    dual warm start: every slice equals its single-slice warm solve bit for
    bit and reports the same gap history to the batch bar."""
    items = _mixed(P, orc, cuda_device)
    betas = [2e-3, 0.0, 5e-3, 3e-3, None]
    opts = P.TvOptions(beta=3e-3, n_iter=10, n_inner=7, lipschitz=6.0, warm_dual=True)
    gaps = [torch.empty(10, dtype=torch.float64, device=cuda_device) for _ in items]
    xs, es, _ = P.pyhst_tv_solve_batch([(g, s, None, b) for (g, s, *_), b in zip(items, betas)], opts, gaps=gaps)
    for k, ((g, s, *_r), b) in enumerate(zip(items, betas)):
        o1 = P.TvOptions(beta=3e-3 if b is None else b, n_iter=10, n_inner=7, lipschitz=6.0, warm_dual=True)
        g1 = torch.empty((1, 10), dtype=torch.float64, device=cuda_device)
        x1, e1, _ = P.pyhst_tv_solve(g, s[None].contiguous(), o1, gap=g1)
        assert torch.equal(xs[k], x1[0]), k
        np.testing.assert_allclose(es[k].cpu().numpy(), e1[0].cpu().numpy(), rtol=ENERGY_BATCH_RTOL)
        np.testing.assert_allclose(gaps[k].cpu().numpy(), g1[0].cpu().numpy(), rtol=1e-6)


def test_warm_dual_tightens_the_prox(P, cuda_device):
    """With few inner steps, starting each prox from the previous field
    leaves it closer to exact once the prox inputs move slowly: the mean
    duality gap over iterations 10-39 is below half the cold start's."""
    fs = acq.foam_slice(96, 30, seed=21, truth=False)
    geo = P.Geometry(fs.angles.to(cuda_device), fs.axis.to(cuda_device), fs.n_bins, fs.nx, fs.ny, fs.pixel_size)
    sino = fs.extra["sino"].to(cuda_device)
    g = {}
    for w in (False, True):
        gp = torch.empty((1, 40), dtype=torch.float64, device=cuda_device)
        P.pyhst_tv_solve(geo, sino, P.TvOptions(beta=3e-3, n_iter=40, n_inner=5, warm_dual=w), gap=gp)
        g[w] = gp[0].cpu().numpy()
    print(f"\nmean prox gap, iterations 10-39: cold {g[False][10:].mean():.3e}, warm {g[True][10:].mean():.3e}")
    assert g[True][0] == g[False][0]
    assert g[True][10:].mean() < 0.5 * g[False][10:].mean()


def test_batch_projector_pairs_with_odd_groups(P, cuda_device):
    """The batched projector walks two slices of one geometry per CTA, paired
    in list order within each geometry: a group of three slices (one pair and
    one slice paired with itself), interleaved with a group of one, gives
    every slice the bits of its single-slice solve."""
    dev = cuda_device
    specs = [(96, 30, 1), (72, 20, 2), (96, 30, 3), (96, 30, 4)]
    geos, items = {}, []
    for n, na, seed in specs:
        if (n, na) not in geos:
            fs = acq.foam_slice(n, na, seed=seed, truth=False)
            geos[(n, na)] = P.Geometry(fs.angles.to(dev), fs.axis.to(dev), n, n, n, fs.pixel_size)
        g = torch.Generator(device=dev).manual_seed(seed)
        items.append((geos[(n, na)], torch.rand((na, n), device=dev, generator=g), None))
    opts = P.TvOptions(beta=2e-3, n_iter=6, n_inner=8, lipschitz=30.0)
    xs, _, _ = P.pyhst_tv_solve_batch(items, opts)
    torch.cuda.synchronize()
    for k, (geo, s, _) in enumerate(items):
        x1, _, _ = P.pyhst_tv_solve(geo, s[None].contiguous(), opts, energy=False)
        assert torch.equal(xs[k], x1[0]), k
