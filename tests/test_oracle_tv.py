"""Pins of the oracle's TV prox, FISTA/ISTA and power iteration (no GPU)."""
import math

import numpy as np
import pytest


def test_grad_div_adjoint_and_tv_closed_forms(orc):
    """div = -grad^T; TV of a ramp a*j is |a| ny (nx-1); TV of a single
    interior spike of height h is h (2 + 2 sqrt(2)) / ... computed from the
    four affected forward differences."""
    g = np.random.default_rng(0)
    x = g.standard_normal((13, 9))
    p1, p2 = g.standard_normal((2, 13, 9))
    g1, g2 = orc.grad(x)
    assert abs(np.vdot(g1, p1) + np.vdot(g2, p2) + np.vdot(x, orc.div(p1, p2))) < 1e-12 * 100
    a = -0.7
    ramp = a * np.arange(9)[None, :] * np.ones((13, 1))
    assert orc.tv(ramp) == pytest.approx(abs(a) * 13 * 8, rel=1e-14)
    spike = np.zeros((7, 7))
    spike[3, 3] = 2.0
    # pixel (3,3): |(-2,-2)| ; (2,3): |(2,0)| ; (3,2): |(0,2)|
    assert orc.tv(spike) == pytest.approx(2 * math.sqrt(2) + 2 + 2, rel=1e-14)


def test_prox_of_constant_is_identity(orc):
    z = np.full((16, 11), 3.25)
    x, p1, p2 = orc.tv_prox(z, 0.7, 20)
    np.testing.assert_array_equal(x, z)
    assert np.all(p1 == 0) and np.all(p2 == 0)


def test_prox_invariants(orc):
    """Mean preserved (div p sums to 0), |p| <= 1, gap >= 0 and decreasing,
    small lam leaves z almost unchanged, large lam flattens to mean(z)."""
    g = np.random.default_rng(1)
    z = g.standard_normal((24, 20))
    lam = 0.3
    gaps = []
    p = None
    for steps in (5, 20, 80, 320):
        x, p1, p2 = orc.tv_prox(z, lam, steps)
        assert abs(x.mean() - z.mean()) < 1e-12
        assert np.all(np.hypot(p1, p2) <= 1 + 1e-12)
        gaps.append(orc.rof_gap(z, lam, p1, p2))
    assert all(gp >= -1e-12 for gp in gaps)
    assert all(b < a for a, b in zip(gaps, gaps[1:])), gaps
    assert gaps[-1] < 1e-2 * gaps[0]
    x, _, _ = orc.tv_prox(z, 1e-6, 20)
    assert np.abs(x - z).max() < 1e-5
    x, _, _ = orc.tv_prox(z, 1e3, 4000)
    assert np.abs(x - z.mean()).max() < 1e-2


def test_prox_two_level_step_closed_form(orc):
    """An image constant along one axis reduces to 1-D ROF per row.  For a
    two-level step (a on m pixels, b < a on n-m pixels) the exact solution
    keeps the step and moves the levels by lam/m and lam/(n-m) toward each
    other while a - b > lam (1/m + 1/(n-m))."""
    ny, nx, m = 6, 20, 8
    a, b, lam = 2.0, 0.5, 0.9
    z = np.where(np.arange(nx)[None, :] < m, a, b) * np.ones((ny, 1))
    x, p1, p2 = orc.tv_prox(z, lam, 6000)
    ref = np.where(np.arange(nx)[None, :] < m, a - lam / m, b + lam / (nx - m)) * np.ones((ny, 1))
    np.testing.assert_allclose(x, ref, atol=1e-6)
    # along the other axis the same (transpose symmetry of Eq. 2)
    xt, _, _ = orc.tv_prox(z.T.copy(), lam, 6000)
    np.testing.assert_allclose(xt, ref.T, atol=1e-6)


def _tiny_geometry(orc, n=8, na=9, nb=12, seed=0):
    g = np.random.default_rng(seed)
    angles = np.arange(na) * math.pi / na + 0.01
    axis = (nb - 1) / 2.0 + g.uniform(-0.3, 0.3, na)
    return orc.Geometry(angles, axis, nb, n, n, 0.25)


def _dense_P(orc, geo):
    n = geo.nx * geo.ny
    cols = []
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        cols.append(geo.P(e.reshape(geo.ny, geo.nx)).ravel())
    return np.stack(cols, 1)


def test_power_iteration_matches_eigenvalue(orc):
    """Power iteration converges to the top eigenvalue of P^T P computed by
    a dense symmetric eigen-solver on a tiny system."""
    geo = _tiny_geometry(orc)
    P = _dense_P(orc, geo)
    lmax = np.linalg.eigvalsh(P.T @ P).max()
    v0 = np.random.default_rng(3).standard_normal((geo.ny, geo.nx))
    lam, v = orc.power_iteration(geo, v0, 400)
    assert lam == pytest.approx(lmax, rel=1e-9)
    lam50, _ = orc.power_iteration(geo, v0, 50)
    assert lam50 <= lmax * (1 + 1e-12) and lam50 > 0.98 * lmax


def test_fista_beta0_converges_to_least_squares(orc):
    """beta = 0 on a fully determined tiny system: FISTA's iterate approaches
    the least-squares solution from a dense solver and the gradient norm
    P^T (P x - y) goes to zero."""
    geo = _tiny_geometry(orc, n=6, na=12, nb=10)
    P = _dense_P(orc, geo)
    g = np.random.default_rng(4)
    xt = g.uniform(0, 1, (geo.ny, geo.nx))
    y = P @ xt.ravel() + 0.01 * g.standard_normal(P.shape[0])
    xls = np.linalg.lstsq(P, y, rcond=None)[0]
    L = 1.01 * np.linalg.eigvalsh(P.T @ P).max()
    x, e = orc.fista(geo, y.reshape(geo.n_bins * 0 + len(geo.angles), geo.n_bins), 0.0, L, 3000, n_inner=1)
    grad = P.T @ (P @ x.ravel() - y)
    assert np.linalg.norm(grad) < 1e-6 * np.linalg.norm(P.T @ y)
    np.testing.assert_allclose(x.ravel(), xls, atol=1e-5)
    assert e[-1] == pytest.approx(0.5 * np.sum((P @ xls - y) ** 2), rel=1e-8)


def test_ista_monotone_and_fista_faster(orc):
    """ISTA's energy (Eq. 3) never increases; FISTA reaches a lower energy
    than ISTA after the same number of iterations (Sec. 3.1)."""
    geo = _tiny_geometry(orc, n=16, na=6, nb=24, seed=2)
    g = np.random.default_rng(5)
    xt = np.zeros((16, 16))
    xt[4:12, 5:11] = 1.0
    y = geo.P(xt) + 0.02 * g.standard_normal((6, 24))
    v0 = g.standard_normal((16, 16))
    L = 1.01 * orc.power_iteration(geo, v0, 100)[0]
    beta = 0.01
    _, ei = orc.fista(geo, y, beta, L, 60, n_inner=40, use_fista=False)
    _, ef = orc.fista(geo, y, beta, L, 60, n_inner=40, use_fista=True)
    assert np.all(np.diff(ei) <= 1e-9 * abs(ei[0]))
    assert ef[-1] < ei[-1]
    # the energy history is Eq. 3 evaluated at the returned iterate
    x, e = orc.fista(geo, y, beta, L, 7, n_inner=20)
    assert e[-1] == pytest.approx(orc.energy(geo, y, x, beta), rel=1e-14)


def test_fista_tv_recovers_piecewise_constant(orc):
    """With few angles and noise, TV-FISTA gets closer to a piecewise-constant
    truth than the unregularised solution at the same iteration count."""
    n = 32
    geo = orc.Geometry(np.arange(8) * math.pi / 8, (n - 1) / 2.0, n, n, n, 2.0 / n)
    xt = np.zeros((n, n))
    xt[8:24, 8:24] = 1.0
    xt[12:18, 14:20] = 0.4
    g = np.random.default_rng(6)
    y = geo.P(xt) + 0.01 * g.standard_normal((8, n))
    L = 1.01 * orc.power_iteration(geo, g.standard_normal((n, n)), 100)[0]
    x0, _ = orc.fista(geo, y, 0.0, L, 150, n_inner=1)
    xb, _ = orc.fista(geo, y, 2e-3, L, 150, n_inner=20)
    assert np.linalg.norm(xb - xt) < 0.7 * np.linalg.norm(x0 - xt)


def test_cosine_and_ecohe_closed_forms(orc):
    """Cos of known vectors (orthogonal 0, parallel 1, 60 degrees 1/2), and
    Eq. 11 on a scaled copy: I(beta) = c I(0+) gives sign((c - 1) c)."""
    a = np.array([1.0, 0.0, 0.0])
    assert orc.cosine(a, np.array([0.0, 2.0, 0.0])) == 0.0
    assert orc.cosine(a, 3 * a) == pytest.approx(1.0, abs=1e-15)
    assert orc.cosine(a, np.array([0.5, math.sqrt(3) / 2, 0.0])) == pytest.approx(0.5, abs=1e-15)
    assert math.isnan(orc.cosine(a, np.zeros(3)))
    g = np.random.default_rng(0)
    I0 = g.standard_normal((9, 7))
    assert orc.ecohe(0.5 * I0, I0) == pytest.approx(-1.0, abs=1e-14)
    assert orc.ecohe(2.0 * I0, I0) == pytest.approx(1.0, abs=1e-14)
    assert math.isnan(orc.ecohe(I0, I0))


def test_cross_validation_is_zero_on_consistent_data(orc):
    """Data generated by the projector itself from an image the solver can
    reach: with beta = 0 and many iterations the held-out projection of the
    reconstruction matches the held-out data (the estimator's zero)."""
    n = 12
    angles = np.arange(30) * math.pi / 30
    geo = orc.Geometry(angles, (n - 1) / 2.0 + 2.0, n + 4, n, n, 0.1)
    g = np.random.default_rng(1)
    x_true = g.uniform(0, 1, (n, n))
    y = geo.P(x_true)
    L = 1.01 * orc.power_iteration(geo, np.ones((n, n)), 200)[0]
    e1, _ = orc.cross_validation(geo, y, 7, [0.0], L, 1000, n_inner=1)
    e3, _ = orc.cross_validation(geo, y, 7, [0.0], L, 3000, n_inner=1)
    assert e3[0] < 1e-8 * np.sum(y[7] ** 2) and e3[0] < 0.1 * e1[0]   # -> 0 as the solve converges


def _np_tv(x):
    """Eq. 2 written with numpy differences (Neumann: zero past the last row
    and column), independent of the oracle's loops."""
    d1 = np.zeros_like(x)
    d2 = np.zeros_like(x)
    d1[:-1, :] = np.diff(x, axis=0)
    d2[:, :-1] = np.diff(x, axis=1)
    return np.sqrt(d1 ** 2 + d2 ** 2).sum()


def test_energy_closed_forms(orc):
    """Eq. 3 at points where it is known exactly: E(0) = 1/2 ||y||^2 for any
    beta (TV(0) = 0); for data y = P x_t of a ramp x_t = a j the data term
    vanishes and E(x_t) = beta |a| ny (nx - 1), the ramp's total variation."""
    geo = _tiny_geometry(orc, n=10, na=7, nb=16, seed=9)
    g = np.random.default_rng(11)
    y = g.standard_normal((7, 16))
    for beta in (0.0, 0.37, 5.0):
        assert orc.energy(geo, y, np.zeros((10, 10)), beta) == pytest.approx(0.5 * np.sum(y ** 2), rel=1e-15)
    a = -1.3
    xt = a * np.arange(10)[None, :] * np.ones((10, 1))
    yt = geo.P(xt)
    for beta in (0.0, 0.25, 3.0):
        assert orc.energy(geo, yt, xt, beta) == pytest.approx(beta * abs(a) * 10 * 9, rel=1e-13, abs=1e-13)


@pytest.mark.parametrize("case", range(3))
def test_energy_equals_dense_system(orc, case):
    """Eq. 3 against the dense hat-function system matrix built entry by
    entry (off-centre, per-angle axes) and a numpy TV: a dropped 1/2, a
    misplaced beta, a sign flip in the residual or a missing pixel-size
    scale of the projector changes the value."""
    from test_oracle_pipeline import _dense_A
    g = np.random.default_rng(40 + case)
    nx, ny = ((7, 9), (11, 6), (8, 8))[case]
    na, nb = int(g.integers(3, 9)), int(g.integers(8, 15))
    angles = g.uniform(0, math.pi, na)
    axis = (nb - 1) / 2.0 + g.uniform(-1.5, 1.5, na)
    s = float(g.uniform(0.05, 0.5))
    geo = orc.Geometry(angles, axis, nb, nx, ny, s)
    A = s * _dense_A(angles, axis, nb, nx, ny, (nx - 1) / 2.0, (ny - 1) / 2.0)
    x = g.standard_normal((ny, nx))
    y = g.standard_normal((na, nb)) + 3.0
    beta = float(g.uniform(0.1, 2.0))
    ref = 0.5 * np.sum((y.ravel() - A @ x.ravel()) ** 2) + beta * _np_tv(x)
    assert orc.energy(geo, y, x, beta) == pytest.approx(ref, rel=1e-13)


def _np_grad(x):
    d1 = np.zeros_like(x)
    d2 = np.zeros_like(x)
    d1[:-1, :] = np.diff(x, axis=0)
    d2[:, :-1] = np.diff(x, axis=1)
    return d1, d2


def test_rof_gap_equals_sum_of_nonnegative_terms(orc):
    """For x = z - lam div p with |p| <= 1, primal minus dual of the ROF
    problem equals lam * sum(|grad x| + p . grad x) (expand the squares and
    use div = -grad^T), a sum of terms that are each >= 0 by Cauchy-Schwarz.
    Checked with numpy differences on random feasible dual fields, so a
    wrong sign, a dropped 1/2 or a wrong lam in the oracle's gap fails."""
    g = np.random.default_rng(21)
    for ny, nx, lam in ((9, 13, 0.4), (20, 7, 2.5), (16, 16, 0.05)):
        z = g.standard_normal((ny, nx))
        p1, p2 = g.standard_normal((2, ny, nx))
        r = np.maximum(1.0, np.hypot(p1, p2)) / g.uniform(0.2, 1.0, (ny, nx))
        p1, p2 = p1 / r, p2 / r
        assert np.all(np.hypot(p1, p2) <= 1.0)
        d1, d2 = _np_grad(z - lam * orc.div(p1, p2))
        terms = np.hypot(d1, d2) + p1 * d1 + p2 * d2
        assert terms.min() >= -1e-12
        assert orc.rof_gap(z, lam, p1, p2) == pytest.approx(lam * terms.sum(), rel=1e-12)


def test_fista_gap_history(orc):
    """The gap history of the solver's proxes: non-negative, zero without a
    penalty, its last entry equal to the gap of the prox recomputed from the
    last prox input, and (first iteration, same z) smaller with more inner
    steps."""
    geo = _tiny_geometry(orc, n=16, na=6, nb=24, seed=2)
    g = np.random.default_rng(22)
    xt = np.zeros((16, 16))
    xt[4:12, 5:11] = 1.0
    y = geo.P(xt) + 0.02 * g.standard_normal((6, 24))
    L = 1.01 * orc.power_iteration(geo, g.standard_normal((16, 16)), 100)[0]
    beta = 0.02
    x, e, z, gp = orc.fista(geo, y, beta, L, 12, n_inner=20, return_z=True, return_gap=True)
    assert np.all(gp >= 0) and np.all(gp > 0)
    _, p1, p2 = orc.tv_prox(z, beta / L, 20)
    assert gp[-1] == pytest.approx(orc.rof_gap(z, beta / L, p1, p2), rel=1e-13)
    _, _, g0 = orc.fista(geo, y, 0.0, L, 5, n_inner=20, return_gap=True)
    assert np.all(g0 == 0)
    first = [orc.fista(geo, y, beta, L, 1, n_inner=m, return_gap=True)[2][0] for m in (2, 8, 32, 128)]
    assert all(b < a for a, b in zip(first, first[1:])), first


def test_fista_dual_warm_start(orc):
    """The dual warm start (each prox's dual field starting at the previous
    prox's final field): its first iteration is the cold start's, bit for bit;
    with near-exact proxes (many inner steps) it reaches the cold-start
    iterates; with few inner steps its proxes end closer to exact (smaller
    duality gaps) once the prox inputs change slowly."""
    geo = _tiny_geometry(orc, n=16, na=6, nb=24, seed=2)
    g = np.random.default_rng(23)
    xt = np.zeros((16, 16))
    xt[3:11, 4:12] = 1.0
    xt[6:9, 6:14] += 0.5
    y = geo.P(xt) + 0.02 * g.standard_normal((6, 24))
    L = 1.01 * orc.power_iteration(geo, g.standard_normal((16, 16)), 100)[0]
    beta = 0.02
    x1c, _ = orc.fista(geo, y, beta, L, 1, n_inner=5)
    x1w, _ = orc.fista(geo, y, beta, L, 1, n_inner=5, warm_dual=True)
    assert np.array_equal(x1c, x1w)
    xc, _ = orc.fista(geo, y, beta, L, 8, n_inner=600)
    xw, _ = orc.fista(geo, y, beta, L, 8, n_inner=600, warm_dual=True)
    assert np.linalg.norm(xw - xc) <= 1e-6 * np.linalg.norm(xc)
    _, _, gc = orc.fista(geo, y, beta, L, 30, n_inner=5, return_gap=True)
    xw5, _, gw = orc.fista(geo, y, beta, L, 30, n_inner=5, return_gap=True, warm_dual=True)
    assert gw[0] == gc[0]
    assert np.mean(gw[10:]) < 0.5 * np.mean(gc[10:]), (np.mean(gw[10:]), np.mean(gc[10:]))
    assert not np.array_equal(xw5, orc.fista(geo, y, beta, L, 30, n_inner=5)[0])
