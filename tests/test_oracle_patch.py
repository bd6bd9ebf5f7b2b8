"""Pins of the oracle's overlapping-patch functional (Sec. 3.2.1, Eqs. 4-9)
and its gradient (Algorithm 1), no GPU: hand-derived patch cores, the DCT
dictionary against scipy's DCT, consistent patches, finite differences of
Eq. 8, and the L1 shrinkage closed form in an orthonormal basis."""
import math

import numpy as np
import pytest
import scipy.fft


def test_grid_cores_and_cover_counts_by_hand(orc):
    """n = 8, m = 4, stride 2: starts 0, 2, 4 with centres 1.5, 3.5, 5.5.
    Nearest centre (Eq. 6) of pixels 0..7 is 0,0,0,1,1,2,2,2 (pixel 2 is 0.5
    from centre 1.5 and 1.5 from 3.5); pixels 0,1,6,7 lie in one patch, the
    others in two.  With constant patches v_ab the image takes v of the core
    patch (Eq. 7), and the penalty of Eq. 8 counts, for patch a along an axis,
    how many of its pixels have core c: n1 = [[3,1,0],[1,2,1],[0,1,3]]."""
    assert orc.patch_grid(8, 8, 4, 2) == (3, 3)
    assert orc.patch_grid(10, 9, 4, 3) == (3, 3)          # 10: starts 0,3,6 ; 9: starts 0,3,5 (clamped)
    assert orc.patch_grid(4, 4, 4, 2) == (1, 1)
    core = [0, 0, 0, 1, 1, 2, 2, 2]
    cover = np.array([1, 1, 2, 2, 2, 2, 1, 1], float)
    g = np.random.default_rng(0)
    v = g.standard_normal((3, 3))
    P = np.repeat(v.reshape(9, 1), 16, axis=1)
    X = orc.patch_assemble(P, 8, 8, 4, 2)
    np.testing.assert_array_equal(X, v[np.ix_(core, core)])
    S, Nv = orc.patch_sum(P, 8, 8, 4, 2)
    np.testing.assert_array_equal(Nv, np.outer(cover, cover))
    n1 = np.array([[3, 1, 0], [1, 2, 1], [0, 1, 3]], float)
    pen = sum(n1[a, c] * n1[b, d] * (v[c, d] - v[a, b]) ** 2
              for a in range(3) for b in range(3) for c in range(3) for d in range(3))
    Dm = np.eye(16)                                         # W = P with the identity dictionary
    prob = orc.PatchProblem(8, 8, 4, 2, Dm, rho=0.7)
    y = g.standard_normal((8, 8))
    assert prob.f(P, y) == pytest.approx(np.sum((y - X) ** 2) + 0.7 * pen, rel=1e-13)


def test_dct_dictionary_is_scipy_orthonormal_dct(orc):
    m = 6
    Dm = orc.dct_dictionary(m)
    np.testing.assert_allclose(Dm @ Dm.T, np.eye(m * m), atol=1e-13)
    B = np.random.default_rng(1).standard_normal((m, m))
    c = scipy.fft.dctn(B, norm="ortho")
    np.testing.assert_allclose(c.ravel() @ Dm, B.ravel(), atol=1e-13)


def _patches_of(x, m, stride):
    ny, nx = x.shape
    kr = (ny - m + stride - 1) // stride + 1
    kc = (nx - m + stride - 1) // stride + 1
    rows = [min(k * stride, ny - m) for k in range(kr)]
    cols = [min(k * stride, nx - m) for k in range(kc)]
    return np.stack([x[r:r + m, c:c + m].ravel() for r in rows for c in cols])


@pytest.mark.parametrize("shape,m,stride", [((8, 8), 4, 2), ((11, 9), 4, 3), ((13, 10), 5, 2)])
def test_consistent_patches_rebuild_the_image(orc, shape, m, stride):
    """Patches cut from one image x (W = patches D^T, D orthonormal) agree
    everywhere, so Eq. 7 returns x, the penalty vanishes and f = ||y - Pi x||^2,
    for denoising and for tomography."""
    g = np.random.default_rng(2)
    x = g.standard_normal(shape)
    Dm = orc.dct_dictionary(m)
    W = _patches_of(x, m, stride) @ Dm.T
    np.testing.assert_allclose(orc.patch_assemble(W @ Dm, *shape, m, stride), x, atol=1e-13)
    y = g.standard_normal(shape)
    prob = orc.PatchProblem(*shape, m, stride, Dm, rho=3.0)
    assert prob.f(W, y) == pytest.approx(np.sum((y - x) ** 2), rel=1e-12)
    na, nb = 7, max(shape) + 3
    geo = orc.Geometry(np.arange(na) * math.pi / na + 0.1, (nb - 1) / 2 + 0.3, nb, shape[1], shape[0], 0.5)
    yt = g.standard_normal((na, nb))
    probt = orc.PatchProblem(*shape, m, stride, Dm, rho=3.0, g=geo)
    assert probt.f(W, yt) == pytest.approx(np.sum((yt - geo.P(x)) ** 2), rel=1e-12)


@pytest.mark.parametrize("tomo", [False, True])
@pytest.mark.parametrize("shape,m,stride,nc", [((8, 8), 4, 2, 16), ((11, 9), 4, 3, 20), ((10, 12), 3, 2, 9)])
def test_gradient_matches_finite_differences_of_eq8(orc, tomo, shape, m, stride, nc):
    """f is quadratic in W, so the central difference (f(W+hV) - f(W-hV)) / 2h
    equals <grad f, V> up to rounding; Algorithm 1's gradient (with the sign of
    Eq. 9 for the residual) must match it for random W, V, y, an
    over-complete random dictionary, ragged grids and both Pi."""
    g = np.random.default_rng(3 + nc)
    Dm = g.standard_normal((nc, m * m))
    geo = None
    if tomo:
        na, nb = 6, max(shape) + 2
        geo = orc.Geometry(np.arange(na) * math.pi / na + 0.05, (nb - 1) / 2 - 0.2, nb, shape[1], shape[0], 0.7)
        y = g.standard_normal((na, nb))
    else:
        y = g.standard_normal(shape)
    prob = orc.PatchProblem(*shape, m, stride, Dm, rho=0.8, g=geo)
    W = g.standard_normal(prob.shape_w)
    G = prob.gradient(W, y)
    for _ in range(4):
        V = g.standard_normal(prob.shape_w)
        h = 1e-3
        fd = (prob.f(W + h * V, y) - prob.f(W - h * V, y)) / (2 * h)
        assert np.vdot(G, V) == pytest.approx(fd, rel=1e-8, abs=1e-8 * abs(prob.f(W, y)))


def test_l1_shrinkage_closed_form_without_overlap(orc):
    """Denoising, stride = m (no overlap), complete orthonormal dictionary:
    every pixel is its own core, the penalty is zero and
    F = sum ||c_p - w_p||^2 + beta ||W||_1 with c_p the DCT of y's patch p,
    minimised by the soft threshold w = sign(c) max(|c| - beta/2, 0).  With
    L = 2 one ISTA/FISTA step from W = 0 lands on it and stays."""
    n, m = 12, 4
    Dm = orc.dct_dictionary(m)
    g = np.random.default_rng(4)
    y = g.standard_normal((n, n))
    prob = orc.PatchProblem(n, n, m, m, Dm, rho=5.0)
    C = _patches_of(y, m, m) @ Dm.T
    beta = 0.6
    Wref = np.sign(C) * np.maximum(np.abs(C) - beta / 2, 0.0)
    for fista in (False, True):
        W, e, X = prob.fista(y, beta, 2.0, 4, use_fista=fista)
        np.testing.assert_allclose(W, Wref, atol=1e-12)
        assert e[-1] == pytest.approx(np.sum((C - Wref) ** 2) + beta * np.abs(Wref).sum(), rel=1e-12)
        np.testing.assert_allclose(X, orc.patch_assemble(Wref @ Dm, n, n, m, m), atol=1e-12)


def _lipschitz(prob, y0):
    """Largest eigenvalue of the (constant) Hessian of f, built densely."""
    nw = prob.shape_w[0] * prob.shape_w[1]
    G0 = prob.gradient(np.zeros(prob.shape_w), y0)
    H = np.empty((nw, nw))
    for k in range(nw):
        e = np.zeros(nw)
        e[k] = 1.0
        H[:, k] = (prob.gradient(e.reshape(prob.shape_w), y0) - G0).ravel()
    assert np.allclose(H, H.T, atol=1e-10)                  # gradient of a quadratic: symmetric Hessian
    return np.linalg.eigvalsh(0.5 * (H + H.T)).max()


def test_ista_monotone_and_beta0_reaches_least_squares(orc):
    """Tomography on a tiny, fully determined system with overlapping patches
    and a complete dictionary: at beta = 0 the minimum of Eq. 8 is the
    least-squares image with consistent patches, so FISTA's image approaches
    the dense least-squares solution; ISTA's F never increases."""
    ny = nx = 6
    m, stride = 4, 2
    na, nb = 10, 9
    geo = orc.Geometry(np.arange(na) * math.pi / na + 0.02, (nb - 1) / 2 + 0.1, nb, nx, ny, 1.0)
    g = np.random.default_rng(5)
    xt = g.uniform(0, 1, (ny, nx))
    y = geo.P(xt) + 0.01 * g.standard_normal((na, nb))
    cols = []
    for k in range(ny * nx):
        e = np.zeros(ny * nx)
        e[k] = 1.0
        cols.append(geo.P(e.reshape(ny, nx)).ravel())
    A = np.stack(cols, 1)
    xls = np.linalg.lstsq(A, y.ravel(), rcond=None)[0].reshape(ny, nx)
    Dm = orc.dct_dictionary(m)
    prob = orc.PatchProblem(ny, nx, m, stride, Dm, rho=1.0, g=geo)
    L = 1.01 * _lipschitz(prob, y)
    _, ei, _ = prob.fista(y, 0.05, L, 80, use_fista=False)
    assert np.all(np.diff(ei) <= 1e-12 * abs(ei[0]))
    W, e, X = prob.fista(y, 0.0, L, 64000)              # ~1 s; the error falls as O(1/k^2)
    np.testing.assert_allclose(X, xls, atol=2e-6)
    assert e[-1] == pytest.approx(np.sum((y.ravel() - A @ xls.ravel()) ** 2), rel=1e-8)
