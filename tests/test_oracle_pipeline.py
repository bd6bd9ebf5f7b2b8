"""Pins of the FP64 oracle's FBP pipeline against closed forms, brute force
and invariants (no GPU).  Each test states what fixes the expected value."""
import math

import numpy as np
import pytest
import torch

from synth import acquisition as acq
from synth import phantoms as ph


# ------------------------------------------------------------- normalisation
def test_normalise_recovers_line_integrals(orc):
    """Noise-free counts I = D + (F - D) exp(-p) give back p (Sec. 2.3)."""
    g = np.random.default_rng(1)
    p = g.uniform(-0.2, 4.0, (7, 33))
    D = g.uniform(90, 110, 33)
    F = D + g.uniform(2e4, 4e4, 33)
    I = D + (F - D) * np.exp(-p)
    np.testing.assert_allclose(orc.normalise(I, F, D), p, rtol=0, atol=1e-11)


def test_normalise_degenerate_counts(orc):
    """Dead flat (F <= D) gives 0; counts at or below dark are clamped to
    ratio 1e-6; counts above the flat give negative p."""
    F = np.array([100.0, 50.0, 1000.0, 1000.0, 1000.0])
    D = np.array([100.0, 80.0, 100.0, 100.0, 100.0])
    I = np.array([[500.0, 500.0, 100.0, 40.0, 1900.0]])
    p = orc.normalise(I, F, D)[0]
    assert p[0] == 0.0 and p[1] == 0.0
    assert p[2] == pytest.approx(-math.log(1e-6)) and p[3] == pytest.approx(-math.log(1e-6))
    assert p[4] == pytest.approx(-math.log(2.0))


# ------------------------------------------------------------- ramp filter
def test_filter_equals_padded_circular_fft(orc):
    """The direct sum equals the circular convolution of the row zero-padded
    to P >= 2 n_bins with h periodised on [-P/2, P/2) (convolution theorem,
    computed here with numpy's FFT)."""
    g = np.random.default_rng(2)
    for nb in (5, 64, 127, 256):
        p = g.standard_normal((3, nb))
        q = orc.ramlak_filter(p)
        for P in (2 * nb, 2 * nb + 6, 4 * nb):
            n = np.arange(P)
            n = np.where(n < (P + 1) // 2, n, n - P)         # periodised offsets
            nf = np.where(n == 0, 1, n).astype(float)
            h = np.where(n == 0, 0.25, np.where(n % 2 != 0, -1.0 / (math.pi ** 2 * nf ** 2), 0.0))
            pad = np.zeros((3, P))
            pad[:, :nb] = p
            ref = np.real(np.fft.ifft(np.fft.fft(pad, axis=1) * np.fft.fft(h)[None], axis=1))[:, :nb]
            np.testing.assert_allclose(q, ref, rtol=0, atol=1e-12 * max(1.0, np.abs(ref).max()))


def test_filter_is_a_ramp_in_frequency(orc):
    """The Ram-Lak kernel's frequency response is |f| (f in cycles per bin,
    |f| <= 1/2): a long cosine row comes out scaled by |f| away from the
    edges (truncation error ~ 1/(pi^2 * distance to the edge))."""
    nb = 4096
    k = np.arange(nb)
    for f in (0.0, 1 / 64, 0.1, 0.25, 0.37):
        row = np.cos(2 * math.pi * f * k + 0.3)
        q = orc.ramlak_filter(row[None])[0]
        mid = slice(1536, 2560)
        np.testing.assert_allclose(q[mid], abs(f) * row[mid], atol=2e-4)


# ------------------------------------------------------------- projector pair
def _dense_A(angles, axis, nb, nx, ny, cx, cy):
    """System matrix from the hat-function definition, entry by entry."""
    A = np.zeros((len(angles) * nb, ny * nx))
    for a, th in enumerate(angles):
        for i in range(ny):
            for j in range(nx):
                t = (j - cx) * math.cos(th) + (i - cy) * math.sin(th) + axis[a]
                for b in range(nb):
                    A[a * nb + b, i * nx + j] = max(0.0, 1.0 - abs(t - b))
    return A


@pytest.mark.parametrize("case", range(8))
def test_projector_pair_brute_force(orc, case):
    """Tiny grids with off-centre axes: the oracle's projector equals the
    dense hat-function matrix and its back-projector equals the transpose."""
    g = np.random.default_rng(100 + case)
    nx, ny = int(g.integers(4, 10)), int(g.integers(4, 10))
    na, nb = int(g.integers(1, 8)), int(g.integers(5, 14))
    angles = np.concatenate([[0.0, math.pi / 2][:min(2, na)], g.uniform(0, math.pi, max(0, na - 2))])
    axis = g.uniform(0.3 * nb, 0.7 * nb, na)
    cx, cy = (nx - 1) / 2 + g.uniform(-1, 1), (ny - 1) / 2 + g.uniform(-1, 1)
    A = _dense_A(angles, axis, nb, nx, ny, cx, cy)
    x = g.standard_normal((ny, nx))
    y = g.standard_normal((na, nb))
    np.testing.assert_allclose(orc.project(x, angles, axis, nb, 1.0, cx, cy).ravel(), A @ x.ravel(),
                               rtol=0, atol=1e-12)
    np.testing.assert_allclose(orc.backproject(y, angles, axis, nx, ny, 1.0, cx, cy).ravel(),
                               A.T @ y.ravel(), rtol=0, atol=1e-12)


def test_adjoint_identity(orc):
    """<P x, y> = <x, P^T y> to 1e-10 relative (spec tolerance)."""
    g = np.random.default_rng(5)
    n, na, nb = 64, 37, 70
    angles = np.sort(g.uniform(0, math.pi, na))
    axis = 34.5 + g.uniform(-2, 2, na)
    x = g.standard_normal((n, n))
    y = g.standard_normal((na, nb))
    s = 0.03
    lhs = np.vdot(orc.project(x, angles, axis, nb, s), y)
    rhs = np.vdot(x, orc.backproject(y, angles, axis, n, n, s))
    assert abs(lhs - rhs) <= 1e-10 * abs(lhs)


def test_zero_angle_is_column_sums(orc):
    """theta = 0 with the axis on the same half-integer grid as cx: every
    pixel lands exactly on a bin, so the projection is the column sums."""
    g = np.random.default_rng(6)
    n = 16
    x = g.standard_normal((n, n))
    sino = orc.project(x, [0.0], [(n - 1) / 2.0 + 3.0], n + 6)
    np.testing.assert_allclose(sino[0, 3:3 + n], x.sum(0), atol=1e-12)
    assert np.all(sino[0, :3] == 0) and np.all(sino[0, 3 + n:] == 0)


def _disk_projection(orc, n, angles, r=0.45, mu=1.5, x0=0.2, y0=-0.3):
    s = 2.0 / n
    ell = ph.Ellipses.from_axes([x0], [y0], [r], [r], [0.0], [mu])
    img = ph.ellipse_image(ell, n, n, s, ss=8).numpy()
    sino = orc.project(img, angles, (n - 1) / 2.0, n, scale=s)
    t = (np.arange(n)[None, :] - (n - 1) / 2.0) * s - (x0 * np.cos(angles) + y0 * np.sin(angles))[:, None]
    ref = 2 * mu * np.sqrt(np.clip(r * r - t * t, 0, None))
    err = np.linalg.norm(sino - ref, axis=1) / np.linalg.norm(ref, axis=1)
    return img, sino, err


def test_projection_of_disk_matches_radon_closed_form(orc):
    """A pixel-averaged disk projects to the closed form 2 mu sqrt(r^2 - t'^2):
    at 0 and 90 degrees pixels land exactly on bins and the error is the
    grid's partial-volume error; at a generic angle it shrinks with the grid;
    at every angle the projection conserves mass exactly (the hat weights of
    a pixel sum to one).  Near 45 degrees a pixel-driven linear-interpolation
    projector has a lattice ripple that does not shrink with the grid; its
    bound was measured once (6.7 %) and is frozen here."""
    angles = np.array([0.0, math.pi / 2, 0.3, math.pi / 4])
    img, sino, err = _disk_projection(orc, 256, angles)
    assert err[0] < 3e-3 and err[1] < 3e-3, err
    assert err[3] < 0.07, err
    s = 2.0 / 256
    np.testing.assert_allclose(sino.sum(1), s * img.sum(), rtol=1e-12)
    _, _, err_lo = _disk_projection(orc, 128, angles[2:3])
    _, _, err_hi = _disk_projection(orc, 512, angles[2:3])
    assert err_hi[0] < err_lo[0] / 3, (err_lo, err_hi)


# ------------------------------------------------------------- FBP end to end
def test_fbp_of_analytic_disk(orc):
    """FBP of the closed-form disk sinogram is mu inside the disk (away from
    the edge), ~0 outside, and centred where the disk is (orientation)."""
    n, s, na = 128, 2.0 / 128, 180
    r, mu, x0, y0 = 0.35, 2.0, 0.3, -0.2
    angles = np.arange(na) * math.pi / na
    t = (np.arange(n)[None, :] - (n - 1) / 2.0) * s - (x0 * np.cos(angles) + y0 * np.sin(angles))[:, None]
    p = 2 * mu * np.sqrt(np.clip(r * r - t * t, 0, None))
    img = orc.fbp_from_sinogram(p, angles, (n - 1) / 2.0, n, n, s)
    yy, xx = np.meshgrid((np.arange(n) - (n - 1) / 2.0) * s, (np.arange(n) - (n - 1) / 2.0) * s, indexing="ij")
    rr = np.hypot(xx - x0, yy - y0)
    inner, outer = rr < r - 6 * s, rr > r + 6 * s
    assert abs(img[inner].mean() - mu) < 0.01 * mu
    assert np.abs(img[inner] - mu).max() < 0.04 * mu
    out = img[outer & (np.hypot(xx, yy) < 0.9)]
    assert np.abs(out).mean() < 0.015 * mu and np.abs(out).max() < 0.06 * mu  # measured 0.010 mu, 0.045 mu
    w = np.clip(img, 0, None)
    assert abs((w * xx).sum() / w.sum() - x0) < s and abs((w * yy).sum() / w.sum() - y0) < s


def test_fbp_single_slice_workload_quality(orc):
    """256^2 / 180 angles head-like phantom from Poisson counts at 1e5
    photons: the reconstruction approximates the phantom (PSNR measured
    once on the noise-free data and frozen with margin)."""
    sl = acq.single_slice_fbp(seed=0, noise=False)
    raw = sl.extra["raw"][:, 0, :].numpy()
    img = orc.fbp_from_raw(raw, sl.extra["flat"][0].numpy(), sl.extra["dark"][0].numpy(),
                           sl.angles.double().numpy(), sl.axis.double().numpy(), sl.nx, sl.ny, sl.pixel_size)
    truth = sl.truth.numpy()
    yy, xx = np.meshgrid(np.arange(256) - 127.5, np.arange(256) - 127.5, indexing="ij")
    disk = np.hypot(xx, yy) <= 127
    mse = np.mean((img - truth)[disk] ** 2)
    psnr = 10 * math.log10((truth.max() - truth.min()) ** 2 / mse)
    assert psnr > 24.0, psnr


@pytest.mark.parametrize("case", range(3))
def test_backproject_at_equals_full_backprojection(orc, case):
    """The spot-check back-projection (used by every full-size parity test)
    evaluates the same sum as the whole-image back-projection at every pixel
    of small non-square, off-centre geometries with per-angle axes, so a
    swapped row/column or a wrong centre in it shows up here."""
    g = np.random.default_rng(300 + case)
    nx, ny = ((23, 17), (31, 12), (9, 40))[case]
    na, nb = int(g.integers(5, 30)), int(g.integers(20, 50))
    angles = g.uniform(0, math.pi, na)
    axis = (nb - 1) / 2.0 + g.uniform(-4, 4, na)
    cx, cy = (nx - 1) / 2 + g.uniform(-3, 3), (ny - 1) / 2 + g.uniform(-3, 3)
    q = g.standard_normal((na, nb))
    w = float(g.uniform(0.5, 2.0))
    full = orc.backproject(q, angles, axis, nx, ny, w, cx, cy)
    ii, jj = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    at = orc.backproject_at(q, angles, axis, nx, ny, ii.ravel(), jj.ravel(), w, cx, cy)
    np.testing.assert_allclose(at, full.ravel(), rtol=0, atol=1e-14 * np.abs(full).max())
    # and both equal the transpose of the dense hat-function matrix
    A = _dense_A(angles, axis, nb, nx, ny, cx, cy)
    np.testing.assert_allclose(at, w * (A.T @ q.ravel()), rtol=0, atol=1e-12 * np.abs(full).max())
