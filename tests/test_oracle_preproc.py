"""Pins of the oracle's preprocessing variants (Sec. 2.3): flats interpolated
in time, the hot-spot median filter and the ring filter (no GPU)."""
import math

import numpy as np
import pytest


def test_flat_interpolation_closed_forms(orc):
    """Two flats with constant values 100 and 300 over a dark of 20: a
    projection at position 0.25 sees F = 150; position 1 picks the second
    flat; a single flat reduces to the one-flat normalisation."""
    na, nz, nb = 3, 2, 5
    flats = np.stack([np.full((nz, nb), 100.0), np.full((nz, nb), 300.0)])
    D = np.full((nz, nb), 20.0)
    I = np.full((na, nz, nb), 85.0)
    r = orc.flatfield(I, flats, np.array([0.25, 1.0, 0.0]), D)
    np.testing.assert_allclose(r[0], (85 - 20) / (150 - 20), rtol=1e-15)
    np.testing.assert_allclose(r[1], (85 - 20) / (300 - 20), rtol=1e-15)
    np.testing.assert_allclose(r[2], (85 - 20) / (100 - 20), rtol=1e-15)
    g = np.random.default_rng(0)
    I = g.uniform(50, 900, (na, nz, nb))
    F = g.uniform(900, 1000, (nz, nb))
    D = g.uniform(0, 40, (nz, nb))
    p = orc.neglog(orc.flatfield(I, F[None], None, D))
    for z in range(nz):
        np.testing.assert_allclose(p[:, z], orc.normalise(I[:, z], F[z], D[z]), rtol=0, atol=1e-14)


def test_hotspot_replaces_only_outliers(orc):
    """A single hot pixel in a smooth field takes its neighbours' median; a
    pixel within the threshold is kept; an even neighbour count (edge) uses
    the mean of the two middle values."""
    r = np.tile(np.linspace(0.5, 0.6, 9)[None, None, :], (2, 7, 1))
    r[0, 3, 4] = 0.95                      # hot
    r[1, 3, 4] += 0.01                     # within threshold
    out = orc.hotspot(r, 0.05)
    neigh = np.sort([r[0, z, b] for z in (2, 3, 4) for b in (3, 4, 5) if (z, b) != (3, 4)])
    assert out[0, 3, 4] == pytest.approx(0.5 * (neigh[3] + neigh[4]), rel=1e-15)
    assert out[1, 3, 4] == r[1, 3, 4]
    mask = np.ones_like(r, bool)
    mask[0, 3, 4] = False
    np.testing.assert_array_equal(out[mask], r[mask])
    # corner pixel: 3 neighbours, odd count -> the middle value
    r2 = np.zeros((1, 3, 3))
    r2[0, 0, 0] = 1.0
    r2[0, 0, 1], r2[0, 1, 0], r2[0, 1, 1] = 0.1, 0.3, 0.2
    assert orc.hotspot(r2, 0.1)[0, 0, 0] == pytest.approx(0.2)


def test_ring_filter_closed_form(orc):
    """A stripe delta on one detector column (a ring artefact) over an
    angularly constant-mean background: the angular mean's high-pass part is
    delta (1 - 1/w) at the column and -delta/w on its w-1 neighbours inside the
    window, so the corrected stripe keeps delta / w and the neighbours get
    +delta / w; a sinogram whose angular mean is locally linear is unchanged."""
    na, nb, w, b0, delta = 16, 40, 5, 20, 0.3
    p = np.zeros((na, nb))
    p[:, b0] = delta
    out = orc.ring(p, w)
    exp = np.zeros(nb)
    exp[b0] = delta / w
    for c in (18, 19, 21, 22):
        exp[c] = delta / w
    np.testing.assert_allclose(out, np.tile(exp, (na, 1)), atol=1e-15)
    g = np.random.default_rng(1)
    noise = g.standard_normal((na, nb))
    lin = noise - noise.mean(0, keepdims=True) + 0.01 * np.arange(nb)[None, :]   # angular mean 0.01 b
    out = orc.ring(lin, w)
    np.testing.assert_allclose(out[:, w:-w], lin[:, w:-w], atol=1e-12)


def test_preprocess_all_off_equals_normalisation(orc):
    g = np.random.default_rng(2)
    na, nz, nb = 4, 3, 6
    I = g.uniform(100, 900, (na, nz, nb))
    F = g.uniform(950, 1000, (nz, nb))
    D = g.uniform(0, 50, (nz, nb))
    p = orc.preprocess(I, F[None], None, D)
    for z in range(nz):
        np.testing.assert_allclose(p[z], orc.normalise(I[:, z], F[z], D[z]), atol=1e-14)
