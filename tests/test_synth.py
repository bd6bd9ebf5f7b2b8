"""The seeded input generators (synth/): closed forms of the phantoms' exact
line integrals, and the determinism that the workloads' seeds rely on."""
import math

import numpy as np
import torch

from synth import acquisition as acq
from synth import phantoms as ph


def test_disk_sinogram_closed_form():
    """An ellipse with equal semi-axes r is a disk: its line integral at
    (theta, t) is 2 mu sqrt(r^2 - (t - x0 cos theta - y0 sin theta)^2)."""
    x0, y0, r, mu = 0.21, -0.13, 0.37, 0.8
    ell = ph.Ellipses.from_axes(x0, y0, r, r, 0.6, mu)
    theta = torch.linspace(0, math.pi, 7, dtype=torch.float64)
    t = torch.linspace(-0.9, 0.9, 41, dtype=torch.float64)[None].repeat(7, 1)
    got = ph.ellipse_sinogram(ell, theta, t)
    u = t - (x0 * torch.cos(theta) + y0 * torch.sin(theta))[:, None]
    ref = 2 * mu * torch.sqrt(torch.clamp(r * r - u * u, min=0.0))
    assert torch.allclose(got, ref, rtol=0, atol=1e-12)


def test_ellipsoid_section_of_a_sphere():
    """The plane z cuts a sphere of radius R centred at (a, b, c) in the disk
    of radius sqrt(R^2 - (z - c)^2) centred at (a, b)."""
    R, C = 0.3, torch.tensor([[0.1, -0.2, 0.05]], dtype=torch.float64)
    E = ph.Ellipsoids(C, torch.eye(3, dtype=torch.float64)[None] / R ** 2, torch.tensor([0.5], dtype=torch.float64))
    sec = ph.ellipsoid_section(E, 0.2)
    rr = R * R - 0.15 ** 2
    assert len(sec) == 1
    assert torch.allclose(sec.c, C[:, :2], atol=1e-15)
    assert torch.allclose(sec.A[0], torch.eye(2, dtype=torch.float64) / rr, rtol=1e-12)
    assert len(ph.ellipsoid_section(E, 0.4)) == 0            # the plane misses the sphere


def test_uniform_foam_is_the_unit_disk():
    """The Voronoi cells partition the unit disk, so with every level set to
    1 the exact cell chords add up to the disk's chord 2 sqrt(1 - t^2)."""
    f = ph.random_foam(40, seed=5)
    f = ph.Foam(f.sites, np.ones_like(f.level), f.nbr)
    theta = torch.linspace(0, math.pi, 9, dtype=torch.float64)[:-1]
    t = torch.linspace(-0.99, 0.99, 57, dtype=torch.float64)[None].repeat(8, 1)
    got = ph.foam_sinogram(f, theta, t)
    ref = 2 * torch.sqrt(1 - t * t)
    assert torch.allclose(got, ref, rtol=0, atol=1e-9)


def test_generators_are_seeded():
    a = acq.foam_slice(64, 24, seed=7, truth=False).extra["sino"]
    b = acq.foam_slice(64, 24, seed=7, truth=False).extra["sino"]
    c = acq.foam_slice(64, 24, seed=8, truth=False).extra["sino"]
    assert torch.equal(a, b) and not torch.equal(a, c)
    e1 = acq.ellipsoid_sinograms(16, 32, 10, seed=4000, slices=[3, 9])
    e2 = acq.ellipsoid_sinograms(16, 32, 10, seed=4000, slices=[9])
    assert torch.equal(e1[1], e2[0])                          # a slice does not depend on which others are made


def test_mixed_batch_plan():
    """128 slices: 43 of 256^2 / 50 angles, 43 of 512^2 / 100, 42 of
    1024^2 / 200, in a seeded order."""
    p = acq.mixed_tv_batch_plan()
    assert len(p) == 128
    assert sorted(set(p)) == [(256, 50), (512, 100), (1024, 200)]
    assert [p.count(s) for s in [(256, 50), (512, 100), (1024, 200)]] == [43, 43, 42]
    assert p == acq.mixed_tv_batch_plan() and p != acq.mixed_tv_batch_plan(seed=3001)
