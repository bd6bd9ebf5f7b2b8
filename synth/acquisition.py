"""Seeded acquisitions: angles, detector geometry, flat/dark fields and
detector counts for the workloads the library is measured on.

Test and benchmark input generation only; no reconstruction arithmetic.  The
counts model follows the paper's raw-data description (radiographies plus an
averaged beam profile ("flat") and an averaged detector background ("dark"),
Sec. 2.3): I = Poisson(F_true * exp(-p)) + D with p the exact line integral.
Random numbers are drawn here and handed to both sides as input.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch

from . import phantoms as ph


def uniform_angles(n_angles: int) -> torch.Tensor:
    """theta_k = k * pi / n_angles (uniform over [0, 180 deg)), float32."""
    return (torch.arange(n_angles, dtype=torch.float64) * (math.pi / n_angles)).to(torch.float32)


def bin_offsets(angles: torch.Tensor, axis: torch.Tensor, n_bins: int, s: float,
                dtype=torch.float64, device=None) -> torch.Tensor:
    """Physical t of every (angle, bin): t = (b - axis(theta)) * s."""
    b = torch.arange(n_bins, dtype=dtype, device=device)
    return (b[None, :] - axis.to(dtype=dtype, device=device)[:, None]) * s


@dataclass
class Slice:
    """One slice's geometry and data (CPU tensors unless stated)."""
    angles: torch.Tensor          # [n_angles] float32 rad
    axis: torch.Tensor            # [n_angles] float32 bin index of the rotation axis
    n_bins: int
    nx: int
    ny: int
    pixel_size: float
    p: torch.Tensor = None        # [n_angles, n_bins] exact line integrals (float64)
    truth: torch.Tensor = None    # [ny, nx] density map
    extra: dict = field(default_factory=dict)


def poisson_counts(rate: torch.Tensor, gen: torch.Generator) -> torch.Tensor:
    return torch.poisson(rate, generator=gen)


# ---------------------------------------------------------------- C1 -------
def single_slice_fbp(seed: int = 0, n: int = 256, n_angles: int = 180, photons: float = 1e5,
                     axis: float = None, noise: bool = True) -> Slice:
    """256^2 grid, 180 angles over [0,180), 256 bins, axis at bin 127.5,
    seeded head-like 10-ellipse phantom, Poisson counts at 1e5 photons/bin,
    flat = 1e5, dark = 0.  Raw counts are float32 [n_angles, 1, n_bins]."""
    s = 2.0 / n
    ang = uniform_angles(n_angles)
    ax = torch.full((n_angles,), (n - 1) / 2.0 if axis is None else axis, dtype=torch.float32)
    ell = ph.head_phantom(seed)
    p = ph.ellipse_sinogram(ell, ang.double(), bin_offsets(ang, ax, n, s))
    gen = torch.Generator().manual_seed(seed)
    rate = photons * torch.exp(-p)
    counts = poisson_counts(rate, gen) if noise else rate
    sl = Slice(ang, ax, n, n, n, s, p=p, truth=ph.ellipse_image(ell, n, n, s, ss=4))
    sl.extra.update(raw=counts.to(torch.float32).reshape(n_angles, 1, n),
                    flat=torch.full((1, n), photons, dtype=torch.float32),
                    dark=torch.zeros((1, n), dtype=torch.float32), ellipses=ell)
    return sl


# ---------------------------------------------------------------- C2 -------
def flat_dark_fields(n_slices: int, n_bins: int, seed: int, level: float = 3e4,
                     ripple: float = 0.05, dark_mean: float = 100.0, dark_sd: float = 3.0):
    """Noise-free averaged fields [n_slices, n_bins]: dark = 100 + N(0, 3) per
    detector pixel; true beam = 3e4 * (1 + 0.05 * smooth low-order cosine
    profile); the recorded flat is beam + dark."""
    g = np.random.default_rng(seed + 7)
    D = dark_mean + dark_sd * g.standard_normal((n_slices, n_bins))
    ph1, ph2 = g.uniform(0, 2 * np.pi, 2)
    zz = (np.arange(n_slices)[:, None] + 0.5) / n_slices
    bb = (np.arange(n_bins)[None, :] + 0.5) / n_bins
    prof = 0.6 * np.cos(2 * np.pi * bb + ph1) * np.cos(np.pi * zz + ph2) + 0.4 * np.cos(4 * np.pi * bb + ph2)
    F_true = level * (1.0 + ripple * prof)
    return (torch.tensor(F_true + D, dtype=torch.float32), torch.tensor(D, dtype=torch.float32),
            torch.tensor(F_true, dtype=torch.float32))


@dataclass
class Volume:
    """A raw radiography stack [n_angles, n_slices, n_bins] (projection-major,
    as a detector writes it) with flat/dark fields [n_slices, n_bins]."""
    raw: torch.Tensor
    flat: torch.Tensor
    dark: torch.Tensor
    angles: torch.Tensor
    axis: torch.Tensor
    n_bins: int
    nx: int
    ny: int
    pixel_size: float
    z: torch.Tensor               # physical z of each slice
    ellipsoids: object = None


def ellipsoid_volume(n_slices: int, n: int, n_angles: int, seed: int, device="cpu",
                     n_ellipsoids: int = 200, slices=None, dtype=None, compact: bool = False) -> Volume:
    """Raw uint16 radiographies of ``n_ellipsoids`` random ellipsoids: the
    detector has n bins of size s = 2/n across [-1,1], the n_slices detector
    rows sit at z = (k - (n_slices-1)/2) * s.  Counts are
    clip(round(Poisson(F_true * exp(-p)) + D), 0, 65535), with the noise of
    detector row k drawn from its own seeded generator (so any subset of rows
    is generated identically on a given device).  ``slices`` restricts
    generation to a subset of rows: the others stay zero, or with
    ``compact`` the stack holds only the listed rows (flat/dark likewise)."""
    device = torch.device(device)
    dtype = dtype or (torch.float64 if device.type == "cpu" else torch.float32)
    s = 2.0 / n
    ang = uniform_angles(n_angles)
    ax = torch.full((n_angles,), (n - 1) / 2.0, dtype=torch.float32)
    E = ph.random_ellipsoids(n_ellipsoids, seed, z_half=0.5 * n_slices * s)
    flat, dark, F_true = flat_dark_fields(n_slices, n, seed)
    rows = list(range(n_slices)) if slices is None else list(slices)
    raw = torch.zeros((n_angles, len(rows) if compact else n_slices, n), dtype=torch.uint16, device=device)
    t = bin_offsets(ang, ax, n, s, dtype=dtype, device=device)
    th = ang.to(dtype=dtype, device=device)
    gen = torch.Generator(device=device)
    zs = (torch.arange(n_slices, dtype=torch.float64) - (n_slices - 1) / 2.0) * s
    Fd = F_true.to(device=device, dtype=dtype)
    Dd = dark.to(device=device, dtype=dtype)
    for o, k in enumerate(rows):
        ell = ph.ellipsoid_section(E, float(zs[k]))
        p = ph.ellipse_sinogram(ell, th, t) if len(ell) else torch.zeros_like(t)
        gen.manual_seed(seed * 1_000_003 + k)
        cnt = torch.poisson(Fd[k][None, :] * torch.exp(-p), generator=gen) + Dd[k][None, :]
        raw[:, o if compact else k, :] = torch.clamp(torch.round(cnt), 0, 65535).to(torch.int32).to(torch.uint16)
    if compact:
        flat, dark, zs = flat[rows], dark[rows], zs[rows]
    return Volume(raw, flat.to(device), dark.to(device), ang, ax, n, n, n, s, zs, E)


def ellipsoid_slice_truth(vol: Volume, k: int, ss: int = 2) -> torch.Tensor:
    ell = ph.ellipsoid_section(vol.ellipsoids, float(vol.z[k]))
    return ph.ellipse_image(ell, vol.nx, vol.ny, vol.pixel_size, ss=ss)


def ellipsoid_sinograms(n_slices: int, n: int, n_angles: int, seed: int, device="cpu",
                        slices=None, dtype=None, n_ellipsoids: int = 200) -> torch.Tensor:
    """Noise-free exact line integrals p [n_slices, n_angles, n] of the
    ellipsoid phantom (pre-normalised sinograms, for the precision study)."""
    device = torch.device(device)
    dtype = dtype or (torch.float64 if device.type == "cpu" else torch.float32)
    s = 2.0 / n
    ang = uniform_angles(n_angles)
    ax = torch.full((n_angles,), (n - 1) / 2.0, dtype=torch.float32)
    E = ph.random_ellipsoids(n_ellipsoids, seed, z_half=0.5 * n_slices * s)
    t = bin_offsets(ang, ax, n, s, dtype=dtype, device=device)
    th = ang.to(dtype=dtype, device=device)
    zs = (torch.arange(n_slices, dtype=torch.float64) - (n_slices - 1) / 2.0) * s
    idx = list(range(n_slices)) if slices is None else list(slices)
    out = torch.zeros((len(idx), n_angles, n), dtype=dtype, device=device)
    for o, k in enumerate(idx):
        ell = ph.ellipsoid_section(E, float(zs[k]))
        if len(ell):
            out[o] = ph.ellipse_sinogram(ell, th, t)
    return out


# ---------------------------------------------------------------- C3 -------
def foam_slice(n: int, n_angles: int, seed: int, photons: float = 1e4, device="cpu",
               truth: bool = True, dtype=None) -> Slice:
    """Reduced-dose slice: Voronoi foam of ~n/8 cells with 4 levels, exact
    line integrals, Poisson counts at ``photons`` per bin, returned as the
    pre-normalised sinogram -ln(max(I,1)/photons) (float32)."""
    device = torch.device(device)
    dtype = dtype or (torch.float64 if device.type == "cpu" else torch.float32)
    s = 2.0 / n
    ang = uniform_angles(n_angles)
    ax = torch.full((n_angles,), (n - 1) / 2.0, dtype=torch.float32)
    f = ph.random_foam(max(8, n // 8), seed)
    p = ph.foam_sinogram(f, ang.to(dtype=dtype, device=device),
                         bin_offsets(ang, ax, n, s, dtype=dtype, device=device))
    gen = torch.Generator(device=device).manual_seed(seed)
    I = torch.poisson(photons * torch.exp(-p), generator=gen)
    sino = -torch.log(torch.clamp(I, min=1.0) / photons)
    sl = Slice(ang, ax, n, n, n, s, p=p,
               truth=ph.foam_image(f, n, n, s, ss=4, device=device) if truth else None)
    sl.extra.update(sino=sino.to(torch.float32), foam=f)
    return sl


def ellipse_slice(n: int, n_angles: int, seed: int, photons: float = 1e4, n_ellipses: int = 12, device="cpu",
                  truth: bool = True, dtype=None) -> Slice:
    """Reduced-dose slice of ``n_ellipses`` random additive ellipses (the
    ellipse counterpart of foam_slice): exact line integrals, Poisson counts
    at ``photons`` per bin, pre-normalised sinogram (float32)."""
    device = torch.device(device)
    dtype = dtype or (torch.float64 if device.type == "cpu" else torch.float32)
    s = 2.0 / n
    ang = uniform_angles(n_angles)
    ax = torch.full((n_angles,), (n - 1) / 2.0, dtype=torch.float32)
    ell = ph.random_ellipses(n_ellipses, seed).to(device=device, dtype=dtype)
    p = ph.ellipse_sinogram(ell, ang.to(dtype=dtype, device=device),
                            bin_offsets(ang, ax, n, s, dtype=dtype, device=device))
    gen = torch.Generator(device=device).manual_seed(seed)
    I = torch.poisson(photons * torch.exp(-p), generator=gen)
    sino = -torch.log(torch.clamp(I, min=1.0) / photons)
    sl = Slice(ang, ax, n, n, n, s, p=p,
               truth=ph.ellipse_image(ell, n, n, s, ss=4, device=device) if truth else None)
    sl.extra.update(sino=sino.to(torch.float32))
    return sl


def mixed_tv_batch_plan(n_slices: int = 128, seed: int = 3000):
    """Sizes of the reduced-dose batch: 256^2/512^2/1024^2 with 50/100/200
    angles (one tenth of the detector width), split 43/43/42 and shuffled."""
    sizes = [(256, 50)] * 43 + [(512, 100)] * 43 + [(1024, 200)] * 42
    sizes = sizes[:n_slices] if n_slices <= 128 else sizes * (n_slices // 128 + 1)
    g = np.random.default_rng(seed)
    order = g.permutation(len(sizes))[:n_slices]
    return [sizes[i] for i in order]
