"""Seeded phantoms and their exact parallel-beam line integrals.

Test and benchmark input generation only.  Nothing here reconstructs: there is
no filtering, no back-projection and no discrete forward projection.  Sinograms
come from closed-form chord lengths (ellipses, ellipsoid cross-sections, convex
Voronoi cells), so they are independent of both the CPU oracle and the CUDA
path, which read their inputs from this module.

Coordinates (shared convention of the whole library):
  image pixel (row i, column j)  <->  physical (x, y) = ((j - cx) * s, (i - cy) * s)
  detector bin b at angle theta  <->  physical t = (b - axis(theta)) * s
  the ray of (theta, t) is the line {(x, y) : x cos(theta) + y sin(theta) = t}.
All functions take and return torch tensors; pass float64 on the CPU for
reference-quality inputs, float32 on a GPU for large volumes.
"""
from __future__ import annotations

import math

import numpy as np
import torch


# --------------------------------------------------------------------------
# ellipses in matrix form:  E = {u : (u - c)^T A (u - c) <= 1},  density mu
# --------------------------------------------------------------------------
class Ellipses:
    """A set of 2-D ellipses (centres ``c`` [E,2], SPD matrices ``A`` [E,2,2],
    densities ``mu`` [E]); densities add where ellipses overlap."""

    def __init__(self, c: torch.Tensor, A: torch.Tensor, mu: torch.Tensor):
        self.c, self.A, self.mu = c, A, mu

    def __len__(self):
        return int(self.mu.shape[0])

    def to(self, device=None, dtype=None):
        return Ellipses(self.c.to(device=device, dtype=dtype),
                        self.A.to(device=device, dtype=dtype),
                        self.mu.to(device=device, dtype=dtype))

    @staticmethod
    def from_axes(cx, cy, a, b, phi, mu, dtype=torch.float64, device=None):
        """Ellipses from centre, semi-axes (a along direction phi, b across) and
        density."""
        t = lambda v: torch.as_tensor(v, dtype=dtype, device=device).reshape(-1)
        cx, cy, a, b, phi, mu = map(t, (cx, cy, a, b, phi, mu))
        co, si = torch.cos(phi), torch.sin(phi)
        ia, ib = 1.0 / (a * a), 1.0 / (b * b)
        A = torch.empty(len(mu), 2, 2, dtype=dtype, device=device)
        A[:, 0, 0] = ia * co * co + ib * si * si
        A[:, 1, 1] = ia * si * si + ib * co * co
        A[:, 0, 1] = A[:, 1, 0] = (ia - ib) * co * si
        return Ellipses(torch.stack([cx, cy], 1), A, mu)


def ellipse_sinogram(ell: Ellipses, theta: torch.Tensor, t: torch.Tensor) -> torch.Tensor:
    """Exact line integrals sum_e mu_e * chord_e(theta, t).

    ``theta`` [n_angles] (rad), ``t`` [n_angles, n_bins] physical offsets.
    For the line u = t*n + tau*d (n = (cos, sin), d = (-sin, cos)) the ellipse
    condition is a quadratic alpha*tau^2 + 2*beta*tau + gamma <= 0, whose root
    spacing 2*sqrt(beta^2 - alpha*gamma)/alpha is the chord length.
    """
    dt, dev = t.dtype, t.device
    th = theta.to(dtype=dt, device=dev)
    n = torch.stack([torch.cos(th), torch.sin(th)], 1)          # [T,2]
    d = torch.stack([-torch.sin(th), torch.cos(th)], 1)
    out = torch.zeros_like(t)
    ell = ell.to(device=dev, dtype=dt)
    for e in range(len(ell)):
        A, c, mu = ell.A[e], ell.c[e], ell.mu[e]
        An, Ad, Ac = n @ A, d @ A, A @ c                       # A symmetric
        alpha = (Ad * d).sum(1)[:, None]
        k1 = (Ad * n).sum(1)[:, None]
        k2 = (d @ Ac)[:, None]
        m1 = (An * n).sum(1)[:, None]
        m2 = (n @ Ac)[:, None]
        m3 = c @ Ac
        beta = t * k1 - k2
        gamma = t * t * m1 - 2.0 * t * m2 + (m3 - 1.0)
        disc = torch.clamp(beta * beta - alpha * gamma, min=0.0)
        out += mu * 2.0 * torch.sqrt(disc) / alpha
    return out


def pixel_centres(nx: int, ny: int, s: float, cx=None, cy=None, ss: int = 1,
                  dtype=torch.float64, device=None):
    """Physical coordinates of ``ss x ss`` sub-samples of every pixel:
    x, y tensors of shape [ny*ss, nx*ss] (sub-pixel grid, row-major)."""
    cx = (nx - 1) / 2.0 if cx is None else cx
    cy = (ny - 1) / 2.0 if cy is None else cy
    off = (torch.arange(ss, dtype=dtype, device=device) + 0.5) / ss - 0.5
    jj = (torch.arange(nx, dtype=dtype, device=device)[:, None] + off[None, :]).reshape(-1)
    ii = (torch.arange(ny, dtype=dtype, device=device)[:, None] + off[None, :]).reshape(-1)
    y, x = torch.meshgrid((ii - cy) * s, (jj - cx) * s, indexing="ij")
    return x, y


def _box_mean(img: torch.Tensor, ss: int) -> torch.Tensor:
    if ss == 1:
        return img
    H, W = img.shape
    return img.reshape(H // ss, ss, W // ss, ss).mean(dim=(1, 3))


def ellipse_image(ell: Ellipses, nx: int, ny: int, s: float, ss: int = 1,
                  dtype=torch.float64, device=None) -> torch.Tensor:
    """Density map averaged over ss x ss sub-samples per pixel."""
    x, y = pixel_centres(nx, ny, s, ss=ss, dtype=dtype, device=device)
    ell = ell.to(device=device, dtype=dtype)
    img = torch.zeros_like(x)
    for e in range(len(ell)):
        ux, uy = x - ell.c[e, 0], y - ell.c[e, 1]
        A = ell.A[e]
        q = A[0, 0] * ux * ux + 2 * A[0, 1] * ux * uy + A[1, 1] * uy * uy
        img += torch.where(q <= 1.0, ell.mu[e], torch.zeros((), dtype=dtype, device=device))
    return _box_mean(img, ss)


def random_ellipses(n: int, seed: int, r_centres: float = 0.7, axes=(0.05, 0.4), density=(0.1, 0.6),
                    dtype=torch.float64) -> Ellipses:
    """``n`` ellipses with centres uniform in the disk r <= r_centres,
    semi-axes U(axes), orientations U(0, pi) and densities U(density)
    (additive where they overlap)."""
    g = np.random.default_rng(seed)
    rad = r_centres * np.sqrt(g.uniform(0, 1, n))
    ang = g.uniform(0, 2 * np.pi, n)
    return Ellipses.from_axes(rad * np.cos(ang), rad * np.sin(ang), g.uniform(*axes, n), g.uniform(*axes, n),
                              g.uniform(0, np.pi, n), g.uniform(*density, n), dtype=dtype)


def head_phantom(seed: int, dtype=torch.float64) -> Ellipses:
    """A seeded 10-ellipse head-like phantom on [-1,1]^2: a dense outer shell,
    a lower-density interior and eight small low-contrast features inside it.
    It has the structure of the classic analytic head phantoms (one skull,
    one brain, small lesions), with its own seeded parameters."""
    g = np.random.default_rng(seed)
    a0, b0 = g.uniform(0.62, 0.72), g.uniform(0.86, 0.94)
    shell = g.uniform(0.05, 0.09)
    cx = [0.0, 0.0]
    cy = [0.0, -g.uniform(0.0, 0.03)]
    a = [a0, a0 - shell]
    b = [b0, b0 - shell]
    phi = [0.0, 0.0]
    mu = [1.0, -0.8]
    for _ in range(8):
        r = g.uniform(0.03, 0.28)
        ratio = g.uniform(0.3, 1.0)
        ang = g.uniform(0, 2 * math.pi)
        rad = g.uniform(0, 1) ** 0.5 * 0.55
        cx.append(rad * math.cos(ang) * (a0 - shell) / b0)
        cy.append(rad * math.sin(ang))
        a.append(r)
        b.append(r * ratio)
        phi.append(g.uniform(0, math.pi))
        mu.append(g.choice([-1, 1]) * g.uniform(0.01, 0.1))
    return Ellipses.from_axes(cx, cy, a, b, phi, mu, dtype=dtype)


# --------------------------------------------------------------------------
# ellipsoids (3-D), sliced by planes z = const
# --------------------------------------------------------------------------
class Ellipsoids:
    """Ellipsoids {X : (X-C)^T M (X-C) <= 1} with densities ``mu``."""

    def __init__(self, C: torch.Tensor, M: torch.Tensor, mu: torch.Tensor):
        self.C, self.M, self.mu = C, M, mu

    def __len__(self):
        return int(self.mu.shape[0])


def random_ellipsoids(n: int, seed: int, r_centres: float = 0.8, z_half: float = 0.5,
                      semi=(0.02, 0.2), dtype=torch.float64) -> Ellipsoids:
    """``n`` ellipsoids with centres uniform in the cylinder r <= r_centres,
    |z| <= z_half, semi-axes uniform in ``semi``, uniformly random 3-D
    orientation and density uniform in (0, 1)."""
    g = np.random.default_rng(seed)
    rad = np.sqrt(g.uniform(0, 1, n)) * r_centres
    ang = g.uniform(0, 2 * np.pi, n)
    C = np.stack([rad * np.cos(ang), rad * np.sin(ang), g.uniform(-z_half, z_half, n)], 1)
    ax = g.uniform(semi[0], semi[1], (n, 3))
    q = g.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    R = np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)], 1),
        np.stack([2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)], 1),
        np.stack([2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)], 1)], 1)
    M = R @ (np.eye(3)[None] / (ax[:, :, None] ** 2)) @ np.transpose(R, (0, 2, 1))
    mu = g.uniform(0, 1, n)
    T = lambda v: torch.tensor(v, dtype=dtype)
    return Ellipsoids(T(C), T(M), T(mu))


def ellipsoid_section(E: Ellipsoids, z: float) -> Ellipses:
    """Cross-section ellipses of the plane z: completing the square in (x, y)
    gives (v)^T M2 v <= kappa with kappa = 1 - dz^2 (m33 - m^T M2^{-1} m)."""
    M2 = E.M[:, :2, :2]
    m = E.M[:, :2, 2]
    dz = z - E.C[:, 2]
    sol = torch.linalg.solve(M2, m.unsqueeze(-1)).squeeze(-1)   # M2^{-1} m
    kappa = 1.0 - dz * dz * (E.M[:, 2, 2] - (m * sol).sum(1))
    keep = kappa > 0
    c = E.C[keep, :2] - dz[keep, None] * sol[keep]
    A = M2[keep] / kappa[keep, None, None]
    return Ellipses(c, A, E.mu[keep])


# --------------------------------------------------------------------------
# foam: Voronoi cells of the unit disk with 4 density levels
# --------------------------------------------------------------------------
class Foam:
    """Voronoi partition of the unit disk; cell k has density ``level[k]``.
    ``nbr`` [K, D] lists Delaunay neighbours (-1 = padding)."""

    def __init__(self, sites: np.ndarray, level: np.ndarray, nbr: np.ndarray):
        self.sites, self.level, self.nbr = sites, level, nbr


def random_foam(n_sites: int, seed: int, levels=(0.0, 1 / 3, 2 / 3, 1.0)) -> Foam:
    from scipy.spatial import Delaunay
    g = np.random.default_rng(seed)
    rad = np.sqrt(g.uniform(0, 1, n_sites))
    ang = g.uniform(0, 2 * np.pi, n_sites)
    sites = np.stack([rad * np.cos(ang), rad * np.sin(ang)], 1)
    level = np.asarray(levels)[g.integers(0, len(levels), n_sites)]
    tri = Delaunay(sites)
    ptr, idx = tri.vertex_neighbor_vertices
    deg = np.diff(ptr)
    nbr = -np.ones((n_sites, deg.max()), dtype=np.int64)
    for k in range(n_sites):
        nbr[k, :deg[k]] = idx[ptr[k]:ptr[k + 1]]
    return Foam(sites, level, nbr)


def foam_sinogram(f: Foam, theta: torch.Tensor, t: torch.Tensor) -> torch.Tensor:
    """Exact line integrals of the foam: for each cell, the chord of the line
    through the convex cell = (unit-disk chord) intersected with the Voronoi
    half-planes 2 (s_j - s_k) . u <= |s_j|^2 - |s_k|^2 of its neighbours."""
    dt, dev = t.dtype, t.device
    th = theta.to(dtype=dt, device=dev)
    n = torch.stack([torch.cos(th), torch.sin(th)], 1)
    d = torch.stack([-torch.sin(th), torch.cos(th)], 1)
    S = torch.as_tensor(f.sites, dtype=dt, device=dev)
    half = torch.sqrt(torch.clamp(1.0 - t * t, min=0.0))
    out = torch.zeros_like(t)
    sq = (S * S).sum(1)
    for k in range(len(f.level)):
        if f.level[k] == 0.0:
            continue
        nb = f.nbr[k][f.nbr[k] >= 0]
        g = 2.0 * (S[nb] - S[k])                          # [D,2]
        h = sq[nb] - sq[k]                                # [D]
        gd = d @ g.T                                      # [T,D]
        gn = n @ g.T
        lo, hi = -half, half.clone()
        for q in range(len(nb)):
            rhs = h[q] - t * gn[:, q:q + 1]               # [T,B]
            gdq = gd[:, q:q + 1]
            bound = rhs / torch.where(gdq == 0, torch.ones_like(gdq), gdq)
            hi = torch.where(gdq > 0, torch.minimum(hi, bound), hi)
            lo = torch.where(gdq < 0, torch.maximum(lo, bound), lo)
            hi = torch.where((gdq == 0) & (rhs < 0), lo, hi)
        out += float(f.level[k]) * torch.clamp(hi - lo, min=0.0)
    return out


def foam_image(f: Foam, nx: int, ny: int, s: float, ss: int = 1,
               dtype=torch.float64, device=None) -> torch.Tensor:
    """Density map (nearest site inside the unit disk), ss x ss sub-samples."""
    x, y = pixel_centres(nx, ny, s, ss=ss, dtype=dtype, device=device)
    S = torch.as_tensor(f.sites, dtype=dtype, device=device)
    L = torch.as_tensor(f.level, dtype=dtype, device=device)
    pts = torch.stack([x.reshape(-1), y.reshape(-1)], 1)
    img = torch.empty(pts.shape[0], dtype=dtype, device=device)
    for s0 in range(0, pts.shape[0], 1 << 20):
        chunk = pts[s0:s0 + (1 << 20)]
        k = torch.cdist(chunk, S).argmin(1)
        inside = (chunk * chunk).sum(1) <= 1.0
        img[s0:s0 + (1 << 20)] = torch.where(inside, L[k], torch.zeros((), dtype=dtype, device=device))
    return _box_mean(img.reshape(x.shape), ss)
