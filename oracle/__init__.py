"""FP64 CPU oracle (test infrastructure only).

Only ``tests/``, the package's ``smoke()`` check and the benchmark's
CPU-baseline leg may import this package; the library itself never does, and
the oracle shares no code with the CUDA path.  The arithmetic lives in
``pyhst_oracle.c`` (plain loops, double precision, each function citing the
passage of the PyHST2 paper it follows); this module only marshals numpy
arrays to it.

Conventions: images are [ny, nx] (row i, column j); sinograms are
[n_angles, n_bins]; the detector coordinate of pixel (i, j) at angle th is
t = (j - cx) cos th + (i - cy) sin th + axis(th) in bin units.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pyhst_oracle.c")
_LIB = os.path.join(_HERE, "_pyhst_oracle.so")
_lib = None

D = ctypes.c_double
I64 = ctypes.c_int64
PD = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, -O2, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Geom(ctypes.Structure):
    _fields_ = [("n_angles", I64), ("n_bins", I64), ("nx", I64), ("ny", I64),
                ("angles", PD), ("axis", PD), ("cx", D), ("cy", D), ("pixel_size", D)]


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        L.orc_tv.restype = D
        L.orc_rof_gap.restype = D
        L.orc_energy.restype = D
        L.orc_power_iteration.restype = D
        L.orc_cosine.restype = D
        L.orc_patch_f.restype = D
        L.orc_ecohe.restype = D
        _lib = L
    return _lib


def _c(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(PD)


def num_threads() -> int:
    """Threads the OpenMP loops of the oracle use."""
    import multiprocessing
    return int(os.environ.get("OMP_NUM_THREADS", multiprocessing.cpu_count()))


# ------------------------------------------------------------------ pipeline
def normalise(I, F, D_):
    """Sec. 2.3 flat/dark correction, p = -ln((I-D)/(F-D)); one slice:
    I [n_rows, n_bins], F and D [n_bins]."""
    I, pI = _c(I)
    F, pF = _c(np.broadcast_to(F, I.shape[-1:]))
    D_, pD = _c(np.broadcast_to(D_, I.shape[-1:]))
    p = np.empty_like(I)
    lib().orc_normalise(pI, pF, pD, I64(I.shape[0]), I64(I.shape[1]), p.ctypes.data_as(PD))
    return p


def ramlak_filter(p):
    """Ram-Lak filtered rows, q[m] = sum_k h(m-k) p[k] (Sec. 2.3)."""
    p, pp = _c(p)
    q = np.empty_like(p)
    lib().orc_ramlak_filter(pp, I64(p.shape[0]), I64(p.shape[1]), q.ctypes.data_as(PD))
    return q


FILTERS = {"ramlak": 0, "shepp-logan": 1, "hann": 2}


def filter_rows(p, kind="ramlak"):
    """Rows filtered with the spatial kernel of `kind` (ramlak, shepp-logan,
    hann): q[m] = sum_k h(m-k) p[k]."""
    p, pp = _c(p)
    q = np.empty_like(p)
    lib().orc_filter(pp, I64(p.shape[0]), I64(p.shape[1]), ctypes.c_int(FILTERS[kind]), q.ctypes.data_as(PD))
    return q


def _centre(n, c):
    return (n - 1) / 2.0 if c is None else float(c)


def backproject(q, angles, axis, nx, ny, weight=1.0, cx=None, cy=None):
    """weight * sum_a L(q_a, t_a(i, j)) (Sec. 2.3)."""
    q, pq = _c(q)
    na, nb = q.shape
    ang, pa = _c(np.asarray(angles, dtype=np.float64).reshape(na))
    ax, px = _c(np.broadcast_to(np.asarray(axis, dtype=np.float64), (na,)))
    img = np.empty((ny, nx))
    lib().orc_backproject(pq, I64(na), I64(nb), pa, px, I64(nx), I64(ny),
                          D(_centre(nx, cx)), D(_centre(ny, cy)), D(weight), img.ctypes.data_as(PD))
    return img


def backproject_at(q, angles, axis, nx, ny, ii, jj, weight=1.0, cx=None, cy=None):
    """The back-projection at pixels (ii[k], jj[k]) only."""
    q, pq = _c(q)
    na, nb = q.shape
    ang, pa = _c(np.asarray(angles, dtype=np.float64).reshape(na))
    ax, px = _c(np.broadcast_to(np.asarray(axis, dtype=np.float64), (na,)))
    ii = np.ascontiguousarray(ii, dtype=np.int64)
    jj = np.ascontiguousarray(jj, dtype=np.int64)
    out = np.empty(len(ii))
    P64 = ctypes.POINTER(ctypes.c_int64)
    lib().orc_backproject_at(pq, I64(na), I64(nb), pa, px, ii.ctypes.data_as(P64), jj.ctypes.data_as(P64),
                             I64(len(ii)), D(_centre(nx, cx)), D(_centre(ny, cy)), D(weight),
                             out.ctypes.data_as(PD))
    return out


def project(img, angles, axis, n_bins, scale=1.0, cx=None, cy=None):
    """scale * (transpose of the unweighted back-projector) applied to img."""
    img, pi = _c(img)
    ny, nx = img.shape
    na = len(angles)
    ang, pa = _c(np.asarray(angles, dtype=np.float64).reshape(na))
    ax, px = _c(np.broadcast_to(np.asarray(axis, dtype=np.float64), (na,)))
    sino = np.empty((na, n_bins))
    lib().orc_project(pi, I64(na), I64(n_bins), pa, px, I64(nx), I64(ny),
                      D(_centre(nx, cx)), D(_centre(ny, cy)), D(scale), sino.ctypes.data_as(PD))
    return sino


def fbp_weight(n_angles, pixel_size):
    """pi / (n_angles * s): uniform angular weight over 180 degrees."""
    return math.pi / (n_angles * pixel_size)


def fbp_from_sinogram(p, angles, axis, nx, ny, pixel_size, cx=None, cy=None):
    """Filter then back-project a normalised sinogram p [n_angles, n_bins]."""
    q = ramlak_filter(p)
    return backproject(q, angles, axis, nx, ny, fbp_weight(len(angles), pixel_size), cx, cy)


def fbp_from_raw(raw, flat, dark, angles, axis, nx, ny, pixel_size, cx=None, cy=None):
    """Full per-slice path: normalise, filter, back-project.  raw is the
    slice's sinogram of counts [n_angles, n_bins], flat/dark [n_bins]."""
    return fbp_from_sinogram(normalise(raw, flat, dark), angles, axis, nx, ny, pixel_size, cx, cy)


# ------------------------------------------------------------------ TV / FISTA
def grad(x):
    x, px = _c(x)
    g1, g2 = np.empty_like(x), np.empty_like(x)
    lib().orc_grad(px, I64(x.shape[0]), I64(x.shape[1]), g1.ctypes.data_as(PD), g2.ctypes.data_as(PD))
    return g1, g2


def div(p1, p2):
    p1, a = _c(p1)
    p2, b = _c(p2)
    d = np.empty_like(p1)
    lib().orc_div(a, b, I64(p1.shape[0]), I64(p1.shape[1]), d.ctypes.data_as(PD))
    return d


def tv(x):
    """Eq. 2."""
    x, px = _c(x)
    return lib().orc_tv(px, I64(x.shape[0]), I64(x.shape[1]))


def tv_prox(z, lam, n_inner, tau=0.125, p=None):
    """prox of lam*TV by Chambolle's fixed point; returns (x, p1, p2)."""
    z, pz = _c(z)
    ny, nx = z.shape
    p1 = np.zeros_like(z) if p is None else np.array(p[0], dtype=np.float64)
    p2 = np.zeros_like(z) if p is None else np.array(p[1], dtype=np.float64)
    x = np.empty_like(z)
    lib().orc_tv_prox(pz, I64(ny), I64(nx), D(lam), D(tau), I64(n_inner),
                      p1.ctypes.data_as(PD), p2.ctypes.data_as(PD), x.ctypes.data_as(PD))
    return x, p1, p2


def rof_gap(z, lam, p1, p2):
    z, pz = _c(z)
    p1, a = _c(p1)
    p2, b = _c(p2)
    return lib().orc_rof_gap(pz, I64(z.shape[0]), I64(z.shape[1]), D(lam), a, b)


class Geometry:
    """One slice's geometry for the solver functions."""

    def __init__(self, angles, axis, n_bins, nx, ny, pixel_size, cx=None, cy=None):
        self.angles = np.ascontiguousarray(np.asarray(angles, dtype=np.float64))
        self.axis = np.ascontiguousarray(np.broadcast_to(np.asarray(axis, dtype=np.float64),
                                                         self.angles.shape))
        self.n_bins, self.nx, self.ny = int(n_bins), int(nx), int(ny)
        self.pixel_size = float(pixel_size)
        self.cx, self.cy = _centre(nx, cx), _centre(ny, cy)

    def _c(self):
        return _Geom(len(self.angles), self.n_bins, self.nx, self.ny,
                     self.angles.ctypes.data_as(PD), self.axis.ctypes.data_as(PD),
                     self.cx, self.cy, self.pixel_size)

    def P(self, x):
        return project(x, self.angles, self.axis, self.n_bins, self.pixel_size, self.cx, self.cy)

    def PT(self, y):
        return backproject(y, self.angles, self.axis, self.nx, self.ny, self.pixel_size, self.cx, self.cy)


def energy(g: Geometry, sino, x, beta):
    """Eq. 3: 1/2 ||sino - P x||^2 + beta TV(x)."""
    sino, ps = _c(sino)
    x, px = _c(x)
    gc = g._c()
    return lib().orc_energy(ctypes.byref(gc), ps, px, D(beta))


def power_iteration(g: Geometry, v0, n_it=50):
    """Largest eigenvalue of P^T P from start vector v0 [ny, nx]."""
    v = np.array(v0, dtype=np.float64, copy=True)
    gc = g._c()
    lam = lib().orc_power_iteration(ctypes.byref(gc), v.ctypes.data_as(PD), I64(n_it))
    return lam, v


def fista(g: Geometry, sino, beta, L, n_iter, n_inner=20, tau=0.125, use_fista=True, x0=None, return_z=False,
          return_gap=False, warm_dual=False):
    """ISTA/FISTA on Eq. 3; returns (x, energy history [n_iter]), then, with
    return_z, the prox input z of the last iteration and, with return_gap,
    the ROF duality gap of every iteration's prox [n_iter].  warm_dual: each
    prox's dual field starts at the previous one's final field instead of
    zero."""
    sino, ps = _c(sino)
    x = np.zeros((g.ny, g.nx)) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    e = np.empty(n_iter)
    z = np.empty((g.ny, g.nx)) if return_z else None
    gp = np.empty(n_iter) if return_gap else None
    gc = g._c()
    lib().orc_fista_z(ctypes.byref(gc), ps, D(beta), D(L), I64(n_iter), I64(n_inner), D(tau),
                      ctypes.c_int(1 if use_fista else 0), x.ctypes.data_as(PD), e.ctypes.data_as(PD),
                      gp.ctypes.data_as(PD) if return_gap else None, z.ctypes.data_as(PD) if return_z else None,
                      ctypes.c_int(1 if warm_dual else 0))
    out = (x, e) + ((z,) if return_z else ()) + ((gp,) if return_gap else ())
    return out


# ------------------------------------------------------------------ beta estimators (Sec. 4)
def cosine(a, b):
    a, pa = _c(a)
    b, pb = _c(b)
    return lib().orc_cosine(pa, pb, I64(a.size))


def ecohe(I_beta, I_0):
    """Eq. 11: Cos(I(beta) - I(0+), I(beta))."""
    a, pa = _c(I_beta)
    b, pb = _c(I_0)
    return lib().orc_ecohe(pa, pb, I64(a.size))


def cross_validation(g: Geometry, sino, held_out, betas, L, n_iter, n_inner=20, tau=0.125):
    """Cross-validation estimator (Sec. 4): reconstruct without the projection
    at angle index held_out, project the result at that angle, return the
    squared distance to the held-out data for each beta, plus the images."""
    keep = [a for a in range(len(g.angles)) if a != held_out]
    gk = Geometry(g.angles[keep], g.axis[keep], g.n_bins, g.nx, g.ny, g.pixel_size, g.cx, g.cy)
    sino = np.asarray(sino, dtype=np.float64)
    errs, imgs = [], []
    for b in betas:
        x, _ = fista(gk, sino[keep], b, L, n_iter, n_inner=n_inner, tau=tau)
        row = project(x, g.angles[held_out:held_out + 1], g.axis[held_out:held_out + 1], g.n_bins,
                      g.pixel_size, g.cx, g.cy)[0]
        errs.append(float(np.sum((row - sino[held_out]) ** 2)))
        imgs.append(x)
    return np.array(errs), imgs


# ------------------------------------------------------------------ preprocessing variants (Sec. 2.3)
def flatfield(I, flats, pos, D):
    """I [na, nz, nb], flats [nf, nz, nb], pos [na] (ignored for one flat),
    D [nz, nb] -> r = (I - D) / (F(pos) - D)."""
    I, pI = _c(I)
    flats, pf = _c(flats)
    na, nz, nb = I.shape
    nf = flats.shape[0]
    pos, pp = _c(np.zeros(na) if pos is None else pos)
    D, pD = _c(D)
    r = np.empty_like(I)
    lib().orc_flatfield(pI, pf, I64(nf), pp, pD, I64(na), I64(nz), I64(nb), r.ctypes.data_as(PD))
    return r


def hotspot(r, threshold):
    r, pr = _c(r)
    out = np.empty_like(r)
    na, nz, nb = r.shape
    lib().orc_hotspot(pr, I64(na), I64(nz), I64(nb), D(threshold), out.ctypes.data_as(PD))
    return out


def neglog(r):
    r, pr = _c(r)
    p = np.empty_like(r)
    lib().orc_log(pr, I64(r.size), p.ctypes.data_as(PD))
    return p


def ring(p, window):
    """Ring filter of one sinogram p [na, nb] (returns a corrected copy)."""
    p = np.array(p, dtype=np.float64, copy=True)
    lib().orc_ring(p.ctypes.data_as(PD), I64(p.shape[0]), I64(p.shape[1]), I64(window))
    return p


def preprocess(I, flats, pos, D, hotspot_threshold=0.0, ring_window=0):
    """Sec. 2.3 order: flat field, hot spots, -ln, rearrangement into
    sinograms, ring filter.  Returns p [nz, na, nb]."""
    r = flatfield(I, flats, pos, D)
    if hotspot_threshold > 0:
        r = hotspot(r, hotspot_threshold)
    p = np.ascontiguousarray(neglog(r).transpose(1, 0, 2))
    if ring_window > 0:
        p = np.stack([ring(pz, ring_window) for pz in p])
    return p


# ------------------------------------------------------------------ overlapping patches (Eqs. 4-9, Algorithm 1)
class _PatchProb(ctypes.Structure):
    _fields_ = [("ny", I64), ("nx", I64), ("m", I64), ("stride", I64), ("nc", I64), ("D", PD), ("rho", D),
                ("denoise", ctypes.c_int), ("g", ctypes.c_void_p)]


def patch_grid(ny, nx, m, stride):
    kr, kc = I64(), I64()
    lib().orc_patch_grid(I64(ny), I64(nx), I64(m), I64(stride), ctypes.byref(kr), ctypes.byref(kc))
    return kr.value, kc.value


def dct_dictionary(m):
    Dm = np.empty((m * m, m * m))
    lib().orc_dct_dictionary(I64(m), Dm.ctypes.data_as(PD))
    return Dm


def patch_assemble(P, ny, nx, m, stride):
    P, pp = _c(P)
    X = np.empty((ny, nx))
    lib().orc_patch_assemble(pp, I64(ny), I64(nx), I64(m), I64(stride), X.ctypes.data_as(PD))
    return X


def patch_sum(P, ny, nx, m, stride):
    P, pp = _c(P)
    S, Nv = np.empty((ny, nx)), np.empty((ny, nx))
    lib().orc_patch_sum(pp, I64(ny), I64(nx), I64(m), I64(stride), S.ctypes.data_as(PD), Nv.ctypes.data_as(PD))
    return S, Nv


class PatchProblem:
    """Eq. 8 on an ny x nx image: patch size m, stride, dictionary Dm [nc, m*m],
    rho; geometry g (tomography) or None (denoising, Pi = identity)."""

    def __init__(self, ny, nx, m, stride, Dm, rho, g: "Geometry" = None):
        self.Dm = np.ascontiguousarray(Dm, dtype=np.float64)
        self.g = g
        self._gc = g._c() if g is not None else None
        self.s = _PatchProb(ny, nx, m, stride, self.Dm.shape[0], self.Dm.ctypes.data_as(PD), rho,
                            1 if g is None else 0,
                            ctypes.cast(ctypes.pointer(self._gc), ctypes.c_void_p) if g is not None else None)
        self.kr, self.kc = patch_grid(ny, nx, m, stride)
        self.shape_w = (self.kr * self.kc, self.Dm.shape[0])

    def f(self, W, y):
        W, pw = _c(W)
        y, py = _c(y)
        return lib().orc_patch_f(ctypes.byref(self.s), pw, py)

    def gradient(self, W, y):
        W, pw = _c(W)
        y, py = _c(y)
        G = np.empty(self.shape_w)
        lib().orc_patch_gradient(ctypes.byref(self.s), pw, py, G.ctypes.data_as(PD))
        return G

    def fista(self, y, beta, L, n_iter, use_fista=True, W0=None):
        y, py = _c(y)
        W = np.zeros(self.shape_w) if W0 is None else np.array(W0, dtype=np.float64, copy=True)
        e = np.empty(n_iter)
        X = np.empty((self.s.ny, self.s.nx))
        lib().orc_patch_fista(ctypes.byref(self.s), py, D(beta), D(L), I64(n_iter), ctypes.c_int(1 if use_fista else 0),
                              W.ctypes.data_as(PD), e.ctypes.data_as(PD), X.ctypes.data_as(PD))
        return W, e, X
