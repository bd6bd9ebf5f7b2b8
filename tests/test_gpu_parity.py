"""GPU parity of the FBP path and the projector pair against the FP64 oracle.

Every comparison goes through the C ABI (the package's binding only marshals
arguments).  Tolerances are the float32 bar: relative L2 <= 1e-5 and
max-abs <= 1e-4 * max|reference|.
"""
import math

import numpy as np
import pytest
import torch

from synth import acquisition as acq

pytestmark = pytest.mark.gpu

REL_L2 = 1e-5
MAX_ABS = 1e-4


def close(got, ref, rel=REL_L2, mx=MAX_ABS):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    scale = np.abs(ref).max()
    e = got - ref
    r = np.linalg.norm(e) / max(np.linalg.norm(ref), 1e-300)
    m = np.abs(e).max() / max(scale, 1e-300)
    assert r <= rel and m <= mx, f"rel L2 {r:.3e} (<= {rel}), max-abs/max {m:.3e} (<= {mx})"
    return r, m


@pytest.fixture(scope="module")
def P():
    import paper_1306_1392_b300 as P
    return P


def geometry(P, angles, axis, n_bins, nx, ny, s, dev, cx=None, cy=None):
    return P.Geometry(torch.as_tensor(np.asarray(angles), dtype=torch.float32, device=dev).contiguous(),
                      torch.as_tensor(np.broadcast_to(np.asarray(axis, dtype=np.float64), (len(angles),)).copy(),
                                      dtype=torch.float32, device=dev),
                      n_bins, nx, ny, s, cx, cy)


def f64(t):
    return t.detach().double().cpu().numpy()


CASES = [
    # (n_angles, n_bins, nx, ny, angles kind, axis offset, seed)
    (180, 256, 256, 256, "uniform", 0.0, 0),
    (37, 131, 100, 77, "random", 3.3, 1),        # ragged tiles, off-centre axis
    (1, 64, 64, 64, "zero", 0.0, 2),              # single angle
    (64, 96, 160, 40, "wide", -2.7, 3),           # angles beyond pi, negative angles
    (33, 300, 129, 257, "random", 10.0, 4),
    (30, 1100, 1024, 1024, "random", 1.5, 5),     # few angles, large image: rows split into 16 segments
    (24, 2400, 96, 2300, "random", -4.0, 10),     # tall image: a walk of 144 chunks (two band windows)
]


def _case(P, dev, na, nb, nx, ny, kind, off, seed):
    g = np.random.default_rng(seed)
    if kind == "uniform":
        ang = np.arange(na) * math.pi / na
    elif kind == "zero":
        ang = np.zeros(na)
    elif kind == "wide":
        ang = g.uniform(-2 * math.pi, 3 * math.pi, na)
    else:
        ang = np.sort(g.uniform(0, math.pi, na))
    ang = ang.astype(np.float32)
    axis = ((nb - 1) / 2.0 + off + g.uniform(-0.5, 0.5, na)).astype(np.float32)
    return g, ang, axis, geometry(P, ang, axis, nb, nx, ny, 2.0 / max(nx, ny), dev)


@pytest.mark.parametrize("case", CASES)
def test_backproject_parity(P, orc, cuda_device, case):
    na, nb, nx, ny, kind, off, seed = case
    g, ang, axis, geo = _case(P, cuda_device, *case)
    sino = g.standard_normal((2, na, nb)).astype(np.float32)
    w = 0.37
    got = P.pyhst_backproject(geo, torch.from_numpy(sino).to(cuda_device), w)
    torch.cuda.synchronize()
    for z in range(2):
        ref = orc.backproject(sino[z].astype(np.float64), ang.astype(np.float64), axis.astype(np.float64),
                              nx, ny, w)
        close(f64(got[z]), ref)


@pytest.mark.parametrize("case", CASES)
def test_project_parity(P, orc, cuda_device, case):
    na, nb, nx, ny, kind, off, seed = case
    g, ang, axis, geo = _case(P, cuda_device, *case)
    img = g.standard_normal((2, ny, nx)).astype(np.float32)
    got = P.pyhst_project(geo, torch.from_numpy(img).to(cuda_device))
    torch.cuda.synchronize()
    for z in range(2):
        ref = orc.project(img[z].astype(np.float64), ang.astype(np.float64), axis.astype(np.float64), nb,
                          geo.pixel_size)
        if np.abs(ref).max() == 0:
            assert np.abs(f64(got[z])).max() == 0
        else:
            close(f64(got[z]), ref)


@pytest.mark.parametrize("na,ns,n_check", [(2000, 4, 24), (150, 1, 30)])
def test_project_full_size_sampled_angles(P, orc, cuda_device, na, ns, n_check):
    """The projector at full size: a 2048^2 grid with 2048 bins, either the
    dense 2000-angle set in 4-slice launches (the back-projector's workload)
    or 150 angles (the sparse variant: 512-column staging and row segments).
    Each sinogram row depends on its own angle only, so sampled angles
    (including the first, the last and those next to 45 and 135 degrees,
    where the walk switches between rows and columns) are checked whole
    against the oracle projecting just those angles."""
    n = 2048
    ang = (np.arange(na) * math.pi / na).astype(np.float32)
    axis = np.full(na, (n - 1) / 2.0 + 0.37, np.float32)
    geo = geometry(P, ang, axis, n, n, n, 2.0 / n, cuda_device)
    g = torch.Generator(device=cuda_device).manual_seed(na)
    img = torch.rand((ns, n, n), device=cuda_device, generator=g)
    got = P.pyhst_project(geo, img)
    torch.cuda.synchronize()
    rng = np.random.default_rng(na)
    near = [int(np.argmin(np.abs(ang - t))) + d for t in (math.pi / 4, 3 * math.pi / 4) for d in (-1, 0, 1)]
    sel = sorted(set([0, na - 1] + [k for k in near if 0 <= k < na] + list(rng.choice(na, n_check, replace=False))))
    for z in sorted({0, ns - 1}):
        ref = orc.project(img[z].double().cpu().numpy(), ang[sel].astype(np.float64), axis[sel].astype(np.float64),
                          n, geo.pixel_size)
        close(f64(got[z][sel]), ref)


def test_projector_pair_is_adjoint(P, cuda_device):
    """<P x, y> = <x, P^T y> for the GPU pair (float32 outputs, float64 dots)."""
    g = np.random.default_rng(9)
    na, nb, n = 90, 200, 160
    ang = np.sort(g.uniform(0, math.pi, na)).astype(np.float32)
    geo = geometry(P, ang, (nb - 1) / 2 + 1.3, nb, n, n, 0.01, cuda_device)
    x = torch.from_numpy(g.standard_normal((1, n, n)).astype(np.float32)).to(cuda_device)
    y = torch.from_numpy(g.standard_normal((1, na, nb)).astype(np.float32)).to(cuda_device)
    px = P.pyhst_project(geo, x)
    pty = P.pyhst_backproject(geo, y, geo.pixel_size)
    lhs = (px.double() * y.double()).sum().item()
    rhs = (x.double() * pty.double()).sum().item()
    assert abs(lhs - rhs) <= 1e-5 * max(abs(lhs), abs(rhs))


def test_project_rays_outside_image_are_zero(P, cuda_device):
    """An axis far off the detector: every ray misses the image."""
    geo = geometry(P, np.array([0.0, 0.7, 2.0], np.float32), 5000.0, 64, 32, 32, 0.1, cuda_device)
    got = P.pyhst_project(geo, torch.ones((1, 32, 32), device=cuda_device))
    assert torch.count_nonzero(got).item() == 0
    back = P.pyhst_backproject(geo, torch.ones((1, 3, 64), device=cuda_device), 1.0)
    assert torch.count_nonzero(back).item() == 0


def test_non_finite_angles_contribute_nothing(P, cuda_device):
    """A NaN or infinite angle/axis entry is skipped, not read out of range."""
    ang = np.array([0.3, np.nan, 1.1, np.inf], np.float32)
    axis = np.array([31.5, 31.5, np.nan, 31.5], np.float32)
    geo = geometry(P, ang, axis, 64, 48, 48, 0.1, cuda_device)
    sino = torch.ones((1, 4, 64), device=cuda_device)
    got = P.pyhst_backproject(geo, sino, 1.0)
    ok = geometry(P, ang[:1], axis[:1], 64, 48, 48, 0.1, cuda_device)
    ref = P.pyhst_backproject(ok, sino[:, :1].contiguous(), 1.0)
    torch.testing.assert_close(got, ref, rtol=0, atol=0)


# ------------------------------------------------------------------ FBP
def test_fbp_single_slice_counts(P, orc, cuda_device):
    """256^2, 180 angles, 256 bins, Poisson counts at 1e5 photons, flat 1e5,
    dark 0, Ram-Lak, padding 512: the single-slice FBP workload."""
    sl = acq.single_slice_fbp(seed=0)
    raw = sl.extra["raw"]                              # [180, 1, 256] float32
    geo = geometry(P, sl.angles.numpy(), sl.axis.numpy(), sl.n_bins, sl.nx, sl.ny, sl.pixel_size, cuda_device)
    got = P.pyhst_fbp(geo, raw.to(cuda_device), "f32_raw", sl.extra["flat"].to(cuda_device),
                      sl.extra["dark"].to(cuda_device), pad_len=512)
    torch.cuda.synchronize()
    ref = orc.fbp_from_raw(raw[:, 0, :].double().numpy(), sl.extra["flat"][0].double().numpy(),
                           sl.extra["dark"][0].double().numpy(), sl.angles.double().numpy(),
                           sl.axis.double().numpy(), sl.nx, sl.ny, sl.pixel_size)
    close(f64(got[0]), ref)


def _oracle_fbp_stack(orc, vol, z):
    raw = vol.raw[:, z, :].to(torch.float64).cpu().numpy()
    return orc.fbp_from_raw(raw, vol.flat[z].double().cpu().numpy(), vol.dark[z].double().cpu().numpy(),
                            vol.angles.double().numpy(), vol.axis.double().numpy(), vol.nx, vol.ny,
                            vol.pixel_size)


@pytest.mark.parametrize("ws_slices", [1, 3, 8])
def test_fbp_uint16_volume_in_place(P, orc, cuda_device, ws_slices):
    """Raw uint16 radiography stack [angles][slices][bins] read in place with
    seeded flat/dark fields; workspaces of 1, 3 and 8 slices per pass."""
    vol = acq.ellipsoid_volume(n_slices=6, n=96, n_angles=120, seed=11, n_ellipsoids=40)
    geo = geometry(P, vol.angles.numpy(), vol.axis.numpy(), vol.n_bins, vol.nx, vol.ny, vol.pixel_size,
                   cuda_device)
    g6 = geo.c(6)
    import ctypes
    from paper_1306_1392_b300 import _lib
    fixed = _lib.lib.pyhst_workspace_size(ctypes.byref(geo.c(1)), _lib.PYHST_OP_FBP) - 120 * 96 * 4
    ws = torch.empty(fixed + ws_slices * 120 * 96 * 4 + 4096, dtype=torch.uint8, device=cuda_device)
    got = P.pyhst_fbp(geo, vol.raw.to(cuda_device), "u16_raw", vol.flat.to(cuda_device),
                      vol.dark.to(cuda_device), workspace=ws)
    torch.cuda.synchronize()
    for z in range(6):
        close(f64(got[z]), _oracle_fbp_stack(orc, vol, z))


@pytest.mark.parametrize("kind,dt", [("f32_sino", torch.float32), ("f16_sino", torch.float16),
                                     ("bf16_sino", torch.bfloat16)])
def test_fbp_sinogram_kinds(P, orc, cuda_device, kind, dt):
    """Pre-normalised sinograms stored in float32 / float16 / bfloat16: the
    GPU converts on load; the oracle gets the same rounded values."""
    p = acq.ellipsoid_sinograms(2, 128, 90, seed=5, n_ellipsoids=30)   # [2, 90, 128] float64
    stored = p.to(dt)
    ang = acq.uniform_angles(90).numpy()
    geo = geometry(P, ang, 63.5, 128, 128, 128, 2 / 128, cuda_device)
    got = P.pyhst_fbp(geo, stored.to(cuda_device).contiguous(), kind)
    torch.cuda.synchronize()
    for z in range(2):
        ref = orc.fbp_from_sinogram(stored[z].double().numpy(), ang.astype(np.float64), 63.5, 128, 128, 2 / 128)
        close(f64(got[z]), ref)


@pytest.mark.parametrize("pad", [0, 1024, 4096])
def test_fbp_padding_lengths_agree(P, orc, cuda_device, pad):
    """Any padding >= 2 n_bins gives the same linear convolution."""
    p = acq.ellipsoid_sinograms(1, 200, 60, seed=6, n_ellipsoids=20)
    ang = acq.uniform_angles(60).numpy()
    geo = geometry(P, ang, 99.5, 200, 150, 170, 0.01, cuda_device)
    got = P.pyhst_fbp(geo, p.float().to(cuda_device), "f32_sino", pad_len=pad)
    torch.cuda.synchronize()
    ref = orc.fbp_from_sinogram(p[0].float().double().numpy(), ang.astype(np.float64), 99.5, 150, 170, 0.01)
    close(f64(got[0]), ref)


def test_fbp_full_size_volume_sampled(P, orc, cuda_device):
    """The batched-volume workload's slice geometry (2048^2 grid, 2000 angles,
    2048 bins, uint16 raw with flat/dark) in the launch configuration the
    benchmark times (passes of 16 slices): sampled pixels of 2 slices of a
    16-slice stack against the oracle evaluated at those pixels."""
    n, na, ns = 2048, 2000, 16
    vol = acq.ellipsoid_volume(n_slices=ns, n=n, n_angles=na, seed=1000, device=cuda_device, slices=[2, 5])
    geo = geometry(P, vol.angles.numpy(), vol.axis.numpy(), n, n, n, vol.pixel_size, cuda_device)
    got = P.pyhst_fbp(geo, vol.raw, "u16_raw", vol.flat, vol.dark)
    torch.cuda.synchronize()
    rng = np.random.default_rng(0)
    for z in (2, 5):
        raw = vol.raw[:, z, :].double().cpu().numpy()
        q = orc.ramlak_filter(orc.normalise(raw, vol.flat[z].double().cpu().numpy(),
                                            vol.dark[z].double().cpu().numpy()))
        ii = np.concatenate([rng.integers(0, n, 1500), [0, n - 1, 0, n - 1, n // 2]])
        jj = np.concatenate([rng.integers(0, n, 1500), [0, 0, n - 1, n - 1, n // 2]])
        ref = orc.backproject_at(q, vol.angles.double().numpy(), vol.axis.double().numpy(), n, n, ii, jj,
                                 orc.fbp_weight(na, vol.pixel_size))
        g = got[z].cpu().numpy()[ii, jj]
        close(g, ref)


def test_filter_only_parity(P, orc, cuda_device):
    """pyhst_filter: normalised and Ram-Lak filtered rows (the first two
    steps of the FBP) against the oracle's, for raw uint16 input."""
    vol = acq.ellipsoid_volume(n_slices=3, n=200, n_angles=50, seed=21, n_ellipsoids=30)
    geo = geometry(P, vol.angles.numpy(), vol.axis.numpy(), vol.n_bins, vol.nx, vol.ny, vol.pixel_size,
                   cuda_device)
    q = P.pyhst_filter(geo, vol.raw.to(cuda_device), "u16_raw", vol.flat.to(cuda_device), vol.dark.to(cuda_device))
    torch.cuda.synchronize()
    for z in range(3):
        ref = orc.ramlak_filter(orc.normalise(vol.raw[:, z, :].double().numpy(), vol.flat[z].double().numpy(),
                                              vol.dark[z].double().numpy()))
        close(f64(q[z]), ref)


@pytest.mark.parametrize("n_slices,chunk", [(7, 1), (7, 3), (7, 8), (40, 16)])
def test_fbp_host_pipeline_matches_device_call(P, cuda_device, n_slices, chunk):
    """pyhst_fbp_host on pinned host buffers gives bitwise the device call's
    slices, for chunk sizes that do and do not divide the stack (40 slices in
    chunks of up to 16: 1, 4, 14, 16, 4, 1)."""
    vol = acq.ellipsoid_volume(n_slices=n_slices, n=128, n_angles=90, seed=31, n_ellipsoids=40)
    geo = geometry(P, vol.angles.numpy(), vol.axis.numpy(), vol.n_bins, vol.nx, vol.ny, vol.pixel_size,
                   cuda_device)
    dev_out = P.pyhst_fbp(geo, vol.raw.to(cuda_device), "u16_raw", vol.flat.to(cuda_device),
                          vol.dark.to(cuda_device))
    host_out = P.pyhst_fbp_host(geo, vol.raw.contiguous().pin_memory(), "u16_raw", vol.flat.pin_memory(),
                                vol.dark.pin_memory(), slices_per_chunk=chunk)
    torch.cuda.synchronize()
    assert torch.equal(host_out, dev_out.cpu())


def test_fbp_slice_range_in_place(P, cuda_device):
    """A slice range of a resident stack, read in place, equals the same
    slices of a whole-stack call."""
    vol = acq.ellipsoid_volume(n_slices=9, n=96, n_angles=60, seed=41, n_ellipsoids=40)
    geo = geometry(P, vol.angles.numpy(), vol.axis.numpy(), vol.n_bins, vol.nx, vol.ny, vol.pixel_size,
                   cuda_device)
    raw, fl, dk = vol.raw.to(cuda_device), vol.flat.to(cuda_device), vol.dark.to(cuda_device)
    full = P.pyhst_fbp(geo, raw, "u16_raw", fl, dk)
    part = P.pyhst_fbp(geo, raw, "u16_raw", fl, dk, slices=(3, 8))
    torch.cuda.synchronize()
    assert torch.equal(full[3:8], part)


@pytest.mark.parametrize("kind,dt", [("f32_sino", torch.float32), ("f16_sino", torch.float16),
                                     ("bf16_sino", torch.bfloat16)])
def test_fbp_4096_geometry_sampled(P, orc, cuda_device, kind, dt):
    """The mixed-precision workload's slice geometry (4096^2 grid, 4000
    angles, 4096 bins, FFT length 8192): stored f32 / f16 / bf16 sinogram, sampled
    pixels against the oracle evaluated on the same stored values."""
    n, na = 4096, 4000
    p = acq.ellipsoid_sinograms(256, n, na, seed=4000, device=cuda_device, slices=[100])
    stored = p.to(dt).contiguous()
    ang = acq.uniform_angles(na)
    geo = geometry(P, ang.numpy(), (n - 1) / 2.0, n, n, n, 2.0 / n, cuda_device)
    got = P.pyhst_fbp(geo, stored, kind)
    torch.cuda.synchronize()
    q = orc.ramlak_filter(stored[0].double().cpu().numpy())
    rng = np.random.default_rng(1)
    ii = np.concatenate([rng.integers(0, n, 1200), [0, n - 1, n // 2]])
    jj = np.concatenate([rng.integers(0, n, 1200), [n - 1, 0, n // 2]])
    ref = orc.backproject_at(q, ang.double().numpy(), (n - 1) / 2.0, n, n, ii, jj, orc.fbp_weight(na, 2.0 / n))
    close(got[0].cpu().numpy()[ii, jj], ref)


def test_fbp_shards_reassemble_the_volume(P, cuda_device):
    """Each rank's contiguous share (computed here one after the other on one
    GPU) equals the same slices of a single whole-stack call."""
    from paper_1306_1392_b300.shard import fbp_shard
    vol = acq.ellipsoid_volume(n_slices=7, n=64, n_angles=40, seed=61, n_ellipsoids=30)
    geo = geometry(P, vol.angles.numpy(), vol.axis.numpy(), vol.n_bins, vol.nx, vol.ny, vol.pixel_size,
                   cuda_device)
    raw, fl, dk = vol.raw.to(cuda_device), vol.flat.to(cuda_device), vol.dark.to(cuda_device)
    full = P.pyhst_fbp(geo, raw, "u16_raw", fl, dk)
    parts = [fbp_shard(geo, raw, "u16_raw", fl, dk, world=3, rank=r) for r in range(3)]
    torch.cuda.synchronize()
    assert [p[:2] for p in parts] == [(0, 3), (3, 5), (5, 7)]
    assert torch.equal(torch.cat([p[2] for p in parts]), full)


# ------------------------------------------------------------------ preprocessing variants (Sec. 2.3)
def test_fbp_pre_all_off_equals_fbp(P, cuda_device):
    vol = acq.ellipsoid_volume(n_slices=5, n=80, n_angles=60, seed=71, n_ellipsoids=30)
    geo = geometry(P, vol.angles.numpy(), vol.axis.numpy(), vol.n_bins, vol.nx, vol.ny, vol.pixel_size,
                   cuda_device)
    raw, fl, dk = vol.raw.to(cuda_device), vol.flat.to(cuda_device), vol.dark.to(cuda_device)
    a = P.pyhst_fbp(geo, raw, "u16_raw", fl, dk)
    b = P.pyhst_fbp_pre(geo, raw, "u16_raw", fl, dk)
    torch.cuda.synchronize()
    assert torch.equal(a, b)


def test_fbp_pre_flats_hotspots_rings_parity(P, orc, cuda_device):
    """Three flats interpolated in time, hot pixels (ratio jumps of ~1.5 far
    above the 0.2 threshold, so float32 and float64 decide alike) and a
    detector column 5 % too sensitive (a ring): the GPU path against the
    oracle's preprocessing, filter and back-projection."""
    ns, n, na = 6, 96, 90
    vol = acq.ellipsoid_volume(n_slices=ns, n=n, n_angles=na, seed=72, n_ellipsoids=40)
    raw = vol.raw.to(torch.float64)
    scale = torch.tensor([0.97, 1.0, 1.04], dtype=torch.float64)
    pos = torch.linspace(0, 2, na, dtype=torch.float64)
    f0 = torch.floor(pos).clamp(max=1)
    w = pos - f0
    s_a = (1 - w) * scale[f0.long()] + w * scale[f0.long() + 1]          # beam drift per projection
    F_true = vol.flat.double() - vol.dark.double()
    counts = (raw - vol.dark.double()[None]) * s_a[:, None, None] + vol.dark.double()[None]
    counts[:, :, 37] = (counts[:, :, 37] - vol.dark.double()[None, :, 37]) * 1.05 + vol.dark.double()[None, :, 37]
    g = np.random.default_rng(3)
    for _ in range(25):
        a, z, b = int(g.integers(0, na)), int(g.integers(0, ns)), int(g.integers(1, n - 1))
        counts[a, z, b] = counts[a, z, b] * 2.5 + 20000
    counts = counts.round().clamp(0, 65535)
    raw16 = counts.to(torch.int32).to(torch.uint16)
    flats = torch.stack([vol.dark.double() + F_true * s for s in scale]).float()
    geo = geometry(P, vol.angles.numpy(), vol.axis.numpy(), n, n, n, vol.pixel_size, cuda_device)
    got = P.pyhst_fbp_pre(geo, raw16.to(cuda_device), "u16_raw", flats.to(cuda_device), vol.dark.to(cuda_device),
                          flat_pos=pos.float().to(cuda_device), hotspot_threshold=0.2, ring_window=9)
    torch.cuda.synchronize()
    p = orc.preprocess(raw16.double().numpy(), flats.double().numpy(), pos.float().double().numpy(),
                       vol.dark.double().numpy(), hotspot_threshold=0.2, ring_window=9)
    for z in range(ns):
        ref = orc.backproject(orc.ramlak_filter(p[z]), vol.angles.double().numpy(), vol.axis.double().numpy(), n, n,
                              orc.fbp_weight(na, vol.pixel_size))
        close(f64(got[z]), ref)


def test_fbp_pre_full_size_sampled(P, orc, cuda_device):
    """The preprocessing study's configuration (Sec. 2.3: three flats
    interpolated by projection position, hot-spot median with threshold 0.2,
    ring filter of window 9) on the batched-volume geometry (2048^2, 2000
    angles, 2048 bins, uint16, an 8-slice stack in one call): sampled pixels
    of two slices against the oracle's preprocessing of the stack, filter and
    back-projection at those pixels."""
    n, na, ns = 2048, 2000, 8
    vol = acq.ellipsoid_volume(n_slices=ns, n=n, n_angles=na, seed=1100, device=cuda_device)
    dev = cuda_device
    scale = torch.tensor([0.97, 1.0, 1.04], dtype=torch.float32, device=dev)
    pos = torch.linspace(0, 2, na, dtype=torch.float32, device=dev)
    f0 = torch.floor(pos).clamp(max=1)
    w = pos - f0
    s_a = (1 - w) * scale[f0.long()] + w * scale[f0.long() + 1]        # beam drift per projection
    dark, flat = vol.dark.to(dev).float(), vol.flat.to(dev).float()
    counts = (vol.raw.to(dev).float() - dark[None]) * s_a[:, None, None] + dark[None]
    counts[:, :, 1001] = (counts[:, :, 1001] - dark[None, :, 1001]) * 1.05 + dark[None, :, 1001]   # a ring
    g = np.random.default_rng(5)
    hot = (torch.from_numpy(g.integers(0, na, 400)).to(dev), torch.from_numpy(g.integers(0, ns, 400)).to(dev),
           torch.from_numpy(g.integers(1, n - 1, 400)).to(dev))
    counts[hot] = counts[hot] * 2.5 + 20000
    raw16 = counts.round().clamp(0, 65535).to(torch.int32).to(torch.uint16)
    flats = torch.stack([dark + (flat - dark) * sc for sc in scale])
    geo = geometry(P, vol.angles.numpy(), vol.axis.numpy(), n, n, n, vol.pixel_size, dev)
    got = P.pyhst_fbp_pre(geo, raw16, "u16_raw", flats, dark, flat_pos=pos, hotspot_threshold=0.2, ring_window=9)
    torch.cuda.synchronize()
    p = orc.preprocess(raw16.cpu().double().numpy(), flats.cpu().double().numpy(), pos.cpu().double().numpy(),
                       dark.cpu().double().numpy(), hotspot_threshold=0.2, ring_window=9)
    rng = np.random.default_rng(1)
    for z in (1, 6):
        ii = np.concatenate([rng.integers(0, n, 800), [0, n - 1, n // 2]])
        jj = np.concatenate([rng.integers(0, n, 800), [0, n - 1, 1001]])
        ref = orc.backproject_at(orc.ramlak_filter(p[z]), vol.angles.double().numpy(), vol.axis.double().numpy(),
                                 n, n, ii, jj, orc.fbp_weight(na, vol.pixel_size))
        close(got[z].cpu().double().numpy()[ii, jj], ref)


@pytest.mark.parametrize("filt", ["shepp-logan", "hann", "ramlak"])
@pytest.mark.parametrize("pad", [0, 2048])
def test_fbp_filters(P, orc, cuda_device, filt, pad):
    """The three ramp filters: FFT filter on the GPU (spectrum of the spatial
    kernel formed in float64) against the oracle's direct-sum filter and
    back-projection, on an ellipsoid sinogram with 77 bins (ragged) and two
    paddings."""
    p = acq.ellipsoid_sinograms(2, 77, 60, seed=9, n_ellipsoids=20).to(torch.float32)
    ang = acq.uniform_angles(60).numpy()
    geo = geometry(P, ang, 38.0, 77, 70, 64, 2 / 77, cuda_device)
    got = P.pyhst_fbp(geo, p.to(cuda_device).contiguous(), "f32_sino", pad_len=pad, filter=filt)
    q = P.pyhst_filter(geo, p.to(cuda_device).contiguous(), "f32_sino", pad_len=pad, filter=filt)
    torch.cuda.synchronize()
    for z in range(2):
        qr = orc.filter_rows(p[z].double().numpy(), filt)
        close(f64(q[z]), qr)
        ref = orc.backproject(qr, ang.astype(np.float64), np.full(60, 38.0), 70, 64, orc.fbp_weight(60, 2 / 77))
        close(f64(got[z]), ref)


# ------------------------------------------------------------------ autotuned back-projector block
@pytest.mark.parametrize("case", [CASES[0], CASES[1], CASES[3], (50, 256, 256, 256, "uniform", 0.0, 7),
                                  (100, 512, 512, 512, "uniform", 0.0, 8)])
def test_backproject_angle_blocks_are_identical(P, orc, cuda_device, case):
    """Every angle block (8, 16, 24 angles staged per CTA) gives the same
    bits, within the oracle bar; the autotuner picks one of them and the
    tuned call still gives the same bits."""
    na, nb, nx, ny, kind, off, seed = case
    g, ang, axis, geo = _case(P, cuda_device, *case)
    sino = torch.from_numpy(g.standard_normal((2, na, nb)).astype(np.float32)).to(cuda_device)
    outs = {}
    try:
        for blk in (8, 16, 24):
            P.pyhst_set_backproject_block(nx, ny, na, blk)
            outs[blk] = P.pyhst_backproject(geo, sino, 0.37)
        torch.cuda.synchronize()
        assert torch.equal(outs[8], outs[16]) and torch.equal(outs[24], outs[16])
        best = P.pyhst_autotune_backproject(geo, sino)
        assert best in (8, 16, 24)
        assert torch.equal(P.pyhst_backproject(geo, sino, 0.37), outs[16])
    finally:
        P.pyhst_set_backproject_block(nx, ny, na, 0)
    ref = orc.backproject(sino[0].double().cpu().numpy(), ang.astype(np.float64), axis.astype(np.float64), nx, ny,
                          0.37)
    close(f64(outs[16][0]), ref)


def test_tv_batch_with_tuned_back_projector_block(P, cuda_device):
    """The batched solver takes the block of its geometry with the most
    updates; its iterates are bitwise those of the default block."""
    dev = cuda_device
    items = []
    for k, (n, na) in enumerate([(256, 50), (128, 30), (256, 50)]):
        fs = acq.foam_slice(n, na, seed=900 + k, truth=False)
        geo = P.Geometry(fs.angles.to(dev), fs.axis.to(dev), n, n, n, fs.pixel_size)
        items.append((geo, fs.extra["sino"].to(dev).contiguous(), None))
    opts = P.TvOptions(beta=2e-3, n_iter=6, n_inner=10, lipschitz=50.0)
    xs0, _, _ = P.pyhst_tv_solve_batch(items, opts)
    try:
        P.pyhst_set_backproject_block(256, 256, 50, 8)
        xs1, _, _ = P.pyhst_tv_solve_batch(items, opts)
    finally:
        P.pyhst_set_backproject_block(256, 256, 50, 0)
    torch.cuda.synchronize()
    assert all(torch.equal(a, b) for a, b in zip(xs0, xs1))


@pytest.mark.parametrize("case", [CASES[0], CASES[1], CASES[5], (50, 256, 256, 256, "uniform", 0.0, 7),
                                  (200, 1024, 1024, 1024, "uniform", 0.0, 9)])
def test_project_staging_widths_are_identical(P, orc, cuda_device, case):
    """Every staging width of the projector (256, 384 and 512 columns) gives
    the same bits, within the oracle bar; the autotuner picks one of them."""
    na, nb, nx, ny, kind, off, seed = case
    g, ang, axis, geo = _case(P, cuda_device, *case)
    img = torch.from_numpy(g.standard_normal((2, ny, nx)).astype(np.float32)).to(cuda_device)
    outs = {}
    try:
        for width in (256, 384, 512):
            P.pyhst_set_project_staging(nx, ny, na, width)
            outs[width] = P.pyhst_project(geo, img)
        torch.cuda.synchronize()
        assert torch.equal(outs[256], outs[512]) and torch.equal(outs[384], outs[512])
        best = P.pyhst_autotune_project(geo, img)
        assert best in (256, 384, 512)
        assert torch.equal(P.pyhst_project(geo, img), outs[256])
    finally:
        P.pyhst_set_project_staging(nx, ny, na, 0)
    ref = orc.project(img[0].double().cpu().numpy(), ang.astype(np.float64), axis.astype(np.float64), nb,
                      geo.pixel_size)
    close(f64(outs[256][0]), ref)


@pytest.mark.parametrize("case,ns", [(CASES[1], 3), (CASES[3], 2), (CASES[6], 5),
                                     ((200, 1024, 1024, 1024, "uniform", 0.0, 9), 9),
                                     ((2000, 2048, 2048, 2048, "uniform", 0.4, 12), 3)])
def test_project_slice_pairs_equal_single_slices(P, cuda_device, case, ns):
    """A stack's projection walks two slices per CTA (one staged plane each,
    ray positions and weights computed once; an odd last slice is paired
    with itself).  Every slice's sinogram equals, bit for bit, the projection
    of that slice alone (one slice per CTA, or row-segment CTAs whose
    partials are added in order), at every staging width.  The cases take
    the paired path: images under 128 pixels on a side (no row segments),
    and stacks with enough CTAs (9 x 1024^2 / 200 angles, 3 x 2048^2 / 2000)."""
    na, nb, nx, ny, kind, off, seed = case
    g, ang, axis, geo = _case(P, cuda_device, *case)
    img = torch.from_numpy(g.standard_normal((ns, ny, nx)).astype(np.float32)).to(cuda_device)
    try:
        for width in (256, 384, 512):
            P.pyhst_set_project_staging(nx, ny, na, width)
            stack = P.pyhst_project(geo, img)
            for z in range(ns):
                one = P.pyhst_project(geo, img[z:z + 1].contiguous())
                assert torch.equal(stack[z], one[0]), (width, z)
    finally:
        P.pyhst_set_project_staging(nx, ny, na, 0)


def test_tv_batch_with_three_projector_widths(P, cuda_device):
    """Slices whose geometries take different staging widths run in one
    batched solve (one projector launch per width); the iterates are bitwise
    those of the batch with every slice at the default width."""
    dev = cuda_device
    items, sizes = [], [(256, 50), (128, 30), (192, 40)]
    for k, (n, na) in enumerate(sizes):
        fs = acq.foam_slice(n, na, seed=950 + k, truth=False)
        geo = P.Geometry(fs.angles.to(dev), fs.axis.to(dev), n, n, n, fs.pixel_size)
        items.append((geo, fs.extra["sino"].to(dev).contiguous(), None))
    opts = P.TvOptions(beta=2e-3, n_iter=5, n_inner=10, lipschitz=40.0)
    xs0, _, _ = P.pyhst_tv_solve_batch(items, opts)
    try:
        for (n, na), w in zip(sizes, (256, 384, 512)):
            P.pyhst_set_project_staging(n, n, na, w)
        xs1, _, _ = P.pyhst_tv_solve_batch(items, opts)
    finally:
        for n, na in sizes:
            P.pyhst_set_project_staging(n, n, na, 0)
    torch.cuda.synchronize()
    assert all(torch.equal(a, b) for a, b in zip(xs0, xs1))
