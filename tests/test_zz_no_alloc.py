"""pyhst_fbp_static, the FBP entry point that allocates nothing.

It serves callers that cannot allocate device memory (a framework that owns
every device allocation, an acquisition loop that may not call cudaMalloc
while it runs): the scratch is a fixed array inside the library.  The GPU
tests call it through the C ABI twice in a row, on different inputs, and
check each result against pyhst_fbp (the workspace entry point): both run the
same kernels on each slice, so the results are equal bit for bit, including
a geometry whose filtered rows need two passes through the fixed scratch.
This file is collected last.
"""
import ctypes

import pytest
import torch

from synth import acquisition as acq


def _geometry(P, vol, dev):
    return P.Geometry(vol.angles.to(dev), vol.axis.to(dev), vol.n_bins, vol.nx, vol.ny, vol.pixel_size)


def test_static_entry_rejects_oversized_geometry():
    """Host-side check: a sinogram too large for the fixed scratch is refused
    before anything runs (no GPU needed)."""
    from paper_1306_1392_b300 import _lib as L
    cap = L.lib.pyhst_fbp_static_max_bytes()
    assert cap == 32 << 20
    g = L.pyhst_geometry(4096, 4096, 64, 64, 1, 8, 8, 31.5, 31.5, 0.1)     # 64 MiB of filtered rows
    rc = L.lib.pyhst_fbp_static(ctypes.byref(g), L.PYHST_F32_SINO, 8, 4096 * 4096, 4096, None, None,
                                L.PYHST_RAMLAK, 0, 8, None)
    assert rc == L.PYHST_ERR_INVALID_ARG
    assert "static" in L.lib.pyhst_last_error().decode()


def test_static_entry_shares_the_fbp_argument_checks():
    """Host-side checks (no GPU needed): raw kinds without flat or dark, an
    unknown kind or filter, and a pad length below 2 n_bins are refused with
    the same messages as pyhst_fbp, before anything runs."""
    from paper_1306_1392_b300 import _lib as L
    g = L.pyhst_geometry(100, 64, 32, 32, 2, 8, 8, 15.5, 15.5, 0.1)
    for kind, flat, dark, filt, pad, what in ((L.PYHST_U16_RAW, None, 8, L.PYHST_RAMLAK, 0, "flat and dark"),
                                              (L.PYHST_F32_RAW, 8, None, L.PYHST_RAMLAK, 0, "flat and dark"),
                                              (17, None, None, L.PYHST_RAMLAK, 0, "input kind"),
                                              (L.PYHST_F32_SINO, None, None, 9, 0, "filter"),
                                              (L.PYHST_F32_SINO, None, None, L.PYHST_RAMLAK, 64, "pad_len")):
        rc_s = L.lib.pyhst_fbp_static(ctypes.byref(g), kind, 8, 6400, 64, flat, dark, filt, pad, 8, None)
        msg_s = L.lib.pyhst_last_error().decode()
        rc_w = L.lib.pyhst_fbp(ctypes.byref(g), kind, 8, 6400, 64, flat, dark, filt, pad, 8, None, 0, None)
        msg_w = L.lib.pyhst_last_error().decode()
        assert rc_s == rc_w == L.PYHST_ERR_INVALID_ARG, (what, rc_s, rc_w)
        assert what in msg_s and msg_s == msg_w, (msg_s, msg_w)


def _c_call(L, geo, kind, data, s_stride, a_stride, fl, dk, out, ns):
    g = geo.c(ns)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    ptr = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None  # noqa: E731
    rc = L.lib.pyhst_fbp_static(ctypes.byref(g), kind, ptr(data), s_stride, a_stride, ptr(fl), ptr(dk),
                                L.PYHST_RAMLAK, 0, ptr(out), stream)
    assert rc == 0, L.lib.pyhst_last_error().decode()


@pytest.mark.gpu
def test_static_entry_matches_workspace_entry_twice(cuda_device):
    import paper_1306_1392_b300 as P
    from paper_1306_1392_b300 import _lib as L
    dev = cuda_device
    for seed, ns in ((51, 5), (52, 3)):
        vol = acq.ellipsoid_volume(n_slices=ns, n=160, n_angles=120, seed=seed, n_ellipsoids=40)
        geo = _geometry(P, vol, dev)
        raw, fl, dk = vol.raw.to(dev), vol.flat.to(dev), vol.dark.to(dev)
        ref = P.pyhst_fbp(geo, raw, "u16_raw", fl, dk)
        out = torch.full((ns, 160, 160), float("nan"), device=dev)
        _c_call(L, geo, L.PYHST_U16_RAW, raw, 160, ns * 160, fl, dk, out, ns)
        torch.cuda.synchronize()
        assert torch.equal(out, ref)


@pytest.mark.gpu
def test_static_entry_multi_pass_matches_workspace_entry(cuda_device):
    """2000 angles x 1024 bins: 8.2 MB of filtered rows per slice, so the
    32 MiB scratch holds 4 slices and 6 slices take two passes (4 + 2); the
    second pass reuses the filtered-row area and writes at a slice offset.
    Called through the C ABI and through the Python binding, twice in a row
    on different stacks."""
    import paper_1306_1392_b300 as P
    from paper_1306_1392_b300 import _lib as L
    dev = cuda_device
    n, na, ns = 1024, 2000, 6
    per = 4 * na * n
    assert L.lib.pyhst_fbp_static_max_bytes() // per == 4
    for seed in (53, 54):
        vol = acq.ellipsoid_volume(n_slices=ns, n=n, n_angles=na, seed=seed, device=dev, n_ellipsoids=40)
        geo = _geometry(P, vol, dev)
        raw, fl, dk = vol.raw.to(dev), vol.flat.to(dev), vol.dark.to(dev)
        ref = P.pyhst_fbp(geo, raw, "u16_raw", fl, dk)
        out = torch.full((ns, n, n), float("nan"), device=dev)
        _c_call(L, geo, L.PYHST_U16_RAW, raw, n, ns * n, fl, dk, out, ns)
        out2 = P.pyhst_fbp_static(geo, raw, "u16_raw", fl, dk)
        torch.cuda.synchronize()
        assert torch.isfinite(ref).all()
        assert torch.equal(out, ref)
        assert torch.equal(out2, ref)


@pytest.mark.gpu
def test_static_binding_refuses_bad_tensors(cuda_device):
    """The binding refuses, before any launch, flat/dark that are on the host,
    of the wrong dtype or shape, and an output too short for the stack."""
    import paper_1306_1392_b300 as P
    dev = cuda_device
    vol = acq.ellipsoid_volume(n_slices=2, n=64, n_angles=40, seed=55, n_ellipsoids=10)
    geo = _geometry(P, vol, dev)
    raw, fl, dk = vol.raw.to(dev), vol.flat.to(dev), vol.dark.to(dev)
    with pytest.raises(TypeError):
        P.pyhst_fbp_static(geo, raw, "u16_raw", vol.flat, dk)
    with pytest.raises(TypeError):
        P.pyhst_fbp_static(geo, raw, "u16_raw", fl, dk.double())
    with pytest.raises(ValueError):
        P.pyhst_fbp_static(geo, raw, "u16_raw", fl[:1], dk)
    with pytest.raises(TypeError):
        P.pyhst_fbp_static(geo, raw, "u16_raw", fl, None)
    with pytest.raises(ValueError):
        P.pyhst_fbp_static(geo, raw, "u16_raw", fl, dk, out=torch.empty((1, 64, 64), device=dev))
