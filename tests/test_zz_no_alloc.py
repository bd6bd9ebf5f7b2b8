"""pyhst_fbp_static, the FBP entry point that allocates nothing.

It serves callers that cannot allocate device memory (a framework that owns
every device allocation, an acquisition loop that may not call cudaMalloc
while it runs): the scratch is a fixed array inside the library.  The test
calls it through the C ABI twice in a row, on different inputs, and checks
each result against pyhst_fbp (the workspace entry point) within the float32
tolerance of the other parity tests.  This file is collected last.
"""
import ctypes

import numpy as np
import pytest
import torch

from synth import acquisition as acq

REL_L2 = 1e-5
MAX_ABS = 1e-4


def _geometry(P, vol, dev):
    return P.Geometry(vol.angles.to(dev), vol.axis.to(dev), vol.n_bins, vol.nx, vol.ny, vol.pixel_size)


def _close(got, ref):
    got, ref = got.double().cpu().numpy(), ref.double().cpu().numpy()
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    mx = np.abs(got - ref).max() / np.abs(ref).max()
    assert rel <= REL_L2 and mx <= MAX_ABS, (rel, mx)


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
        g = geo.c(ns)
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        rc = L.lib.pyhst_fbp_static(ctypes.byref(g), L.PYHST_U16_RAW, ctypes.c_void_p(raw.data_ptr()), 160,
                                    ns * 160, ctypes.c_void_p(fl.data_ptr()), ctypes.c_void_p(dk.data_ptr()),
                                    L.PYHST_RAMLAK, 0, ctypes.c_void_p(out.data_ptr()), stream)
        assert rc == 0, L.lib.pyhst_last_error().decode()
        torch.cuda.synchronize()
        assert torch.isfinite(out).all()
        _close(out, ref)
