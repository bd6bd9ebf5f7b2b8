"""B300 (sm_103a) parallel-beam reconstruction: PyHST2's per-slice hot path.

Thin Python binding of the C ABI in include/pyhst.h.  Every function has the
name of the C entry point it calls and only marshals arguments: tensors are
checked (CUDA, dtype, contiguity, shape) and their device pointers, the
caller-owned workspace and PyTorch's current stream are passed through.
Every step of the computation runs in the library's CUDA kernels; there is
no CPU path.

Conventions (the library's): images [n_slices, ny, nx]; sinograms
[n_slices, n_angles, n_bins]; raw radiography stacks [n_angles, n_slices,
n_bins]; detector coordinate t = (j - cx) cos th + (i - cy) sin th + axis(th).
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass

import torch

from . import _lib as L
from ._lib import (PYHST_BF16_SINO, PYHST_F16_SINO, PYHST_F32_RAW, PYHST_F32_SINO,  # noqa: F401
                   PYHST_OP_BACKPROJECT, PYHST_OP_FBP, PYHST_OP_PROJECT, PYHST_OP_TV_SOLVE, PYHST_RAMLAK,
                   PYHST_U16_RAW)

__all__ = ["Geometry", "TvOptions", "PyhstError", "pyhst_fbp", "pyhst_filter", "pyhst_fbp_host",
           "pyhst_profile_enable", "pyhst_profile_read", "pyhst_fbp_static", "pyhst_fbp_pre", "pyhst_backproject", "pyhst_project",
           "pyhst_tv_solve", "pyhst_tv_solve_batch", "pyhst_beta_scan", "pyhst_tv_prox", "pyhst_workspace_size", "pyhst_fbp_workspace_size", "pyhst_fbp_host_workspace_size", "pyhst_tv_workspace_size", "pyhst_last_error",
           "pyhst_version", "library_path"]


class PyhstError(RuntimeError):
    def __init__(self, code, message):
        super().__init__(f"pyhst status {code}: {message}")
        self.code = code


def library_path() -> str:
    return L.LIB_PATH


def pyhst_last_error() -> str:
    return L.lib.pyhst_last_error().decode()


def pyhst_version() -> str:
    return L.lib.pyhst_version().decode()


def _check(rc):
    if rc != 0:
        raise PyhstError(rc, pyhst_last_error())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _cuda(t, name, dtypes):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype not in dtypes:
        raise TypeError(f"{name} has dtype {t.dtype}, expected one of {dtypes}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


@dataclass
class Geometry:
    """Angles and axis positions are float32 CUDA tensors [n_angles]."""
    angles: torch.Tensor
    axis: torch.Tensor
    n_bins: int
    nx: int
    ny: int
    pixel_size: float
    cx: float = None
    cy: float = None

    def __post_init__(self):
        _cuda(self.angles, "angles", (torch.float32,))
        _cuda(self.axis, "axis", (torch.float32,))
        if self.axis.shape != self.angles.shape or self.angles.dim() != 1:
            raise ValueError("angles and axis must be 1-D tensors of the same length")

    @property
    def n_angles(self) -> int:
        return int(self.angles.shape[0])

    def c(self, n_slices: int = 1) -> L.pyhst_geometry:
        cx = (self.nx - 1) / 2.0 if self.cx is None else self.cx
        cy = (self.ny - 1) / 2.0 if self.cy is None else self.cy
        return L.pyhst_geometry(self.n_angles, self.n_bins, self.nx, self.ny, n_slices,
                                self.angles.data_ptr(), self.axis.data_ptr(), cx, cy, self.pixel_size)


@dataclass
class TvOptions:
    beta: float
    n_iter: int = 200
    n_inner: int = 20
    tau: float = 0.125
    use_fista: bool = True
    warm_start: bool = False
    lipschitz: float = 0.0
    n_power_iter: int = 50
    warm_dual: bool = False

    def c(self) -> L.pyhst_tv_opts:
        return L.pyhst_tv_opts(self.beta, self.n_iter, self.n_inner, self.tau, int(bool(self.use_fista)),
                               int(bool(self.warm_start)), self.lipschitz, self.n_power_iter,
                               int(bool(self.warm_dual)))


def pyhst_fbp_workspace_size(geom: Geometry, n_slices: int = 1, pad_len: int = 0, slices_per_pass: int = 4) -> int:
    g = geom.c(n_slices)
    return int(L.lib.pyhst_fbp_workspace_size(ctypes.byref(g), pad_len, slices_per_pass))


def pyhst_fbp_host_workspace_size(geom: Geometry, kind: str, n_slices: int, pad_len: int = 0,
                                  slices_per_chunk: int = 16) -> int:
    g = geom.c(n_slices)
    return int(L.lib.pyhst_fbp_host_workspace_size(ctypes.byref(g), _KINDS[kind][0], pad_len, slices_per_chunk))


def pyhst_workspace_size(geom: Geometry, op: int, n_slices: int = 1) -> int:
    g = geom.c(n_slices)
    return int(L.lib.pyhst_workspace_size(ctypes.byref(g), op))


def pyhst_tv_workspace_size(geom: Geometry, opts: TvOptions, n_slices: int = 1) -> int:
    g, o = geom.c(n_slices), opts.c()
    return int(L.lib.pyhst_tv_workspace_size(ctypes.byref(g), ctypes.byref(o)))


def _workspace(nbytes, device, workspace):
    if workspace is None:
        return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)
    return workspace


def _stack3(t, name):
    return t.unsqueeze(0) if t.dim() == 2 else t


_KINDS = {"u16_raw": (PYHST_U16_RAW, torch.uint16), "f32_raw": (PYHST_F32_RAW, torch.float32),
          "f32_sino": (PYHST_F32_SINO, torch.float32), "f16_sino": (PYHST_F16_SINO, torch.float16),
          "bf16_sino": (PYHST_BF16_SINO, torch.bfloat16)}


_FILTERS = {"ramlak": 0, "shepp-logan": 1, "hann": 2}


def _filter_code(name: str) -> int:
    if name not in _FILTERS:
        raise ValueError(f"filter must be one of {sorted(_FILTERS)}")
    return _FILTERS[name]


def pyhst_fbp(geom: Geometry, data: torch.Tensor, kind: str, flat=None, dark=None, layout: str = None,
              pad_len: int = 0, out=None, workspace=None, ws_bytes: int = None,
              slices_per_pass: int = 16, slices: tuple = None, filter: str = "ramlak") -> torch.Tensor:
    """Filtered back-projection of every slice in ``data``.

    ``layout`` "projections": data [n_angles, n_slices, n_bins] (a raw
    radiography stack, read in place through strides); "sinograms": data
    [n_slices, n_angles, n_bins].  Default: projections for raw kinds,
    sinograms otherwise.  flat/dark [n_slices, n_bins] float32 for raw kinds.
    Without a ``workspace`` one is allocated for ``slices_per_pass`` slices
    (their filtered rows; more slices per pass fill the back-projector's last
    wave of CTAs better).
    ``slices=(z0, z1)`` reconstructs only that range of the stack (read in
    place); ``out`` then holds z1 - z0 slices.
    """
    code, raw, data, ns, na, nb, s_stride, a_stride = _fbp_inputs(geom, data, kind, flat, dark, layout)
    z0, z1 = (0, ns) if slices is None else slices
    if not 0 <= z0 < z1 <= ns:
        raise ValueError(f"slice range {slices} outside [0, {ns}]")
    out = _fbp_out(geom, out, z1 - z0, data.device)
    g = geom.c(z1 - z0)
    need = L.lib.pyhst_fbp_workspace_size(ctypes.byref(g), pad_len, slices_per_pass)
    ws = _workspace(need, data.device, workspace)
    nbytes = ws.numel() * ws.element_size() if ws_bytes is None else ws_bytes
    es = data.element_size()
    dptr = ctypes.c_void_p(data.data_ptr() + z0 * s_stride * es)
    fptr = ctypes.c_void_p(flat.data_ptr() + z0 * nb * 4) if raw else None
    kptr = ctypes.c_void_p(dark.data_ptr() + z0 * nb * 4) if raw else None
    _check(L.lib.pyhst_fbp(ctypes.byref(g), code, dptr, s_stride, a_stride, fptr, kptr,
                           _filter_code(filter), pad_len, _ptr(out), _ptr(ws), nbytes, _stream()))
    return out


def _fbp_inputs(geom, data, kind, flat, dark, layout):
    """Checks shared by the FBP entry points: data of the kind's dtype on the
    geometry's device and of its shape; flat/dark float32 [n_slices, n_bins]
    on that device for raw kinds."""
    if kind not in _KINDS:
        raise ValueError(f"kind must be one of {sorted(_KINDS)}")
    code, dt = _KINDS[kind]
    _cuda(data, "data", (dt,))
    if geom.angles.device != data.device:
        raise ValueError(f"geometry tensors on {geom.angles.device}, data on {data.device}")
    raw = kind.endswith("raw")
    data, ns, na, nb, s_stride, a_stride = _layout(data, kind, layout)
    if na != geom.n_angles or nb != geom.n_bins:
        raise ValueError(f"data shape {tuple(data.shape)} does not match the geometry")
    if raw:
        for t, nm in ((flat, "flat"), (dark, "dark")):
            _cuda(t, nm, (torch.float32,))
            if t.device != data.device:
                raise ValueError(f"{nm} is on {t.device}, data on {data.device}")
            if tuple(t.shape) != (ns, nb):
                raise ValueError("flat/dark must be [n_slices, n_bins]")
    return code, raw, data, ns, na, nb, s_stride, a_stride


def _fbp_out(geom, out, n_slices, device):
    """The output stack [n_slices, ny, nx] float32 on ``device`` (allocated
    when None; a caller's tensor must hold every slice)."""
    if out is None:
        return torch.empty((n_slices, geom.ny, geom.nx), dtype=torch.float32, device=device)
    _cuda(out, "out", (torch.float32,))
    if out.device != device:
        raise ValueError(f"out is on {out.device}, data on {device}")
    if out.numel() < n_slices * geom.ny * geom.nx:
        raise ValueError(f"out holds {out.numel()} floats, {n_slices} slices of {geom.ny} x {geom.nx} need more")
    return out


def _layout(data, kind, layout):
    raw = kind.endswith("raw")
    layout = layout or ("projections" if raw else "sinograms")
    if data.dim() == 2:
        data = data.unsqueeze(1 if layout == "projections" else 0)
    if layout == "projections":
        na, ns, nb = data.shape
        return data, ns, na, nb, nb, ns * nb
    if layout == "sinograms":
        ns, na, nb = data.shape
        return data, ns, na, nb, na * nb, nb
    raise ValueError(f"unknown layout {layout}")


def pyhst_filter(geom: Geometry, data: torch.Tensor, kind: str, flat=None, dark=None, layout: str = None,
                 pad_len: int = 0, out=None, workspace=None, filter: str = "ramlak") -> torch.Tensor:
    """Normalised, ramp-filtered (``filter``: ramlak, shepp-logan, hann) sinograms q [n_slices, n_angles, n_bins]
    (the first two steps of pyhst_fbp; same data conventions)."""
    code, dt = _KINDS[kind]
    _cuda(data, "data", (dt,))
    data, ns, na, nb, s_stride, a_stride = _layout(data, kind, layout)
    if na != geom.n_angles or nb != geom.n_bins:
        raise ValueError(f"data shape {tuple(data.shape)} does not match the geometry")
    if out is None:
        out = torch.empty((ns, na, nb), dtype=torch.float32, device=data.device)
    _cuda(out, "out", (torch.float32,))
    g = geom.c(ns)
    ws = _workspace(L.lib.pyhst_filter_workspace_size(ctypes.byref(g), pad_len), data.device, workspace)
    _check(L.lib.pyhst_filter(ctypes.byref(g), code, _ptr(data), s_stride, a_stride, _ptr(flat), _ptr(dark),
                              _filter_code(filter), pad_len, _ptr(out), _ptr(ws), ws.numel(), _stream()))
    return out


def pyhst_fbp_host(geom: Geometry, data: torch.Tensor, kind: str, flat=None, dark=None, out=None,
                   layout: str = None, pad_len: int = 0, slices_per_chunk: int = 16, workspace=None,
                   device=None, filter: str = "ramlak") -> torch.Tensor:
    """pyhst_fbp on HOST tensors (pin them for overlap): chunks are streamed
    through the device by the library.  Returns the host output; the work is
    queued on the current stream (synchronise before reading it)."""
    code, dt = _KINDS[kind]
    if data.is_cuda or data.dtype != dt or not data.is_contiguous():
        raise TypeError("data must be a contiguous host tensor of the kind's dtype")
    data, ns, na, nb, s_stride, a_stride = _layout(data, kind, layout)
    if kind.endswith("raw"):
        for t, nm in ((flat, "flat"), (dark, "dark")):
            if t is None or t.is_cuda or t.dtype != torch.float32 or tuple(t.shape) != (ns, nb) or not t.is_contiguous():
                raise TypeError(f"{nm} must be a contiguous float32 host tensor [n_slices, n_bins]")
    if out is None:
        out = torch.empty((ns, geom.ny, geom.nx), dtype=torch.float32, pin_memory=True)
    g = geom.c(ns)
    need = L.lib.pyhst_fbp_host_workspace_size(ctypes.byref(g), code, pad_len, slices_per_chunk)
    ws = _workspace(need, device or geom.angles.device, workspace)
    _check(L.lib.pyhst_fbp_host(ctypes.byref(g), code, _ptr(data), s_stride, a_stride, _ptr(flat), _ptr(dark),
                                _filter_code(filter), pad_len, _ptr(out), slices_per_chunk, _ptr(ws), ws.numel(),
                                _stream()))
    return out


def pyhst_fbp_static(geom: Geometry, data: torch.Tensor, kind: str, flat=None, dark=None, layout: str = None,
                     pad_len: int = 0, out=None, filter: str = "ramlak") -> torch.Tensor:
    """pyhst_fbp for callers that cannot allocate device scratch: the library
    uses its own fixed device array (see include/pyhst.h); calls that overlap
    on the GPU race on it."""
    code, raw, data, ns, na, nb, s_stride, a_stride = _fbp_inputs(geom, data, kind, flat, dark, layout)
    out = _fbp_out(geom, out, ns, data.device)
    g = geom.c(ns)
    _check(L.lib.pyhst_fbp_static(ctypes.byref(g), code, _ptr(data), s_stride, a_stride,
                                  _ptr(flat) if raw else None, _ptr(dark) if raw else None,
                                  _filter_code(filter), pad_len, _ptr(out), _stream()))
    return out


def pyhst_fbp_pre(geom: Geometry, data: torch.Tensor, kind: str, flats: torch.Tensor, dark: torch.Tensor,
                  flat_pos: torch.Tensor = None, hotspot_threshold: float = 0.0, ring_window: int = 0,
                  pad_len: int = 0, out=None, workspace=None, slices_per_pass: int = 4,
                  filter: str = "ramlak") -> torch.Tensor:
    """FBP with the preprocessing of Sec. 2.3: data [n_angles, n_slices,
    n_bins] raw counts, flats [n_flats, n_slices, n_bins] (or [n_slices,
    n_bins] for one flat), flat_pos [n_angles] (more than one flat), dark
    [n_slices, n_bins]."""
    code, dt = _KINDS[kind]
    if not kind.endswith("raw"):
        raise ValueError("pyhst_fbp_pre needs raw counts")
    _cuda(data, "data", (dt,))
    data, ns, na, nb, s_stride, a_stride = _layout(data, kind, "projections")
    flats = _cuda(flats, "flats", (torch.float32,))
    if flats.dim() == 2:
        flats = flats.unsqueeze(0)
    _cuda(dark, "dark", (torch.float32,))
    if flat_pos is not None:
        _cuda(flat_pos, "flat_pos", (torch.float32,))
    if out is None:
        out = torch.empty((ns, geom.ny, geom.nx), dtype=torch.float32, device=data.device)
    _cuda(out, "out", (torch.float32,))
    g = geom.c(ns)
    pre = L.pyhst_preproc(int(flats.shape[0]), flats.data_ptr(), flat_pos.data_ptr() if flat_pos is not None else None,
                          float(hotspot_threshold), int(ring_window))
    ws = _workspace(L.lib.pyhst_fbp_pre_workspace_size(ctypes.byref(g), pad_len, slices_per_pass), data.device,
                    workspace)
    _check(L.lib.pyhst_fbp_pre(ctypes.byref(g), code, _ptr(data), s_stride, a_stride, _ptr(dark), ctypes.byref(pre),
                               _filter_code(filter), pad_len, _ptr(out), _ptr(ws), ws.numel(), _stream()))
    return out


def pyhst_profile_enable(on: bool = True) -> None:
    _check(L.lib.pyhst_profile_enable(int(bool(on))))


def pyhst_profile_read(kernel: str):
    """(total ms, launches) of the recorded launches of "backproject",
    "filter", "project" or "chambolle" since the last read."""
    ms, n = ctypes.c_double(), ctypes.c_int64()
    _check(L.lib.pyhst_profile_read(kernel.encode(), ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


_MICROBENCH = {"smem_read": 0, "fp32_fma": 1, "fp32_fma2": 2, "mufu": 3}


def pyhst_microbench(kind: str, iters: int = 4096, device=None) -> float:
    """Rate of one microbenchmark launch on ``device`` (default: the current
    CUDA device): "smem_read" in bytes/s of shared-memory reads, "fp32_fma"
    and "fp32_fma2" (paired) in flop/s, "mufu" in MUFU operations/s.  One warm-up launch, then one timed
    with CUDA events on the current stream."""
    if kind not in _MICROBENCH:
        raise ValueError(f"kind must be one of {sorted(_MICROBENCH)}")
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    with torch.cuda.device(dev):
        sink = torch.empty(int(L.lib.pyhst_microbench_sink_floats()), dtype=torch.float32, device=dev)
        units = ctypes.c_double()
        run = lambda: _check(L.lib.pyhst_microbench(_MICROBENCH[kind], iters, _ptr(sink), ctypes.byref(units),  # noqa: E731
                                                    _stream()))
        run()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        run()
        e1.record()
        e1.synchronize()
        return units.value / (e0.elapsed_time(e1) * 1e-3)


def pyhst_backproject(geom: Geometry, sino: torch.Tensor, weight: float, out=None, workspace=None):
    """img = weight * sum_a L(sino_a, t_a); sino [n_slices, n_angles, n_bins]."""
    sino = _stack3(_cuda(sino, "sino", (torch.float32,)), "sino")
    ns = sino.shape[0]
    if tuple(sino.shape[1:]) != (geom.n_angles, geom.n_bins):
        raise ValueError("sinogram shape does not match the geometry")
    if out is None:
        out = torch.empty((ns, geom.ny, geom.nx), dtype=torch.float32, device=sino.device)
    _cuda(out, "out", (torch.float32,))
    g = geom.c(ns)
    need = L.lib.pyhst_workspace_size(ctypes.byref(g), PYHST_OP_BACKPROJECT)
    ws = _workspace(need, sino.device, workspace)
    _check(L.lib.pyhst_backproject(ctypes.byref(g), _ptr(sino), _ptr(out), float(weight), _ptr(ws),
                                   ws.numel(), _stream()))
    return out


def pyhst_project(geom: Geometry, img: torch.Tensor, out=None, workspace=None):
    """sino = pixel_size * A img, A the transpose of the unweighted back-projector."""
    img = _stack3(_cuda(img, "img", (torch.float32,)), "img")
    ns = img.shape[0]
    if tuple(img.shape[1:]) != (geom.ny, geom.nx):
        raise ValueError("image shape does not match the geometry")
    if out is None:
        out = torch.empty((ns, geom.n_angles, geom.n_bins), dtype=torch.float32, device=img.device)
    _cuda(out, "out", (torch.float32,))
    g = geom.c(ns)
    need = L.lib.pyhst_workspace_size(ctypes.byref(g), PYHST_OP_PROJECT)
    ws = _workspace(need, img.device, workspace)
    _check(L.lib.pyhst_project(ctypes.byref(g), _ptr(img), _ptr(out), _ptr(ws), ws.numel(), _stream()))
    return out


def _gap_out(gap, shape, device):
    """A caller's float64 CUDA tensor of ``shape`` for the prox duality gaps (or None)."""
    if gap is None:
        return None
    _cuda(gap, "gap", (torch.float64,))
    if tuple(gap.shape) != tuple(shape) or gap.device != device:
        raise ValueError(f"gap must be a float64 tensor {tuple(shape)} on {device}")
    return gap


def pyhst_tv_solve(geom: Geometry, sino: torch.Tensor, opts: TvOptions, x=None, energy: bool = True,
                   workspace=None, gap=None):
    """Eq. 3 by ISTA/FISTA for each slice; returns (x, energy [n_slices, n_iter]
    float64 or None, lipschitz [n_slices] float64).  ``gap``: None, or a
    float64 CUDA tensor [n_slices, n_iter] that receives the duality gap of
    each iteration's TV prox."""
    sino = _stack3(_cuda(sino, "sino", (torch.float32,)), "sino")
    ns = sino.shape[0]
    if tuple(sino.shape[1:]) != (geom.n_angles, geom.n_bins):
        raise ValueError("sinogram shape does not match the geometry")
    if x is None:
        x = torch.zeros((ns, geom.ny, geom.nx), dtype=torch.float32, device=sino.device)
    _cuda(x, "x", (torch.float32,))
    e = torch.empty((ns, opts.n_iter), dtype=torch.float64, device=sino.device) if energy else None
    lip = torch.empty((ns,), dtype=torch.float64, device=sino.device)
    g, o = geom.c(ns), opts.c()
    need = L.lib.pyhst_tv_workspace_size(ctypes.byref(g), ctypes.byref(o))
    ws = _workspace(need, sino.device, workspace)
    gp = _gap_out(gap, (ns, opts.n_iter), sino.device)
    _check(L.lib.pyhst_tv_solve(ctypes.byref(g), _ptr(sino), ctypes.byref(o), _ptr(x), _ptr(e), _ptr(gp), _ptr(lip),
                                _ptr(ws), ws.numel(), _stream()))
    return x, e, lip


def pyhst_tv_solve_capture(geom: Geometry, sino: torch.Tensor, opts: TvOptions, capture_iters, x=None,
                           workspace=None):
    """pyhst_tv_solve that also returns the prox inputs z_k of the given
    (1-based) iterations: (x [n_slices, ny, nx], z [n_capture, n_slices, ny, nx])."""
    sino = _stack3(_cuda(sino, "sino", (torch.float32,)), "sino")
    ns = sino.shape[0]
    if tuple(sino.shape[1:]) != (geom.n_angles, geom.n_bins):
        raise ValueError("sinogram shape does not match the geometry")
    if x is None:
        x = torch.zeros((ns, geom.ny, geom.nx), dtype=torch.float32, device=sino.device)
    _cuda(x, "x", (torch.float32,))
    its = list(capture_iters)
    cap = torch.empty((len(its), ns, geom.ny, geom.nx), dtype=torch.float32, device=sino.device)
    arr = (ctypes.c_int32 * max(1, len(its)))(*its)
    g, o = geom.c(ns), opts.c()
    ws = _workspace(L.lib.pyhst_tv_workspace_size(ctypes.byref(g), ctypes.byref(o)), sino.device, workspace)
    _check(L.lib.pyhst_tv_solve_capture(ctypes.byref(g), _ptr(sino), ctypes.byref(o), _ptr(x), len(its), arr,
                                        _ptr(cap), _ptr(ws), ws.numel(), _stream()))
    return x, cap


def pyhst_pnp_solve(geom: Geometry, sino: torch.Tensor, params: torch.Tensor, opts: TvOptions, x=None,
                    energy: bool = True, workspace=None):
    """FISTA/ISTA with the learned prox for each slice; returns (x, data-term
    energy [n_slices, n_iter] float64 or None, lipschitz [n_slices])."""
    sino = _stack3(_cuda(sino, "sino", (torch.float32,)), "sino")
    params = _cuda(params, "params", (torch.float32,))
    if params.numel() != pyhst_cnn_param_count():
        raise ValueError(f"params must hold {pyhst_cnn_param_count()} values")
    ns = sino.shape[0]
    if tuple(sino.shape[1:]) != (geom.n_angles, geom.n_bins):
        raise ValueError("sinogram shape does not match the geometry")
    if x is None:
        x = torch.zeros((ns, geom.ny, geom.nx), dtype=torch.float32, device=sino.device)
    _cuda(x, "x", (torch.float32,))
    e = torch.empty((ns, opts.n_iter), dtype=torch.float64, device=sino.device) if energy else None
    lip = torch.empty((ns,), dtype=torch.float64, device=sino.device)
    g, o = geom.c(ns), opts.c()
    ws = _workspace(L.lib.pyhst_pnp_workspace_size(ctypes.byref(g)), sino.device, workspace)
    _check(L.lib.pyhst_pnp_solve(ctypes.byref(g), _ptr(sino), _ptr(params), ctypes.byref(o), _ptr(x), _ptr(e),
                                 _ptr(lip), _ptr(ws), ws.numel(), _stream()))
    return x, e, lip


def pyhst_tv_prox(z: torch.Tensor, lam: float, n_inner: int = 20, tau: float = 0.125, out=None, workspace=None,
                  gap=None):
    """prox of lam * TV (Eq. 2) for images z [n_slices, ny, nx] (or [ny, nx]).
    ``gap``: None, or a float64 CUDA tensor [n_slices] that receives the ROF
    duality gap of each result."""
    z3 = _stack3(_cuda(z, "z", (torch.float32,)), "z")
    ns, ny, nx = z3.shape
    if out is None:
        out = torch.empty_like(z3)
    _cuda(out, "out", (torch.float32,))
    need = L.lib.pyhst_tv_prox_workspace_size(nx, ny, ns)
    ws = _workspace(need, z3.device, workspace)
    gp = _gap_out(gap, (ns,), z3.device)
    _check(L.lib.pyhst_tv_prox(_ptr(z3), nx, ny, ns, float(lam), int(n_inner), float(tau), _ptr(out), _ptr(gp),
                               _ptr(ws), ws.numel(), _stream()))
    return out


def pyhst_autotune_tv_prox(z: torch.Tensor, lam: float, n_inner: int = 20, tau: float = 0.125,
                           workspace=None) -> int:
    """Time the Chambolle steps fused per launch (2, 3, 4, 5, 6, 8; same
    results) on z [n_slices, ny, nx] and record the fastest for ny x nx;
    returns it."""
    z3 = _stack3(_cuda(z, "z", (torch.float32,)), "z").contiguous()
    ns, ny, nx = z3.shape
    ws = _workspace(L.lib.pyhst_tv_prox_workspace_size(nx, ny, ns), z3.device, workspace)
    best = ctypes.c_int32(0)
    _check(L.lib.pyhst_autotune_tv_prox(_ptr(z3), nx, ny, ns, float(lam), int(n_inner), float(tau), _ptr(ws),
                                        ws.numel(), ctypes.byref(best), _stream()))
    return best.value


def pyhst_set_tv_prox_steps(nx: int, ny: int, steps: int) -> None:
    """Record the Chambolle steps fused per launch for ny x nx images (0: default)."""
    _check(L.lib.pyhst_set_tv_prox_steps(nx, ny, steps))


def pyhst_tv_solve_batch(slices, opts: TvOptions, energy: bool = True, workspace=None, gaps=None):
    """Eq. 3 for a mixed batch: ``slices`` is a list of (Geometry, sino
    [n_angles, n_bins], x or None[, beta]) (beta defaults to opts.beta).
    Returns (list of x, list of energy [n_iter] float64 or None,
    lipschitz [n] float64).  ``gaps``: None, or a list with, per slice, None or
    a float64 CUDA tensor [n_iter] that receives its prox duality gaps."""
    if gaps is not None and len(gaps) != len(slices):
        raise ValueError("gaps needs one entry per slice")
    items = (L.pyhst_tv_item * len(slices))()
    xs, es = [], []
    dev = None
    for k, entry in enumerate(slices):
        geom, sino, x = entry[:3]
        beta = float(entry[3]) if len(entry) > 3 and entry[3] is not None else -1.0
        sino = _cuda(sino, "sino", (torch.float32,))
        if tuple(sino.shape[-2:]) != (geom.n_angles, geom.n_bins):
            raise ValueError(f"slice {k}: sinogram shape does not match its geometry")
        dev = sino.device
        if x is None:
            x = torch.zeros((geom.ny, geom.nx), dtype=torch.float32, device=dev)
        _cuda(x, "x", (torch.float32,))
        e = torch.empty((opts.n_iter,), dtype=torch.float64, device=dev) if energy else None
        gp = _gap_out(gaps[k], (opts.n_iter,), dev) if gaps is not None else None
        items[k] = L.pyhst_tv_item(geom.c(1), sino.data_ptr(), x.data_ptr(), e.data_ptr() if e is not None else None,
                                   gp.data_ptr() if gp is not None else None, beta)
        xs.append(x)
        es.append(e)
    o = opts.c()
    lip = torch.empty((len(slices),), dtype=torch.float64, device=dev)
    need = L.lib.pyhst_tv_batch_workspace_size(items, len(slices), ctypes.byref(o))
    ws = _workspace(need, dev, workspace)
    _check(L.lib.pyhst_tv_solve_batch(items, len(slices), ctypes.byref(o), _ptr(lip), _ptr(ws), ws.numel(),
                                      _stream()))
    return xs, es, lip


def pyhst_beta_scan(geom: Geometry, sino: torch.Tensor, betas, opts: TvOptions, held_out: int = -1,
                    workspace=None):
    """Sec. 4 estimators over a beta grid: returns (x [n_beta, ny, nx],
    cross-validation error [n_beta] float64 or None, E_cohe [n_beta] float64)."""
    sino = _cuda(sino, "sino", (torch.float32,))
    if tuple(sino.shape[-2:]) != (geom.n_angles, geom.n_bins):
        raise ValueError("sinogram shape does not match the geometry")
    nbeta = len(betas)
    bh = (ctypes.c_float * nbeta)(*[float(b) for b in betas])
    x = torch.empty((nbeta, geom.ny, geom.nx), dtype=torch.float32, device=sino.device)
    cv = torch.empty((nbeta,), dtype=torch.float64, device=sino.device) if held_out >= 0 else None
    ec = torch.empty((nbeta,), dtype=torch.float64, device=sino.device)
    g, o = geom.c(1), opts.c()
    need = L.lib.pyhst_beta_scan_workspace_size(ctypes.byref(g), nbeta, held_out, ctypes.byref(o))
    ws = _workspace(need, sino.device, workspace)
    _check(L.lib.pyhst_beta_scan(ctypes.byref(g), _ptr(sino), bh, nbeta, held_out, ctypes.byref(o), _ptr(x), _ptr(cv),
                                 _ptr(ec), _ptr(ws), ws.numel(), _stream()))
    return x, cv, ec


def pyhst_cnn_param_count() -> int:
    return int(L.lib.pyhst_cnn_param_count())


def pyhst_cnn_forward(params: torch.Tensor, z: torch.Tensor, out=None, workspace=None):
    """Residual CNN prox on images z [n, ny, nx] (or [ny, nx]) with the flat
    float32 parameter vector ``params`` (device)."""
    params = _cuda(params, "params", (torch.float32,))
    if params.numel() != pyhst_cnn_param_count():
        raise ValueError(f"params must hold {pyhst_cnn_param_count()} values")
    z3 = _stack3(_cuda(z, "z", (torch.float32,)), "z")
    n, ny, nx = z3.shape
    if out is None:
        out = torch.empty_like(z3)
    _cuda(out, "out", (torch.float32,))
    ws = _workspace(L.lib.pyhst_cnn_workspace_size(n, ny, nx), z3.device, workspace)
    _check(L.lib.pyhst_cnn_forward(_ptr(params), _ptr(z3), _ptr(out), n, ny, nx, _ptr(ws), ws.numel(), _stream()))
    return out.view(z.shape)


def pyhst_cnn_grad(params: torch.Tensor, z: torch.Tensor, target: torch.Tensor, grad=None, loss=None,
                   workspace=None):
    """Mean squared error of the network on the batch z [n, ny, nx] against
    target and its gradient; returns (grad [param_count] float32, loss
    [1] float64), both on the device."""
    params = _cuda(params, "params", (torch.float32,))
    z3 = _stack3(_cuda(z, "z", (torch.float32,)), "z")
    t3 = _stack3(_cuda(target, "target", (torch.float32,)), "target")
    if t3.shape != z3.shape:
        raise ValueError("target must have the shape of z")
    n, ny, nx = z3.shape
    if grad is None:
        grad = torch.empty_like(params)
    if loss is None:
        loss = torch.empty((1,), dtype=torch.float64, device=z3.device)
    ws = _workspace(L.lib.pyhst_cnn_train_workspace_size(n, ny, nx), z3.device, workspace)
    _check(L.lib.pyhst_cnn_grad(_ptr(params), _ptr(z3), _ptr(t3), n, ny, nx, _ptr(grad), _ptr(loss), _ptr(ws),
                                ws.numel(), _stream()))
    return grad, loss


def pyhst_cnn_adam(params: torch.Tensor, grad: torch.Tensor, m: torch.Tensor, v: torch.Tensor, step: int,
                   lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8) -> None:
    """One Adam step in place on params, m, v (device float32)."""
    for t, nm in ((params, "params"), (grad, "grad"), (m, "m"), (v, "v")):
        _cuda(t, nm, (torch.float32,))
    _check(L.lib.pyhst_cnn_adam(_ptr(params), _ptr(grad), _ptr(m), _ptr(v), params.numel(), int(step), float(lr),
                                float(beta1), float(beta2), float(eps), _stream()))


@dataclass
class PatchProblem:
    """Overlapping-patch functional (Eq. 8): image ny x nx, m x m patches on a
    grid of step ``stride``, dictionary ``dict`` [n_atoms, m*m] (device
    float32), weight ``rho``."""
    ny: int
    nx: int
    m: int
    stride: int
    dict: torch.Tensor
    rho: float

    def __post_init__(self):
        _cuda(self.dict, "dict", (torch.float32,))
        if self.dict.dim() != 2 or self.dict.shape[1] != self.m * self.m:
            raise ValueError("dict must be [n_atoms, m*m]")
        self.dict = self.dict.contiguous()

    def c(self) -> L.pyhst_patch_problem:
        return L.pyhst_patch_problem(self.ny, self.nx, self.m, self.stride, self.dict.shape[0],
                                     self.dict.data_ptr(), self.rho)

    def grid(self):
        return pyhst_patch_grid(self.ny, self.nx, self.m, self.stride)

    def coef_shape(self):
        kr, kc = self.grid()
        return (kr * kc, self.dict.shape[0])


def pyhst_patch_grid(ny: int, nx: int, m: int, stride: int):
    kr, kc = ctypes.c_int32(), ctypes.c_int32()
    _check(L.lib.pyhst_patch_grid(ny, nx, m, stride, ctypes.byref(kr), ctypes.byref(kc)))
    return kr.value, kc.value


def _patch_ws(pp: PatchProblem, geom, device, workspace):
    pc = pp.c()
    gc = geom.c(1) if geom is not None else None
    need = L.lib.pyhst_patch_workspace_size(ctypes.byref(pc), ctypes.byref(gc) if gc is not None else None)
    return pc, gc, _workspace(need, device, workspace)


def pyhst_patch_image(pp: PatchProblem, W: torch.Tensor, out=None, workspace=None):
    """The image of the coefficients W [N, n_atoms] (Eq. 7)."""
    W = _cuda(W, "W", (torch.float32,)).contiguous()
    out = torch.empty((pp.ny, pp.nx), dtype=torch.float32, device=W.device) if out is None else out
    pc, _, ws = _patch_ws(pp, None, W.device, workspace)
    _check(L.lib.pyhst_patch_image(ctypes.byref(pc), _ptr(W), _ptr(out), _ptr(ws), ws.numel(), _stream()))
    return out


def pyhst_patch_gradient(pp: PatchProblem, geom, W: torch.Tensor, y: torch.Tensor, workspace=None):
    """Gradient of Eq. 8 (Algorithm 1) at W and f(W); geom None: denoising.
    Returns (G [N, n_atoms], f [1] float64)."""
    W = _cuda(W, "W", (torch.float32,)).contiguous()
    y = _cuda(y, "y", (torch.float32,)).contiguous()
    G = torch.empty_like(W)
    f = torch.empty((1,), dtype=torch.float64, device=W.device)
    pc, gc, ws = _patch_ws(pp, geom, W.device, workspace)
    _check(L.lib.pyhst_patch_gradient(ctypes.byref(pc), ctypes.byref(gc) if gc is not None else None, _ptr(W),
                                      _ptr(y), _ptr(G), _ptr(f), _ptr(ws), ws.numel(), _stream()))
    return G, f


def pyhst_patch_solve(pp: PatchProblem, geom, y: torch.Tensor, beta: float, n_iter: int, lipschitz: float = 0.0,
                      n_power_iter: int = 50, use_fista: bool = True, W=None, energy: bool = True, workspace=None):
    """ISTA/FISTA on F(W) = f(W) + beta ||W||_1; returns (W, x, energy
    [n_iter] float64 or None, L [1] float64)."""
    y = _cuda(y, "y", (torch.float32,)).contiguous()
    W = torch.zeros(pp.coef_shape(), dtype=torch.float32, device=y.device) if W is None else W
    _cuda(W, "W", (torch.float32,))
    x = torch.empty((pp.ny, pp.nx), dtype=torch.float32, device=y.device)
    e = torch.empty((n_iter,), dtype=torch.float64, device=y.device) if energy else None
    lip = torch.empty((1,), dtype=torch.float64, device=y.device)
    pc, gc, ws = _patch_ws(pp, geom, y.device, workspace)
    _check(L.lib.pyhst_patch_solve(ctypes.byref(pc), ctypes.byref(gc) if gc is not None else None, _ptr(y),
                                   float(beta), float(lipschitz), int(n_power_iter), int(n_iter), int(bool(use_fista)),
                                   _ptr(W), _ptr(x), _ptr(e), _ptr(lip), _ptr(ws), ws.numel(), _stream()))
    return W, x, e, lip


def pyhst_device_status(clear: bool = True) -> int:
    """Error bits recorded by kernels whose bounded waits gave up (0: none)."""
    v = ctypes.c_uint32(0)
    _check(L.lib.pyhst_device_status(ctypes.byref(v), 1 if clear else 0))
    return int(v.value)


def pyhst_autotune_backproject(geom: Geometry, sino: torch.Tensor, out=None, workspace=None) -> int:
    """Time the back-projector's angle blocks (8, 16, 24 angles; identical
    results) on sino [n_slices, n_angles, n_bins] and record the fastest for
    the geometry; returns it."""
    sino = _stack3(_cuda(sino, "sino", (torch.float32,)), "sino")
    ns = sino.shape[0]
    if tuple(sino.shape[1:]) != (geom.n_angles, geom.n_bins):
        raise ValueError("sinogram shape does not match the geometry")
    if out is None:
        out = torch.empty((ns, geom.ny, geom.nx), dtype=torch.float32, device=sino.device)
    _cuda(out, "out", (torch.float32,))
    g = geom.c(ns)
    ws = _workspace(L.lib.pyhst_workspace_size(ctypes.byref(g), PYHST_OP_BACKPROJECT), sino.device, workspace)
    best = ctypes.c_int32(0)
    _check(L.lib.pyhst_autotune_backproject(ctypes.byref(g), _ptr(sino), _ptr(out), _ptr(ws), ws.numel(),
                                            ctypes.byref(best), _stream()))
    return int(best.value)


def pyhst_autotune_project(geom: Geometry, img: torch.Tensor, out=None, workspace=None) -> int:
    """Time the projector's staging widths (256, 384, 512 columns; identical
    results) on img [n_slices, ny, nx] and record the fastest for the
    geometry; returns it."""
    img = _stack3(_cuda(img, "img", (torch.float32,)), "img")
    ns = img.shape[0]
    if tuple(img.shape[1:]) != (geom.ny, geom.nx):
        raise ValueError("image shape does not match the geometry")
    if out is None:
        out = torch.empty((ns, geom.n_angles, geom.n_bins), dtype=torch.float32, device=img.device)
    _cuda(out, "out", (torch.float32,))
    g = geom.c(ns)
    ws = _workspace(L.lib.pyhst_workspace_size(ctypes.byref(g), PYHST_OP_PROJECT), img.device, workspace)
    best = ctypes.c_int32(0)
    _check(L.lib.pyhst_autotune_project(ctypes.byref(g), _ptr(img), _ptr(out), _ptr(ws), ws.numel(),
                                        ctypes.byref(best), _stream()))
    return int(best.value)


def pyhst_set_project_staging(nx: int, ny: int, n_angles: int, width: int) -> None:
    """Record the projector's staging width (256, 384 or 512) for a geometry (0 clears)."""
    _check(L.lib.pyhst_set_project_staging(int(nx), int(ny), int(n_angles), int(width)))


def pyhst_set_backproject_block(nx: int, ny: int, n_angles: int, angles_per_block: int) -> None:
    """Record the back-projector's angle block for a geometry (0 clears)."""
    _check(L.lib.pyhst_set_backproject_block(int(nx), int(ny), int(n_angles), int(angles_per_block)))


def pyhst_set_wait_limit(polls: int = -1) -> None:
    """Polls after which the tensor-core kernels' pipeline waits give up
    (negative: the default; 0: give up without polling); for tests of
    failure detection."""
    _check(L.lib.pyhst_set_wait_limit(int(polls)))


def fbp_weight(n_angles: int, pixel_size: float) -> float:
    """pi / (n_angles * s), the FBP angular weight over 180 degrees."""
    return math.pi / (n_angles * pixel_size)
