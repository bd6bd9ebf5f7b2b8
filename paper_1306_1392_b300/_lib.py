"""ctypes view of the C ABI declared in include/pyhst.h.

Loads the in-tree libpyhst_b300.so (building it with nvcc when it is missing
or older than its sources).  There is no fallback: if the library cannot be
built or loaded, importing this module raises.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

c_int32, c_int64, c_size_t, c_void_p, c_float, c_double = (
    ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_float, ctypes.c_double)

PYHST_OK = 0
PYHST_ERR_INVALID_ARG = -1
PYHST_ERR_CUDA = -2
PYHST_ERR_WORKSPACE = -3
PYHST_ERR_TIMEOUT = -4
PYHST_ERR_NUMERIC = -5

PYHST_U16_RAW, PYHST_F32_RAW, PYHST_F32_SINO, PYHST_F16_SINO, PYHST_BF16_SINO = range(5)
PYHST_RAMLAK, PYHST_SHEPP_LOGAN, PYHST_HANN = range(3)
PYHST_OP_FBP, PYHST_OP_BACKPROJECT, PYHST_OP_PROJECT, PYHST_OP_TV_SOLVE = range(4)


class pyhst_geometry(ctypes.Structure):
    _fields_ = [("n_angles", c_int32), ("n_bins", c_int32), ("nx", c_int32), ("ny", c_int32),
                ("n_slices", c_int32), ("angles", c_void_p), ("axis", c_void_p),
                ("cx", c_float), ("cy", c_float), ("pixel_size", c_float)]


class pyhst_patch_problem(ctypes.Structure):
    _fields_ = [("ny", c_int32), ("nx", c_int32), ("m", c_int32), ("stride", c_int32), ("n_atoms", c_int32),
                ("dict", c_void_p), ("rho", c_float)]


class pyhst_tv_opts(ctypes.Structure):
    _fields_ = [("beta", c_float), ("n_iter", c_int32), ("n_inner", c_int32), ("tau", c_float),
                ("use_fista", c_int32), ("warm_start", c_int32), ("lipschitz", c_double),
                ("n_power_iter", c_int32), ("warm_dual", c_int32)]


class pyhst_preproc(ctypes.Structure):
    _fields_ = [("n_flats", c_int32), ("flats", c_void_p), ("flat_pos", c_void_p), ("hotspot_threshold", c_float),
                ("ring_window", c_int32)]


class pyhst_tv_item(ctypes.Structure):
    _fields_ = [("geom", pyhst_geometry), ("sino", c_void_p), ("x", c_void_p), ("energy", c_void_p),
                ("gap", c_void_p), ("beta", c_float)]


# (name, restype, argtypes) of every exported entry point
SIGNATURES = [
    ("pyhst_workspace_size", c_size_t, [ctypes.POINTER(pyhst_geometry), c_int32]),
    ("pyhst_fbp_workspace_size", c_size_t, [ctypes.POINTER(pyhst_geometry), c_int32, c_int32]),
    ("pyhst_fbp", c_int32, [ctypes.POINTER(pyhst_geometry), c_int32, c_void_p, c_int64, c_int64, c_void_p,
                            c_void_p, c_int32, c_int32, c_void_p, c_void_p, c_size_t, c_void_p]),
    ("pyhst_filter_workspace_size", c_size_t, [ctypes.POINTER(pyhst_geometry), c_int32]),
    ("pyhst_filter", c_int32, [ctypes.POINTER(pyhst_geometry), c_int32, c_void_p, c_int64, c_int64, c_void_p,
                               c_void_p, c_int32, c_int32, c_void_p, c_void_p, c_size_t, c_void_p]),
    ("pyhst_fbp_host_workspace_size", c_size_t, [ctypes.POINTER(pyhst_geometry), c_int32, c_int32, c_int32]),
    ("pyhst_fbp_host", c_int32, [ctypes.POINTER(pyhst_geometry), c_int32, c_void_p, c_int64, c_int64, c_void_p,
                                 c_void_p, c_int32, c_int32, c_void_p, c_int32, c_void_p, c_size_t, c_void_p]),
    ("pyhst_fbp_static_max_bytes", c_size_t, []),
    ("pyhst_fbp_static", c_int32, [ctypes.POINTER(pyhst_geometry), c_int32, c_void_p, c_int64, c_int64, c_void_p,
                                   c_void_p, c_int32, c_int32, c_void_p, c_void_p]),
    ("pyhst_backproject", c_int32, [ctypes.POINTER(pyhst_geometry), c_void_p, c_void_p, c_float, c_void_p,
                                    c_size_t, c_void_p]),
    ("pyhst_project", c_int32, [ctypes.POINTER(pyhst_geometry), c_void_p, c_void_p, c_void_p, c_size_t,
                                c_void_p]),
    ("pyhst_tv_solve", c_int32, [ctypes.POINTER(pyhst_geometry), c_void_p, ctypes.POINTER(pyhst_tv_opts),
                                 c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    ("pyhst_tv_workspace_size", c_size_t, [ctypes.POINTER(pyhst_geometry), ctypes.POINTER(pyhst_tv_opts)]),
    ("pyhst_tv_prox_workspace_size", c_size_t, [c_int32, c_int32, c_int32]),
    ("pyhst_tv_prox", c_int32, [c_void_p, c_int32, c_int32, c_int32, c_float, c_int32, c_float, c_void_p,
                                c_void_p, c_void_p, c_size_t, c_void_p]),
    ("pyhst_profile_enable", c_int32, [c_int32]),
    ("pyhst_profile_read", c_int32, [ctypes.c_char_p, ctypes.POINTER(c_double), ctypes.POINTER(c_int64)]),
    ("pyhst_microbench_sink_floats", c_size_t, []),
    ("pyhst_microbench", c_int32, [c_int32, c_int32, c_void_p, ctypes.POINTER(c_double), c_void_p]),
    ("pyhst_tv_batch_workspace_size", c_size_t, [ctypes.POINTER(pyhst_tv_item), c_int32,
                                                 ctypes.POINTER(pyhst_tv_opts)]),
    ("pyhst_tv_solve_batch", c_int32, [ctypes.POINTER(pyhst_tv_item), c_int32, ctypes.POINTER(pyhst_tv_opts),
                                       c_void_p, c_void_p, c_size_t, c_void_p]),
    ("pyhst_cnn_param_count", c_int64, []),
    ("pyhst_cnn_workspace_size", c_size_t, [c_int32, c_int32, c_int32]),
    ("pyhst_cnn_forward", c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_int32, c_int32, c_void_p, c_size_t,
                                    c_void_p]),
    ("pyhst_device_status", c_int32, [ctypes.POINTER(ctypes.c_uint32), c_int32]),
    ("pyhst_set_wait_limit", c_int32, [c_int64]),
    ("pyhst_autotune_backproject", c_int32, [ctypes.POINTER(pyhst_geometry), c_void_p, c_void_p, c_void_p, c_size_t,
                                             ctypes.POINTER(c_int32), c_void_p]),
    ("pyhst_set_backproject_block", c_int32, [c_int32, c_int32, c_int32, c_int32]),
    ("pyhst_autotune_project", c_int32, [ctypes.POINTER(pyhst_geometry), c_void_p, c_void_p, c_void_p, c_size_t,
                                         ctypes.POINTER(c_int32), c_void_p]),
    ("pyhst_set_project_staging", c_int32, [c_int32, c_int32, c_int32, c_int32]),
    ("pyhst_autotune_tv_prox", c_int32, [c_void_p, c_int32, c_int32, c_int32, c_float, c_int32, c_float, c_void_p,
                                         c_size_t, ctypes.POINTER(c_int32), c_void_p]),
    ("pyhst_set_tv_prox_steps", c_int32, [c_int32, c_int32, c_int32]),
    ("pyhst_patch_grid", c_int32, [c_int32, c_int32, c_int32, c_int32, ctypes.POINTER(c_int32), ctypes.POINTER(c_int32)]),
    ("pyhst_patch_workspace_size", c_size_t, [ctypes.POINTER(pyhst_patch_problem), ctypes.POINTER(pyhst_geometry)]),
    ("pyhst_patch_image", c_int32, [ctypes.POINTER(pyhst_patch_problem), c_void_p, c_void_p, c_void_p, c_size_t,
                                    c_void_p]),
    ("pyhst_patch_gradient", c_int32, [ctypes.POINTER(pyhst_patch_problem), ctypes.POINTER(pyhst_geometry), c_void_p,
                                       c_void_p, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    ("pyhst_patch_solve", c_int32, [ctypes.POINTER(pyhst_patch_problem), ctypes.POINTER(pyhst_geometry), c_void_p,
                                    c_float, c_double, c_int32, c_int32, c_int32, c_void_p, c_void_p, c_void_p,
                                    c_void_p, c_void_p, c_size_t, c_void_p]),
    ("pyhst_pnp_workspace_size", c_size_t, [ctypes.POINTER(pyhst_geometry)]),
    ("pyhst_pnp_solve", c_int32, [ctypes.POINTER(pyhst_geometry), c_void_p, c_void_p, ctypes.POINTER(pyhst_tv_opts),
                                  c_void_p, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    ("pyhst_tv_solve_capture", c_int32, [ctypes.POINTER(pyhst_geometry), c_void_p, ctypes.POINTER(pyhst_tv_opts),
                                         c_void_p, c_int32, ctypes.POINTER(c_int32), c_void_p, c_void_p, c_size_t,
                                         c_void_p]),
    ("pyhst_cnn_train_workspace_size", c_size_t, [c_int32, c_int32, c_int32]),
    ("pyhst_cnn_grad", c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_int32, c_int32, c_void_p, c_void_p,
                                 c_void_p, c_size_t, c_void_p]),
    ("pyhst_cnn_adam", c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_int32, c_float, c_float, c_float,
                                 c_float, c_void_p]),
    ("pyhst_beta_scan_workspace_size", c_size_t, [ctypes.POINTER(pyhst_geometry), c_int32, c_int32,
                                                  ctypes.POINTER(pyhst_tv_opts)]),
    ("pyhst_beta_scan", c_int32, [ctypes.POINTER(pyhst_geometry), c_void_p, ctypes.POINTER(c_float), c_int32, c_int32,
                                  ctypes.POINTER(pyhst_tv_opts), c_void_p, c_void_p, c_void_p, c_void_p, c_size_t,
                                  c_void_p]),
    ("pyhst_fbp_pre_workspace_size", c_size_t, [ctypes.POINTER(pyhst_geometry), c_int32, c_int32]),
    ("pyhst_fbp_pre", c_int32, [ctypes.POINTER(pyhst_geometry), c_int32, c_void_p, c_int64, c_int64, c_void_p,
                                ctypes.POINTER(pyhst_preproc), c_int32, c_int32, c_void_p, c_void_p, c_size_t,
                                c_void_p]),
    ("pyhst_last_error", ctypes.c_char_p, []),
    ("pyhst_version", ctypes.c_char_p, []),
]


def _load():
    path = _build.LIB
    if _build.stale():
        path = _build.build_library()
    if not os.path.exists(path):
        raise ImportError(f"CUDA library {path} is missing and could not be built")
    lib = ctypes.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()
LIB_PATH = _build.LIB
