"""ctypes declarations of the C ABI in include/sr.h (libsr.so, built in-tree).

Loading fails loudly: there is no fallback implementation. Call
``paper_2409_05734_gb300.buildlib.build()`` (or ``__graft_entry__.build()``) first.
"""
from __future__ import annotations

import ctypes as C
import os

from . import buildlib as _build

SR_OK = 0
STATUS_NAMES = {0: "SR_OK", 1: "SR_ERR_INVALID_ARG", 2: "SR_ERR_UNSUPPORTED", 3: "SR_ERR_OOM",
                4: "SR_ERR_CUDA", 5: "SR_ERR_TIMEOUT", 6: "SR_ERR_NUMERIC"}

SR_WEIGHT_IDENTITY = 0
SR_WEIGHT_OPTIMAL = 1


class SpectralOpts(C.Structure):
    _fields_ = [("weight_mode", C.c_int), ("lambda_", C.c_float)]


class GdOpts(C.Structure):
    _fields_ = [("mu0", C.c_float), ("tau0", C.c_float)]


class SrError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {message}")


# (name, restype, argtypes) of every exported entry point
_VP = C.c_void_p
SIGNATURES = [
    ("sr_phases", C.c_int, [C.c_uint64, C.c_int, C.c_int64, C.POINTER(C.c_double)]),
    ("sr_plan_create", C.c_int, [C.c_int64, C.c_int64, C.c_int, C.c_uint64, C.POINTER(_VP)]),
    ("sr_plan_set_batch_phases", C.c_int, [_VP, C.c_int, C.POINTER(C.c_uint64)]),
    ("sr_plan_create_2d", C.c_int, [C.c_int64, C.c_int64, C.c_int64, C.c_int, C.c_uint64, C.POINTER(_VP)]),
    ("sr_plan_destroy", C.c_int, [_VP]),
    ("sr_plan_get_phases", C.c_int, [_VP, C.POINTER(C.c_double)]),
    ("sr_plan_set_phases", C.c_int, [_VP, C.POINTER(C.c_double)]),
    ("sr_plan_info", C.c_int, [_VP, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int)]),
    ("sr_plan_reserve", C.c_int, [_VP, C.c_int]),
    ("sr_forward", C.c_int, [_VP, _VP, _VP, C.c_int, _VP]),
    ("sr_adjoint", C.c_int, [_VP, _VP, _VP, C.c_int, _VP]),
    ("sr_loss_grad", C.c_int, [_VP, _VP, _VP, _VP, _VP, C.c_int, _VP]),
    ("sr_spectral_init", C.c_int, [_VP, _VP, _VP, C.c_int, C.POINTER(SpectralOpts), _VP, C.c_int, _VP]),
    ("sr_spectral_init_early_stop", C.c_int, [_VP, _VP, _VP, C.c_int, C.POINTER(SpectralOpts), C.c_float, C.c_int,
                                              _VP, C.POINTER(C.c_int), C.c_int, _VP]),
    ("sr_gd_solve", C.c_int, [_VP, _VP, _VP, C.c_int, C.POINTER(GdOpts), _VP, C.c_int, _VP]),
    ("sr_gd_solve_early_stop", C.c_int, [_VP, _VP, _VP, C.c_int, C.POINTER(GdOpts), C.c_float, C.c_int, _VP,
                                         C.POINTER(C.c_int), C.c_int, _VP]),
    ("sr_plan_set_phases_device", C.c_int, [_VP, _VP, _VP]),
    ("sr_backward", C.c_int, [_VP, _VP, _VP, _VP, _VP, C.c_int, _VP]),
    ("sr_forward_noalloc", C.c_int, [_VP, _VP, _VP, C.c_int, _VP]),
    ("sr_metrics", C.c_int, [_VP, _VP, C.c_int64, C.c_int, _VP, _VP, _VP]),
    ("sr_dense_create", C.c_int, [C.c_int64, C.c_int64, _VP, C.POINTER(_VP)]),
    ("sr_dense_create_format", C.c_int, [C.c_int64, C.c_int64, _VP, C.c_int, C.POINTER(_VP)]),
    ("sr_dense_destroy", C.c_int, [_VP]),
    ("sr_dense_forward", C.c_int, [_VP, _VP, _VP, C.c_int, _VP]),
    ("sr_dense_adjoint", C.c_int, [_VP, _VP, _VP, C.c_int, _VP]),
    ("sr_dense_gd_solve", C.c_int, [_VP, _VP, _VP, C.c_int, C.POINTER(GdOpts), _VP, C.c_int, _VP]),
    ("sr_dense_spectral_init", C.c_int, [_VP, _VP, _VP, C.c_int, C.POINTER(SpectralOpts), _VP, C.c_int, _VP]),
    ("sr_dense_check", C.c_int, [_VP]),
    ("sr_plan_check", C.c_int, [_VP]),
    ("sr_plan_autotune", C.c_int, [_VP, C.c_int, _VP]),
    ("sr_plan_set_split", C.c_int, [_VP, C.c_int]),
    ("sr_plan_tuning", C.c_int, [_VP, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    ("sr_plan_selftest_timeout", C.c_int, [_VP, _VP]),
    ("sr_ragged_create", C.c_int, [C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int),
                                   C.POINTER(C.c_uint64), C.c_int, C.POINTER(_VP)]),
    ("sr_ragged_destroy", C.c_int, [_VP]),
    ("sr_ragged_layout", C.c_int, [_VP, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                   C.POINTER(C.c_int64), C.POINTER(C.c_int)]),
    ("sr_ragged_forward", C.c_int, [_VP, _VP, _VP, _VP]),
    ("sr_ragged_spectral_init", C.c_int, [_VP, _VP, _VP, C.c_int, C.POINTER(SpectralOpts), _VP, _VP]),
    ("sr_ragged_reserve", C.c_int, [_VP, C.c_int]),
    ("sr_ragged_gd_solve", C.c_int, [_VP, _VP, _VP, C.c_int, C.POINTER(GdOpts), _VP, _VP]),
    ("sr_ragged_check", C.c_int, [_VP]),
    ("sr_ragged_selftest_timeout", C.c_int, [_VP, _VP]),
    ("sr_kernel_launches", C.c_uint64, []),
    ("sr_plan_set_timing", C.c_int, [_VP, C.c_int]),
    ("sr_plan_get_timing", C.c_int, [_VP, C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
    ("sr_status_string", C.c_char_p, [C.c_int]),
    ("sr_last_error", C.c_char_p, []),
]

_LIB = None


def load(path: str | None = None):
    """Load libsr.so (once) and declare the signatures. Raises if it is missing."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = path or _build.library_path()
    if not os.path.exists(path):
        raise ImportError(f"libsr.so not found at {path}: build it with paper_2409_05734_gb300.buildlib.build()")
    lib = C.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def check(status: int, where: str):
    if status != SR_OK:
        msg = load().sr_last_error().decode(errors="replace")
        raise SrError(status, where, msg)
