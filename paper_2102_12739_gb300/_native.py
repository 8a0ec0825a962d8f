"""ctypes binding of libdegrid.so (argument marshalling only).

Every entry point declared in include/degrid.h is bound here under the same
name.  The library is loaded from this package's ``_build`` directory; if it
is missing it is built with nvcc, and if that is impossible the import fails
loudly: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

DG_OK = 0
DG_ERR_ARG = 1
DG_ERR_CUDA = 2
DG_ERR_OOM = 3
DG_ERR_DTYPE = 4
DG_ERR_OFFSETS = 5
DG_ERR_UNSUPPORTED = 6
DG_ERR_SCRATCH_LIMIT = 7
DG_ERR_TIMEOUT = 8
DG_ERR_BOUNDS = 9

DG_C64 = 0
DG_C32_F16 = 1
DG_C32_BF16 = 2

DG_TABLE2D_MAX_OVERSAMPLE = 256
DG_DIRECT_RUNS_NEVER = 33
DG_DIRECT_RUNS_DEFAULT = DG_DIRECT_RUNS_NEVER
DG_DIRECT_RUNS_SHORT = 9

# name -> (restype, argtypes); mirrors include/degrid.h
_P = ctypes.c_void_p
_I = ctypes.c_int
_I64 = ctypes.c_int64
SIGNATURES = {
    "degrid_status_string": (ctypes.c_char_p, [_I]),
    "degrid_version": (ctypes.c_char_p, []),
    "degrid_schedule_reserve": (_I, [_I, _I, _I, _I64, ctypes.POINTER(_I), ctypes.POINTER(_I64)]),
    "degrid_plan_create": (_I, [ctypes.POINTER(_P), _I, _I, _I, _P, _I, _I, _P, _I, _I, _I, _I]),
    "degrid_plan_destroy": (None, [_P]),
    "degrid_plan_set_tuning": (_I, [_P, _I, _I, _I]),
    "degrid_plan_get_tuning": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "degrid_plan_create_2d": (_I, [ctypes.POINTER(_P), _I, _I, _I, _P, _I, _P, _I, _I, _I, _I]),
    "degrid_execute_host": (_I, [_P, _I, _P, _P, _P, _P, _I64, _P]),
    "degrid_plan_set_compensated": (_I, [_P, _I]),
    "degrid_plan_set_direct_runs": (_I, [_P, _I]),
    "degrid_plan_get_direct_runs": (_I, [_P, ctypes.POINTER(_I)]),
    "degrid_plan_get_compensated": (_I, [_P, ctypes.POINTER(_I)]),
    "degrid_plan_set_gather": (_I, [_P, _I]),
    "degrid_plan_set_host_direct": (_I, [_P, _I]),
    "degrid_plan_get_host_direct": (_I, [_P, ctypes.POINTER(_I)]),
    "degrid_plan_get_gather": (_I, [_P, ctypes.POINTER(_I)]),
    "degrid_measure_fp32_peak": (_I, [_I, _I, ctypes.POINTER(ctypes.c_double)]),
    "degrid_measure_l2_read_bw": (_I, [_I, ctypes.POINTER(ctypes.c_double)]),
    "degrid_measure_l2_reduce_bw": (_I, [_I, ctypes.POINTER(ctypes.c_double)]),
    "degrid_plan_enable_timing": (_I, [_P, _I]),
    "degrid_plan_kernel_times_ms": (_I, [_P, ctypes.POINTER(ctypes.c_float), _I,
                                         ctypes.POINTER(_I)]),
    "degrid_execute": (_I, [_P, _P, _I, _P, _P, _P, _P, _I64, _P]),
    "grid_adjoint_execute": (_I, [_P, _P, _I, _P, _P, _I64, _P, _P, _I]),
    "degrid_coords_execute": (_I, [_P, _P, _P, _I64, _P]),
    "degrid_pack_subgrids": (_I, [_P, _I, _I, _I64, _P, _P, _P]),
    "degrid_get_status": (_I, [_P, _P, ctypes.POINTER(_I64)]),
    "degrid_execute_noalloc": (_I, [_P, _I, _I, _I, _P, _I, _P, _I, _I, _I, _P, _P, _P, _P,
                                    _I64, _P, _P]),
    "subgrid_predict_plan_create": (_I, [ctypes.POINTER(_P), _I, _I, _I, _I]),
    "subgrid_predict_execute": (_I, [_P, _P, ctypes.c_double, _P, _P, _I, _P, _P, _P]),
    "subgrid_predict_plan_destroy": (None, [_P]),
}

_lock = threading.Lock()
_lib = None


class DegridError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} (status {status})")


def _variant() -> str:
    """The library variant named by $DEGRID_LIBRARY_VARIANT ("" = the product library)."""
    v = os.environ.get("DEGRID_LIBRARY_VARIANT", "")
    if v and v not in _build.VARIANTS:
        raise RuntimeError(f"unknown DEGRID_LIBRARY_VARIANT {v!r}; known: {sorted(_build.VARIANTS)}")
    return v


def lib_path() -> str:
    v = _variant()
    return _build.variant_path(v) if v else _build.LIB_PATH


def load(build_if_missing: bool = True):
    """Load libdegrid.so (building it first if needed) and bind signatures."""
    global _lib
    with _lock:
        if _lib is None:
            variant = _variant()
            path = lib_path()
            if variant:
                if build_if_missing:
                    _build.build_variant(variant)
            elif build_if_missing and not _build.up_to_date():
                _build.build()
            if not os.path.exists(path):
                raise RuntimeError(f"libdegrid.so not found at {path}; run "
                                   "python -m paper_2102_12739_gb300.build")
            lib = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def status_string(status: int) -> str:
    return load().degrid_status_string(int(status)).decode()


def check(status: int, where: str) -> None:
    if status != DG_OK:
        raise DegridError(status, where)
