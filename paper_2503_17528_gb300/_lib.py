"""ctypes loader for libbta.so (the C ABI declared in include/bta.h).

Loading fails loudly: there is no fallback path. Build the library with
``python -m paper_2503_17528_gb300.build`` (or ``__graft_entry__.build()``).
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbta.so")

_i64 = ctypes.c_int64
_p = ctypes.c_void_p
_sz = ctypes.c_size_t

# name -> argtypes (every entry point returns int, except bta_workspace_bytes)
_SIGS = {
    "bta_factor": [_i64, _i64, _i64, _p, _p, _p, _p, _p],
    "bta_selinv": [_i64, _i64, _i64, _p, _p, _p, _p, _p],
    "bta_solve": [_i64, _i64, _i64, _p, _p, _p, _p, _p, _i64, _p],
    "bta_logdet": [_i64, _i64, _i64, _p, _p, _p, _p],
    "bta_get_info": [_p, ctypes.POINTER(_i64)],
    "bta_workspace_bytes": [ctypes.c_int, _i64, _i64, _i64, _i64],
    "bta_factor_ws": [_i64, _i64, _i64, _p, _p, _p, _p, _p, _sz, _p],
    "bta_selinv_ws": [_i64, _i64, _i64, _p, _p, _p, _p, _p, _sz, _p],
    "bta_solve_ws": [_i64, _i64, _i64, _p, _p, _p, _p, _p, _i64, _p, _sz, _p],
    "bta_logdet_ws": [_i64, _i64, _i64, _p, _p, _p, _p, _sz, _p],
    "bta_logdet_noalloc": [_i64, _i64, _i64, _p, _p, _p, _p],
    "bta_timing_enable": [ctypes.c_int],
    "bta_timing_read": [ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                        ctypes.POINTER(_i64)],
    "bta_probe_fp64_peak": [_p, _i64, ctypes.POINTER(ctypes.c_double), _p],
    "bta_batch_workspace_bytes": [_i64, _i64, _i64, ctypes.c_int],
    "bta_factor_selinv_batched": [_i64, ctypes.c_void_p, ctypes.c_int, _p],
    "bta_partitioned_workspace_bytes": [_i64, _i64, _i64, _i64, ctypes.c_double],
    "bta_factor_selinv_partitioned": [_i64, _i64, _i64, _p, _p, _p, _p, _i64, ctypes.c_double, _p, _p,
                                      _sz, _p],
    "bta_grad_blocks": [_i64, _i64, _i64, _p, _p, _p, _p, _p, ctypes.c_double, ctypes.c_double,
                        _p, _p, _p, _p, _p, _p],
    "bta_dot": [_i64, _p, _p, _p, _p, _sz, _p],
    "bta_set_precision": [ctypes.c_int],
    "bta_get_precision": [],
    "bta_gemm_workspace_bytes": [ctypes.c_int, _i64, _i64, _i64],
    "bta_gemm": [ctypes.c_int, _i64, _i64, _i64, ctypes.c_double, _p, _i64, ctypes.c_int, _p, _i64,
                 ctypes.c_int, ctypes.c_double, _p, _i64, _p, _sz, _p],
    "bta_tc_status": [ctypes.POINTER(ctypes.c_int)],
    "bta_wait_selftest": [_i64, ctypes.POINTER(ctypes.c_int)],
    "bta_host_pipeline_workspace_bytes": [_i64, _i64, _i64, _i64],
    "bta_all_workspace_bytes": [_i64, _i64, _i64, _i64],
    "bta_factor_selinv_all": [_i64, _i64, _i64, _p, _p, _p, _p, _p, _i64, _p, _p, _sz, _p],
    "bta_factor_selinv_host": [_i64, _i64, _i64, _p, _p, _p, _p, _p, _i64, _p, _p, _p, _p, _p, _p,
                               _p, _sz, _p],
    "bta_plan_entry_workspace_bytes": [_i64, _i64, _i64],
    "bta_plan_create": [_i64, _p, _p, _p],
    "bta_plan_run": [_p, _p],
    "bta_plan_status": [_p, ctypes.POINTER(ctypes.c_int), _p, _p],
    "bta_plan_describe": [_p, ctypes.POINTER(_i64), ctypes.c_int],
    "bta_plan_destroy": [_p],
    "bta_version": [],
}

class BatchEntry(ctypes.Structure):
    _fields_ = [("n", _i64), ("b", _i64), ("a", _i64), ("diag", _p), ("lower", _p), ("arrow", _p),
                ("tip", _p), ("logdet_out", _p), ("prec", ctypes.c_int), ("ws", _p), ("ws_bytes", _sz)]


class PlanParams(ctypes.Structure):
    _fields_ = [("ctas_per_sm", ctypes.c_int), ("levels", ctypes.c_int), ("rows_per_item", ctypes.c_int),
                ("reserved", ctypes.c_int)]


_lib = None


def load() -> ctypes.CDLL:
    """Load libbta.so once; raises if it is missing or lacks a symbol."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it first (paper_2503_17528_gb300.build)")
    lib = ctypes.CDLL(LIB_PATH)
    for name, args in _SIGS.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = _sz if name.endswith("workspace_bytes") else ctypes.c_int
    _lib = lib
    return lib


def exported_symbols() -> list[str]:
    return list(_SIGS)
