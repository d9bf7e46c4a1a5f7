"""Torch-facing binding of the C ABI (argument marshalling only).

Each function takes FP64 CUDA tensors in block storage, checks shapes and
device placement, and calls the same-named C entry point on the current torch
stream with a workspace tensor from torch's allocator. No computation happens
here.
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib

OP_FACTOR, OP_SELINV, OP_SOLVE, OP_LOGDET = 1, 2, 3, 4


class BTAError(RuntimeError):
    pass


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None and t.numel() else None


def _stream(device):
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _check(rc: int, name: str):
    if rc != 0:
        if rc < 0:
            raise BTAError(f"{name}: invalid argument {-rc} (return code {rc})")
        raise BTAError(f"{name}: CUDA error {rc}")


def _dims(diag, lower, arrow, tip, on_host=False):
    if diag.dim() != 3 or diag.shape[1] != diag.shape[2]:
        raise ValueError("diag must be [n, b, b]")
    n, b = diag.shape[0], diag.shape[1]
    a = tip.shape[0] if tip is not None else 0
    for name, t, shape in (("lower", lower, (n - 1, b, b)), ("arrow", arrow, (n, a, b)),
                           ("tip", tip, (a, a))):
        if t is None:
            if (name == "lower" and n > 1) or (name != "lower" and a > 0):
                raise ValueError(f"{name} is required")
            continue
        if tuple(t.shape) != shape:
            raise ValueError(f"{name} must have shape {shape}, got {tuple(t.shape)}")
    for t in (diag, lower, arrow, tip):
        if t is None:
            continue
        if t.dtype != torch.float64 or t.is_cuda == on_host or not t.is_contiguous():
            raise ValueError("blocks must be contiguous float64 " + ("CPU" if on_host else "CUDA")
                             + " tensors")
        if t.device != diag.device:
            raise ValueError("all blocks must be on one device")
    return n, b, a


def workspace_bytes(op: int, n: int, b: int, a: int, nrhs: int = 1) -> int:
    return int(_lib.load().bta_workspace_bytes(op, n, b, a, nrhs))


def _workspace(op, n, b, a, device, nrhs=1):
    nbytes = workspace_bytes(op, n, b, a, nrhs)
    ws = torch.empty(max(nbytes, 256) + 256, dtype=torch.uint8, device=device)
    off = (-ws.data_ptr()) % 256
    return ws, ctypes.c_void_p(ws.data_ptr() + off), nbytes


def factor(diag, lower, arrow, tip):
    """In place: A -> L (Algorithm 1). Returns the same tensors."""
    n, b, a = _dims(diag, lower, arrow, tip)
    lib = _lib.load()
    with torch.cuda.device(diag.device):
        ws, wp, nb = _workspace(OP_FACTOR, n, b, a, diag.device)
        _check(lib.bta_factor_ws(n, b, a, _ptr(diag), _ptr(lower), _ptr(arrow), _ptr(tip),
                                 wp, nb, _stream(diag.device)), "bta_factor")
    return diag, lower, arrow, tip


def selinv(diag, lower, arrow, tip):
    """In place: L -> X, the selected inverse on the BTA pattern (Algorithm 2)."""
    n, b, a = _dims(diag, lower, arrow, tip)
    lib = _lib.load()
    with torch.cuda.device(diag.device):
        ws, wp, nb = _workspace(OP_SELINV, n, b, a, diag.device)
        _check(lib.bta_selinv_ws(n, b, a, _ptr(diag), _ptr(lower), _ptr(arrow), _ptr(tip),
                                 wp, nb, _stream(diag.device)), "bta_selinv")
    return diag, lower, arrow, tip


def solve(diag, lower, arrow, tip, rhs):
    """In place on rhs [N, nrhs] (or [N]): rhs <- A^{-1} rhs, given the factor L."""
    n, b, a = _dims(diag, lower, arrow, tip)
    if rhs.dtype != torch.float64 or not rhs.is_cuda or not rhs.is_contiguous():
        raise ValueError("rhs must be a contiguous float64 CUDA tensor")
    nrhs = 1 if rhs.dim() == 1 else rhs.shape[1]
    if rhs.shape[0] != n * b + a:
        raise ValueError("rhs must have n*b + a rows")
    lib = _lib.load()
    with torch.cuda.device(diag.device):
        ws, wp, nb = _workspace(OP_SOLVE, n, b, a, diag.device, nrhs)
        _check(lib.bta_solve_ws(n, b, a, _ptr(diag), _ptr(lower), _ptr(arrow), _ptr(tip),
                                _ptr(rhs), nrhs, wp, nb, _stream(diag.device)), "bta_solve")
    return rhs


def logdet(diag, tip, out=None):
    """log det A from the factor; returns a 0-d float64 CUDA tensor (no host sync)."""
    n, b = diag.shape[0], diag.shape[1]
    a = tip.shape[0] if tip is not None else 0
    if out is None:
        out = torch.empty((), dtype=torch.float64, device=diag.device)
    lib = _lib.load()
    with torch.cuda.device(diag.device):
        ws, wp, nb = _workspace(OP_LOGDET, n, b, a, diag.device)
        _check(lib.bta_logdet_ws(n, b, a, _ptr(diag), _ptr(tip), _ptr(out), wp, nb,
                                 _stream(diag.device)), "bta_logdet")
    return out


def get_info(device=None) -> int:
    """Synchronizes the current stream and returns (and clears) the info word."""
    lib = _lib.load()
    v = ctypes.c_int64(0)
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else device
    with torch.cuda.device(dev):
        _check(lib.bta_get_info(_stream(dev), ctypes.byref(v)), "bta_get_info")
    return int(v.value)


PREC_FP64, PREC_OZAKI, PREC_BF16X3 = 0, 1, 2
_PREC_NAMES = {"fp64": PREC_FP64, "ozaki": PREC_OZAKI, "bf16x3": PREC_BF16X3}


def set_precision(prec) -> None:
    """Precision of the large block products of factor/selinv: "fp64" (DMMA),
    "ozaki" (FP64 emulated on BF16 tensor cores) or "bf16x3" (mixed)."""
    p = _PREC_NAMES[prec] if isinstance(prec, str) else int(prec)
    _check(_lib.load().bta_set_precision(p), "bta_set_precision")


def get_precision() -> int:
    return int(_lib.load().bta_get_precision())


def gemm(A, B, C=None, *, alpha=1.0, beta=0.0, trans_a=False, trans_b=False, precision="fp64"):
    """C = alpha op(A) op(B) + beta C through bta_gemm (FP64 tensors on one device)."""
    p = _PREC_NAMES[precision] if isinstance(precision, str) else int(precision)
    for t in (A, B):
        if t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous() or t.dim() != 2:
            raise ValueError("A and B must be contiguous 2-D float64 CUDA tensors")
    M = A.shape[1] if trans_a else A.shape[0]
    K = A.shape[0] if trans_a else A.shape[1]
    Kb = B.shape[1] if trans_b else B.shape[0]
    N = B.shape[0] if trans_b else B.shape[1]
    if K != Kb:
        raise ValueError("inner dimensions differ")
    if C is None:
        C = torch.zeros((M, N), dtype=torch.float64, device=A.device)
    lib = _lib.load()
    with torch.cuda.device(A.device):
        nbytes = int(lib.bta_gemm_workspace_bytes(p, M, N, K))
        ws = torch.empty(max(nbytes, 256) + 256, dtype=torch.uint8, device=A.device)
        wp = ctypes.c_void_p(ws.data_ptr() + (-ws.data_ptr()) % 256)
        _check(lib.bta_gemm(p, M, N, K, alpha, _ptr(A), A.shape[1], int(trans_a), _ptr(B), B.shape[1],
                            int(trans_b), beta, _ptr(C), C.shape[1], wp, nbytes, _stream(A.device)),
               "bta_gemm")
    return C


def tc_status() -> int:
    """1 if a tensor-core kernel gave up on a bounded wait since the last read."""
    v = ctypes.c_int(0)
    _check(_lib.load().bta_tc_status(ctypes.byref(v)), "bta_tc_status")
    return int(v.value)


def factor_selinv_all(diag, lower, arrow, tip, rhs=None, logdet_out=None):
    """factor + logdet + solve (if rhs is given, in place) + selinv (A -> X in
    place) in one call, the solve overlapped with the selected inversion's
    prologue. Returns log det A as a 0-d CUDA tensor."""
    n, b, a = _dims(diag, lower, arrow, tip)
    nrhs = 0
    if rhs is not None:
        if rhs.dtype != torch.float64 or not rhs.is_cuda or not rhs.is_contiguous():
            raise ValueError("rhs must be a contiguous float64 CUDA tensor")
        if rhs.shape[0] != n * b + a:
            raise ValueError("rhs must have n*b + a rows")
        nrhs = rhs.shape[1] if rhs.dim() == 2 else 1
    if logdet_out is None:
        logdet_out = torch.empty((), dtype=torch.float64, device=diag.device)
    lib = _lib.load()
    with torch.cuda.device(diag.device):
        nbytes = int(lib.bta_all_workspace_bytes(n, b, a, nrhs))
        if nbytes == 0:
            raise BTAError("bta_all_workspace_bytes: invalid arguments")
        ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=diag.device)
        wp = ctypes.c_void_p(ws.data_ptr() + (-ws.data_ptr()) % 256)
        _check(lib.bta_factor_selinv_all(n, b, a, _ptr(diag), _ptr(lower), _ptr(arrow), _ptr(tip),
                                         _ptr(rhs), nrhs, _ptr(logdet_out), wp, nbytes,
                                         _stream(diag.device)), "bta_factor_selinv_all")
    return logdet_out


def factor_selinv_host(diag, lower, arrow, tip, rhs=None, out=None, device=None):
    """Factor, log det, solve (if rhs is given) and selected inversion of a matrix
    held in host memory (CPU tensors; pinned ones let the copies overlap the
    sweeps). Returns (x_diag, x_lower, x_arrow, x_tip, x, logdet) as CPU tensors
    (`out`, if given, is that tuple preallocated); they are valid once the
    current stream of `device` has finished (torch.cuda.synchronize)."""
    n, b, a = _dims(diag, lower, arrow, tip, on_host=True)
    for name, t in (("diag", diag), ("lower", lower), ("arrow", arrow), ("tip", tip), ("rhs", rhs)):
        if t is not None and (t.device.type != "cpu" or t.dtype != torch.float64 or not t.is_contiguous()):
            raise ValueError(f"{name} must be a contiguous float64 CPU tensor")
    nrhs = 0 if rhs is None else (rhs.shape[1] if rhs.dim() == 2 else 1)
    if rhs is not None and rhs.shape[0] != n * b + a:
        raise ValueError("rhs must have n*b + a rows")
    device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    if out is None:
        pin = diag.is_pinned()
        def _e(t):
            return None if t is None else torch.empty(t.shape, dtype=torch.float64, pin_memory=pin)
        out = (_e(diag), _e(lower), _e(arrow), _e(tip), _e(rhs), torch.empty((), dtype=torch.float64,
                                                                         pin_memory=pin))
    lib = _lib.load()
    with torch.cuda.device(device):
        nbytes = int(lib.bta_host_pipeline_workspace_bytes(n, b, a, nrhs))
        if nbytes == 0:
            raise BTAError("bta_host_pipeline_workspace_bytes: invalid arguments")
        ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
        wp = ctypes.c_void_p(ws.data_ptr() + (-ws.data_ptr()) % 256)
        _check(lib.bta_factor_selinv_host(n, b, a, _ptr(diag), _ptr(lower), _ptr(arrow), _ptr(tip),
                                          _ptr(rhs), nrhs, _ptr(out[0]), _ptr(out[1]), _ptr(out[2]),
                                          _ptr(out[3]), _ptr(out[4]), _ptr(out[5]), wp, nbytes,
                                          _stream(device)), "bta_factor_selinv_host")
    return out


def wait_selftest(polls: int = 1000) -> int:
    """Runs the bounded-wait timeout self-test; 1 if the timeout was recorded."""
    v = ctypes.c_int(0)
    _check(_lib.load().bta_wait_selftest(int(polls), ctypes.byref(v)), "bta_wait_selftest")
    return int(v.value)


def factor_selinv_partitioned(diag, lower, arrow, tip, parts=4, lb=1.8, logdet_out=None):
    """In place A -> X by the partitioned scheme (P concurrent partitions plus a
    reduced system); returns log det A as a 0-d CUDA tensor."""
    n, b, a = _dims(diag, lower, arrow, tip)
    lib = _lib.load()
    if logdet_out is None:
        logdet_out = torch.empty((), dtype=torch.float64, device=diag.device)
    with torch.cuda.device(diag.device):
        nbytes = int(lib.bta_partitioned_workspace_bytes(n, b, a, parts, lb))
        if nbytes == 0:
            raise BTAError("bta_partitioned_workspace_bytes: invalid arguments")
        ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=diag.device)
        wp = ctypes.c_void_p(ws.data_ptr() + (-ws.data_ptr()) % 256)
        _check(lib.bta_factor_selinv_partitioned(n, b, a, _ptr(diag), _ptr(lower), _ptr(arrow), _ptr(tip),
                                                 parts, lb, _ptr(logdet_out), wp, nbytes,
                                                 _stream(diag.device)), "bta_factor_selinv_partitioned")
    return logdet_out
