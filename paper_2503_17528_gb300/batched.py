"""Batched form: many independent BTA matrices of uneven n, b, a factored,
log-det'ed and inverted in one library call (bta_factor_selinv_batched), which
can be captured once into a CUDA graph and replayed.

The call assigns matrices largest first to the least-loaded of `nstreams`
library streams forked from the caller's stream; the streams join back, so a
capture of the caller's stream records the whole batch. The number of streams
and the engine per block size (FP64 DMMA or the tensor-core FP64 emulation)
come from the autotuner in tune.py.
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib
from .api import PREC_BF16X3, PREC_FP64, PREC_OZAKI, _check, _stream

_PREC = {"fp64": PREC_FP64, "ozaki": PREC_OZAKI, "bf16x3": PREC_BF16X3}

# Engine policies: block size b -> precision mode.
POLICIES = {
    "fp64": lambda b: PREC_FP64,
    "ozaki": lambda b: PREC_OZAKI,
    "ozaki_b256": lambda b: PREC_OZAKI if b >= 256 else PREC_FP64,
}


def _p(t):
    return t.data_ptr() if t is not None and t.numel() else None


class Batch:
    """Holds the entry table and per-matrix workspaces for a list of matrices.

    mats: list of (diag, lower, arrow, tip) contiguous float64 CUDA tensors on
    one device; they are overwritten in place with the selected inverse.
    """

    def __init__(self, mats, policy="fp64", nstreams=8):
        self.mats = mats
        self.nstreams = int(nstreams)
        self.policy = policy
        pick = POLICIES[policy] if isinstance(policy, str) else policy
        dev = mats[0][0].device
        self.device = dev
        lib = _lib.load()
        self.logdets = torch.empty(len(mats), dtype=torch.float64, device=dev)
        self.entries = (_lib.BatchEntry * len(mats))()
        self.ws = []
        for k, (d, l, ar, t) in enumerate(mats):
            n, b = d.shape[0], d.shape[1]
            a = t.shape[0] if t is not None else 0
            prec = pick(b)
            nbytes = int(lib.bta_batch_workspace_bytes(n, b, a, prec))
            if nbytes == 0:
                raise ValueError(f"invalid batch entry {k}: n={n} b={b} a={a}")
            w = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
            self.ws.append(w)
            e = self.entries[k]
            e.n, e.b, e.a = n, b, a
            e.diag, e.lower, e.arrow, e.tip = _p(d), _p(l), _p(ar), _p(t)
            e.logdet_out = self.logdets.data_ptr() + 8 * k
            e.prec = prec
            e.ws = w.data_ptr() + (-w.data_ptr()) % 256
            e.ws_bytes = nbytes

    def run(self):
        """Enqueue the batch on the current stream; returns the log-det tensor."""
        lib = _lib.load()
        with torch.cuda.device(self.device):
            _check(lib.bta_factor_selinv_batched(len(self.mats), ctypes.addressof(self.entries),
                                                 self.nstreams, _stream(self.device)),
                   "bta_factor_selinv_batched")
        return self.logdets

    def capture(self):
        """Record one run into a CUDA graph (call run() once before, outside capture)."""
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.run()
        return g


class PersistentBatch:
    """The batched form as ONE persistent kernel launch (bta_plan_*), FP64.

    mats: list of (diag, lower, arrow, tip) contiguous float64 CUDA tensors on
    one device, overwritten in place with the selected inverse by run(). The plan
    (schedule and device tables) is built once here, for exactly these buffers;
    run() enqueues one launch on the current stream and can be captured in a
    CUDA graph. Tuning parameters (0 = automatic): ctas_per_sm, levels (priority
    levels 1..8 of the device queues: operations of the matrices with the most
    remaining work first; 1 = ready order), rows_per_item (1 or 2).
    """

    def __init__(self, mats, ctas_per_sm=0, levels=0, rows_per_item=0):
        self.mats = mats
        dev = mats[0][0].device
        self.device = dev
        lib = _lib.load()
        self.logdets = torch.empty(len(mats), dtype=torch.float64, device=dev)
        self.entries = (_lib.BatchEntry * len(mats))()
        self.ws = []
        for k, (d, l, ar, t) in enumerate(mats):
            n, b = d.shape[0], d.shape[1]
            a = t.shape[0] if t is not None else 0
            nbytes = int(lib.bta_plan_entry_workspace_bytes(n, b, a))
            if nbytes == 0:
                raise ValueError(f"invalid batch entry {k}: n={n} b={b} a={a}")
            w = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
            self.ws.append(w)
            e = self.entries[k]
            e.n, e.b, e.a = n, b, a
            e.diag, e.lower, e.arrow, e.tip = _p(d), _p(l), _p(ar), _p(t)
            e.logdet_out = self.logdets.data_ptr() + 8 * k
            e.prec = PREC_FP64
            e.ws = w.data_ptr() + (-w.data_ptr()) % 256
            e.ws_bytes = nbytes
        self.params = _lib.PlanParams(int(ctas_per_sm), int(levels), int(rows_per_item), 0)
        self._plan = ctypes.c_void_p()
        with torch.cuda.device(dev):
            _check(lib.bta_plan_create(len(mats), ctypes.addressof(self.entries),
                                       ctypes.addressof(self.params), ctypes.byref(self._plan)),
                   "bta_plan_create")

    def run(self):
        """Enqueue one run on the current stream; returns the log-det tensor."""
        lib = _lib.load()
        with torch.cuda.device(self.device):
            _check(lib.bta_plan_run(self._plan, _stream(self.device)), "bta_plan_run")
        return self.logdets

    def capture(self):
        """Record one run into a CUDA graph."""
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.run()
        return g

    def status(self):
        """(timed_out, per-matrix info) of the last run (synchronizes)."""
        lib = _lib.load()
        to = ctypes.c_int(0)
        info = (ctypes.c_int64 * len(self.mats))()
        with torch.cuda.device(self.device):
            _check(lib.bta_plan_status(self._plan, ctypes.byref(to), info, _stream(self.device)),
                   "bta_plan_status")
        return int(to.value), [int(x) for x in info]

    def describe(self):
        lib = _lib.load()
        out = (ctypes.c_int64 * 8)()
        _check(lib.bta_plan_describe(self._plan, out, 8), "bta_plan_describe")
        keys = ("grid", "ctas_per_sm", "levels", "rows_per_item", "ops", "items", "flops", "ready_at_start")
        return dict(zip(keys, [int(x) for x in out]))

    def close(self):
        if self._plan:
            lib = _lib.load()
            with torch.cuda.device(self.device):
                lib.bta_plan_destroy(self._plan)
            self._plan = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
