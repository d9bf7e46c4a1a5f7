#!/usr/bin/env python3
"""Benchmark of the BTA hot path on GB300: factor + log-det + solve + selected inversion.

One step = one pass of the whole path over one synthetic BTA matrix resident in
HBM: reset the working blocks from a pristine device copy, bta_factor,
bta_logdet, bta_solve (4 right-hand sides), bta_selinv. The metric is ms per
matrix (lower is better); TFLOP/s of the algorithmic FP64 flop count is reported
beside it. Multi-GPU (torchrun): every rank factors and inverts its own matrix
(independent problems, weak scaling, no collective on the data path).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]

Default workload: n=365, b=1024, a=8, dominance shift 1.01 (inputs ~6.1 GB, far
above the 129 MB L2, so no L2 flush is needed between steps).
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bta_inputs as gen  # noqa: E402

METRIC = "BTA factor+selinv ms/matrix & TFLOP/s vs FP64 peak; batched/mixed speedup"
WORKLOADS = {
    "n365_b1024_a8": dict(n=365, b=1024, a=8, shift=gen.SHIFT_1_01, shift_name="1.01 x row sum"),
    "n16_b32_a4": dict(n=16, b=32, a=4, shift=gen.SHIFT_PLUS_ONE, shift_name="1 + row sum"),
    "n256_b2048_a16": dict(n=256, b=2048, a=16, shift=gen.SHIFT_1_001, shift_name="1.001 x row sum"),
}
NRHS = 4


# Algorithmic FP64 flops (LAPACK counts of the method itself).
def flops_factor(n, b, a):
    return n * b**3 / 3 + (n - 1) * 2 * b**3 + n * a * b**2 + (n - 1) * 2 * a * b**2 + n * a**2 * b + a**3 / 3


def flops_selinv(n, b, a):
    return 2 * a**3 / 3 + n * 2 * b**3 / 3 + (n - 1) * 4 * b**3 + n * (2 * a * b**2 + 2 * a**2 * b) + (n - 1) * 4 * a * b**2


def flops_solve(n, b, a, r):
    return 2 * r * (n * b * b + 2 * (n - 1) * b * b + 2 * n * a * b + a * a)


def pattern_bytes(n, b, a):
    return 8 * (n * b * b + (n - 1) * b * b + n * a * b + a * a)


# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    @staticmethod
    def _die_with_parent():
        # The sampler must never outlive the benchmark (a profiler waits for
        # every process of the tree): ask the kernel to SIGTERM it when the
        # parent exits.
        try:
            import signal
            ctypes.CDLL("libc.so.6", use_errno=True).prctl(1, signal.SIGTERM)  # PR_SET_PDEATHSIG
        except Exception:
            pass

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["timeout", "900", "nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True,
                preexec_fn=self._die_with_parent)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
def cpu_oracle_sample(w, arrays, target_s=8.0, max_blocks=None):
    """Time the oracle (factor, logdet, solve, selinv) on leading principal block
    sub-matrices of the workload, doubling the block count until one run takes
    >= target_s. Returns (ms per full matrix, sample description, cores)."""
    import oracle
    d, l, ar, t, r = arrays
    n, b, a = w["n"], w["b"], w["a"]
    ns = min(n, 2)
    while True:
        rs = np.concatenate([r[: ns * b], r[n * b:]])
        t0 = time.perf_counter()
        F = oracle.pobtaf(d[:ns], l[: ns - 1], ar[:ns], t)
        oracle.logdet(F)
        oracle.solve(F, rs)
        oracle.pobtasi(F)
        dt = time.perf_counter() - t0
        if dt >= target_s or ns >= n or (max_blocks and ns >= max_blocks):
            break
        ns = min(n, ns * 2)
    per_full = dt * 1e3 * n / ns
    desc = (f"oracle (NumPy/SciPy FP64) on the leading {ns} of {n} block rows plus the arrowhead "
            f"({dt:.1f} s), scaled by n/{ns} to one full matrix")
    return per_full, desc, os.cpu_count()


def make_workload(w, seed):
    d, l, ar, t = gen.make_bta(w["n"], w["b"], w["a"], seed=seed, shift=w["shift"])
    r = gen.make_rhs(w["n"], w["b"], w["a"], NRHS, seed=seed + 1000)
    return d, l, ar, t, r


# ---------------------------------------------------------------------------
def run_reference(args, w, rank, world):
    if rank != 0:
        return 0
    arrays = make_workload(w, seed=0)
    t_steps = []
    desc = cores = None
    for i in range(args.warmup + args.steps):
        per_full, desc, cores = cpu_oracle_sample(w, arrays, target_s=args.ref_target_s)
        if i >= args.warmup:
            t_steps.append(per_full)
    v = statistics.median(t_steps)
    line = {
        "impl": "reference", "metric": METRIC, "value": round(v, 3), "unit": "ms/matrix",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(v, 3),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(w),
        "cpu_baseline": {"value": round(v, 3), "unit": "ms/matrix", "cores": cores, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": round(v, 3), "unit": "ms/matrix", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def workload_config(w):
    n, b, a = w["n"], w["b"], w["a"]
    return {"workload": f"n{n}_b{b}_a{a}", "n": n, "b": b, "a": a, "nrhs": NRHS,
            "dominance_shift": w["shift_name"], "generator": "seeded N(0,1)/sqrt(b) blocks, diagonally dominant",
            "l2": f"inputs {pattern_bytes(n, b, a) / 1e9:.2f} GB per matrix > 129 MB L2; no flush",
            "steps_include": "device reset copy + factor + logdet + solve + selinv"}


def run_ours(args, w, rank, world, local_rank):
    import torch
    import paper_2503_17528_gb300 as bta
    from paper_2503_17528_gb300 import _lib

    dist = None
    if world > 1:
        import torch.distributed as dist
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    lib = _lib.load()
    n, b, a = w["n"], w["b"], w["a"]

    arrays = make_workload(w, seed=rank)
    d, l, ar, t, r = arrays
    P = [torch.from_numpy(x).to(dev) for x in (d, l, ar, t, r)]
    W = [torch.empty_like(x) for x in P]
    ld_out = torch.empty((), dtype=torch.float64, device=dev)

    def step():
        for dst, src in zip(W, P):
            dst.copy_(src, non_blocking=True)
        D, Lo, Ar, Ti, R = W
        bta.factor(D, Lo, Ar, Ti)
        bta.logdet(D, Ti, out=ld_out)
        bta.solve(D, Lo, Ar, Ti, R)
        bta.selinv(D, Lo, Ar, Ti)

    def barrier():
        if dist is not None:
            dist.barrier()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    if bta.get_info(dev) != 0:
        raise RuntimeError("non-positive pivot in the benchmark matrix")

    sampler = ClockSampler(local_rank)
    barrier()
    torch.cuda.synchronize(dev)
    if not args.no_clocks:
        sampler.start()
    time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        step()
    e1.record()
    torch.cuda.synchronize(dev)
    barrier()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    if dist is not None:
        tt = torch.tensor([ms], dtype=torch.float64, device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms = float(tt.item())
    ms_per_step = ms / args.steps
    value = ms_per_step / world  # whole job: `world` matrices per step

    # End to end through the public API with host buffers (pinned).
    e2e = None
    if not args.no_e2e:
        H = [torch.from_numpy(x).pin_memory() for x in (d, l, ar, t, r)]
        O = [torch.empty(x.shape, dtype=torch.float64).pin_memory() for x in (d, l, ar, t, r)]
        O_ld = torch.empty((), dtype=torch.float64).pin_memory()

        def e2e_step():
            for dst, src in zip(W, H):
                dst.copy_(src, non_blocking=True)
            D, Lo, Ar, Ti, R = W
            bta.factor(D, Lo, Ar, Ti)
            bta.logdet(D, Ti, out=ld_out)
            bta.solve(D, Lo, Ar, Ti, R)
            bta.selinv(D, Lo, Ar, Ti)
            for dst, src in zip(O, W):
                dst.copy_(src, non_blocking=True)
            O_ld.copy_(ld_out, non_blocking=True)

        e2e_step()
        torch.cuda.synchronize(dev)
        barrier()
        k2 = max(1, min(args.steps, 2))
        e0.record()
        for _ in range(k2):
            e2e_step()
        e1.record()
        torch.cuda.synchronize(dev)
        barrier()
        ms2 = e0.elapsed_time(e1)
        if dist is not None:
            tt = torch.tensor([ms2], dtype=torch.float64, device=dev)
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            ms2 = float(tt.item())
        h2d = sum(x.numel() * 8 for x in H)
        d2h = sum(x.numel() * 8 for x in O) + 8
        e2e = {"value": round(ms2 / k2 / world, 3), "unit": "ms/matrix", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h}
        del H, O

    F = flops_factor(n, b, a) + flops_selinv(n, b, a)
    out = None
    if rank == 0:
        # Kernel-level measurement pass (after the timed steps): per-launch events
        # around every library kernel of one step, then the FP64 DMMA peak probe.
        stream = torch.cuda.current_stream(dev)
        # Phase split of one step (events between the C calls on the stream).
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
        for dst, src in zip(W, P):
            dst.copy_(src, non_blocking=True)
        D, Lo, Ar, Ti, R = W
        ev[0].record()
        bta.factor(D, Lo, Ar, Ti)
        ev[1].record()
        bta.logdet(D, Ti, out=ld_out)
        ev[2].record()
        bta.solve(D, Lo, Ar, Ti, R)
        ev[3].record()
        bta.selinv(D, Lo, Ar, Ti)
        ev[4].record()
        torch.cuda.synchronize(dev)
        phases = {nm: round(ev[i].elapsed_time(ev[i + 1]), 3)
                  for i, nm in enumerate(["factor", "logdet", "solve", "selinv"])}
        lib.bta_timing_enable(1)
        step()
        torch.cuda.synchronize(dev)
        stats = {}
        for kid, name in enumerate(["gemm_f64", "potrf_tile", "trsm_panel", "tile_inv", "zero_upper",
                                    "mirror", "logdet", "trsv", "gemv", "arrow"]):
            tms, fl, cnt = ctypes.c_double(), ctypes.c_double(), ctypes.c_int64()
            lib.bta_timing_read(kid, ctypes.byref(tms), ctypes.byref(fl), ctypes.byref(cnt))
            stats[name] = (tms.value, fl.value, cnt.value)
        lib.bta_timing_enable(0)
        probe_out = torch.zeros(1, dtype=torch.float64, device=dev)
        pf = ctypes.c_double()
        lib.bta_probe_fp64_peak(ctypes.c_void_p(probe_out.data_ptr()), 200, ctypes.byref(pf),
                                ctypes.c_void_p(stream.cuda_stream))
        torch.cuda.synchronize(dev)
        e0.record()
        lib.bta_probe_fp64_peak(ctypes.c_void_p(probe_out.data_ptr()), 20000, ctypes.byref(pf),
                                ctypes.c_void_p(stream.cuda_stream))
        e1.record()
        torch.cuda.synchronize(dev)
        peak_tf = pf.value / (e0.elapsed_time(e1) * 1e-3) / 1e12

        g_ms, g_fl, g_cnt = stats["gemm_f64"]
        total_kernel_ms = sum(v[0] for v in stats.values())
        launches_per_step = sum(v[2] for v in stats.values())
        achieved = g_fl / (g_ms * 1e-3) / 1e12 if g_ms > 0 else None
        tflops = F / (ms_per_step * 1e-3 / 1.0) / 1e12 * 1.0
        out = {
            "metric": METRIC, "value": round(value, 3), "unit": "ms/matrix", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 3),
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(w),
            "tflops_per_gpu": round(F / (ms_per_step * 1e-3) / 1e12, 4),
            "fp64_peak_tflops_measured": round(peak_tf, 4),
            "frac_of_fp64_peak": round(tflops / peak_tf, 4),
            "roofline": {
                "bound": "alu", "achieved": round(achieved, 4) if achieved else None,
                "peak": round(peak_tf, 4), "unit": "TFLOP/s",
                "frac": round(achieved / peak_tf, 4) if achieved else None, "traffic": None,
                "kernel": "gemm_f64_kernel (DMMA m8n8k4)",
                "peak_source": "measured live: bta_probe_fp64_peak DMMA loop on all SMs",
                "kernel_share_of_step": round(g_ms / total_kernel_ms, 4) if total_kernel_ms else None,
                "avg_launch_ms": round(g_ms / max(g_cnt, 1), 5),
            },
            "kernel_ms_per_step": {k: round(v[0], 3) for k, v in stats.items()},
            "phase_ms": phases,
            "gpu_launches": int(launches_per_step * args.steps),
            "e2e": e2e,
        }
        if clocks:
            out["clocks"] = clocks
        if world == 1 and not args.no_cpu_baseline:
            per_full, desc, cores = cpu_oracle_sample(w, arrays, target_s=args.cpu_target_s)
            out["cpu_baseline"] = {"value": round(per_full, 3), "unit": "ms/matrix", "cores": cores,
                                   "kind": "oracle", "sample": desc}
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.barrier()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="n365_b1024_a8")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-clocks", action="store_true", help="skip nvidia-smi clock sampling (profiler runs)")
    ap.add_argument("--cpu-target-s", type=float, default=10.0)
    ap.add_argument("--ref-target-s", type=float, default=5.0)
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    w = WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, w, rank, world)
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    rc = run_ours(args, w, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return rc


if __name__ == "__main__":
    sys.exit(main())
