#!/usr/bin/env python3
"""Benchmark of the BTA hot path on GB300: factor + log-det + solve + selected inversion.

One step = one pass of the whole path over one synthetic BTA matrix resident in
HBM: reset the working blocks from a pristine device copy, then factor, log-det,
solve (4 right-hand sides) and selected inversion in one bta_factor_selinv_all
call (the same results as bta_factor, bta_logdet, bta_solve, bta_selinv in a
row). The metric is ms per matrix (lower is better); TFLOP/s of the algorithmic
FP64 flop count is reported beside it. `e2e` times bta_factor_selinv_host from
pinned host buffers (inputs in, X, x and log det out, inside the timed region).
Multi-GPU (torchrun): every rank factors and inverts its own matrix (independent
problems, weak scaling, no collective on the data path).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]

Default workload: n=256, b=2048, a=16, dominance shift 1.001 (inputs 17.2 GB, far
above the 129 MB L2, so no L2 flush is needed between steps). Beside the FP64
line: the tensor-core precision modes on the same matrix (speedup and per-block
error against the FP64 result), and the batched form (64 uneven matrices, one
call replayed from a CUDA graph, against 64 sequential plain FP64 calls, with a
sample checked against the oracle). Wall-clock progress goes to stderr.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
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
    # small cases with the same block shapes, for profiler captures (under 1 GB on the device)
    "n48_b1024_a8": dict(n=48, b=1024, a=8, shift=gen.SHIFT_1_01, shift_name="1.01 x row sum"),
    "n8_b2048_a16": dict(n=8, b=2048, a=16, shift=gen.SHIFT_1_001, shift_name="1.001 x row sum"),
    # the block shape of the paper's weak-scaling dataset (4) at one process (Section 5.2, 5.4)
    "n90_b2865_a4": dict(n=90, b=2865, a=4, shift=gen.SHIFT_1_01, shift_name="1.01 x row sum"),
}
# The paper's one single-GPU factorization time: block-sequential POBTAF on dataset (4) at one
# process, n=90, b=2865, a=4, FP64, on one GH200 (Section 5.4). Context, not a target.
PAPER_POBTAF_GH200_MS = 2510.0
NRHS = 4
BATCH_WORKLOAD = "batch64_n20-200_b128-512_a2-8"
# a 16-matrix sample of the same kind, about 1 GB on the device: the persistent
# kernel alone, for profiler captures
BATCH_SMALL = "batch16_n20-40_b128-512_a2-8"


# Algorithmic FP64 flops (LAPACK counts of the method itself).
def flops_factor(n, b, a):
    return n * b**3 / 3 + (n - 1) * 2 * b**3 + n * a * b**2 + (n - 1) * 2 * a * b**2 + n * a**2 * b + a**3 / 3


def flops_selinv(n, b, a):
    return 2 * a**3 / 3 + n * 2 * b**3 / 3 + (n - 1) * 4 * b**3 + n * (2 * a * b**2 + 2 * a**2 * b) + (n - 1) * 4 * a * b**2


def flops_solve(n, b, a, r):
    return 2 * r * (n * b * b + 2 * (n - 1) * b * b + 2 * n * a * b + a * a)


KERNELS = ["gemm_f64", "potrf_panel", "trsm_panel", "tile_inv", "zero_upper", "mirror", "logdet", "trsv",
           "gemv", "arrow", "probe", "gemm_tc", "tc_split", "tc_final", "factor_step", "persistent"]
# tensor-core products per FP64 product in each precision mode
TC_PAIRS = {"ozaki": 28, "bf16x3": 3}
PREC_DTYPE = {"fp64": "f64", "ozaki": "bf16 slices x7 (FP64-emulated, Ozaki splitting)",
              "bf16x3": "bf16x3 (FP32 accumulation) + f64"}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return {"bf16_burst": float(d["bf16_tflops"]), "bf16_sustained": float(d["bf16_tflops_sustained"]),
                "hbm_gbs": float(d["hbm_gbs"]), "source": "MEASURED_PEAKS.json (measured)"}
    except (OSError, KeyError, ValueError):
        return {"bf16_burst": 1900.0, "bf16_sustained": 1700.0, "hbm_gbs": 6800.0,
                "source": "profiling-recipe fallback"}


# DRAM traffic per launch of the dominant kernels (dram__bytes_read.sum +
# dram__bytes_write.sum, summed over the kernel's launches of one step in one ncu
# capture and divided by their number), keyed by kernel name. Each entry names
# the source file of the kernel and a digest of the kernel's own source text
# (its __global__ definition, brace-matched) at capture time: once that text
# changes, the figure no longer describes the kernel and the bench line reports
# traffic as null.
TRAFFIC = {
    "gemm_f64": {"workload": "n256_b2048_a16", "source": "kernels_f64.cu", "symbol": "gemm_f64_kernel",
                 "digest": "780b5ba4e92474a9", "bytes_per_launch": 180.3e6,
                 "capture": "profiles/launches_n256_b2048_a16_fp64.md: 526 launches of one step, "
                            "132.5 MB read + 47.8 MB written per launch on average"},
}


def kernel_source(src, symbol):
    """Text of the __global__ function `symbol` in `src` (brace-matched)."""
    i = src.index(symbol + "(")
    i = src.rfind("__global__", 0, i)
    j = src.index("{", i)
    depth = 0
    for k in range(j, len(src)):
        if src[k] == "{":
            depth += 1
        elif src[k] == "}":
            depth -= 1
            if depth == 0:
                return src[i:k + 1]
    raise ValueError(symbol)


def kernel_digest(rel, symbol):
    with open(os.path.join(ROOT, "paper_2503_17528_gb300", "csrc", rel)) as f:
        return hashlib.sha256(kernel_source(f.read(), symbol).encode()).hexdigest()[:16]


def traffic_of(kernel, workload):
    e = TRAFFIC.get(kernel)
    if not e or e.get("workload") != workload:
        return None
    try:
        if kernel_digest(e["source"], e["symbol"]) != e["digest"]:
            return None
    except (OSError, ValueError):
        return None
    return {"bytes_per_launch": e["bytes_per_launch"], "capture": e["capture"]}


def solve_bytes(n, b, a, nrhs):
    """Algorithmic bytes of one solve: each sweep reads the factor once (lower
    triangles of the diagonal blocks and of the tip, full off-diagonal and arrow
    blocks) and reads and writes the right-hand sides once."""
    factor = n * b * (b + 1) // 2 + (n - 1) * b * b + n * a * b + a * (a + 1) // 2
    return 8 * (2 * factor + 4 * (n * b + a) * nrhs)


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
def cpu_oracle_sample(w, arrays, target_s=8.0, max_blocks=None, ns_fixed=None):
    """Time the oracle (factor, logdet, solve, selinv) on a leading principal block
    sub-matrix of the workload (the first ns block rows plus the arrowhead, itself
    an SPD BTA matrix), doubling ns until one run takes >= target_s (or using
    ns_fixed). Every block step of the method costs the same, so the full matrix
    costs n/ns times the sample, up to the tip. Returns (ms per full matrix,
    sample description, cores, ns, sample seconds)."""
    import oracle
    d, l, ar, t, r = arrays
    n, b, a = w["n"], w["b"], w["a"]
    ns = ns_fixed or min(n, 2)
    while True:
        rs = np.concatenate([r[: ns * b], r[n * b:]])
        t0 = time.perf_counter()
        F = oracle.pobtaf(d[:ns], l[: ns - 1], ar[:ns], t)
        oracle.logdet(F)
        oracle.solve(F, rs)
        oracle.pobtasi(F)
        dt = time.perf_counter() - t0
        if ns_fixed or dt >= target_s or ns >= n or (max_blocks and ns >= max_blocks):
            break
        ns = min(n, ns * 2)
    per_full = dt * 1e3 * n / ns
    desc = (f"oracle (NumPy/SciPy FP64) on the leading {ns} of {n} block rows plus the arrowhead "
            f"({dt:.1f} s), scaled by n/{ns} to one full matrix (extrapolated, not run on the whole matrix)")
    return per_full, desc, os.cpu_count(), ns, dt


def rank_seed(rank: int) -> int:
    """Each rank factors its own seeded matrix (independent problems)."""
    return rank


def max_over_ranks(ms: float, dist, device=None) -> float:
    """The job's time is the slowest rank's (all_reduce MAX; no-op for one rank)."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def shard_batch(flops, world: int):
    """Largest-first greedy assignment of independent matrices to ranks (by
    algorithmic flops); returns one index list per rank. No data crosses ranks."""
    order = sorted(range(len(flops)), key=lambda k: -flops[k])
    load = [0.0] * world
    parts = [[] for _ in range(world)]
    for k in order:
        r = min(range(world), key=lambda j: load[j])
        parts[r].append(k)
        load[r] += flops[k]
    return parts


def make_workload(w, seed):
    d, l, ar, t = gen.make_bta(w["n"], w["b"], w["a"], seed=seed, shift=w["shift"])
    r = gen.make_rhs(w["n"], w["b"], w["a"], NRHS, seed=seed + 1000)
    return d, l, ar, t, r


# ---------------------------------------------------------------------------
def run_reference(args, w, rank, world):
    """The reference arm: the oracle as it stands, on the host cores, on a bounded
    sample of the workload per step (see cpu_oracle_sample). `ms_per_step` is the
    time one step really took; `value` is that sample scaled to one full matrix."""
    if rank != 0:
        return 0
    arrays = make_workload(w, seed=0)
    per, secs = [], []
    desc = cores = ns = None
    for i in range(args.warmup + args.steps):
        per_full, desc, cores, ns, dt = cpu_oracle_sample(w, arrays, target_s=args.ref_target_s, ns_fixed=ns)
        if i >= args.warmup:
            per.append(per_full)
            secs.append(dt)
    v = statistics.median(per)
    line = {
        "impl": "reference", "metric": METRIC, "value": round(v, 3), "unit": "ms/matrix",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * statistics.median(secs), 3),
        "value_is_extrapolated": f"each step runs the oracle on {ns} of {w['n']} block rows; value = n/{ns} x that",
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(w),
        "cpu_baseline": {"value": round(v, 3), "unit": "ms/matrix", "cores": cores, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": round(v, 3), "unit": "ms/matrix", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def make_batch(count=64, seed=2026):
    """64 seeded matrices: n ~ U[20, 200], b in {128, 256, 512}, a in {2, 4, 8},
    generator seed base + k (the batched workload)."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        n = int(rng.integers(20, 201))
        b = int(rng.choice([128, 256, 512]))
        a = int(rng.choice([2, 4, 8]))
        out.append(gen.make_bta(n, b, a, seed=seed + k, shift=gen.SHIFT_1_01))
    return out


def _log(msg):
    print(f"[bench {time.strftime('%H:%M:%S')}] {msg}", file=sys.stderr, flush=True)


def batch_measure(steps, warmup, dev, rank=0, world=1, oracle_sample=0, quick_tune=False):
    """Batched form on this rank's shard of the 64-matrix batch: sequential plain
    FP64 calls against one tuned batched call replayed from a CUDA graph (the
    reset copy of the inputs is in both). Returns the measurements as a dict."""
    import torch
    import paper_2503_17528_gb300 as bta
    from paper_2503_17528_gb300 import tune
    from paper_2503_17528_gb300.batched import Batch, PersistentBatch
    raw_all = make_batch()
    fl_all = [flops_factor(m[0].shape[0], m[0].shape[1], m[3].shape[0]) +
              flops_selinv(m[0].shape[0], m[0].shape[1], m[3].shape[0]) for m in raw_all]
    mine = sorted(shard_batch(fl_all, world)[rank])
    raw = [raw_all[k] for k in mine]
    flops = sum(fl_all[k] for k in mine)
    P = [tuple(torch.from_numpy(x).to(dev) for x in m) for m in raw]
    W = [tuple(x.clone() for x in m) for m in P]

    def reset():
        for w, p in zip(W, P):
            for x, y in zip(w, p):
                if x.numel():
                    x.copy_(y, non_blocking=True)

    bta.set_precision("fp64")
    lds = torch.empty(len(W), dtype=torch.float64, device=dev)

    def sequential():
        reset()
        for k, (d, l, ar, t) in enumerate(W):
            bta.factor(d, l, ar, t)
            bta.logdet(d, t, out=lds[k])
            bta.selinv(d, l, ar, t)

    def timed(fn, k):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(k):
            fn()
        e1.record()
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / k

    seq_ms = timed(sequential, steps)
    seq_out = [tuple(x.clone() for x in w) for w in W]
    seq_ld = lds.clone()
    cfg = tune.lookup(W)
    tuned_now = cfg is None
    if cfg is None:
        if quick_tune:
            cfg = tune.tune(W, P, policies=["fp64", "ozaki_b256"], streams=(8, 16), reps=1, save=False)
        else:
            cfg = tune.tune(W, P)
    batch = Batch(W, policy=cfg["policy"], nstreams=cfg["nstreams"])
    reset()
    batch.run()
    torch.cuda.synchronize(dev)
    side = torch.cuda.Stream(dev)
    side.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(side):
        graph = batch.capture()
    torch.cuda.current_stream(dev).wait_stream(side)

    def replay():
        reset()
        graph.replay()

    graph_ms = timed(replay, steps)
    worst = 0.0
    for w, r in zip(W, seq_out):
        for x, y in zip(w, r):
            if y.numel():
                worst = max(worst, blockerr(x, y))
    out = {"ms_per_batch": round(graph_ms, 3), "matrices": len(raw), "total_flops": flops,
           "sequential_plain_fp64_ms": round(seq_ms, 3), "speedup_vs_sequential": round(seq_ms / graph_ms, 3),
           "tflops": round(flops / (graph_ms * 1e-3) / 1e12, 4),
           "tuned": {k: cfg[k] for k in ("nstreams", "policy", "ms")}, "tuned_in_this_run": tuned_now,
           "dtype": "f64" if cfg["policy"] == "fp64" else
           "f64 + bf16-slice FP64 emulation (b >= 256)" if cfg["policy"] == "ozaki_b256"
           else "bf16 slices (FP64-emulated)",
           "max_block_rel_err_vs_sequential_fp64": float(f"{worst:.3e}")}
    if oracle_sample:
        out["oracle_check"] = _batch_oracle_check(raw, W, batch.logdets, oracle_sample)
    # The persistent form: the whole batch in one cooperative launch (FP64),
    # parameters from the autotuner (cached, else a short search now).
    pcfg = tune.lookup_persistent(W)
    ptuned_now = pcfg is None
    if pcfg is None:
        pcfg = tune.tune_persistent(W, P, candidates=PERSISTENT_QUICK if quick_tune else None, reps=1,
                                    save=not quick_tune)
    pb = PersistentBatch(W, **pcfg["params"])
    reset()
    pb.run()
    torch.cuda.synchronize(dev)
    with torch.cuda.stream(side):
        pgraph = pb.capture()
    torch.cuda.current_stream(dev).wait_stream(side)

    def preplay():
        reset()
        pgraph.replay()

    pers_ms = timed(preplay, steps)
    timed_out, info = pb.status()
    pworst = 0.0
    for w, r in zip(W, seq_out):
        for x, y in zip(w, r):
            if y.numel():
                pworst = max(pworst, blockerr(x, y))
    pers = {"ms_per_batch": round(pers_ms, 3), "speedup_vs_sequential": round(seq_ms / pers_ms, 3),
            "speedup_vs_multistream_graph": round(graph_ms / pers_ms, 3),
            "tflops": round(flops / (pers_ms * 1e-3) / 1e12, 4), "dtype": "f64",
            "launches_per_batch": 1, "plan": pb.describe(), "tuned": pcfg["params"],
            "tuned_in_this_run": ptuned_now, "tuning_table": pcfg.get("table"),
            "timed_out": timed_out, "failed_matrices": sum(1 for v in info if v),
            "max_block_rel_err_vs_sequential_fp64": float(f"{pworst:.3e}"),
            "logdet_max_rel_err_vs_sequential_fp64": float(f"{float(((pb.logdets - seq_ld).abs() / seq_ld.abs()).max()):.3e}")}
    if oracle_sample:
        pers["oracle_check"] = _batch_oracle_check(raw, W, pb.logdets, oracle_sample)
    out["persistent"] = pers
    del pgraph
    pb.close()
    del seq_ld
    return out


PERSISTENT_QUICK = ((4, 8, 1), (4, 4, 1), (3, 8, 1), (4, 8, 2))


def _batch_oracle_check(raw, W, logdets, sample):
    """The first few matrices of a batched result against the oracle."""
    import torch
    import oracle
    ow = 0.0
    ld_err = 0.0
    lds = logdets.cpu().numpy()
    for k in range(min(sample, len(raw))):
        F = oracle.pobtaf(*raw[k])
        X = oracle.pobtasi(F)
        for x, y in zip(W[k], X):
            if y.size:
                ow = max(ow, blockerr(x.cpu(), torch.from_numpy(y)))
        ldo = oracle.logdet(F)
        ld_err = max(ld_err, abs(float(lds[k]) - ldo) / abs(ldo))
    return {"matrices": min(sample, len(raw)), "max_block_rel_err_vs_oracle": float(f"{ow:.3e}"),
            "max_logdet_rel_err_vs_oracle": float(f"{ld_err:.3e}")}


def run_batch_small(args):
    """The persistent batched kernel on the 16-matrix sample (default plan
    parameters): W warm-up and K timed launches, one JSON line."""
    import torch
    from paper_2503_17528_gb300.batched import PersistentBatch
    rng = np.random.default_rng(77)
    shapes = [(int(rng.integers(20, 41)), int(rng.choice([128, 256, 512])), int(rng.choice([2, 4, 8])))
              for _ in range(16)]
    raw = [gen.make_bta(n, b, a, seed=900 + k, shift=gen.SHIFT_1_01) for k, (n, b, a) in enumerate(shapes)]
    dev = torch.device("cuda", 0)
    P = [tuple(torch.from_numpy(x).to(dev) for x in m) for m in raw]
    W = [tuple(x.clone() for x in m) for m in P]
    pb = PersistentBatch(W)

    def step():
        for w, p in zip(W, P):
            for x, y in zip(w, p):
                if x.numel():
                    x.copy_(y, non_blocking=True)
        pb.run()

    ms = _timed_steps(step, args.steps, args.warmup, dev)
    to, info = pb.status()
    fl = sum(flops_factor(n, b, a) + flops_selinv(n, b, a) for n, b, a in shapes)
    print(json.dumps({"metric": "BTA persistent batched factor+logdet+selinv ms/batch", "value": round(ms, 3),
                      "unit": "ms/batch", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
                      "higher_is_better": False, "dtype": "f64", "data": "synthetic",
                      "config": {"workload": BATCH_SMALL, "shapes": shapes, "plan": pb.describe(),
                                 "steps_include": "device reset copy + one persistent launch"},
                      "tflops": round(fl / (ms * 1e-3) / 1e12, 4), "timed_out": to,
                      "failed_matrices": sum(1 for v in info if v)}), flush=True)
    pb.close()
    return 0


def run_batch(args, rank=0, world=1, local_rank=0):
    """The batched workload as its own bench line: each rank runs its shard of the
    64 matrices (largest-first bin-pack on algorithmic flops, no data-path
    collective); the job time is the slowest rank's."""
    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    res = batch_measure(args.steps, args.warmup, dev, rank, world)
    ms = max_over_ranks(res["ms_per_batch"], dist, dev)
    if rank == 0:
        line = {"metric": "BTA batched factor+logdet+selinv ms/batch (64 uneven matrices)",
                "value": round(ms, 3), "unit": "ms/batch", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": False,
                "scaling": "strong", "vs_baseline": None, "dtype": res["dtype"], "data": "synthetic",
                "config": {"workload": BATCH_WORKLOAD, "matrices": 64,
                           "steps_include": "device reset copy + every matrix of this rank's shard"},
                "rank0": res}
        print(json.dumps(line), flush=True)
    return 0


def workload_config(w):
    n, b, a = w["n"], w["b"], w["a"]
    return {"workload": f"n{n}_b{b}_a{a}", "n": n, "b": b, "a": a, "nrhs": NRHS,
            "dominance_shift": w["shift_name"], "generator": "seeded N(0,1)/sqrt(b) blocks, diagonally dominant",
            "l2": f"inputs {pattern_bytes(n, b, a) / 1e9:.2f} GB per matrix > 129 MB L2; no flush",
            "steps_include": "device reset copy + factor + logdet + solve + selinv (one bta_factor_selinv_all call)"}


def read_kernel_stats(lib):
    stats = {}
    for kid, name in enumerate(KERNELS):
        tms, fl, cnt = ctypes.c_double(), ctypes.c_double(), ctypes.c_int64()
        lib.bta_timing_read(kid, ctypes.byref(tms), ctypes.byref(fl), ctypes.byref(cnt))
        if cnt.value:
            stats[name] = (tms.value, fl.value, cnt.value)
    return stats


def roofline_of(stats, prec, fp64_peak, peaks, workload=None):
    """Roofline of the dominant kernel of one step (largest summed device time).
    `achieved` is its algorithmic flops summed over the step's launches divided by
    their summed device time (CUDA events around each launch on its stream)."""
    top = max(stats.items(), key=lambda kv: kv[1][0])
    name, (ms, fl, cnt) = top
    total = sum(v[0] for v in stats.values())
    tr = traffic_of(name, workload)
    base = {"kernel": name, "kernel_share_of_step": round(ms / total, 4) if total else None,
            "avg_launch_ms": round(ms / max(cnt, 1), 5), "launches_per_step": int(cnt),
            "traffic": tr["bytes_per_launch"] if tr else None}
    if tr:
        base["traffic_capture"] = tr["capture"]
    if name == "gemm_tc":
        pairs = TC_PAIRS.get(prec, 1)
        ach = pairs * fl / (ms * 1e-3) / 1e12
        base.update({"bound": "tensor", "achieved": round(ach, 3), "peak": peaks["bf16_sustained"],
                     "unit": "TFLOP/s", "frac": round(ach / peaks["bf16_sustained"], 4),
                     "peak_source": peaks["source"] + ", bf16 sustained",
                     "fp64_equivalent_tflops": round(fl / (ms * 1e-3) / 1e12, 3),
                     "achieved_counts": f"{pairs} BF16 slice products per FP64 product"})
    else:
        ach = fl / (ms * 1e-3) / 1e12 if ms > 0 and fl > 0 else None
        base.update({"bound": "alu", "achieved": round(ach, 4) if ach else None, "peak": round(fp64_peak, 4),
                     "unit": "TFLOP/s", "frac": round(ach / fp64_peak, 4) if ach else None,
                     "peak_source": "measured live: bta_probe_fp64_peak DMMA loop on all SMs"})
    return base


def blockerr(x, y):
    """Largest per-block relative Frobenius error of x against y (torch tensors)."""
    import torch
    if x.numel() == 0:
        return 0.0
    if x.dim() == 3:
        num = torch.linalg.norm((x - y).flatten(1), dim=1)
        den = torch.linalg.norm(y.flatten(1), dim=1).clamp_min(1e-300)
        return float((num / den).max())
    return float(torch.linalg.norm(x - y) / torch.linalg.norm(y).clamp_min(1e-300))


def _timed_steps(fn, steps, warmup, dev):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        fn()
    e1.record()
    torch.cuda.synchronize(dev)
    return e0.elapsed_time(e1) / steps


def run_modes(args, bta, lib, step, step_seq, W, ld_out, base_ms, dev, ref_inputs, base_phases,
              peak_tf, workload):
    """Time the other precision modes on the same matrix; state each one's error
    against the main mode's result (per block, relative Frobenius) and its speedup."""
    import torch
    ref = [x.clone() for x in W]
    ref_ld = float(ld_out.item())
    res = {}
    ms_steps, ms_warm = max(1, min(args.steps, args.mode_steps)), max(1, min(args.warmup, args.mode_warmup))
    for mode in [m for m in (args.modes or "").split(",") if m and m != args.precision]:
        _log(f"mode {mode}")
        bta.set_precision(mode)
        ms = _timed_steps(step, ms_steps, ms_warm, dev)
        errs = {nm: blockerr(W[i], ref[i]) for i, nm in enumerate(["X_diag", "X_lower", "X_arrow", "X_tip"])}
        errs["solve"] = blockerr(W[4], ref[4])
        errs["logdet"] = abs(float(ld_out.item()) - ref_ld) / abs(ref_ld)
        # phase split of one step in this mode
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        for dst, src in zip(W, ref_inputs):
            dst.copy_(src)
        D, Lo, Ar, Ti, R = W
        evs[0].record()
        bta.factor(D, Lo, Ar, Ti)
        evs[1].record()
        bta.solve(D, Lo, Ar, Ti, R)
        evs[2].record()
        bta.selinv(D, Lo, Ar, Ti)
        evs[3].record()
        torch.cuda.synchronize(dev)
        phases = {nm: round(evs[i].elapsed_time(evs[i + 1]), 3) for i, nm in enumerate(["factor", "solve", "selinv"])}
        lib.bta_timing_enable(1)
        step_seq()
        torch.cuda.synchronize(dev)
        stats = read_kernel_stats(lib)
        lib.bta_timing_enable(0)
        peaks = measured_peaks()
        res[mode] = {"phase_ms": phases, "ms_per_matrix": round(ms, 3), "steps": ms_steps, "warmup": ms_warm,
                     "speedup_vs_" + args.precision: round(base_ms / ms, 3),
                     "max_block_rel_err_vs_" + args.precision: {k: float(f"{v:.3e}") for k, v in errs.items()},
                     "dtype": PREC_DTYPE[mode],
                     "roofline": roofline_of(stats, mode, peak_tf, peaks, workload),
                     "kernel_ms_per_step": {k: round(v[0], 3) for k, v in stats.items()}}
    # Partitioned form (the paper's P-way scheme on one device): factor + logdet + selinv.
    for spec in [x for x in (args.partitioned or "").split(",") if x]:
        prec, P = spec.split(":")
        P = int(P)
        _log(f"partitioned {prec} P={P}")
        bta.set_precision(prec)

        def pstep():
            for dst, src in zip(W, ref_inputs):
                dst.copy_(src, non_blocking=True)
            bta.factor_selinv_partitioned(W[0], W[1], W[2], W[3], parts=P, lb=1.8, logdet_out=ld_out)

        ms = _timed_steps(pstep, ms_steps, ms_warm, dev)
        errs = {nm: blockerr(W[i], ref[i]) for i, nm in enumerate(["X_diag", "X_lower", "X_arrow", "X_tip"])}
        errs["logdet"] = abs(float(ld_out.item()) - ref_ld) / abs(ref_ld)
        base_fls = base_phases["factor"] + base_phases["logdet"] + base_phases["selinv"]
        res[f"partitioned_{prec}_P{P}"] = {
            "ms_per_matrix_factor_logdet_selinv": round(ms, 3),
            "speedup_vs_" + args.precision + "_factor_logdet_selinv": round(base_fls / ms, 3),
            "max_block_rel_err_vs_" + args.precision: {k: float(f"{v:.3e}") for k, v in errs.items()},
            "parts": P, "load_balance_top": 1.8}
    return res


def run_context(dev, steps, peak_tf):
    """The dataset-4 block shape (n=90, b=2865, a=4: a ragged 17-row last tile)
    beside the paper's 2.51 s POBTAF on GH200: factor alone (POBTAF) and the
    whole path (factor + log det + solve + selinv), in FP64 and in the Ozaki
    mode, each after one warm-up, with the Ozaki result's largest per-block
    error against the FP64 one."""
    import torch
    import paper_2503_17528_gb300 as bta
    w = WORKLOADS["n90_b2865_a4"]
    n, b, a = w["n"], w["b"], w["a"]
    arrays = make_workload(w, seed=0)
    P = [torch.from_numpy(x).to(dev) for x in arrays]
    del arrays
    W = [torch.empty_like(x) for x in P]
    ld = torch.empty((), dtype=torch.float64, device=dev)

    def reset():
        for dst, src in zip(W, P):
            dst.copy_(src, non_blocking=True)

    def factor_only():
        reset()
        bta.factor(*W[:4])

    def whole():
        reset()
        bta.factor_selinv_all(*W[:4], rhs=W[4], logdet_out=ld)

    def copy_ms():
        return _timed_steps(reset, steps, 1, dev)

    out = {"workload": "n90_b2865_a4", "n": n, "b": b, "a": a,
           "paper_pobtaf_gh200_ms": PAPER_POBTAF_GH200_MS,
           "note": "paper: block-sequential POBTAF, dataset (4) at P=1, FP64, 1 GH200 (67 TFLOP/s FP64 "
                   "tensor); here synthetic blocks of the same shape; times exclude the reset copy"}
    reset_ms = copy_ms()
    res = {}
    for prec in ("fp64", "ozaki"):
        bta.set_precision(prec)
        f_ms = _timed_steps(factor_only, steps, 1, dev) - reset_ms
        a_ms = _timed_steps(whole, steps, 1, dev) - reset_ms
        res[prec] = {"factor_ms": round(f_ms, 1), "factor_tflops": round(flops_factor(n, b, a) / (f_ms * 1e-3) / 1e12, 4),
                     "factor_selinv_logdet_solve_ms": round(a_ms, 1),
                     "factor_vs_paper_gh200": round(PAPER_POBTAF_GH200_MS / f_ms, 3)}
        if prec == "fp64":
            ref = [x.clone() for x in W[:4]]
        else:
            res[prec]["max_block_rel_err_vs_fp64"] = float(f"{max(blockerr(x, y) for x, y in zip(W[:4], ref) if y.numel()):.3e}")
    bta.set_precision("fp64")
    res["fp64"]["factor_frac_of_fp64_peak"] = round(res["fp64"]["factor_tflops"] / peak_tf, 4)
    out.update(res)
    del P, W
    torch.cuda.empty_cache()
    return out


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
    bta.set_precision(args.precision)
    wname = f"n{n}_b{b}_a{a}"

    _log(f"generating {wname} (seed {rank_seed(rank)})")
    arrays = make_workload(w, seed=rank_seed(rank))
    d, l, ar, t, r = arrays
    P = [torch.from_numpy(x).to(dev) for x in (d, l, ar, t, r)]
    W = [torch.empty_like(x) for x in P]
    ld_out = torch.empty((), dtype=torch.float64, device=dev)

    def step():
        # One call: factor + logdet + solve + selinv (the solve overlapped with
        # the selected inversion's prologue).
        for dst, src in zip(W, P):
            dst.copy_(src, non_blocking=True)
        D, Lo, Ar, Ti, R = W
        bta.factor_selinv_all(D, Lo, Ar, Ti, rhs=R, logdet_out=ld_out)

    def step_seq():
        # The same work as four calls in a row (no overlap): per-kernel times
        # free of interference, comparable with a serialized ncu launch list.
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

    _log(f"warmup x{args.warmup}")
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    if bta.get_info(dev) != 0:
        raise RuntimeError("non-positive pivot in the benchmark matrix")

    _log(f"timed x{args.steps}")
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
    ms = max_over_ranks(e0.elapsed_time(e1), dist, dev)
    ms_per_step = ms / args.steps
    value = ms_per_step / world  # whole job: `world` matrices per step

    # End to end through the public API with host buffers (pinned): one call
    # (bta_factor_selinv_host) copies the pattern and right-hand sides in, runs
    # factor + logdet + solve + selinv, and copies X, x and log det back, the
    # copies overlapped with the block sweeps. Timed over the same K steps.
    e2e = None
    if not args.no_e2e:
        _log(f"e2e x{args.steps}")
        H = [torch.from_numpy(x).pin_memory() for x in (d, l, ar, t, r)]
        O = tuple([torch.empty(x.shape, dtype=torch.float64).pin_memory() for x in (d, l, ar, t, r)]
                  + [torch.empty((), dtype=torch.float64).pin_memory()])

        def e2e_step():
            bta.factor_selinv_host(*H[:4], rhs=H[4], out=O, device=dev)

        e2e_step()
        torch.cuda.synchronize(dev)
        barrier()
        e0.record()
        for _ in range(args.steps):
            e2e_step()
        e1.record()
        torch.cuda.synchronize(dev)
        barrier()
        ms2 = max_over_ranks(e0.elapsed_time(e1), dist, dev)
        h2d = sum(x.numel() * 8 for x in H)
        d2h = sum(x.numel() * 8 for x in O)
        # The host results against the device path's (W holds X after the timed steps).
        idx = sorted({0, n // 2, n - 1})
        sel = torch.tensor(idx)
        e2e_err = blockerr(O[0][sel], W[0][sel.to(dev)].cpu())
        if n > 1:
            sl = sel.clamp(max=n - 2)
            e2e_err = max(e2e_err, blockerr(O[1][sl], W[1][sl.to(dev)].cpu()))
        e2e = {"value": round(ms2 / args.steps / world, 3), "unit": "ms/matrix", "steps": args.steps,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "max_block_rel_err_vs_device_path": float(f"{e2e_err:.3e}")}
        del H, O

    F = flops_factor(n, b, a) + flops_selinv(n, b, a)
    modes = {}
    batched = None
    out = None
    if rank == 0:
        # Kernel-level measurement pass (after the timed steps): per-launch events
        # around every library kernel of one step, then the FP64 DMMA peak probe.
        _log("phase split and per-kernel pass")
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
        step_seq()
        torch.cuda.synchronize(dev)
        stats = read_kernel_stats(lib)
        lib.bta_timing_enable(0)
        peaks = measured_peaks()
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
        if args.modes or args.partitioned:
            modes = run_modes(args, bta, lib, step, step_seq, W, ld_out, ms_per_step, dev, P, phases,
                              peak_tf, wname)
            bta.set_precision(args.precision)

        total_kernel_ms = sum(v[0] for v in stats.values())
        launches_per_step = sum(v[2] for v in stats.values())
        tflops = F / (ms_per_step * 1e-3) / 1e12
        out = {
            "metric": METRIC, "value": round(value, 3), "unit": "ms/matrix", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 3),
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": PREC_DTYPE[args.precision], "precision_mode": args.precision,
            "data": "synthetic", "config": workload_config(w),
            "tflops_per_gpu": round(tflops, 4),
            "fp64_peak_tflops_measured": round(peak_tf, 4),
            "frac_of_fp64_peak": round(tflops / peak_tf, 4),
            "roofline": roofline_of(stats, args.precision, peak_tf, peaks, wname),
            # the solve (a sequential chain of latency-bound triangular solves) against HBM
            "solve_roofline": {
                "bound": "latency", "unit": "GB/s", "peak": peaks["hbm_gbs"],
                "achieved": round(solve_bytes(n, b, a, NRHS) / (phases["solve"] * 1e-3) / 1e9, 2),
                "frac": round(solve_bytes(n, b, a, NRHS) / (phases["solve"] * 1e-3) / 1e9
                              / peaks["hbm_gbs"], 4),
                "traffic": None, "peak_source": peaks["source"]},
            "kernel_ms_per_step": {k: round(v[0], 3) for k, v in stats.items()},
            "kernel_launches_per_step": {k: int(v[2]) for k, v in stats.items()},
            "kernel_total_ms_per_step": round(total_kernel_ms, 3),
            "phase_ms": phases,
            "gpu_launches": int(launches_per_step * args.steps),
            "modes": modes or None,
            "e2e": e2e,
        }
        if clocks:
            out["clocks"] = clocks
    # The main workload's device buffers are no longer needed.
    del P, W
    torch.cuda.empty_cache()
    if rank == 0 and world == 1 and args.context:
        _log("context workload n90_b2865_a4")
        out["context"] = run_context(dev, 1, peak_tf)
    if rank == 0 and world == 1 and not args.no_batch:
        _log("batched form")
        batched = batch_measure(max(1, min(args.steps, args.mode_steps)), max(1, min(args.warmup, args.mode_warmup)),
                                dev, oracle_sample=args.batch_oracle_sample, quick_tune=True)
        out["batched"] = dict(batched, workload=BATCH_WORKLOAD)
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            _log("cpu baseline (oracle)")
            per_full, desc, cores, _, _ = cpu_oracle_sample(w, arrays, target_s=args.cpu_target_s)
            out["cpu_baseline"] = {"value": round(per_full, 3), "unit": "ms/matrix", "cores": cores,
                                   "kind": "oracle", "sample": desc}
        _log("done")
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
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + [BATCH_WORKLOAD, BATCH_SMALL], default="n256_b2048_a16")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-clocks", action="store_true", help="skip nvidia-smi clock sampling (profiler runs)")
    ap.add_argument("--precision", choices=["fp64", "ozaki", "bf16x3"], default="fp64")
    ap.add_argument("--modes", default="ozaki,bf16x3",
                    help="other precision modes timed on the same matrix ('' to skip)")
    ap.add_argument("--partitioned", default="",
                    help="partitioned runs 'precision:P,...' timed on the same matrix (e.g. ozaki:8)")
    ap.add_argument("--mode-steps", type=int, default=3, help="timed steps per extra precision mode")
    ap.add_argument("--mode-warmup", type=int, default=1, help="warm-up steps per extra precision mode")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-form sub-record")
    ap.add_argument("--no-context", dest="context", action="store_false",
                    help="skip the dataset-4-shaped context record (n=90, b=2865, a=4)")
    ap.add_argument("--batch-oracle-sample", type=int, default=4,
                    help="matrices of the batched result checked against the oracle")
    ap.add_argument("--cpu-target-s", type=float, default=10.0)
    ap.add_argument("--ref-target-s", type=float, default=5.0)
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.workload in (BATCH_WORKLOAD, BATCH_SMALL) and args.impl == "reference":
        return 0
    if args.workload == BATCH_SMALL:
        return run_batch_small(args)
    if args.impl == "reference":
        return run_reference(args, WORKLOADS[args.workload], rank, world)
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    if args.workload == BATCH_WORKLOAD:
        rc = run_batch(args, rank, world, local_rank)
    else:
        rc = run_ours(args, WORKLOADS[args.workload], rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return rc


if __name__ == "__main__":
    sys.exit(main())
