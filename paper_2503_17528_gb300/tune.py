"""Autotuner for the batched form: measures every (streams, engine policy)
candidate on the actual batch, as it is deployed (captured once in a CUDA
graph, timed over graph replays: eager runs of thousands of small launches
measure host enqueue time, not the GPU), and caches the fastest per device and
batch signature (count and the multiset of (b, a)) in tuning_cache.json beside
this file.
"""
from __future__ import annotations

import json
import os

import torch

from .batched import POLICIES, Batch

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning_cache.json")
STREAMS = (1, 4, 8, 16, 32)


def signature(mats) -> str:
    name = torch.cuda.get_device_name(mats[0][0].device)
    shapes = sorted((int(d.shape[1]), int(t.shape[0])) for d, _, _, t in mats)
    return f"{name}|{len(mats)}|{shapes}"


def _load():
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def lookup(mats):
    return _load().get(signature(mats))


def tune(mats, pristine, policies=None, streams=STREAMS, reps=2, save=True):
    """mats: working tensors (overwritten); pristine: matching copies to restore.
    Returns {"nstreams", "policy", "ms", "table"} and stores it in the cache."""
    policies = list(policies or POLICIES)
    table = []

    def restore():
        for w, p in zip(mats, pristine):
            for x, y in zip(w, p):
                if x is not None and x.numel():
                    x.copy_(y)

    for pol in policies:
        for ns in streams:
            batch = Batch(mats, policy=pol, nstreams=ns)
            restore()
            batch.run()  # first use on the device: library set-up happens outside capture
            torch.cuda.synchronize()
            side = torch.cuda.Stream()
            side.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(side):
                graph = batch.capture()
            torch.cuda.current_stream().wait_stream(side)
            restore()
            graph.replay()  # warm
            torch.cuda.synchronize()
            times = []
            for _ in range(reps):
                restore()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                graph.replay()
                e1.record()
                torch.cuda.synchronize()
                times.append(e0.elapsed_time(e1))
            del graph
            table.append({"policy": pol, "nstreams": ns, "ms": min(times)})
    best = min(table, key=lambda r: r["ms"])
    res = {"nstreams": best["nstreams"], "policy": best["policy"], "ms": best["ms"], "table": table}
    if save:
        cache = _load()
        cache[signature(mats)] = res
        with open(CACHE, "w") as f:
            json.dump(cache, f, indent=1)
    restore()
    return res


# Candidates of the persistent kernel: (CTAs per SM, priority levels, tile rows
# per item). Both builds of the kernel hold at most 4 CTAs per SM.
PERSISTENT_CANDIDATES = tuple((c, w, r) for r in (1, 2) for c in ((2, 3, 4) if r == 1 else (2, 4))
                              for w in (1, 4, 8))


def tune_persistent(mats, pristine, candidates=None, reps=2, save=True):
    """Times each (ctas_per_sm, levels, rows_per_item) candidate of the persistent
    batched kernel on the actual batch (graph replays) and caches the fastest
    under the key 'persistent|' + signature. Returns {"params", "ms", "table"}."""
    from .batched import PersistentBatch
    table = []

    def restore():
        for w, p in zip(mats, pristine):
            for x, y in zip(w, p):
                if x is not None and x.numel():
                    x.copy_(y)

    for cps, levels, rows in (candidates or PERSISTENT_CANDIDATES):
        pb = PersistentBatch(mats, ctas_per_sm=cps, levels=levels, rows_per_item=rows)
        restore()
        pb.run()
        torch.cuda.synchronize()
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            graph = pb.capture()
        torch.cuda.current_stream().wait_stream(side)
        times = []
        for _ in range(reps):
            restore()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            graph.replay()
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        desc = pb.describe()
        del graph
        pb.close()
        table.append({"ctas_per_sm": desc["ctas_per_sm"], "levels": desc["levels"],
                      "rows_per_item": rows, "ms": min(times)})
    best = min(table, key=lambda r: r["ms"])
    res = {"params": {"ctas_per_sm": best["ctas_per_sm"], "levels": best["levels"],
                      "rows_per_item": best["rows_per_item"]}, "ms": best["ms"], "table": table}
    if save:
        cache = _load()
        cache["persistent|" + signature(mats)] = res
        with open(CACHE, "w") as f:
            json.dump(cache, f, indent=1)
    restore()
    return res


def lookup_persistent(mats):
    return _load().get("persistent|" + signature(mats))
