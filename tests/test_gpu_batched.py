"""Batched form: one call for matrices of uneven n, b, a; results equal those of
the per-matrix calls (oracle parity at 1e-10 per block), also when captured in a
CUDA graph and replayed; the autotuner returns a measured configuration."""
import numpy as np
import pytest
import torch

import bta_inputs as gen
import oracle
import paper_2503_17528_gb300 as bta
from paper_2503_17528_gb300.batched import Batch
from gpu_util import TOL, dev, host, worst_block_error

pytestmark = pytest.mark.gpu

SHAPES = [(5, 128, 2), (9, 64, 8), (3, 256, 4), (12, 33, 0), (2, 300, 8), (7, 128, 4)]


def _make():
    raw = [gen.make_bta(n, b, a, seed=100 + k, shift=gen.SHIFT_1_01) for k, (n, b, a) in enumerate(SHAPES)]
    return raw, [tuple(dev(x) for x in m) for m in raw]


@pytest.mark.parametrize("policy", ["fp64", "ozaki_b256"])
def test_batched_matches_oracle(policy):
    raw, mats = _make()
    lds = Batch(mats, policy=policy, nstreams=4).run()
    torch.cuda.synchronize()
    assert bta.get_info() == 0 and bta.tc_status() == 0
    for (d, l, ar, t), m, ld in zip(raw, mats, host(lds)):
        F = oracle.pobtaf(d, l, ar, t)
        assert abs(ld - oracle.logdet(F)) <= TOL * abs(oracle.logdet(F))
        assert worst_block_error([host(x) for x in m], oracle.pobtasi(F)) <= TOL


def test_graph_replay_equals_direct_call():
    raw, mats = _make()
    batch = Batch(mats, policy="fp64", nstreams=4)
    batch.run()
    torch.cuda.synchronize()
    direct = [[host(x) for x in m] for m in mats] + [host(batch.logdets)]
    for m, r in zip(mats, raw):
        for x, y in zip(m, r):
            x.copy_(torch.from_numpy(y))
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        g = batch.capture()
    torch.cuda.current_stream().wait_stream(s)
    for m, r in zip(mats, raw):  # capture does not execute; restore and replay
        for x, y in zip(m, r):
            x.copy_(torch.from_numpy(y))
    g.replay()
    torch.cuda.synchronize()
    replay = [[host(x) for x in m] for m in mats] + [host(batch.logdets)]
    for a_, b_ in zip(direct[:-1], replay[:-1]):
        for x, y in zip(a_, b_):
            assert np.array_equal(x, y)
    assert np.array_equal(direct[-1], replay[-1])


def test_autotuner_measures_and_caches(tmp_path, monkeypatch):
    from paper_2503_17528_gb300 import tune
    monkeypatch.setattr(tune, "CACHE", str(tmp_path / "cache.json"))
    raw, mats = _make()
    pristine = [tuple(x.clone() for x in m) for m in mats]
    res = tune.tune(mats, pristine, policies=["fp64", "ozaki_b256"], streams=(1, 4), reps=1)
    assert res["nstreams"] in (1, 4) and res["policy"] in ("fp64", "ozaki_b256")
    assert len(res["table"]) == 4 and all(r["ms"] > 0 for r in res["table"])
    assert tune.lookup(mats)["nstreams"] == res["nstreams"]


def test_many_streams_uneven_batch_matches_oracle():
    """Shapes drawn like the benchmark batch (b in {128, 256, 512}) on 16
    concurrent library streams. Under that load the CTAs of one launch start at
    different times, which exposes any kernel that reads in one CTA what another
    CTA of the same launch writes (the small-b POTRF step once did)."""
    rng = np.random.default_rng(5)
    shapes = [(int(rng.integers(20, 41)), int(rng.choice([128, 256, 512])), int(rng.choice([2, 4, 8])))
              for _ in range(24)]
    raw = [gen.make_bta(n, b, a, seed=700 + k, shift=gen.SHIFT_1_01) for k, (n, b, a) in enumerate(shapes)]
    mats = [tuple(dev(x) for x in m) for m in raw]
    lds = Batch(mats, policy="fp64", nstreams=16).run()
    torch.cuda.synchronize()
    assert bta.get_info() == 0 and bta.tc_status() == 0
    for (d, l, ar, t), m, ld in zip(raw, mats, host(lds)):
        F = oracle.pobtaf(d, l, ar, t)
        assert abs(ld - oracle.logdet(F)) <= TOL * abs(oracle.logdet(F))
        assert worst_block_error([host(x) for x in m], oracle.pobtasi(F)) <= TOL
