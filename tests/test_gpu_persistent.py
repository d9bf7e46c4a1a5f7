"""Persistent batched form (bta_plan_*): one cooperative launch factors, log-dets
and inverts a batch of matrices of uneven n, b, a. Checked against the FP64
oracle at 1e-10 per block (ragged b, several arrow tiles, a = 0, n = 1), for
every tuning parameter (bit-identical results: the schedule changes the order
of items, never the arithmetic of a tile), under CUDA-graph replay, and with a
non-SPD matrix whose failure is reported for that matrix alone."""
import numpy as np
import pytest
import torch

import bta_inputs as gen
import oracle
from paper_2503_17528_gb300.batched import PersistentBatch
from gpu_util import TOL, dev, host, worst_block_error

pytestmark = pytest.mark.gpu

# (n, b, a): ragged b (33, 100, 70), arrow tips over one tile (a = 40), a = 0, n = 1
SHAPES = [(5, 128, 2), (9, 64, 8), (3, 100, 40), (12, 33, 0), (1, 70, 5), (7, 128, 4), (4, 256, 16),
          (2, 32, 0)]


def _make(shapes=SHAPES, seed=300):
    raw = [gen.make_bta(n, b, a, seed=seed + k, shift=gen.SHIFT_1_01) for k, (n, b, a) in enumerate(shapes)]
    return raw, [tuple(dev(x) for x in m) for m in raw]


def _restore(mats, raw):
    for m, r in zip(mats, raw):
        for x, y in zip(m, r):
            x.copy_(torch.from_numpy(y))


def _check_oracle(raw, mats, lds):
    for (d, l, ar, t), m, ld in zip(raw, mats, host(lds)):
        F = oracle.pobtaf(d, l, ar, t)
        ldo = oracle.logdet(F)
        assert abs(ld - ldo) <= TOL * abs(ldo)
        assert worst_block_error([host(x) for x in m], oracle.pobtasi(F)) <= TOL


def test_persistent_matches_oracle():
    raw, mats = _make()
    pb = PersistentBatch(mats)
    lds = pb.run()
    torch.cuda.synchronize()
    to, info = pb.status()
    assert to == 0 and info == [0] * len(mats)
    _check_oracle(raw, mats, lds)
    desc = pb.describe()
    assert desc["grid"] >= desc["ctas_per_sm"] >= 1 and desc["ops"] > 0 and desc["items"] >= desc["ops"]


@pytest.mark.parametrize("params", [dict(rows_per_item=2), dict(levels=1),
                                    dict(levels=3, ctas_per_sm=2),
                                    dict(ctas_per_sm=1, levels=8, rows_per_item=2)])
def test_parameters_change_schedule_not_results(params):
    raw, mats = _make()
    base = PersistentBatch(mats)
    base.run()
    torch.cuda.synchronize()
    want = [[host(x) for x in m] for m in mats] + [host(base.logdets)]
    _restore(mats, raw)
    pb = PersistentBatch(mats, **params)
    pb.run()
    torch.cuda.synchronize()
    assert pb.status()[0] == 0
    got = [[host(x) for x in m] for m in mats] + [host(pb.logdets)]
    for g, w in zip(got[:-1], want[:-1]):
        for x, y in zip(g, w):
            assert np.array_equal(x, y)
    assert np.array_equal(got[-1], want[-1])


def test_graph_replay_and_repeat():
    raw, mats = _make()
    pb = PersistentBatch(mats)
    pb.run()
    torch.cuda.synchronize()
    direct = [[host(x) for x in m] for m in mats] + [host(pb.logdets)]
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        g = pb.capture()
    torch.cuda.current_stream().wait_stream(s)
    for _ in range(2):
        _restore(mats, raw)
        g.replay()
        torch.cuda.synchronize()
        assert pb.status()[0] == 0
        replay = [[host(x) for x in m] for m in mats] + [host(pb.logdets)]
        for a_, b_ in zip(direct[:-1], replay[:-1]):
            for x, y in zip(a_, b_):
                assert np.array_equal(x, y)
        assert np.array_equal(direct[-1], replay[-1])


def test_failure_reported_per_matrix():
    shapes = [(3, 64, 4), (4, 96, 2), (2, 64, 0)]
    raw, mats = _make(shapes, seed=500)
    # matrix 1: break positive definiteness at global row 96 + 40 + 1 (block 1, row 40)
    d = raw[1][0].copy()
    d[1, 40, 40] = -1e3
    mats[1][0].copy_(torch.from_numpy(d))
    pb = PersistentBatch(mats)
    pb.run()
    torch.cuda.synchronize()
    to, info = pb.status()
    assert to == 0
    assert info[0] == 0 and info[2] == 0 and info[1] == 96 + 40 + 1
    for k in (0, 2):
        r = raw[k]
        F = oracle.pobtaf(*r)
        assert worst_block_error([host(x) for x in mats[k]], oracle.pobtasi(F)) <= TOL


def test_uneven_batch_like_the_benchmark():
    """A 16-matrix sample drawn like the 64-matrix benchmark batch (n in
    [20, 200], b in {128, 256, 512}, a in {2, 4, 8}), against the oracle."""
    rng = np.random.default_rng(77)
    shapes = [(int(rng.integers(20, 41)), int(rng.choice([128, 256, 512])), int(rng.choice([2, 4, 8])))
              for _ in range(16)]
    raw, mats = _make(shapes, seed=900)
    pb = PersistentBatch(mats)
    lds = pb.run()
    torch.cuda.synchronize()
    to, info = pb.status()
    assert to == 0 and not any(info)
    _check_oracle(raw, mats, lds)
