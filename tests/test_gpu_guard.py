"""Out-of-bounds writes: every block array of a call sits inside one device buffer
between guard regions filled with a sentinel value, and after factor, log det,
solve and selected inversion (and a persistent batched run) every guard word must
still hold the sentinel. Shapes with ragged block orders (33, 70, 100, 130, 300),
arrow tips of one to two tiles and a = 0 reach the edge-tile code of each kernel.
"""
import pytest
import torch

import bta_inputs as gen
import oracle
import paper_2503_17528_gb300 as bta
from paper_2503_17528_gb300.batched import PersistentBatch
from gpu_util import TOL, host, worst_block_error

pytestmark = pytest.mark.gpu

GUARD = 4096            # doubles before, between and after the arrays
SENTINEL = -7.25e300    # a value none of the kernels writes


@pytest.fixture(autouse=True)
def _restore_precision():
    yield
    bta.set_precision("fp64")


def _guarded(arrays):
    """One device buffer holding the arrays between sentinel guards; returns the
    buffer, the views (same shapes) and the guard slices."""
    sizes = [a.size for a in arrays]
    total = GUARD * (len(arrays) + 1) + sum(sizes)
    buf = torch.full((total,), SENTINEL, dtype=torch.float64, device="cuda")
    views, guards, at = [], [], 0
    for a in arrays:
        guards.append((at, at + GUARD))
        at += GUARD
        v = buf[at:at + a.size].view(a.shape)
        v.copy_(torch.from_numpy(a))
        views.append(v)
        at += a.size
    guards.append((at, at + GUARD))
    return buf, views, guards


def _guards_intact(buf, guards):
    want = torch.full((GUARD,), SENTINEL, dtype=torch.float64, device="cuda")
    return all(torch.equal(buf[s:e], want) for s, e in guards)


@pytest.mark.parametrize("prec,n,b,a", [("fp64", 3, 33, 3), ("fp64", 1, 70, 5), ("fp64", 4, 100, 40),
                                        ("fp64", 2, 130, 0), ("fp64", 3, 256, 8), ("ozaki", 3, 300, 20)])
def test_no_write_outside_the_blocks(prec, n, b, a):
    bta.set_precision(prec)
    d, l, ar, t = gen.make_bta(n, b, a, seed=4242 + b, shift=gen.SHIFT_1_01)
    r = gen.make_rhs(n, b, a, nrhs=3, seed=4243)
    buf, (D, Lo, Ar, Ti, R), guards = _guarded([d, l, ar, t, r])
    ld_buf = torch.full((3,), SENTINEL, dtype=torch.float64, device="cuda")
    bta.factor(D, Lo, Ar, Ti)
    bta.logdet(D, Ti, out=ld_buf[1])
    bta.solve(D, Lo, Ar, Ti, R)
    bta.selinv(D, Lo, Ar, Ti)
    torch.cuda.synchronize()
    assert bta.get_info() == 0 and bta.tc_status() == 0
    assert _guards_intact(buf, guards)
    assert float(ld_buf[0]) == SENTINEL and float(ld_buf[2]) == SENTINEL
    F = oracle.pobtaf(d, l, ar, t)
    assert worst_block_error([host(x) for x in (D, Lo, Ar, Ti)], oracle.pobtasi(F)) <= TOL


def test_persistent_batch_writes_only_its_blocks():
    shapes = [(3, 33, 3), (2, 64, 0), (2, 100, 40)]
    raws = [gen.make_bta(n, b, a, seed=777 + k, shift=gen.SHIFT_1_01) for k, (n, b, a) in enumerate(shapes)]
    flat = [x for m in raws for x in m]
    buf, views, guards = _guarded(flat)
    mats = [tuple(views[4 * k:4 * k + 4]) for k in range(len(shapes))]
    pb = PersistentBatch(mats)
    pb.run()
    torch.cuda.synchronize()
    timed_out, info = pb.status()
    assert timed_out == 0 and not any(info)
    assert _guards_intact(buf, guards)
    for m, raw in zip(mats, raws):
        F = oracle.pobtaf(*raw)
        assert worst_block_error([host(x) for x in m], oracle.pobtasi(F)) <= TOL
    pb.close()
