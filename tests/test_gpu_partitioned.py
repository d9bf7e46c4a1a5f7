"""Partitioned form (P concurrent partitions + reduced system) against the FP64
oracle: X on the whole pattern and log det, at the 1e-10 per-block bound."""
import numpy as np
import pytest
import torch

import bta_inputs as gen
import oracle
import paper_2503_17528_gb300 as bta
from gpu_util import TOL, dev, host, worst_block_error

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _restore_precision():
    yield
    bta.set_precision("fp64")


@pytest.mark.parametrize("n,b,a,P", [
    (12, 32, 4, 3), (20, 48, 0, 4), (9, 40, 5, 2), (30, 64, 8, 6), (7, 33, 3, 3),
    (16, 128, 8, 4), (5, 20, 2, 1), (13, 96, 17, 5),
])
def test_partitioned_matches_oracle(n, b, a, P):
    d, l, ar, t = gen.make_bta(n, b, a, seed=n * 7 + b + P, shift=gen.SHIFT_1_01)
    D, Lo, Ar, Ti = dev(d), dev(l), dev(ar), dev(t)
    ld = bta.factor_selinv_partitioned(D, Lo, Ar, Ti, parts=P, lb=1.8)
    torch.cuda.synchronize()
    assert bta.get_info() == 0 and bta.tc_status() == 0
    F = oracle.pobtaf(d, l, ar, t)
    assert abs(ld.item() - oracle.logdet(F)) <= TOL * abs(oracle.logdet(F))
    assert worst_block_error([host(x) for x in (D, Lo, Ar, Ti)], oracle.pobtasi(F)) <= TOL


def test_partitioned_ozaki_n365_b256():
    bta.set_precision("ozaki")
    n, b, a = 365, 256, 8
    d, l, ar, t = gen.make_bta(n, b, a, seed=5, shift=gen.SHIFT_1_01)
    D, Lo, Ar, Ti = dev(d), dev(l), dev(ar), dev(t)
    ld = bta.factor_selinv_partitioned(D, Lo, Ar, Ti, parts=8, lb=1.8)
    torch.cuda.synchronize()
    assert bta.tc_status() == 0
    F = oracle.pobtaf(d, l, ar, t)
    assert abs(ld.item() - oracle.logdet(F)) <= TOL * abs(oracle.logdet(F))
    assert worst_block_error([host(x) for x in (D, Lo, Ar, Ti)], oracle.pobtasi(F)) <= TOL
