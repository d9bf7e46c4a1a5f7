"""Parity at block order b = 2048 (the n=256, b=2048, a=16 workload, dominance
shift 1.001), through the C ABI, against the FP64 CPU oracle.

At b = 2048, a = 16 the FP64 step kernel runs 64 tile steps over 129 extended
tile rows (two blocks of 64 tiles and one arrow tile), and the Ozaki mode takes
its inverse + tensor-core product route (b above 1024). The small shape (n = 3)
covers both at the 1e-10 per-block bound; the full-size case runs the one call
the benchmark times (bta_factor_selinv_all: factor, log det, solve with 4
right-hand sides, selected inversion) on the whole n = 256 matrix and compares
every block of X, the log-determinant and the solution.
"""
import numpy as np
import pytest
import torch

import bta_inputs as gen
import oracle
import paper_2503_17528_gb300 as bta
from gpu_util import TOL, dev, host, rel_fro, worst_block_error

pytestmark = pytest.mark.gpu

# Split-BF16x3 products (hi*hi + hi*lo + lo*hi, FP32 accumulation) carry a relative
# error of about u = 2^-16 of the operands' scale, and a relative perturbation eta of
# A moves the blocks of A^{-1} by up to kappa * eta: the bound is 4 kappa u with
# kappa <= 4 for this generator (measured 3.1), 2.4e-4; measured up to 3.5e-5.
BF16X3_BOUND = 4 * 4.0 * 2.0 ** -16


@pytest.fixture(autouse=True)
def _restore_precision():
    yield
    bta.set_precision("fp64")


def _run_four_calls(d, l, ar, t, r):
    D, Lo, Ar, Ti, R = dev(d), dev(l), dev(ar), dev(t), dev(r)
    bta.factor(D, Lo, Ar, Ti)
    ld = bta.logdet(D, Ti)
    bta.solve(D, Lo, Ar, Ti, R)
    Lg = [host(x) for x in (D, Lo, Ar, Ti)]
    bta.selinv(D, Lo, Ar, Ti)
    torch.cuda.synchronize()
    return Lg, float(ld.item()), host(R), [host(x) for x in (D, Lo, Ar, Ti)]


@pytest.mark.parametrize("prec", ["fp64", "ozaki"])
def test_b2048_parity(prec):
    bta.set_precision(prec)
    n, b, a = 3, 2048, 16
    d, l, ar, t = gen.make_bta(n, b, a, seed=2048, shift=gen.SHIFT_1_001)
    r = gen.make_rhs(n, b, a, nrhs=4, seed=2049)
    Lg, ldg, xg, Xg = _run_four_calls(d, l, ar, t, r)
    assert bta.tc_status() == 0 and bta.get_info() == 0
    F = oracle.pobtaf(d, l, ar, t)
    assert worst_block_error(Lg, (F.diag, F.lower, F.arrow, F.tip)) <= TOL
    ldo = oracle.logdet(F)
    assert abs(ldg - ldo) <= TOL * abs(ldo)
    assert rel_fro(xg, oracle.solve(F, r)) <= TOL
    assert worst_block_error(Xg, oracle.pobtasi(F)) <= TOL
    assert np.array_equal(Xg[0], np.swapaxes(Xg[0], 1, 2))


def test_b2048_bf16x3_bound():
    bta.set_precision("bf16x3")
    n, b, a = 3, 2048, 16
    d, l, ar, t = gen.make_bta(n, b, a, seed=2050, shift=gen.SHIFT_1_001)
    r = gen.make_rhs(n, b, a, nrhs=4, seed=2051)
    Lg, ldg, xg, Xg = _run_four_calls(d, l, ar, t, r)
    assert bta.tc_status() == 0 and bta.get_info() == 0
    F = oracle.pobtaf(d, l, ar, t)
    assert worst_block_error(Lg, (F.diag, F.lower, F.arrow, F.tip)) <= BF16X3_BOUND
    assert worst_block_error(Xg, oracle.pobtasi(F)) <= BF16X3_BOUND
    ldo = oracle.logdet(F)
    assert abs(ldg - ldo) <= BF16X3_BOUND * abs(ldo)


def test_n256_b2048_a16_full_parity():
    """The whole n=256, b=2048, a=16 matrix in the benchmark's launch configuration
    (one bta_factor_selinv_all call, FP64): every block of X, log det and the
    solution of 4 right-hand sides against the oracle, at 1e-10 per block."""
    n, b, a = 256, 2048, 16
    d, l, ar, t = gen.make_bta(n, b, a, seed=0, shift=gen.SHIFT_1_001)
    r = gen.make_rhs(n, b, a, nrhs=4, seed=1000)
    D, Lo, Ar, Ti, R = dev(d), dev(l), dev(ar), dev(t), dev(r)
    ld = bta.factor_selinv_all(D, Lo, Ar, Ti, rhs=R)
    torch.cuda.synchronize()
    assert bta.get_info() == 0
    F = oracle.pobtaf(d, l, ar, t)
    del d, l
    ldo = oracle.logdet(F)
    assert abs(ld.item() - ldo) <= TOL * abs(ldo)
    assert rel_fro(host(R), oracle.solve(F, r)) <= TOL
    Xd, Xl, Xa, Xt = oracle.pobtasi(F)
    del F
    worst = 0.0
    for i in range(n):  # one block at a time from the device
        worst = max(worst, rel_fro(host(D[i]), Xd[i]), rel_fro(host(Ar[i]), Xa[i]))
        if i + 1 < n:
            worst = max(worst, rel_fro(host(Lo[i]), Xl[i]))
    worst = max(worst, rel_fro(host(Ti), Xt))
    assert worst <= TOL, worst


@pytest.mark.parametrize("prec", ["fp64", "ozaki"])
def test_dataset4_block_shape_parity(prec):
    """Block order b = 2865, a = 4 (the shape of the paper's weak-scaling dataset,
    Section 5.2): 90 tiles per block row with a 17-row ragged last tile, so every
    tile kernel runs its ragged edges at scale (Ozaki: halves of 1432 and 1433)."""
    bta.set_precision(prec)
    n, b, a = 3, 2865, 4
    d, l, ar, t = gen.make_bta(n, b, a, seed=2865, shift=gen.SHIFT_1_01)
    r = gen.make_rhs(n, b, a, nrhs=4, seed=2866)
    Lg, ldg, xg, Xg = _run_four_calls(d, l, ar, t, r)
    assert bta.tc_status() == 0 and bta.get_info() == 0
    F = oracle.pobtaf(d, l, ar, t)
    assert worst_block_error(Lg, (F.diag, F.lower, F.arrow, F.tip)) <= TOL
    ldo = oracle.logdet(F)
    assert abs(ldg - ldo) <= TOL * abs(ldo)
    assert rel_fro(xg, oracle.solve(F, r)) <= TOL
    assert worst_block_error(Xg, oracle.pobtasi(F)) <= TOL
