"""Tensor-core (tcgen05) paths against FP64 references.

* bta_gemm in the OZAKI mode (FP64 emulated on BF16 slices) against the FP64
  product: relative Frobenius error <= 1e-12 (the splitting keeps ~48 bits per
  operand and accumulates the leading slice groups exactly).
* bta_gemm in the BF16X3 mode: error <= 1e-4 (split-BF16 with FP32 accumulation).
* factor + selinv + logdet + solve in the OZAKI mode against the FP64 oracle at
  the same 1e-10 per-block bound as the FP64 path.
"""
import numpy as np
import pytest
import torch

import bta_inputs as gen
import oracle
import paper_2503_17528_gb300 as bta
from gpu_util import TOL, dev, host, rel_fro, worst_block_error

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _restore_precision():
    yield
    bta.set_precision("fp64")


GEMM_SHAPES = [
    (128, 128, 64, False, False),
    (1024, 1024, 1024, False, True),
    (300, 200, 1000, True, False),
    (256, 384, 2048, False, False),   # two k chunks
    (129, 65, 97, True, True),        # ragged everything
    (1024, 8, 1024, False, False),    # narrow
    (2048, 2048, 2048, False, False),  # the b = 2048 block product: 512 tiles, all SMs, no k split
]


@pytest.mark.parametrize("M,N,K,ta,tb", GEMM_SHAPES)
def test_gemm_ozaki_matches_fp64(M, N, K, ta, tb):
    rng = np.random.default_rng(M + N + K)
    A = rng.standard_normal((K, M) if ta else (M, K)) / np.sqrt(K)
    B = rng.standard_normal((N, K) if tb else (K, N))
    A[0, 0] = 3.0  # a spread of magnitudes within a row
    C0 = rng.standard_normal((M, N))
    want = 1.5 * ((A.T if ta else A) @ (B.T if tb else B)) - 0.5 * C0
    got = bta.gemm(dev(A), dev(B), dev(C0), alpha=1.5, beta=-0.5, trans_a=ta, trans_b=tb,
                   precision="ozaki")
    torch.cuda.synchronize()
    assert bta.tc_status() == 0
    err = rel_fro(host(got), want)
    assert err <= 1e-12, err


@pytest.mark.parametrize("M,N,K,ta,tb", GEMM_SHAPES[:3])
def test_gemm_bf16x3_error_bound(M, N, K, ta, tb):
    rng = np.random.default_rng(7 + M)
    A = rng.standard_normal((K, M) if ta else (M, K))
    B = rng.standard_normal((N, K) if tb else (K, N))
    want = (A.T if ta else A) @ (B.T if tb else B)
    got = bta.gemm(dev(A), dev(B), trans_a=ta, trans_b=tb, precision="bf16x3")
    torch.cuda.synchronize()
    assert bta.tc_status() == 0
    assert rel_fro(host(got), want) <= 1e-4


def test_gemm_zero_and_nan_rows():
    A = np.zeros((256, 128))
    A[5, :] = np.nan
    A[7, 3] = 2.0
    B = np.ones((128, 128))
    got = host(bta.gemm(dev(A), dev(B), precision="ozaki"))
    torch.cuda.synchronize()
    assert np.all(np.isnan(got[5]))
    assert np.all(got[0] == 0) and np.allclose(got[7], 2.0)


@pytest.mark.parametrize("n,b,a", [(6, 256, 8), (4, 300, 20), (3, 1024, 8), (2, 1100, 4), (2, 130, 0), (5, 64, 70)])
def test_ozaki_factor_selinv_parity(n, b, a):
    bta.set_precision("ozaki")
    d, l, ar, t = gen.make_bta(n, b, a, seed=n + b + a, shift=gen.SHIFT_1_01)
    r = gen.make_rhs(n, b, a, nrhs=4, seed=2)
    D, Lo, Ar, Ti, R = dev(d), dev(l), dev(ar), dev(t), dev(r)
    bta.factor(D, Lo, Ar, Ti)
    ld = bta.logdet(D, Ti)
    bta.solve(D, Lo, Ar, Ti, R)
    Lg = [host(x) for x in (D, Lo, Ar, Ti)]
    bta.selinv(D, Lo, Ar, Ti)
    torch.cuda.synchronize()
    assert bta.tc_status() == 0 and bta.get_info() == 0
    F = oracle.pobtaf(d, l, ar, t)
    assert worst_block_error(Lg, (F.diag, F.lower, F.arrow, F.tip)) <= TOL
    assert abs(ld.item() - oracle.logdet(F)) <= TOL * abs(oracle.logdet(F))
    assert rel_fro(host(R), oracle.solve(F, r)) <= TOL
    assert worst_block_error([host(x) for x in (D, Lo, Ar, Ti)], oracle.pobtasi(F)) <= TOL


def test_bf16x3_mixed_error_is_bounded():
    """Mixed precision: stated bound on the per-block error against the FP64 oracle,
    4 kappa u with u = 2^-16 (split-BF16x3 products) and kappa <= 4 for this
    generator (1.001 dominance shift, measured kappa about 3): 2.4e-4."""
    bta.set_precision("bf16x3")
    n, b, a = 6, 256, 8
    d, l, ar, t = gen.make_bta(n, b, a, seed=5, shift=gen.SHIFT_1_001)
    D, Lo, Ar, Ti = dev(d), dev(l), dev(ar), dev(t)
    bta.factor(D, Lo, Ar, Ti)
    Lg = [host(x) for x in (D, Lo, Ar, Ti)]
    bta.selinv(D, Lo, Ar, Ti)
    torch.cuda.synchronize()
    F = oracle.pobtaf(d, l, ar, t)
    bound = 4 * 4.0 * 2.0 ** -16
    assert worst_block_error(Lg, (F.diag, F.lower, F.arrow, F.tip)) <= bound
    assert worst_block_error([host(x) for x in (D, Lo, Ar, Ti)], oracle.pobtasi(F)) <= bound


def test_gemm_ozaki_self_product_after_another_call():
    """A A^T splits A once: op(B)^T has the same rows, scales and slices. With
    fewer output tiles than SMs (1024 x 1024: 128 tiles) the k-units of a tile are
    split over CTAs and a finalize kernel applies the scales. A previous call with
    very different scales must leave nothing behind that this product reads."""
    rng = np.random.default_rng(5)
    B0 = rng.standard_normal((1024, 1024)) * 1e6
    bta.gemm(dev(B0), dev(B0.T.copy()), precision="ozaki")
    torch.cuda.synchronize()
    s = 2.0 ** rng.integers(-20, 21, 1024).astype(np.float64)
    An = rng.standard_normal((1024, 1024))
    A = An * s[:, None]
    got = host(bta.gemm(dev(A), dev(A), trans_b=True, precision="ozaki"))
    torch.cuda.synchronize()
    assert bta.tc_status() == 0
    # compare on the unscaled rows: C_ij / (s_i s_j) against An An^T
    err = rel_fro(got / np.outer(s, s), An @ An.T)
    assert err <= 1e-12, err
