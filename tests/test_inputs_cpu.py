"""The stress-conditioning generator: its condition number is the requested one,
and the oracle stays consistent with the dense definitions on such matrices
(log det exactly the dense one to rounding; the factor within kappa times
machine precision of the dense Cholesky factor restricted to the pattern)."""
import numpy as np
import pytest

import bta_inputs as gen
import oracle
from oracle import dense


@pytest.mark.parametrize("n,b,a,kappa", [(3, 20, 2, 1e4), (4, 16, 0, 1e6), (1, 30, 5, 1e8), (5, 8, 3, 1e3)])
def test_stress_generator_hits_the_condition_number(n, b, a, kappa):
    d, l, ar, t, got = gen.make_bta_stress(n, b, a, seed=n + b, kappa=kappa)
    A = dense.assemble(d, l, ar, t)
    assert np.array_equal(A, A.T)
    lam = np.linalg.eigvalsh(A)
    assert lam[0] > 0
    assert abs(lam[-1] / lam[0] / kappa - 1) < 1e-6
    assert abs(got / kappa - 1) < 1e-6  # lambda_min + shift cancels: ~1e-16 / lambda_min


@pytest.mark.parametrize("kappa", [1e4, 1e7])
def test_oracle_on_stress_matrices(kappa):
    n, b, a = 4, 24, 3
    d, l, ar, t, _ = gen.make_bta_stress(n, b, a, seed=5, kappa=kappa)
    A = dense.assemble(d, l, ar, t)
    F = oracle.pobtaf(d, l, ar, t)
    assert F.info == 0
    sign, ld = np.linalg.slogdet(A)
    assert sign > 0 and abs(oracle.logdet(F) - ld) <= 1e-12 * max(1.0, abs(ld)) * np.log10(kappa)
    L = np.linalg.cholesky(A)
    Ld, Ll, La, Lt = dense.extract(L, n, b, a)
    scale = np.linalg.norm(L)
    for got, want in ((F.diag, Ld), (F.lower, Ll), (F.arrow, La), (F.tip, Lt)):
        assert np.linalg.norm(got - want) <= 1e-15 * kappa * scale
    X = oracle.pobtasi(F)
    Xd = dense.extract(np.linalg.inv(A), n, b, a)
    for got, want in zip(X, Xd):
        assert np.linalg.norm(got - want) <= 1e-14 * kappa * np.linalg.norm(Xd[0])


def test_stress_generator_rejects_large_or_bad_inputs():
    with pytest.raises(ValueError):
        gen.make_bta_stress(100, 100, 0)
    with pytest.raises(ValueError):
        gen.make_bta_stress(2, 8, 1, kappa=1.0)
