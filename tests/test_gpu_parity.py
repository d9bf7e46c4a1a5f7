"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Per-block relative Frobenius error <= 1e-10 for L and X; the same relative bound
for log-det and for the solve. Shapes span several 32-wide tiles, ragged tails,
n = 1 and 2, a = 0 (plain block-tridiagonal) and a tip wider than one tile.
"""
import numpy as np
import pytest
import torch

import bta_inputs as gen
import oracle
import paper_2503_17528_gb300 as bta
from gpu_util import TOL, dev, host, rel_fro, worst_block_error

pytestmark = pytest.mark.gpu

SHAPES = [
    (16, 32, 4),    # the n=16, b=32, a=4 workload
    (1, 5, 3), (1, 40, 0), (2, 33, 1), (3, 45, 7), (4, 64, 0), (5, 70, 13),
    (7, 100, 33), (3, 96, 40), (9, 17, 2), (6, 128, 8), (2, 1, 1), (4, 1, 0),
    (3, 200, 5), (2, 300, 0), (4, 160, 17),  # one fused launch per block step, ragged last tile
    (1, 128, 0), (1, 150, 9), (2, 130, 40), (3, 256, 70),  # one block; arrow rows over 2-3 tiles
    (2, 520, 3),  # 17 row tiles: 16-CTA solve clusters, two tiles on one CTA, ragged last tile
]


def _shift(b):
    return (1.0, 3.0) if b < 8 else gen.SHIFT_PLUS_ONE


def _run(n, b, a, seed):
    d, l, ar, t = gen.make_bta(n, b, a, seed=seed, shift=_shift(b))
    D, Lo, Ar, Ti = dev(d), dev(l), dev(ar), dev(t)
    bta.factor(D, Lo, Ar, Ti)
    ld = bta.logdet(D, Ti)
    r = gen.make_rhs(n, b, a, nrhs=4, seed=seed + 1)
    R = dev(r)
    bta.solve(D, Lo, Ar, Ti, R)
    Lg = [host(x) for x in (D, Lo, Ar, Ti)]
    bta.selinv(D, Lo, Ar, Ti)
    torch.cuda.synchronize()
    Xg = [host(x) for x in (D, Lo, Ar, Ti)]
    return (d, l, ar, t, r), Lg, float(ld.item()), host(R), Xg


@pytest.mark.parametrize("n,b,a", SHAPES)
def test_factor_selinv_logdet_solve(n, b, a):
    (d, l, ar, t, r), Lg, ldg, xg, Xg = _run(n, b, a, seed=n * 1000 + b + a)
    F = oracle.pobtaf(d, l, ar, t)
    assert F.info == 0 and bta.get_info() == 0
    assert worst_block_error(Lg, (F.diag, F.lower, F.arrow, F.tip)) <= TOL
    ldo = oracle.logdet(F)
    assert abs(ldg - ldo) <= TOL * max(1.0, abs(ldo))
    assert rel_fro(xg, oracle.solve(F, r)) <= TOL
    Xo = oracle.pobtasi(F)
    assert worst_block_error(Xg, Xo) <= TOL
    # X_ii is returned full and exactly symmetric
    assert np.array_equal(Xg[0], np.swapaxes(Xg[0], 1, 2))


def test_upper_triangles_are_not_read():
    n, b, a = 3, 40, 5
    d, l, ar, t = gen.make_bta(n, b, a, seed=3)
    d2, t2 = d.copy(), t.copy()
    iu = np.triu_indices(b, 1)
    for i in range(n):
        d2[i][iu] = 1e30
    t2[np.triu_indices(a, 1)] = -7.0
    D, Lo, Ar, Ti = dev(d2), dev(l), dev(ar), dev(t2)
    bta.factor(D, Lo, Ar, Ti)
    F = oracle.pobtaf(d, l, ar, t)
    assert worst_block_error([host(x) for x in (D, Lo, Ar, Ti)], (F.diag, F.lower, F.arrow, F.tip)) <= TOL
    assert np.all(np.triu(host(D)[1], 1) == 0)


def test_non_default_stream_and_repeat_bits():
    n, b, a = 5, 64, 6
    d, l, ar, t = gen.make_bta(n, b, a, seed=8)
    outs = []
    s = torch.cuda.Stream()
    for _ in range(2):
        with torch.cuda.stream(s):
            D, Lo, Ar, Ti = dev(d), dev(l), dev(ar), dev(t)
            bta.factor(D, Lo, Ar, Ti)
            ld = bta.logdet(D, Ti)
            bta.selinv(D, Lo, Ar, Ti)
        s.synchronize()
        outs.append([host(x) for x in (D, Lo, Ar, Ti)] + [host(ld)])
    for x, y in zip(*outs):
        assert np.array_equal(x, y)  # deterministic: identical bits on a repeat


@pytest.mark.parametrize("b", [40, 160])
@pytest.mark.parametrize("where", ["block0", "block2", "tip"])
def test_non_spd_reports_lapack_info(where, b):
    n, a = 4, 3
    d, l, ar, t = gen.make_bta(n, b, a, seed=9)
    if where == "block0":
        d[0][5, 5] = -50.0
        d[0][b - 3, b - 3] = -50.0  # a later failure in the same block must not win
    elif where == "block2":
        d[2] = -d[2]
    else:
        t[1, 1] = -1e3
    F = oracle.pobtaf(d, l, ar, t)
    assert F.info > 0
    D, Lo, Ar, Ti = dev(d), dev(l), dev(ar), dev(t)
    bta.factor(D, Lo, Ar, Ti)
    assert bta.get_info() == F.info
    assert bta.get_info() == 0  # reading clears the word
    k = (F.info - 1) // b
    Dg = host(D)
    for i in range(min(k, n)):
        assert rel_fro(Dg[i], F.diag[i]) <= TOL
    if k < n:
        assert np.isnan(Dg[k]).any()


def test_plain_entry_points_allocate_stream_ordered():
    """The plain C calls (no _ws) through ctypes, with their own scratch."""
    import ctypes
    from paper_2503_17528_gb300 import _lib
    lib = _lib.load()
    n, b, a = 4, 50, 5
    d, l, ar, t = gen.make_bta(n, b, a, seed=12)
    D, Lo, Ar, Ti = dev(d), dev(l), dev(ar), dev(t)
    p = lambda x: ctypes.c_void_p(x.data_ptr())  # noqa: E731
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.bta_factor(n, b, a, p(D), p(Lo), p(Ar), p(Ti), s) == 0
    out = torch.empty((), dtype=torch.float64, device="cuda")
    assert lib.bta_logdet(n, b, a, p(D), p(Ti), p(out), s) == 0
    r = gen.make_rhs(n, b, a, 2, seed=3)
    R = dev(r)
    assert lib.bta_solve(n, b, a, p(D), p(Lo), p(Ar), p(Ti), p(R), 2, s) == 0
    assert lib.bta_selinv(n, b, a, p(D), p(Lo), p(Ar), p(Ti), s) == 0
    torch.cuda.synchronize()
    F = oracle.pobtaf(d, l, ar, t)
    assert abs(out.item() - oracle.logdet(F)) <= TOL * abs(oracle.logdet(F))
    assert rel_fro(host(R), oracle.solve(F, r)) <= TOL
    assert worst_block_error([host(x) for x in (D, Lo, Ar, Ti)], oracle.pobtasi(F)) <= TOL


def test_n365_b1024_a8_full_parity():
    """The n=365, b=1024, a=8 workload (dominance shift 1.01): every block against the oracle."""
    n, b, a = 365, 1024, 8
    d, l, ar, t = gen.make_bta(n, b, a, seed=0, shift=gen.SHIFT_1_01)
    r = gen.make_rhs(n, b, a, nrhs=4, seed=1)
    D, Lo, Ar, Ti = dev(d), dev(l), dev(ar), dev(t)
    bta.factor(D, Lo, Ar, Ti)
    ld = bta.logdet(D, Ti)
    R = dev(r)
    bta.solve(D, Lo, Ar, Ti, R)
    F = oracle.pobtaf(d, l, ar, t)
    assert bta.get_info() == 0
    assert worst_block_error([host(x) for x in (D, Lo, Ar, Ti)], (F.diag, F.lower, F.arrow, F.tip)) <= TOL
    assert abs(ld.item() - oracle.logdet(F)) <= TOL * abs(oracle.logdet(F))
    assert rel_fro(host(R), oracle.solve(F, r)) <= TOL
    bta.selinv(D, Lo, Ar, Ti)
    Xo = oracle.pobtasi(F)
    assert worst_block_error([host(x) for x in (D, Lo, Ar, Ti)], Xo) <= TOL


@pytest.mark.parametrize("b", [40, 160])
@pytest.mark.parametrize("e", [140, -160])
def test_power_of_two_scaled_matrix(b, e):
    """A matrix scaled by 2^140 (pivots above the float range) or 2^-160 (below
    it) factors, inverts and solves like the unscaled one: L scales by 2^(e/2),
    X by 2^-e, exactly. Covers the step kernel (b = 160), the panel kernel
    (b = 40) and the tip."""
    n, a = 3, 5
    d, l, ar, t = gen.make_bta(n, b, a, seed=21 + b)
    s = 2.0 ** e
    d, l, ar, t = d * s, l * s, ar * s, t * s
    (d, l, ar, t, r), Lg, ldg, xg, Xg = _run_scaled(d, l, ar, t, seed=22)
    F = oracle.pobtaf(d, l, ar, t)
    assert F.info == 0 and bta.get_info() == 0
    assert np.isfinite(Lg[0]).all() and np.isfinite(Xg[0]).all()
    assert worst_block_error(Lg, (F.diag, F.lower, F.arrow, F.tip)) <= TOL
    ldo = oracle.logdet(F)
    assert abs(ldg - ldo) <= TOL * abs(ldo)
    assert rel_fro(xg, oracle.solve(F, r)) <= TOL
    assert worst_block_error(Xg, oracle.pobtasi(F)) <= TOL


def _run_scaled(d, l, ar, t, seed):
    n, b, a = d.shape[0], d.shape[1], t.shape[0]
    D, Lo, Ar, Ti = dev(d), dev(l), dev(ar), dev(t)
    bta.factor(D, Lo, Ar, Ti)
    ld = bta.logdet(D, Ti)
    r = gen.make_rhs(n, b, a, nrhs=2, seed=seed)
    R = dev(r)
    bta.solve(D, Lo, Ar, Ti, R)
    Lg = [host(x) for x in (D, Lo, Ar, Ti)]
    bta.selinv(D, Lo, Ar, Ti)
    torch.cuda.synchronize()
    return (d, l, ar, t, r), Lg, float(ld.item()), host(R), [host(x) for x in (D, Lo, Ar, Ti)]
