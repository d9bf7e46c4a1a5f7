"""Pins for the CPU oracle, independent of the oracle's own block recursion.

Each test checks the block recursion (Algorithms 1 and 2 of the paper, plus
log-det and solve) against something the mathematics fixes: brute-force dense
linear algebra on tiny inputs, closed forms, identities that hold at any size,
and special cases that reduce to textbook formulas.
"""
import numpy as np
import pytest

import bta_inputs as gen
import oracle
from oracle import dense

TOL = 1e-12


def mk(n, b, a, seed, shift=None):
    """Generator input; very small b gets a larger additive shift, since one
    N(0,1)/sqrt(b) diagonal entry can then outweigh the +1 dominance margin."""
    if shift is None:
        shift = (1.0, 3.0) if b < 8 else gen.SHIFT_PLUS_ONE
    return gen.make_bta(n, b, a, seed=seed, shift=shift)


def rel(x, y):
    ny = np.linalg.norm(y)
    return np.linalg.norm(x - y) / (ny if ny > 0 else 1.0)


def assert_blocks_close(got, want, tol=TOL):
    for name, g, w in zip(("diag", "lower", "arrow", "tip"), got, want):
        assert g.shape == w.shape, name
        for k in range(g.shape[0] if g.ndim == 3 else 1):
            gk, wk = (g[k], w[k]) if g.ndim == 3 else (g, w)
            if wk.size:
                assert rel(gk, wk) <= tol, (name, k, rel(gk, wk))


SHAPES = [(1, 3, 2), (1, 4, 0), (2, 4, 3), (3, 5, 2), (5, 4, 0), (4, 1, 1),
          (3, 1, 0), (6, 7, 7), (16, 32, 4), (7, 9, 13)]


@pytest.mark.parametrize("n,b,a", SHAPES)
def test_factor_matches_dense_cholesky(n, b, a):
    d, l, ar, t = mk(n, b, a, seed=n * 100 + b * 10 + a)
    F = oracle.pobtaf(d, l, ar, t)
    assert F.info == 0
    assert_blocks_close((F.diag, F.lower, F.arrow, F.tip), dense.dense_factor(d, l, ar, t))


@pytest.mark.parametrize("n,b,a", SHAPES)
def test_selinv_matches_dense_inverse(n, b, a):
    d, l, ar, t = mk(n, b, a, seed=n * 100 + b * 10 + a + 1)
    X = oracle.pobtasi(oracle.pobtaf(d, l, ar, t))
    assert_blocks_close(X, dense.dense_selinv(d, l, ar, t))


@pytest.mark.parametrize("n,b,a", SHAPES)
def test_logdet_and_solve_match_dense(n, b, a):
    d, l, ar, t = mk(n, b, a, seed=7 + n + b + a)
    F = oracle.pobtaf(d, l, ar, t)
    assert abs(oracle.logdet(F) - dense.dense_logdet(d, l, ar, t)) <= 1e-12 * max(1.0, abs(oracle.logdet(F)))
    r = gen.make_rhs(n, b, a, nrhs=3, seed=5)
    assert rel(oracle.solve(F, r), dense.dense_solve(d, l, ar, t, r)) <= TOL
    assert rel(oracle.solve(F, r[:, 0]), dense.dense_solve(d, l, ar, t, r[:, 0])) <= TOL


@pytest.mark.parametrize("N", [1, 2, 5, 12])
def test_laplacian_closed_form(N):
    """b=1, a=0: the 1-D Laplacian tridiag(-1, 2, -1) of order N.

    Closed forms (1-based k): L_kk = sqrt((k+1)/k), L_{k+1,k} = -sqrt(k/(k+1)),
    (A^{-1})_{ij} = min(i,j) (N+1-max(i,j)) / (N+1), det A = N+1.
    """
    d = np.full((N, 1, 1), 2.0)
    l = np.full((N - 1, 1, 1), -1.0)
    ar = np.zeros((N, 0, 1))
    t = np.zeros((0, 0))
    F = oracle.pobtaf(d, l, ar, t)
    k = np.arange(1, N + 1, dtype=float)
    np.testing.assert_allclose(F.diag[:, 0, 0], np.sqrt((k + 1) / k), rtol=1e-14)
    np.testing.assert_allclose(F.lower[:, 0, 0], -np.sqrt(k[:-1] / k[1:]), rtol=1e-14)
    Xd, Xl, _, _ = oracle.pobtasi(F)
    np.testing.assert_allclose(Xd[:, 0, 0], k * (N + 1 - k) / (N + 1), rtol=1e-13)
    np.testing.assert_allclose(Xl[:, 0, 0], k[:-1] * (N - k[:-1]) / (N + 1), rtol=1e-13)
    assert abs(oracle.logdet(F) - np.log(N + 1)) <= 1e-13
    x = oracle.solve(F, np.ones(N))
    np.testing.assert_allclose(x, k * (N + 1 - k) / 2.0, rtol=1e-12)  # A x = 1 -> x_k = k(N+1-k)/2


def test_kronecker_similarity_closed_form():
    """A = D (T kron I_b) D^T with D = blockdiag(D_0..D_n), D_i lower triangular.

    For a scalar (n+1)x(n+1) SPD matrix T on the arrowhead-tridiagonal pattern
    (so a = b here): L_ij = (chol T)_ij D_i, (A^{-1})_ij = (T^{-1})_ij D_i^{-T} D_j^{-1},
    log det A = b log det T + 2 sum_i log det D_i. The D_i make every block of A
    non-symmetric, so a transposed operand anywhere shows up.
    """
    n, b = 5, 3
    rng = np.random.default_rng(11)
    T = np.zeros((n + 1, n + 1))
    for i in range(n):
        T[i, i] = 4.0 + i
        if i + 1 < n:
            T[i + 1, i] = T[i, i + 1] = -1.0 + 0.1 * i
        T[n, i] = T[i, n] = 0.3 + 0.05 * i
    T[n, n] = 6.0
    D = [np.tril(rng.standard_normal((b, b))) + np.diag(1.5 + rng.random(b)) for _ in range(n + 1)]
    blk = lambda i, j: T[i, j] * D[i] @ D[j].T  # noqa: E731
    d = np.stack([blk(i, i) for i in range(n)])
    l = np.stack([blk(i + 1, i) for i in range(n - 1)])
    ar = np.stack([blk(n, i) for i in range(n)])
    t = blk(n, n)

    F = oracle.pobtaf(d, l, ar, t)
    LT = np.linalg.cholesky(T)
    np.testing.assert_allclose(F.diag, np.stack([LT[i, i] * D[i] for i in range(n)]), atol=1e-12)
    np.testing.assert_allclose(F.lower, np.stack([LT[i + 1, i] * D[i + 1] for i in range(n - 1)]), atol=1e-12)
    np.testing.assert_allclose(F.arrow, np.stack([LT[n, i] * D[n] for i in range(n)]), atol=1e-12)
    np.testing.assert_allclose(F.tip, LT[n, n] * D[n], atol=1e-12)

    Ti = np.linalg.inv(T)
    Di = [np.linalg.inv(x) for x in D]
    xb = lambda i, j: Ti[i, j] * Di[i].T @ Di[j]  # noqa: E731
    Xd, Xl, Xa, Xt = oracle.pobtasi(F)
    np.testing.assert_allclose(Xd, np.stack([xb(i, i) for i in range(n)]), atol=1e-12)
    np.testing.assert_allclose(Xl, np.stack([xb(i + 1, i) for i in range(n - 1)]), atol=1e-12)
    np.testing.assert_allclose(Xa, np.stack([xb(n, i) for i in range(n)]), atol=1e-12)
    np.testing.assert_allclose(Xt, xb(n, n), atol=1e-12)

    want = b * np.linalg.slogdet(T)[1] + 2 * sum(np.sum(np.log(np.diag(x))) for x in D)
    assert abs(oracle.logdet(F) - want) <= 1e-11


@pytest.mark.parametrize("b,a", [(4, 3), (6, 2), (5, 5)])
def test_two_block_textbook_inverse(b, a):
    """n = 1: A = [[A00, A10^T], [A10, A11]] and the textbook 2x2 block formulas.

    L00 = chol(A00), L10 = A10 L00^{-T}, L11 = chol(S) with S = A11 - A10 A00^{-1} A10^T;
    X11 = S^{-1}, X10 = -S^{-1} A10 A00^{-1}, X00 = A00^{-1} + A00^{-1} A10^T S^{-1} A10 A00^{-1}.
    """
    d, l, ar, t = mk(1, b, a, seed=3)
    A00, A10, A11 = d[0], ar[0], t
    iA00 = np.linalg.inv(A00)
    S = A11 - A10 @ iA00 @ A10.T
    iS = np.linalg.inv(S)
    F = oracle.pobtaf(d, l, ar, t)
    np.testing.assert_allclose(F.diag[0], np.linalg.cholesky(A00), atol=1e-13)
    np.testing.assert_allclose(F.arrow[0] @ F.diag[0].T, A10, atol=1e-13)
    np.testing.assert_allclose(F.tip, np.linalg.cholesky(S), atol=1e-13)
    Xd, Xl, Xa, Xt = oracle.pobtasi(F)
    np.testing.assert_allclose(Xt, iS, atol=1e-13)
    np.testing.assert_allclose(Xa[0], -iS @ A10 @ iA00, atol=1e-13)
    np.testing.assert_allclose(Xd[0], iA00 + iA00 @ A10.T @ iS @ A10 @ iA00, atol=1e-13)
    assert Xl.shape == (0, b, b)


def test_block_diagonal_input():
    """Zero off-diagonal and arrow blocks: L_ii = chol(A_ii) and X_ii = A_ii^{-1}."""
    n, b, a = 4, 6, 3
    d, l, ar, t = mk(n, b, a, seed=21)
    l[:] = 0.0
    ar[:] = 0.0
    F = oracle.pobtaf(d, l, ar, t)
    Xd, Xl, Xa, Xt = oracle.pobtasi(F)
    for i in range(n):
        np.testing.assert_allclose(F.diag[i], np.linalg.cholesky(d[i]), atol=1e-13)
        np.testing.assert_allclose(Xd[i], np.linalg.inv(d[i]), atol=1e-13)
    assert np.all(Xl == 0) and np.all(Xa == 0)
    np.testing.assert_allclose(Xt, np.linalg.inv(t), atol=1e-13)


def test_invariants_medium():
    """LL^T = A on the pattern and (A X)_ii = I, (A X)_nn = I on a size past dense comfort."""
    n, b, a = 30, 20, 5
    d, l, ar, t = gen.make_bta(n, b, a, seed=4, shift=gen.SHIFT_1_01)
    F = oracle.pobtaf(d, l, ar, t)
    Ld, Ll, La, Lt = F.diag, F.lower, F.arrow, F.tip
    for i in range(n):
        llt = Ld[i] @ Ld[i].T + (Ll[i - 1] @ Ll[i - 1].T if i else 0)
        assert rel(llt, d[i]) < 1e-13
        if i + 1 < n:
            assert rel(Ll[i] @ Ld[i].T, l[i]) < 1e-13
        na = La[i] @ Ld[i].T + (La[i - 1] @ Ll[i - 1].T if i else 0)
        assert rel(na, ar[i]) < 1e-13
    assert rel(sum(La[i] @ La[i].T for i in range(n)) + Lt @ Lt.T, t) < 1e-13

    Xd, Xl, Xa, Xt = oracle.pobtasi(F)
    I_b = np.eye(b)
    for i in range(n):
        ax = d[i] @ Xd[i] + ar[i].T @ Xa[i]
        if i > 0:
            ax += l[i - 1] @ Xl[i - 1].T
        if i + 1 < n:
            ax += l[i].T @ Xl[i]
        assert np.abs(ax - I_b).max() < 1e-12
    axn = t @ Xt + sum(ar[i] @ Xa[i].T for i in range(n))
    assert np.abs(axn - np.eye(a)).max() < 1e-12


@pytest.mark.parametrize("where", ["block0", "block2", "last", "tip"])
def test_failure_info_matches_lapack_on_dense(where):
    """A non-SPD input gives the dense LAPACK dpotrf info (first bad global row, 1-based)."""
    from scipy.linalg import lapack
    n, b, a = 4, 5, 3
    d, l, ar, t = mk(n, b, a, seed=9)
    if where == "block0":
        d[0][2, 2] = -50.0
    elif where == "block2":
        d[2] = -d[2]
    elif where == "last":
        d[n - 1][4, 4] = 1e-3
        d[n - 1][4, :4] = d[n - 1][:4, 4] = 3.0
    else:
        t[1, 1] = -1.0
    F = oracle.pobtaf(d, l, ar, t)
    _, info = lapack.dpotrf(dense.assemble(d, l, ar, t), lower=1)
    assert info > 0 and F.info == info


def test_generator_properties():
    d, l, ar, t = gen.make_bta(6, 8, 3, seed=2)
    d2, l2, ar2, t2 = gen.make_bta(6, 8, 3, seed=2)
    assert all(np.array_equal(x, y) for x, y in zip((d, l, ar, t), (d2, l2, ar2, t2)))
    assert np.array_equal(d, np.swapaxes(d, 1, 2)) and np.array_equal(t, t.T)
    A = dense.assemble(d, l, ar, t)
    off = np.abs(A).sum(axis=1) - np.abs(np.diag(A))
    assert np.all(np.diag(A) > off)              # strictly diagonally dominant -> SPD
    assert np.all(np.linalg.eigvalsh(A) > 0)


def test_psd_factor_generator_has_bta_pattern():
    n, b, a = 4, 3, 2
    fd, fl, fa, ft = gen.make_bta_psd_factor_blocks(n, b, a, seed=1)
    N = n * b + a
    F = np.zeros((N, N))
    for i in range(n):
        F[i * b:(i + 1) * b, i * b:(i + 1) * b] = fd[i]
        if i + 1 < n:
            F[(i + 1) * b:(i + 2) * b, i * b:(i + 1) * b] = fl[i]
        F[n * b:, i * b:(i + 1) * b] = fa[i]
    F[n * b:, n * b:] = ft
    G = F @ F.T
    blocks = gen.gram_of_factor_blocks(fd, fl, fa, ft)
    np.testing.assert_allclose(dense.assemble(*blocks), G, atol=1e-13)
    assert rel(dense.assemble(*dense.extract(G, n, b, a)), G) < 1e-15  # nothing outside the pattern


# Planted mistakes: each variant of a recursion step below is a plausible slip,
# and at least one pin above must reject it.
def _mutants():
    from scipy.linalg import solve_triangular as st
    return {
        "_trsm_right": lambda L, U: st(L, U.T, lower=True).T,                   # L^{-T} instead of L^{-1}
        "_trsm_right_trans": lambda L, B: st(L, B.T, lower=True, trans="T").T,  # L^{-1} instead of L^{-T}
        "_tri_inv": lambda L: st(L, np.eye(L.shape[0]), lower=True).T,          # transposed inverse
    }


@pytest.mark.parametrize("name", ["_trsm_right", "_trsm_right_trans", "_tri_inv"])
def test_planted_mistake_is_caught(monkeypatch, name):
    import oracle.bta_oracle as ob
    monkeypatch.setattr(ob, name, _mutants()[name])
    d, l, ar, t = mk(3, 5, 2, seed=1)
    F = ob.pobtaf(d, l, ar, t)
    X = ob.pobtasi(F)
    bad_f = any(rel(g, w) > 1e-8 for g, w in zip((F.diag, F.lower, F.arrow, F.tip), dense.dense_factor(d, l, ar, t)))
    bad_x = any(rel(g, w) > 1e-8 for g, w in zip(X, dense.dense_selinv(d, l, ar, t)))
    assert bad_f or bad_x
