"""Block-sequential FP64 oracle for the BTA path (test infrastructure only).

Follows the paper's listings in their order and notation, with LAPACK POTRF
(scipy.linalg.lapack.dpotrf) and triangular solves (scipy.linalg.solve_triangular)
as library steps; no blocking, fusion or reordering beyond what the listings state.

  pobtaf   Algorithm 1 (POBTAF), Section 2.2.
  pobtasi  Algorithm 2 (POBTASI), Section 2.2.
  logdet   log det A = 2 * sum log diag(L); not in the paper (a property of the
           Cholesky factor: det A = det(L)^2).
  solve    A x = r through L y = r, then L^T x = y over the BTA pattern; not in
           the paper (block forward / backward substitution on the factor).

Readings of the paper used here:
  * "TRSM(L_ii, B)" in Algorithm 1 means B L_ii^{-T} (right side, transposed),
    and in Algorithm 2 it means U L_ii^{-1} (right side, not transposed): the
    first solves L_{i+1,i} L_ii^T = A_{i+1,i}; the second follows from X L = L^{-T}.
  * The dagger is the (conjugate) transpose; all data here are real.
  * a = 0 is the plain block-tridiagonal case: every arrow and tip step is skipped.
  * A non-positive pivot returns LAPACK-style info = global 1-based row of the
    failing leading minor (block i, local row j -> i*b + j; tip -> n*b + j); the
    blocks from the failing one on are returned as NaN.
"""
from __future__ import annotations

from typing import NamedTuple

import numpy as np
from scipy.linalg import lapack, solve_triangular


class BTAFactor(NamedTuple):
    diag: np.ndarray   # L_ii            [n, b, b] (lower triangular)
    lower: np.ndarray  # L_{i+1,i}       [n-1, b, b]
    arrow: np.ndarray  # L_{n,i}         [n, a, b]
    tip: np.ndarray    # L_{n,n}         [a, a] (lower triangular)
    info: int


def _potrf(A: np.ndarray):
    """Lower Cholesky factor (LAPACK dpotrf, uplo='L'); reads only tril(A)."""
    c, info = lapack.dpotrf(A, lower=1, clean=1)
    return c, int(info)


def _trsm_right_trans(L: np.ndarray, B: np.ndarray) -> np.ndarray:
    """B L^{-T}: the X with X L^T = B, i.e. L X^T = B^T."""
    return solve_triangular(L, B.T, lower=True).T


def _trsm_right(L: np.ndarray, U: np.ndarray) -> np.ndarray:
    """U L^{-1}: the X with X L = U, i.e. L^T X^T = U^T."""
    return solve_triangular(L, U.T, lower=True, trans="T").T


def _tri_inv(L: np.ndarray) -> np.ndarray:
    """L^{-1} for lower-triangular L (triangular solve against the identity)."""
    return solve_triangular(L, np.eye(L.shape[0]), lower=True)


def _fail(Ld, Ll, La, Lt, i, info):
    """NaN-fill every block from block column i on and return the failed factor."""
    Ld[i:] = np.nan
    Ll[i:] = np.nan
    La[i:] = np.nan
    Lt[...] = np.nan
    return BTAFactor(Ld, Ll, La, Lt, info)


def pobtaf(diag, lower, arrow, tip) -> BTAFactor:
    """Algorithm 1 (POBTAF): block-sequential block Cholesky of a BTA matrix.

    For i = 0..n-2: L_ii = POTRF(A_ii); L_{i+1,i} = A_{i+1,i} L_ii^{-T};
    L_{n,i} = A_{n,i} L_ii^{-T}; A_{i+1,i+1} -= L_{i+1,i} L_{i+1,i}^T;
    A_{n,i+1} -= L_{n,i} L_{i+1,i}^T; A_{n,n} -= L_{n,i} L_{n,i}^T.
    Then the last block column and POTRF of the updated tip.
    Inputs are not modified.
    """
    n, b = diag.shape[0], diag.shape[1]
    a = tip.shape[0]
    Ad = np.array(diag, dtype=np.float64, copy=True)
    Al = np.array(lower, dtype=np.float64, copy=True).reshape(max(n - 1, 0), b, b)
    Aa = np.array(arrow, dtype=np.float64, copy=True).reshape(n, a, b)
    At = np.array(tip, dtype=np.float64, copy=True).reshape(a, a)

    for i in range(n - 1):
        Ad[i], info = _potrf(Ad[i])
        if info:
            return _fail(Ad, Al, Aa, At, i, i * b + info)
        Al[i] = _trsm_right_trans(Ad[i], Al[i])
        if a:
            Aa[i] = _trsm_right_trans(Ad[i], Aa[i])
        Ad[i + 1] -= Al[i] @ Al[i].T
        if a:
            Aa[i + 1] -= Aa[i] @ Al[i].T
            At -= Aa[i] @ Aa[i].T

    last = n - 1
    Ad[last], info = _potrf(Ad[last])
    if info:
        return _fail(Ad, Al, Aa, At, last, last * b + info)
    if a:
        Aa[last] = _trsm_right_trans(Ad[last], Aa[last])
        At -= Aa[last] @ Aa[last].T
        At, info = _potrf(At)
        if info:
            At[...] = np.nan
            return BTAFactor(Ad, Al, Aa, At, n * b + info)
    return BTAFactor(Ad, Al, Aa, At, 0)


def pobtasi(F: BTAFactor):
    """Algorithm 2 (POBTASI): selected inverse X of A from its block Cholesky factor.

    Returns (Xd [n,b,b], Xl [n-1,b,b], Xa [n,a,b], Xt [a,a]) = the blocks of A^{-1}
    at the positions of A's lower non-zero blocks. X_ii is returned as computed
    (not symmetrized).
    """
    Ld, Ll, La, Lt = F.diag, F.lower, F.arrow, F.tip
    n, b = Ld.shape[0], Ld.shape[1]
    a = Lt.shape[0]
    Xd = np.empty_like(Ld)
    Xl = np.empty_like(Ll)
    Xa = np.empty_like(La)
    Xt = np.empty_like(Lt)

    if a:
        Lt_inv = _tri_inv(Lt)
        Xt[...] = Lt_inv.T @ Lt_inv                       # X_nn = L_nn^{-T} L_nn^{-1}

    last = n - 1
    U = _tri_inv(Ld[last]).T                              # L_{n-1,n-1}^{-T}
    if a:
        Xa[last] = _trsm_right(Ld[last], -Xt @ La[last])  # X_{n,n-1}
        U = U - Xa[last].T @ La[last]
    Xd[last] = _trsm_right(Ld[last], U)                   # X_{n-1,n-1}

    for i in range(n - 2, -1, -1):
        U = -Xd[i + 1] @ Ll[i]
        if a:
            U -= Xa[i + 1].T @ La[i]
        Xl[i] = _trsm_right(Ld[i], U)                     # X_{i+1,i}
        if a:
            U = -Xa[i + 1] @ Ll[i] - Xt @ La[i]
            Xa[i] = _trsm_right(Ld[i], U)                 # X_{n,i}
        U = _tri_inv(Ld[i]).T - Xl[i].T @ Ll[i]
        if a:
            U -= Xa[i].T @ La[i]
        Xd[i] = _trsm_right(Ld[i], U)                     # X_{i,i}
    return Xd, Xl, Xa, Xt


def logdet(F: BTAFactor) -> float:
    """log det A = 2 * (sum_i sum_k log (L_ii)_kk + sum_k log (L_nn)_kk), in block then row order."""
    total = 0.0
    for i in range(F.diag.shape[0]):
        total += float(np.sum(np.log(np.diagonal(F.diag[i]))))
    if F.tip.shape[0]:
        total += float(np.sum(np.log(np.diagonal(F.tip))))
    return 2.0 * total


def solve(F: BTAFactor, rhs: np.ndarray) -> np.ndarray:
    """x = A^{-1} rhs by block forward substitution (L y = r) and backward (L^T x = y).

    Forward:  y_0 = L_00^{-1} r_0;  y_i = L_ii^{-1} (r_i - L_{i,i-1} y_{i-1});
              y_n = L_nn^{-1} (r_n - sum_i L_{n,i} y_i).
    Backward: x_n = L_nn^{-T} y_n;
              x_i = L_ii^{-T} (y_i - L_{i+1,i}^T x_{i+1} - L_{n,i}^T x_n).
    rhs: [n*b + a, nrhs] (a 1-D vector is accepted).
    """
    Ld, Ll, La, Lt = F.diag, F.lower, F.arrow, F.tip
    n, b = Ld.shape[0], Ld.shape[1]
    a = Lt.shape[0]
    r = np.array(rhs, dtype=np.float64, copy=True)
    vec = r.ndim == 1
    if vec:
        r = r[:, None]
    y = np.empty_like(r)
    for i in range(n):
        t = r[i * b:(i + 1) * b].copy()
        if i > 0:
            t -= Ll[i - 1] @ y[(i - 1) * b:i * b]
        y[i * b:(i + 1) * b] = solve_triangular(Ld[i], t, lower=True)
    if a:
        t = r[n * b:].copy()
        for i in range(n):
            t -= La[i] @ y[i * b:(i + 1) * b]
        y[n * b:] = solve_triangular(Lt, t, lower=True)

    x = np.empty_like(y)
    if a:
        x[n * b:] = solve_triangular(Lt, y[n * b:], lower=True, trans="T")
    for i in range(n - 1, -1, -1):
        t = y[i * b:(i + 1) * b].copy()
        if i + 1 < n:
            t -= Ll[i].T @ x[(i + 1) * b:(i + 2) * b]
        if a:
            t -= La[i].T @ x[n * b:]
        x[i * b:(i + 1) * b] = solve_triangular(Ld[i], t, lower=True, trans="T")
    return x[:, 0] if vec else x
