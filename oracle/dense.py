"""Dense definitions of what the BTA path computes (test infrastructure only).

The selected inversion is exact (Section 2.2 of the paper: POBTASI returns the
"true inverse" blocks of A on the non-zero block pattern of A), so its result
is, up to rounding order, the dense inverse of the assembled matrix restricted
to that pattern. Likewise the block Cholesky factor has no fill-in outside the
pattern (Section 1), so it equals the dense Cholesky factor restricted to it.
These functions write those definitions out with numpy.linalg and are the
brute-force truth for small N.
"""
from __future__ import annotations

import numpy as np


def assemble(diag, lower, arrow, tip) -> np.ndarray:
    """Full symmetric N x N matrix (N = n*b + a) from the lower-pattern blocks.

    Only the lower triangles of diag[i] and tip are used (mirrored), matching
    what a lower Cholesky factorization reads.
    """
    n, b = diag.shape[0], diag.shape[1]
    a = tip.shape[0]
    N = n * b + a
    A = np.zeros((N, N))
    for i in range(n):
        d = np.tril(diag[i])
        A[i * b:(i + 1) * b, i * b:(i + 1) * b] = d + np.tril(d, -1).T
        if i + 1 < n:
            A[(i + 1) * b:(i + 2) * b, i * b:(i + 1) * b] = lower[i]
            A[i * b:(i + 1) * b, (i + 1) * b:(i + 2) * b] = lower[i].T
        if a:
            A[n * b:, i * b:(i + 1) * b] = arrow[i]
            A[i * b:(i + 1) * b, n * b:] = arrow[i].T
    if a:
        t = np.tril(tip)
        A[n * b:, n * b:] = t + np.tril(t, -1).T
    return A


def extract(M: np.ndarray, n: int, b: int, a: int):
    """Blocks of a dense N x N matrix on the (lower) BTA pattern."""
    diag = np.stack([M[i * b:(i + 1) * b, i * b:(i + 1) * b] for i in range(n)])
    lower = np.stack([M[(i + 1) * b:(i + 2) * b, i * b:(i + 1) * b] for i in range(n - 1)]) \
        if n > 1 else np.zeros((0, b, b))
    arrow = np.stack([M[n * b:, i * b:(i + 1) * b] for i in range(n)])
    tip = M[n * b:, n * b:].copy()
    return diag, lower, arrow, tip


def dense_factor(diag, lower, arrow, tip):
    """L = chol(A) restricted to the pattern (numpy.linalg.cholesky of the assembly)."""
    n, b = diag.shape[0], diag.shape[1]
    a = tip.shape[0]
    return extract(np.linalg.cholesky(assemble(diag, lower, arrow, tip)), n, b, a)


def dense_selinv(diag, lower, arrow, tip):
    """X = A^{-1} restricted to the BTA pattern (numpy.linalg.inv of the assembly)."""
    n, b = diag.shape[0], diag.shape[1]
    a = tip.shape[0]
    return extract(np.linalg.inv(assemble(diag, lower, arrow, tip)), n, b, a)


def dense_logdet(diag, lower, arrow, tip) -> float:
    sign, ld = np.linalg.slogdet(assemble(diag, lower, arrow, tip))
    if sign <= 0:
        raise np.linalg.LinAlgError("matrix is not positive definite")
    return float(ld)


def dense_solve(diag, lower, arrow, tip, rhs) -> np.ndarray:
    return np.linalg.solve(assemble(diag, lower, arrow, tip), rhs)
