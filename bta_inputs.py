"""Seeded synthetic inputs for BTA (block-tridiagonal with arrowhead) matrices.

This module is shared by the tests, the benchmark and the smoke check. It only
draws random numbers and assembles inputs; it contains none of the method's
arithmetic (no factorization, no inversion), so both the CPU oracle and the
CUDA path can take their inputs from here without sharing any computation.

Block storage (FP64, C-contiguous), with N = n*b + a:
    diag  [n, b, b]    A_{i,i}            (symmetric)
    lower [n-1, b, b]  A_{i+1,i}          (A_{i,i+1} = lower[i]^T)
    arrow [n, a, b]    A_{n,i}            (the arrowhead block row; column = transpose)
    tip   [a, a]       A_{n,n}            (symmetric)

Generator (the workloads of the paper's Section 5.2 are INLA precision matrices
that are not available; these matrices stand in for them with the same block
shapes): off-diagonal and arrow blocks are N(0,1)/sqrt(b); each diagonal block
is a symmetric N(0,1)/sqrt(b) block (lower triangle drawn, mirrored) plus c*I
with c = scale * R + add, where R is the largest absolute off-diagonal row sum
over the block's rows of the assembled matrix (in-block, sub-, super-diagonal
and arrow-column entries). The tip is a symmetric N(0,1)/sqrt(b) block plus its
own shift computed the same way over the arrowhead rows. Draw order from
numpy.random.default_rng(seed): diag, lower, arrow, tip.
"""
from __future__ import annotations

import numpy as np

# Dominance presets (scale, add) for the three plain workloads.
SHIFT_PLUS_ONE = (1.0, 1.0)      # c = 1 + R     (n=16, b=32, a=4)
SHIFT_1_01 = (1.01, 0.0)         # c = 1.01 R    (n=365, b=1024, a=8)
SHIFT_1_001 = (1.001, 0.0)       # c = 1.001 R   (n=256, b=2048, a=16)


def _symmetric_from_lower(g: np.ndarray) -> np.ndarray:
    """Keep tril(g) and mirror it (works on a stack of square blocks)."""
    lo = np.tril(g)
    return lo + np.swapaxes(np.tril(g, -1), -1, -2)


def make_bta(n: int, b: int, a: int, seed: int = 0, shift=SHIFT_PLUS_ONE):
    """Return (diag, lower, arrow, tip) of a seeded, diagonally dominant SPD BTA matrix."""
    if n < 1 or b < 1 or a < 0:
        raise ValueError("need n >= 1, b >= 1, a >= 0")
    scale, add = shift
    rng = np.random.default_rng(seed)
    s = 1.0 / np.sqrt(b)
    diag = _symmetric_from_lower(rng.standard_normal((n, b, b)) * s)
    lower = rng.standard_normal((n - 1, b, b)) * s
    arrow = rng.standard_normal((n, a, b)) * s
    tip = _symmetric_from_lower(rng.standard_normal((a, a)) * s)

    absd = np.abs(diag)
    r = absd.sum(axis=2) - np.abs(np.diagonal(diag, axis1=1, axis2=2))  # [n, b]
    if n > 1:
        absl = np.abs(lower)
        r[1:] += absl.sum(axis=2)   # row k of A_{i,i-1} = row k of lower[i-1]
        r[:-1] += absl.sum(axis=1)  # row k of A_{i,i+1} = column k of lower[i]
    if a > 0:
        r += np.abs(arrow).sum(axis=1)  # row k of A_{i,n} = column k of arrow[i]
    c = scale * r.max(axis=1) + add
    idx = np.arange(b)
    diag[:, idx, idx] += c[:, None]

    if a > 0:
        rt = np.abs(tip).sum(axis=1) - np.abs(np.diagonal(tip)) + np.abs(arrow).sum(axis=(0, 2))
        tip[np.arange(a), np.arange(a)] += scale * rt.max() + add
    return diag, lower, arrow, tip


def make_rhs(n: int, b: int, a: int, nrhs: int, seed: int = 1) -> np.ndarray:
    """N(0,1) right-hand sides, shape [n*b + a, nrhs]."""
    return np.random.default_rng(seed).standard_normal((n * b + a, nrhs))


def make_bta_psd_factor_blocks(n: int, b: int, a: int, seed: int):
    """Random factor F (block lower bidiagonal + arrowhead row + tip), N(0,1)/sqrt(b).

    Returns (fd [n,b,b], fl [n-1,b,b], fa [n,a,b], ft [a,a]); F F^T has exactly
    the BTA pattern and is positive semidefinite. Used to build the T and S
    matrices of the differentiable workload Q(theta) = t1*T + t2*S + t3*I.
    """
    rng = np.random.default_rng(seed)
    s = 1.0 / np.sqrt(b)
    fd = rng.standard_normal((n, b, b)) * s
    fl = rng.standard_normal((n - 1, b, b)) * s
    fa = rng.standard_normal((n, a, b)) * s
    ft = rng.standard_normal((a, a)) * s
    return fd, fl, fa, ft


def gram_of_factor_blocks(fd, fl, fa, ft):
    """Blocks of F F^T for the factor blocks above (input construction only)."""
    n, b = fd.shape[0], fd.shape[1]
    a = ft.shape[0]
    diag = np.einsum("nij,nkj->nik", fd, fd)
    if n > 1:
        diag[1:] += np.einsum("nij,nkj->nik", fl, fl)
    lower = np.einsum("nij,nkj->nik", fl, fd[:-1]) if n > 1 else np.zeros((0, b, b))
    arrow = np.einsum("nij,nkj->nik", fa, fd) if a else np.zeros((n, 0, b))
    if a and n > 1:
        arrow[1:] += np.einsum("nij,nkj->nik", fa[:-1], fl)
    tip = np.einsum("nij,nkj->ik", fa, fa) + ft @ ft.T if a else np.zeros((0, 0))
    return diag, lower, arrow, tip


def _assemble_symmetric(diag, lower, arrow, tip):
    """Dense N x N symmetric matrix with the given blocks (input construction)."""
    n, b = diag.shape[0], diag.shape[1]
    a = tip.shape[0]
    N = n * b + a
    A = np.zeros((N, N))
    for i in range(n):
        A[i * b:(i + 1) * b, i * b:(i + 1) * b] = diag[i]
        if i + 1 < n:
            A[(i + 1) * b:(i + 2) * b, i * b:(i + 1) * b] = lower[i]
            A[i * b:(i + 1) * b, (i + 1) * b:(i + 2) * b] = lower[i].T
        if a:
            A[n * b:, i * b:(i + 1) * b] = arrow[i]
            A[i * b:(i + 1) * b, n * b:] = arrow[i].T
    if a:
        A[n * b:, n * b:] = tip
    return A


def make_bta_stress(n: int, b: int, a: int, seed: int = 0, kappa: float = 1e6):
    """A badly conditioned SPD BTA matrix for error statements of the reduced-
    precision modes (the dominance-shifted generator gives condition numbers of
    only 3 to 8). The blocks are drawn as in make_bta, without the dominance
    shift; then every diagonal entry gets the shift s that sets the spectral
    condition number of the whole matrix to `kappa`:
    (lambda_max + s) / (lambda_min + s) = kappa, with lambda_min, lambda_max the
    extreme eigenvalues of the random symmetric part. Dense eigenvalues: for
    N = n*b + a up to 6000. Returns (diag, lower, arrow, tip, kappa_achieved).
    """
    if n < 1 or b < 1 or a < 0:
        raise ValueError("need n >= 1, b >= 1, a >= 0")
    if n * b + a > 6000:
        raise ValueError("make_bta_stress computes dense eigenvalues: N = n*b + a must be <= 6000")
    if not kappa > 1.0:
        raise ValueError("kappa must exceed 1")
    rng = np.random.default_rng(seed)
    s = 1.0 / np.sqrt(b)
    diag = _symmetric_from_lower(rng.standard_normal((n, b, b)) * s)
    lower = rng.standard_normal((n - 1, b, b)) * s
    arrow = rng.standard_normal((n, a, b)) * s
    tip = _symmetric_from_lower(rng.standard_normal((a, a)) * s)
    lam = np.linalg.eigvalsh(_assemble_symmetric(diag, lower, arrow, tip))
    lo, hi = float(lam[0]), float(lam[-1])
    shift = (hi - kappa * lo) / (kappa - 1.0)
    idx = np.arange(b)
    diag[:, idx, idx] += shift
    if a:
        tip[np.arange(a), np.arange(a)] += shift
    return diag, lower, arrow, tip, (hi + shift) / (lo + shift)
