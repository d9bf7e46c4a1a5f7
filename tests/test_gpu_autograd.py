"""Differentiation: L(theta) = log det Q(theta) - x^T Q(theta)^{-1} x with
Q(theta) = t1 T + t2 S + t3 I over a BTA pattern (T, S = F F^T of random
block-bidiagonal-plus-arrowhead factors), through BTALogdetQuad, whose backward
is the selected inverse plus one solve.

Checks: dL/dtheta against central finite differences (h = 1e-6) of the forward,
against the gradient assembled from the CPU oracle's selected inverse and
solve, and (tiny sizes) against dense tr(Q^{-1} dQ) + y^T dQ y.
"""
import numpy as np
import pytest
import torch

import bta_inputs as gen
import oracle
from oracle import dense
import paper_2503_17528_gb300 as bta
from gpu_util import dev

pytestmark = pytest.mark.gpu


def _problem(n, b, a, seed):
    T = gen.gram_of_factor_blocks(*gen.make_bta_psd_factor_blocks(n, b, a, seed=seed))
    S = gen.gram_of_factor_blocks(*gen.make_bta_psd_factor_blocks(n, b, a, seed=seed + 1))
    x = np.random.default_rng(seed + 2).standard_normal(n * b + a)
    return T, S, x


def _q_blocks(theta, T, S, eye_d, eye_t):
    Td, Tl, Ta, Tt = T
    Sd, Sl, Sa, St = S
    return (theta[0] * Td + theta[1] * Sd + theta[2] * eye_d,
            theta[0] * Tl + theta[1] * Sl,
            theta[0] * Ta + theta[1] * Sa,
            theta[0] * Tt + theta[1] * St + theta[2] * eye_t)


def _loss_and_grad(theta_np, T, S, x):
    n, b = T[0].shape[0], T[0].shape[1]
    a = T[3].shape[0]
    Tg = [dev(t) for t in T]
    Sg = [dev(t) for t in S]
    eye_d = torch.eye(b, dtype=torch.float64, device="cuda").expand(n, b, b)
    eye_t = torch.eye(a, dtype=torch.float64, device="cuda")
    theta = torch.tensor(theta_np, dtype=torch.float64, device="cuda", requires_grad=True)
    Q = [q.contiguous() for q in _q_blocks(theta, Tg, Sg, eye_d, eye_t)]
    ld, quad = bta.logdet_quad(*Q, dev(x))
    L = ld - quad
    L.backward()
    torch.cuda.synchronize()
    return float(L.item()), theta.grad.detach().cpu().numpy()


def _loss_only(theta_np, T, S, x):
    Q = [np.ascontiguousarray(q) for q in _q_blocks(theta_np, T, S, np.eye(T[0].shape[1]), np.eye(T[3].shape[0]))]
    with torch.no_grad():
        ld, quad = bta.logdet_quad(*[dev(q) for q in Q], dev(x))
    return float(ld.item()) - float(quad.item())


def _oracle_grad(theta, T, S, x):
    n, b = T[0].shape[0], T[0].shape[1]
    a = T[3].shape[0]
    Q = _q_blocks(theta, T, S, np.eye(b), np.eye(a))
    F = oracle.pobtaf(*Q)
    Xd, Xl, Xa, Xt = oracle.pobtasi(F)
    y = oracle.solve(F, x)
    yb = y[: n * b].reshape(n, b)
    yn = y[n * b:]
    # dL/dQ = Q^{-1} + y y^T on the pattern; off-diagonal blocks counted twice
    Gd = Xd + np.einsum("ir,ic->irc", yb, yb)
    Gl = Xl + np.einsum("ir,ic->irc", yb[1:], yb[:-1])
    Ga = Xa + np.einsum("r,ic->irc", yn, yb)
    Gt = Xt + np.outer(yn, yn)
    dQ = [T, S, (np.broadcast_to(np.eye(b), (n, b, b)), np.zeros_like(T[1]), np.zeros_like(T[2]), np.eye(a))]
    out = []
    for d in dQ:
        out.append(np.sum(Gd * d[0]) + 2 * np.sum(Gl * d[1]) + 2 * np.sum(Ga * d[2]) + np.sum(Gt * d[3]))
    return np.array(out)


@pytest.mark.parametrize("n,b,a", [(3, 40, 5), (6, 64, 8), (2, 33, 0)])
def test_grad_small_vs_dense_fd_and_oracle(n, b, a):
    T, S, x = _problem(n, b, a, seed=n + b)
    theta = np.array([1.0, 0.5, 0.1])
    L, g = _loss_and_grad(theta, T, S, x)
    # dense definition
    Qd = dense.assemble(*_q_blocks(theta, T, S, np.eye(b), np.eye(a)))
    Qi = np.linalg.inv(Qd)
    y = Qi @ x
    Ld = np.linalg.slogdet(Qd)[1] - x @ y
    assert abs(L - Ld) <= 1e-10 * abs(Ld)
    for k, dQb in enumerate([dense.assemble(*T), dense.assemble(*S), np.eye(n * b + a)]):
        want = np.trace(Qi @ dQb) + y @ dQb @ y
        assert abs(g[k] - want) <= 1e-9 * max(1.0, abs(want)), (k, g[k], want)
    np.testing.assert_allclose(g, _oracle_grad(theta, T, S, x), rtol=1e-9)
    h = 1e-6
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        fd = (_loss_only(theta + e, T, S, x) - _loss_only(theta - e, T, S, x)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(g[k])), (k, fd, g[k])


def test_grad_n128_b512_a8_vs_fd_and_oracle():
    """The differentiable workload: n=128, b=512, a=8, theta = (1.0, 0.5, 0.1)."""
    n, b, a = 128, 512, 8
    T, S, x = _problem(n, b, a, seed=0)
    theta = np.array([1.0, 0.5, 0.1])
    L, g = _loss_and_grad(theta, T, S, x)
    np.testing.assert_allclose(g, _oracle_grad(theta, T, S, x), rtol=1e-9)
    h = 1e-6
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        fd = (_loss_only(theta + e, T, S, x) - _loss_only(theta - e, T, S, x)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(g[k])), (k, fd, g[k])


def test_block_gradients_match_oracle():
    n, b, a = 4, 48, 6
    d, l, ar, t = gen.make_bta(n, b, a, seed=13)
    x = np.random.default_rng(3).standard_normal(n * b + a)
    blocks = [dev(v).requires_grad_(True) for v in (d, l, ar, t)]
    xg = dev(x).requires_grad_(True)
    ld, quad = bta.logdet_quad(*blocks, xg)
    (2.0 * ld + 3.0 * quad).backward()
    F = oracle.pobtaf(d, l, ar, t)
    Xd, Xl, Xa, Xt = oracle.pobtasi(F)
    y = oracle.solve(F, x)
    yb, yn = y[: n * b].reshape(n, b), y[n * b:]
    want = [2 * Xd - 3 * np.einsum("ir,ic->irc", yb, yb),
            2 * (2 * Xl - 3 * np.einsum("ir,ic->irc", yb[1:], yb[:-1])),
            2 * (2 * Xa - 3 * np.einsum("r,ic->irc", yn, yb)),
            2 * Xt - 3 * np.outer(yn, yn)]
    for gtens, w in zip(blocks, want):
        np.testing.assert_allclose(gtens.grad.cpu().numpy(), w, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(xg.grad.cpu().numpy(), 6.0 * y, rtol=1e-10)
