"""torch.autograd binding: log det Q and x^T Q^{-1} x of an SPD BTA matrix Q.

Forward: bta_factor, bta_logdet, bta_solve (y = Q^{-1} x) and bta_dot.
Backward: bta_selinv on the saved factor (the selected inverse X) and
bta_grad_blocks, which forms d/d blocks = g_ld X - g_q y y^T on the pattern
(off-diagonal blocks doubled) and d/dx = 2 g_q y. The diagonal and tip blocks
are read through their lower triangles and take the symmetric gradient, so the
blocks of a symmetric Q should be passed symmetric (as a BTA precision matrix is).
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib
from . import api


def _p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None and t.numel() else None


class BTALogdetQuad(torch.autograd.Function):
    @staticmethod
    def forward(ctx, diag, lower, arrow, tip, x):
        L = [t.detach().clone() for t in (diag, lower, arrow, tip)]
        api.factor(*L)
        ld = api.logdet(L[0], L[3])
        y = x.detach().clone()
        api.solve(*L, y)
        quad = torch.empty((), dtype=torch.float64, device=x.device)
        ws = torch.empty(1024, dtype=torch.float64, device=x.device)
        lib = _lib.load()
        with torch.cuda.device(x.device):
            api._check(lib.bta_dot(x.numel(), _p(x.detach()), _p(y), _p(quad), _p(ws), ws.numel() * 8,
                                   api._stream(x.device)), "bta_dot")
        ctx.save_for_backward(*L, y)
        return ld, quad

    @staticmethod
    def backward(ctx, g_ld, g_q):
        Ld, Ll, La, Lt, y = ctx.saved_tensors
        X = [t.clone() for t in (Ld, Ll, La, Lt)]
        api.selinv(*X)
        G = [torch.empty_like(t) for t in X]
        gx = torch.empty_like(y)
        n, b = Ld.shape[0], Ld.shape[1]
        a = Lt.shape[0]
        alpha = float(g_ld) if g_ld is not None else 0.0
        beta = float(g_q) if g_q is not None else 0.0
        lib = _lib.load()
        with torch.cuda.device(y.device):
            api._check(lib.bta_grad_blocks(n, b, a, _p(X[0]), _p(X[1]), _p(X[2]), _p(X[3]), _p(y),
                                           alpha, beta, _p(G[0]), _p(G[1]), _p(G[2]), _p(G[3]),
                                           _p(gx), api._stream(y.device)), "bta_grad_blocks")
        return G[0], G[1], G[2], G[3], gx


def logdet_quad(diag, lower, arrow, tip, x):
    """(log det Q, x^T Q^{-1} x), differentiable in the blocks and in x."""
    return BTALogdetQuad.apply(diag, lower, arrow, tip, x)
