"""Helpers shared by the GPU tests (device transfer and block comparisons)."""
import numpy as np
import torch

TOL = 1e-10  # relative Frobenius error per block, FP64


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


def host(t):
    return t.detach().cpu().numpy()


def rel_fro(got, want):
    nw = np.linalg.norm(want)
    return np.linalg.norm(got - want) / (nw if nw > 0 else 1.0)


def worst_block_error(got_blocks, want_blocks):
    """Largest per-block relative Frobenius error over (diag, lower, arrow, tip)."""
    worst = 0.0
    for g, w in zip(got_blocks, want_blocks):
        g = np.asarray(g)
        w = np.asarray(w)
        assert g.shape == w.shape, (g.shape, w.shape)
        if w.size == 0:
            continue
        if w.ndim == 3:
            for k in range(w.shape[0]):
                worst = max(worst, rel_fro(g[k], w[k]))
        else:
            worst = max(worst, rel_fro(g, w))
    return worst
