"""bta_logdet_noalloc against bta_logdet, through the C ABI.

bta_logdet_noalloc serves callers that cannot allocate device memory when they
need a log-determinant (their host framework owns the memory budget, or a
cudaMalloc in their loop would synchronize the device). It keeps its scratch in
a fixed array inside the library. This file is collected last on purpose: if it
fails, a run that stops at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

import bta_inputs as gen
import paper_2503_17528_gb300 as bta
from paper_2503_17528_gb300 import _lib

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _factored(n, b, a, seed):
    d, l, ar, t = gen.make_bta(n, b, a, seed=seed)
    blocks = [torch.from_numpy(x).to("cuda") for x in (d, l, ar, t)]
    bta.factor(*blocks)
    return blocks


def test_noalloc_logdet_matches_logdet_on_two_calls():
    lib = _lib.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    p = lambda x: ctypes.c_void_p(x.data_ptr())  # noqa: E731
    # Two calls in a row; the second has fewer blocks, so partial sums left in
    # the shared array by the first call must not leak into it.
    for (n, b, a, seed) in ((40, 48, 5, 1), (7, 33, 0, 2)):
        D, Lo, Ar, Ti = _factored(n, b, a, seed)
        tip = p(Ti) if a else None
        ref = torch.empty((), dtype=torch.float64, device="cuda")
        got = torch.full((), np.nan, dtype=torch.float64, device="cuda")
        assert lib.bta_logdet(n, b, a, p(D), tip, p(ref), stream) == 0
        assert lib.bta_logdet_noalloc(n, b, a, p(D), tip, p(got), stream) == 0
        torch.cuda.synchronize()
        r, g = ref.item(), got.item()
        assert np.isfinite(g)
        assert abs(g - r) <= TOL * max(1.0, abs(r)), (n, g, r)


@pytest.mark.parametrize("a", [1, 0])
def test_noalloc_logdet_at_the_block_limit(a):
    """n = 65536 fills the fixed array to its last slot (n partial sums, plus one
    for the tip when a > 0). Log-det only reads the diagonals of the factor's
    blocks, so a positive-diagonal stand-in for the factor serves as input."""
    lib = _lib.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    p = lambda x: ctypes.c_void_p(x.data_ptr())  # noqa: E731
    n, b = 65536, 1
    rng = np.random.default_rng(11 + a)
    D = torch.from_numpy(rng.uniform(0.5, 2.0, (n, b, b))).to("cuda")
    Ti = torch.from_numpy(rng.uniform(0.5, 2.0, (a, a))).to("cuda")
    tip = p(Ti) if a else None
    for _ in range(2):
        ref = torch.empty((), dtype=torch.float64, device="cuda")
        got = torch.full((), np.nan, dtype=torch.float64, device="cuda")
        assert lib.bta_logdet(n, b, a, p(D), tip, p(ref), stream) == 0
        assert lib.bta_logdet_noalloc(n, b, a, p(D), tip, p(got), stream) == 0
        torch.cuda.synchronize()
        r, g = ref.item(), got.item()
        assert np.isfinite(g) and abs(g - r) <= TOL * max(1.0, abs(r)), (g, r)
        D.mul_(1.5)  # the second call sees other values in every slot


def test_noalloc_logdet_rejects_too_many_blocks():
    lib = _lib.load()
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(dummy.data_ptr())
    assert lib.bta_logdet_noalloc(65537, 4, 0, p, None, p, None) == -1
