"""bta_factor_selinv_host / bta_factor_selinv_all: the whole per-matrix sequence
in one call (from host memory with the copies overlapped, or on device buffers).
The solve there uses the block inverses L_ii^{-1} of the selected inversion's
prologue and runs beside the rest of it, so its result agrees with bta_solve's
(substitution) to rounding, while X and log det are bit-identical.

Checked against the oracle (X on the pattern, log det, solve) and against the
device-buffer entry points, over the fused FP64 step (b >= 128), the small-b
path, several input chunks (b = 520: 7 blocks per ~32 MB chunk), a = 0, n = 1
and no right-hand side.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import bta_inputs as gen  # noqa: E402
import oracle  # noqa: E402
import paper_2503_17528_gb300 as bta  # noqa: E402
from gpu_util import TOL, dev, host, rel_fro, worst_block_error  # noqa: E402


def _pinned(x):
    return torch.from_numpy(np.ascontiguousarray(x)).pin_memory()


@pytest.mark.parametrize("n,b,a,nrhs", [(4, 160, 5, 3), (3, 40, 2, 1), (9, 520, 3, 4), (3, 130, 0, 2),
                                        (1, 200, 7, 1), (2, 128, 4, 0)])
def test_host_pipeline_matches_oracle_and_device_path(n, b, a, nrhs):
    d, l, ar, t = gen.make_bta(n, b, a, seed=100 + n + b + a)
    r = gen.make_rhs(n, b, a, max(nrhs, 1), seed=7)
    H = [_pinned(x) for x in (d, l, ar, t)]
    hr = _pinned(r) if nrhs else None
    out = bta.factor_selinv_host(*H, rhs=hr)
    torch.cuda.synchronize()
    assert bta.get_info() == 0
    F = oracle.pobtaf(d, l, ar, t)
    Xo = oracle.pobtasi(F)
    got = tuple(o.numpy() for o in out[:4])
    assert worst_block_error(got, Xo) <= TOL
    ldo = oracle.logdet(F)
    assert abs(float(out[5]) - ldo) <= TOL * max(1.0, abs(ldo))
    if nrhs:
        assert rel_fro(out[4].numpy(), oracle.solve(F, r)) <= TOL
    # the inputs are untouched
    assert np.array_equal(H[0].numpy(), d) and np.array_equal(H[2].numpy(), ar)
    # same as the device-buffer path
    D, Lw, A, Tp = dev(d), dev(l), dev(ar), dev(t)
    bta.factor(D, Lw, A, Tp)
    bta.selinv(D, Lw, A, Tp)
    torch.cuda.synchronize()
    assert worst_block_error(got, (host(D), host(Lw), host(A), host(Tp))) <= 1e-13


def test_host_pipeline_twice_in_a_row_is_bitwise_repeatable():
    d, l, ar, t = gen.make_bta(5, 256, 6, seed=3)
    r = gen.make_rhs(5, 256, 6, 2, seed=4)
    H = [_pinned(x) for x in (d, l, ar, t)]
    o1 = bta.factor_selinv_host(*H, rhs=_pinned(r))
    torch.cuda.synchronize()
    o1 = [x.clone() for x in o1 if x is not None]
    o2 = bta.factor_selinv_host(*H, rhs=_pinned(r))
    torch.cuda.synchronize()
    for a_, b_ in zip(o1, [x for x in o2 if x is not None]):
        assert torch.equal(a_, b_)


@pytest.mark.parametrize("n,b,a,nrhs", [(4, 160, 5, 3), (3, 40, 2, 1), (2, 256, 0, 2), (1, 130, 9, 0)])
def test_device_all_in_one_matches_separate_calls(n, b, a, nrhs):
    d, l, ar, t = gen.make_bta(n, b, a, seed=200 + n + b + a)
    r = gen.make_rhs(n, b, a, max(nrhs, 1), seed=9)
    D, Lw, A, Tp = dev(d), dev(l), dev(ar), dev(t)
    R = dev(r) if nrhs else None
    ld = bta.factor_selinv_all(D, Lw, A, Tp, rhs=R)
    torch.cuda.synchronize()
    assert bta.get_info() == 0
    F = oracle.pobtaf(d, l, ar, t)
    assert worst_block_error((host(D), host(Lw), host(A), host(Tp)), oracle.pobtasi(F)) <= TOL
    ldo = oracle.logdet(F)
    assert abs(float(ld.item()) - ldo) <= TOL * max(1.0, abs(ldo))
    if nrhs:
        assert rel_fro(host(R), oracle.solve(F, r)) <= TOL
    # X and log det bit-identical to the four separate calls; the solution to rounding
    D2, L2, A2, T2 = dev(d), dev(l), dev(ar), dev(t)
    bta.factor(D2, L2, A2, T2)
    ld2 = bta.logdet(D2, T2)
    if nrhs:
        R2 = dev(r)
        bta.solve(D2, L2, A2, T2, R2)
    bta.selinv(D2, L2, A2, T2)
    torch.cuda.synchronize()
    for x1, x2 in ((D, D2), (Lw, L2), (A, A2), (Tp, T2)):
        assert torch.equal(x1, x2)
    assert float(ld.item()) == float(ld2.item())
    if nrhs:
        assert rel_fro(host(R), host(R2)) <= 1e-13
