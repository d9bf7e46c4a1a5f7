"""Failure reporting on the GPU without faulting it.

Every spin-wait of the library's cooperative and tensor-core kernels is bounded:
on timeout it records an error word, lets the kernel end, and bta_tc_status
reports it. Here a wait on a flag that nothing raises runs out (small poll
limit), the timeout is reported once, and the context stays usable for a
normal factorization afterwards. Non-SPD input (the numerical failure) is
covered in test_gpu_parity.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import bta_inputs as gen  # noqa: E402
import oracle  # noqa: E402
import paper_2503_17528_gb300 as bta  # noqa: E402
from gpu_util import TOL, dev, host, worst_block_error  # noqa: E402


def test_bounded_wait_timeout_is_reported_and_context_survives():
    assert bta.tc_status() == 0  # nothing pending from earlier tests
    assert bta.wait_selftest(1000) == 1
    assert bta.tc_status() == 0  # the flag was read and cleared
    d, l, ar, t = gen.make_bta(3, 160, 5, seed=11)
    D, Lw, A, Tp = dev(d), dev(l), dev(ar), dev(t)
    bta.factor(D, Lw, A, Tp)
    torch.cuda.synchronize()
    F = oracle.pobtaf(d, l, ar, t)
    got = (host(D), host(Lw), host(A), host(Tp))
    assert worst_block_error(got, (F.diag, F.lower, F.arrow, F.tip)) <= TOL
    assert bta.tc_status() == 0


def test_wait_selftest_argument_checks():
    with pytest.raises(bta.BTAError):
        bta.wait_selftest(0)
