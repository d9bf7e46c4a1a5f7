"""The benchmark's algorithmic flop and byte models, checked without a GPU.

Every TFLOP/s figure divides these counts by a measured time, so they are pinned
here: against the closed-form totals of the five workloads (4.06e6, 2.77e12,
1.55e13 and 1.22e11 flops for factor + selected inversion), against the leading
order 7 n b^3 of the method, and against hand counts on tiny cases.
"""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


@pytest.mark.parametrize("n,b,a,total", [(16, 32, 4, 4.06e6), (365, 1024, 8, 2.77e12),
                                         (256, 2048, 16, 1.55e13), (128, 512, 8, 1.22e11)])
def test_flop_model_matches_the_workload_totals(bench, n, b, a, total):
    f = bench.flops_factor(n, b, a) + bench.flops_selinv(n, b, a)
    assert abs(f / total - 1) < 5e-3


def test_flop_model_leading_order(bench):
    # per block: POTRF b^3/3 + TRSM b^3 + SYRK b^3 in the factor, TRTRI-based
    # M_i 2b^3/3 + G_i b^3 + the chain 3b^3 in the selected inversion: 7 b^3
    n, b = 50, 8192
    f = bench.flops_factor(n, b, 0) + bench.flops_selinv(n, b, 0)
    assert abs(f / (7 * n * b**3) - 1) < 0.03
    # one dense block: Cholesky b^3/3 and L^{-T} L^{-1} 2b^3/3
    assert bench.flops_factor(1, 64, 0) + bench.flops_selinv(1, 64, 0) == pytest.approx(64**3)


def test_solve_byte_model_hand_count(bench):
    # n=2, b=2, a=1, one right-hand side: per sweep the factor's lower
    # triangles (2 x 3), the off-diagonal block (4), the arrow blocks (2 x 2)
    # and the tip (1): 15 doubles; the right-hand side (5 doubles) is read and
    # written in each of the two sweeps.
    assert bench.solve_bytes(2, 2, 1, 1) == 8 * (2 * 15 + 4 * 5)
    assert bench.solve_bytes(365, 1024, 8, 4) == pytest.approx(9.27e9, rel=1e-3)


def test_traffic_table_names_live_kernels(bench):
    """Every stored DRAM-traffic figure names a kernel whose source text is found,
    and is reported only while that text is unchanged since the capture."""
    for name, e in bench.TRAFFIC.items():
        assert e["bytes_per_launch"] > 0 and e["capture"].startswith("profiles/")
        assert os.path.exists(os.path.join(ROOT, e["capture"].split(":")[0]))
        assert len(bench.kernel_digest(e["source"], e["symbol"])) == 16
        live = bench.kernel_digest(e["source"], e["symbol"]) == e["digest"]
        assert (bench.traffic_of(name, e["workload"]) is not None) == live
        assert bench.traffic_of(name, "another_workload") is None
