"""CPU checks of the C ABI: the library loads, exports every declared symbol,
sizes its workspaces, and rejects bad arguments before touching the GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bta.h")


def _declared():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|size_t)\s+(bta_\w+)\s*\(", src, re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2503_17528_gb300 import _lib
    if not os.path.exists(_lib.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    return _lib.load()


def test_every_declared_symbol_is_exported(lib):
    from paper_2503_17528_gb300 import _lib
    names = _declared()
    assert len(names) >= 11
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(_lib.exported_symbols())


def test_version(lib):
    assert lib.bta_version() == 100


def test_workspace_sizes(lib):
    n, b, a = 365, 1024, 8
    f = lib.bta_workspace_bytes(1, n, b, a, 1)
    s = lib.bta_workspace_bytes(2, n, b, a, 1)
    assert f >= 2 * b * b * 8 + a * b * 8
    assert s >= (2 * n - 1) * b * b * 8 + n * a * b * 8
    assert lib.bta_workspace_bytes(3, n, b, a, 4) > 0
    assert lib.bta_workspace_bytes(4, n, b, a, 1) >= (n + 1) * 8
    assert lib.bta_workspace_bytes(9, n, b, a, 1) == 0
    assert lib.bta_workspace_bytes(1, 0, b, a, 1) == 0
    assert lib.bta_workspace_bytes(3, n, b, a, 65) == 0


def test_argument_errors_need_no_gpu(lib):
    v = ctypes.c_void_p
    good = v(4096)
    assert lib.bta_factor(0, 4, 1, good, good, good, good, None) == -1
    assert lib.bta_factor(2, 0, 1, good, good, good, good, None) == -2
    assert lib.bta_factor(2, 4, -1, good, good, good, good, None) == -3
    assert lib.bta_factor(2, 4, 1, None, good, good, good, None) == -4
    assert lib.bta_factor(2, 4, 1, v(4097), good, good, good, None) == -4
    assert lib.bta_factor(2, 4, 1, good, None, good, good, None) == -5
    assert lib.bta_factor(2, 4, 1, good, good, None, good, None) == -6
    assert lib.bta_factor(2, 4, 1, good, good, good, None, None) == -7
    assert lib.bta_selinv(2, 4, 1, good, good, good, None, None) == -7
    assert lib.bta_solve(2, 4, 1, good, good, good, good, None, 1, None) == -8
    assert lib.bta_solve(2, 4, 1, good, good, good, good, good, 0, None) == -9
    assert lib.bta_logdet(2, 4, 1, good, good, None, None) == -6
    assert lib.bta_factor_ws(2, 4, 1, good, good, good, good, None, 0, None) == -8
    assert lib.bta_factor_ws(2, 4, 1, good, good, good, good, v(4096), 16, None) == -9
    assert lib.bta_get_info(None, None) == -2


def test_one_call_forms_check_arguments_before_the_gpu(lib):
    v = ctypes.c_void_p
    good = v(4096)
    n, b, a = 3, 200, 4
    # workspace sizes: the device form holds the scratch only, the host form adds
    # the device copy of the pattern and the right-hand sides
    dw = lib.bta_all_workspace_bytes(n, b, a, 2)
    hw = lib.bta_host_pipeline_workspace_bytes(n, b, a, 2)
    pattern = 8 * (n * b * b + (n - 1) * b * b + n * a * b + a * a + (n * b + a) * 2)
    assert dw > 0 and hw >= dw + pattern
    assert lib.bta_all_workspace_bytes(n, b, a, 65) == 0
    assert lib.bta_host_pipeline_workspace_bytes(0, b, a, 1) == 0
    # device form: rhs, logdet and workspace checks
    assert lib.bta_factor_selinv_all(n, b, a, good, good, good, good, None, 1, good, good, dw, None) == -8
    assert lib.bta_factor_selinv_all(n, b, a, good, good, good, good, good, 65, good, good, dw, None) == -9
    assert lib.bta_factor_selinv_all(n, b, a, good, good, good, good, None, 0, None, good, dw, None) == -10
    assert lib.bta_factor_selinv_all(n, b, a, good, good, good, good, None, 0, good, v(4100), dw,
                                     None) == -11
    assert lib.bta_factor_selinv_all(n, b, a, good, good, good, good, None, 0, good, good, 16, None) == -12
    # host form: each host pointer is checked in argument order
    args = [n, b, a, good, good, good, good, good, 2, good, good, good, good, good, good, good, hw, None]
    assert lib.bta_factor_selinv_host(*args[:3], None, *args[4:]) == -4
    assert lib.bta_factor_selinv_host(*args[:4], None, *args[5:]) == -5
    assert lib.bta_factor_selinv_host(*args[:7], None, *args[8:]) == -8
    assert lib.bta_factor_selinv_host(*args[:9], None, *args[10:]) == -10
    assert lib.bta_factor_selinv_host(*args[:14], None, *args[15:]) == -15
    assert lib.bta_factor_selinv_host(*args[:15], v(4100), *args[16:]) == -16
    assert lib.bta_factor_selinv_host(*args[:16], 16, None) == -17
    # the wait self-test's own checks
    t = ctypes.c_int(0)
    assert lib.bta_wait_selftest(0, ctypes.byref(t)) == -1
    assert lib.bta_wait_selftest(10, None) == -2


def test_persistent_plan_checks_arguments_before_the_gpu(lib):
    """bta_plan_* reject bad arguments without touching the GPU, and the per-matrix
    workspace holds L^{-1}, G, H, L_nn^{-1}, the pivot reciprocals and log sums."""
    from paper_2503_17528_gb300 import _lib
    v = ctypes.c_void_p
    n, b, a = 5, 100, 3
    nt, na = 4, 1
    need = lib.bta_plan_entry_workspace_bytes(n, b, a)
    parts = [n * b * b, (n - 1) * b * b, n * a * b, a * a, max(nt, na) * 32, n * nt + na]
    assert need == sum(-(-8 * p // 256) * 256 for p in parts)
    assert lib.bta_plan_entry_workspace_bytes(0, b, a) == 0
    assert lib.bta_plan_entry_workspace_bytes(n, 0, a) == 0
    ents = (_lib.BatchEntry * 1)()
    e = ents[0]
    e.n, e.b, e.a = n, b, a
    e.diag, e.lower, e.arrow, e.tip = 4096, 4096, 4096, 4096
    e.prec, e.ws, e.ws_bytes = 0, 4096, need
    plan = v()
    ok = _lib.PlanParams(0, 0, 0, 0)
    assert lib.bta_plan_create(0, ctypes.addressof(ents), None, ctypes.byref(plan)) == -1
    assert lib.bta_plan_create(1, None, None, ctypes.byref(plan)) == -2
    assert lib.bta_plan_create(1, ctypes.addressof(ents), None, None) == -4
    for bad in (_lib.PlanParams(0, 0, 3, 0), _lib.PlanParams(0, 9, 0, 0), _lib.PlanParams(-1, 0, 0, 0)):
        assert lib.bta_plan_create(1, ctypes.addressof(ents), ctypes.addressof(bad), ctypes.byref(plan)) == -3
    for field, value in (("prec", 1), ("ws_bytes", need - 1), ("ws", 4097), ("tip", 0), ("b", 0)):
        old = getattr(e, field)
        setattr(e, field, value)
        assert lib.bta_plan_create(1, ctypes.addressof(ents), ctypes.addressof(ok), ctypes.byref(plan)) == -2, field
        setattr(e, field, old)
    assert lib.bta_plan_run(None, None) == -1
    assert lib.bta_plan_status(None, None, None, None) == -1
    assert lib.bta_plan_describe(None, None, 0) == -1
    assert lib.bta_plan_destroy(None) == 0


def test_persistent_plan_rejects_item_counts_past_int_range(lib):
    """One product over all blocks has n (b/32)^2 tile items, indexed by ints."""
    from paper_2503_17528_gb300 import _lib
    ents = (_lib.BatchEntry * 1)()
    e = ents[0]
    e.n, e.b, e.a = 1 << 20, 2048, 0
    e.diag, e.lower = 4096, 4096
    e.prec, e.ws, e.ws_bytes = 0, 4096, 1 << 62
    plan = ctypes.c_void_p()
    assert lib.bta_plan_create(1, ctypes.addressof(ents), None, ctypes.byref(plan)) == -2
