"""GB300 (sm_103a) block Cholesky, selected inversion, log-det and solve for
symmetric positive-definite block-tridiagonal-with-arrowhead (BTA) matrices.

The Python layer only marshals torch tensors (device memory, current stream)
into the C ABI of libbta.so; every step of the computation runs in the
library's CUDA kernels. Block storage, FP64, contiguous, on one CUDA device:
    diag [n, b, b], lower [n-1, b, b], arrow [n, a, b], tip [a, a].
"""
from __future__ import annotations

from .api import (  # noqa: F401
    BTAError,
    OP_FACTOR,
    PREC_BF16X3,
    PREC_FP64,
    PREC_OZAKI,
    OP_LOGDET,
    OP_SELINV,
    OP_SOLVE,
    factor,
    factor_selinv_all,
    factor_selinv_host,
    factor_selinv_partitioned,
    gemm,
    get_info,
    get_precision,
    logdet,
    selinv,
    set_precision,
    solve,
    tc_status,
    wait_selftest,
    workspace_bytes,
)
from .autograd import BTALogdetQuad, logdet_quad  # noqa: F401,E402
