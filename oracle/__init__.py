"""CPU oracle for the BTA block-Cholesky / selected-inversion path.

TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the benchmark's
CPU-baseline leg may import this package. The product path (the CUDA library
and its Python binding) never calls into it, and this package never imports the
product path.

Two layers:
  * ``dense``: the plain definitions (assemble the N x N matrix, dense Cholesky,
    dense inverse restricted to the BTA pattern, slogdet, dense solve). Usable
    for N up to a few thousand.
  * ``bta_oracle``: the block-sequential recursions of the paper, Algorithm 1
    (POBTAF) and Algorithm 2 (POBTASI), in FP64 with LAPACK POTRF and TRSM as
    library steps, plus the log-determinant and the block triangular solves.
"""
from .bta_oracle import pobtaf, pobtasi, logdet, solve, BTAFactor  # noqa: F401
from . import dense  # noqa: F401
