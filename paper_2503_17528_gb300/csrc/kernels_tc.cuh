// Interface of the tensor-core (tcgen05) GEMM of kernels_tc.cu.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include "bta_internal.cuh"

namespace bta {

enum { TC_OZ = 1, TC_X3 = 2 };
constexpr int kOzSlices = 7;     // BF16 digit slices per FP64 operand (7 bits each)

int tc_slices(int mode);
// Scratch bytes for one call of gemm_tc with these sizes and batch (K <= 16384).
size_t tc_workspace_bytes(int mode, int M, int N, int K, int batch);
// GEMM on the tensor cores; ws: >= tc_workspace_bytes. Terms that share alpha
// and have no triangular operand run as one product over the concatenated k.
// reuse_b: op(B) is the one the previous call on this workspace split (same
// parts, N, k extent and batch, the data unchanged since; M may differ), so it
// is not split again. A self-product (op(B)^T is op(A)) leaves its operand's
// split in op(B)'s place, where a following product with that op(B) can reuse it.
cudaError_t gemm_tc(const GemmArgs& g, int mode, void* ws, size_t ws_bytes, cudaStream_t s,
                    bool reuse_b = false);
// Reads and clears the bounded-wait timeout flag of the tensor-core kernels.
cudaError_t tc_error_read_reset(int* out);

}  // namespace bta
