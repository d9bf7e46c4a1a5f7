/*
 * bta.h -- C ABI of the GB300 (sm_103a) BTA block-Cholesky / selected-inversion library.
 *
 * A BTA matrix (paper, Section 2.1, Table 2) is symmetric positive definite, with
 * n diagonal blocks of size b, the sub/super-diagonal blocks, and an arrowhead of
 * a rows and columns whose a x a corner is the "arrow tip"; N = n*b + a. a = 0 is
 * the plain block-tridiagonal case.
 *
 * Storage (all entry points): FP64, row-major, C-contiguous DEVICE memory owned
 * by the caller. Only the lower block pattern is stored:
 *   diag  [n][b][b]     A_{i,i}
 *   lower [n-1][b][b]   A_{i+1,i}        (may be NULL when n == 1)
 *   arrow [n][a][b]     A_{n,i}          (may be NULL when a == 0)
 *   tip   [a][a]        A_{n,n}          (may be NULL when a == 0)
 *   rhs   [N][nrhs]     right-hand sides, row-major
 * Every pointer must be 8-byte aligned. All calls are asynchronous on `stream`
 * (a cudaStream_t; NULL means the legacy default stream) and only enqueue work.
 *
 * Return codes (synchronous, about the arguments and the launch only):
 *   0                   enqueued
 *   -k (k = 1, 2, ...)  argument k is invalid (out of range, NULL where a
 *                       buffer is needed, misaligned, or workspace too small)
 *   > 0                 a CUDA error code raised while enqueueing
 * Numerical failure is asynchronous: a non-positive pivot in bta_factor sets the
 * library's per-device info word (read it with bta_get_info) and the outputs from
 * the failing block column on become NaN. Nothing traps.
 *
 * Ordering: bta_factor -> { bta_logdet, bta_solve } -> bta_selinv. bta_selinv
 * overwrites the factor with the selected inverse (like LAPACK POTRI), so call
 * logdet and solve before it, or on a copy.
 *
 * Scratch memory: the plain entry points allocate their scratch stream-ordered
 * (cudaMallocAsync / cudaFreeAsync on `stream`). The *_ws variants take a
 * caller-owned device workspace of at least bta_workspace_bytes(...) bytes
 * (256-byte aligned) and allocate nothing; a workspace must not be shared by
 * calls that can run concurrently.
 */
#ifndef BTA_H_
#define BTA_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* bta_stream_t; /* same type as cudaStream_t */

/* Operation selectors for bta_workspace_bytes. */
#define BTA_OP_FACTOR 1
#define BTA_OP_SELINV 2
#define BTA_OP_SOLVE 3
#define BTA_OP_LOGDET 4

/*
 * bta_factor -- block Cholesky A = L L^T in place (paper, Algorithm 1, POBTAF;
 * Section 2.2). For i = 0..n-2: L_ii = POTRF(A_ii); L_{i+1,i} = A_{i+1,i} L_ii^{-T};
 * L_{n,i} = A_{n,i} L_ii^{-T}; A_{i+1,i+1} -= L_{i+1,i} L_{i+1,i}^T;
 * A_{n,i+1} -= L_{n,i} L_{i+1,i}^T; A_{n,n} -= L_{n,i} L_{n,i}^T; then the last
 * block column and L_nn = POTRF(A_nn).
 * In: the lower triangles of diag[i] and tip (upper triangles are not read),
 * lower, arrow. Out: L in the same buffers; the strict upper triangles of diag[i]
 * and tip are set to zero. In FP64 (b >= 128) each block step is one cooperative
 * launch: a tile Cholesky of the block column [A_ii; A_{i+1,i}; A_{n,i}] whose
 * trailing tile updates are the step's Schur products; the triangular solves are
 * tile substitutions. In the tensor-core precision modes the triangular solves
 * run as L_ii^{-1} followed by products (the inverse-plus-GEMM substitution of
 * Sections 4 and 5.1).
 * Errors: see the header comment; info = 1-based global row of the first
 * non-positive leading minor (block i, local row j -> i*b + j; tip -> n*b + j).
 */
int bta_factor(int64_t n, int64_t b, int64_t a, double* diag, double* lower,
               double* arrow, double* tip, bta_stream_t stream);

/*
 * bta_selinv -- selected inversion (paper, Algorithm 2, POBTASI; Section 2.2):
 * overwrites the factor L (as left by bta_factor) with X = A^{-1} restricted to
 * the BTA pattern: X_{i,i} (returned full and symmetric), X_{i+1,i}, X_{n,i} and
 * X_{n,n}. X_nn = L_nn^{-T} L_nn^{-1}; for i = n-1..0:
 *   X_{i+1,i} = -(X_{i+1,i+1} L_{i+1,i} + X_{n,i+1}^T L_{n,i}) L_ii^{-1}
 *   X_{n,i}   = -(X_{n,i+1}  L_{i+1,i} + X_{n,n}     L_{n,i}) L_ii^{-1}
 *   X_{i,i}   = (L_ii^{-T} - X_{i+1,i}^T L_{i+1,i} - X_{n,i}^T L_{n,i}) L_ii^{-1}
 * evaluated with G_i = L_{i+1,i} L_ii^{-1}, H_i = L_{n,i} L_ii^{-1} and
 * M_i = L_ii^{-T} L_ii^{-1} formed for all i before the backward sweep.
 */
int bta_selinv(int64_t n, int64_t b, int64_t a, double* diag, double* lower,
               double* arrow, double* tip, bta_stream_t stream);

/*
 * bta_solve -- solves A x = rhs in place given the factor L (block forward
 * substitution L y = rhs, then backward L^T x = y). Not in the paper; it is the
 * standard use of a Cholesky factor.
 *   y_i = L_ii^{-1}(r_i - L_{i,i-1} y_{i-1}),  y_n = L_nn^{-1}(r_n - sum_i L_{n,i} y_i)
 *   x_n = L_nn^{-T} y_n,  x_i = L_ii^{-T}(y_i - L_{i+1,i}^T x_{i+1} - L_{n,i}^T x_n)
 * rhs: [N][nrhs] row-major device buffer, 1 <= nrhs <= 64. Inside a block the
 * triangular solve is blocked by diagonal sub-blocks of order ds = min(b, 256),
 * whose inverses are formed first in the workspace (n * ceil(b/ds) * ds^2
 * doubles, besides the arrow partial sums and one block of staging): each block
 * step is then ceil(b/ds) dependent pairs of matrix-vector products.
 */
int bta_solve(int64_t n, int64_t b, int64_t a, const double* diag,
              const double* lower, const double* arrow, const double* tip,
              double* rhs, int64_t nrhs, bta_stream_t stream);

/*
 * bta_logdet -- log det A = 2 * (sum_i sum_k log (L_ii)_kk + sum_k log (L_nn)_kk)
 * from the factor (not in the paper: det A = det(L)^2). Summed in FP64 in a fixed
 * order (per-block tree sums, then blocks in order, then the tip), so repeated
 * calls give identical bits. out_dev: one double in device memory.
 */
int bta_logdet(int64_t n, int64_t b, int64_t a, const double* diag,
               const double* tip, double* out_dev, bta_stream_t stream);

/*
 * bta_get_info -- synchronizes `stream`, returns the current device's info word
 * in *info (0: every pivot positive since the last read; k > 0: LAPACK-style
 * global row of the first failed pivot) and resets it to 0. The word is shared by
 * all calls on the device: failures of concurrent calls on different streams are
 * not told apart.
 */
int bta_get_info(bta_stream_t stream, int64_t* info);

/*
 * bta_workspace_bytes -- scratch bytes the *_ws variant of operation `op`
 * (BTA_OP_*) needs for these sizes; nrhs is used by BTA_OP_SOLVE only.
 * Returns 0 for invalid arguments or an operation that needs no scratch.
 */
size_t bta_workspace_bytes(int op, int64_t n, int64_t b, int64_t a, int64_t nrhs);

/* The same operations on a caller-owned workspace (see bta_workspace_bytes);
 * they allocate nothing. */
int bta_factor_ws(int64_t n, int64_t b, int64_t a, double* diag, double* lower,
                  double* arrow, double* tip, void* ws, size_t ws_bytes,
                  bta_stream_t stream);
int bta_selinv_ws(int64_t n, int64_t b, int64_t a, double* diag, double* lower,
                  double* arrow, double* tip, void* ws, size_t ws_bytes,
                  bta_stream_t stream);
int bta_solve_ws(int64_t n, int64_t b, int64_t a, const double* diag,
                 const double* lower, const double* arrow, const double* tip,
                 double* rhs, int64_t nrhs, void* ws, size_t ws_bytes,
                 bta_stream_t stream);
int bta_logdet_ws(int64_t n, int64_t b, int64_t a, const double* diag,
                  const double* tip, double* out_dev, void* ws, size_t ws_bytes,
                  bta_stream_t stream);

/*
 * bta_logdet_noalloc -- the same result as bta_logdet, for callers that cannot
 * allocate device memory when they need it (a host framework that owns the
 * device-memory budget, or a latency-critical loop where cudaMalloc/cudaFree
 * would synchronize the device). It allocates nothing: its scratch is a fixed
 * 512 KiB array inside the library, present on every GPU that loads the library
 * until the process exits. The paper has no counterpart; this is an interface
 * convenience.
 * Limits: n <= 65536 (larger n returns -1, nothing is enqueued).
 * `stream` must belong to the current device (else -7, nothing enqueued).
 * The first call on each device looks up the array's device address (with that
 * device current); make that first call before any stream capture. The address
 * is kept for the life of the process, so do not call this entry point on a
 * device after cudaDeviceReset there. All calls on a device share the array:
 * calls that overlap on the GPU race and must be ordered by the caller (same
 * stream, or events).
 */
int bta_logdet_noalloc(int64_t n, int64_t b, int64_t a, const double* diag,
                       const double* tip, double* out_dev, bta_stream_t stream);

/* ---- Batched form -------------------------------------------------------- */

/* One matrix of a batch: its blocks (in place: A -> X), an optional device
 * double for its log-determinant, its precision mode and a workspace of at
 * least bta_batch_workspace_bytes(n, b, a, prec) bytes (256-byte aligned). */
typedef struct bta_batch_entry {
  int64_t n, b, a;
  double* diag;
  double* lower;
  double* arrow;
  double* tip;
  double* logdet_out;
  int prec;
  void* ws;
  size_t ws_bytes;
} bta_batch_entry;

size_t bta_batch_workspace_bytes(int64_t n, int64_t b, int64_t a, int prec);

/*
 * bta_factor_selinv_batched -- factor, log-det and selected inversion of
 * `count` independent BTA matrices of any sizes (not in the paper; a batch of
 * the Algorithm 1 + Algorithm 2 pipeline). Matrices are taken largest first and
 * each goes to whichever of `nstreams` (1..64) library streams has the least work
 * so far; the streams fork from `stream` and join back into it, so the whole
 * batch is ordered on `stream` and can be captured in one CUDA graph (capture
 * `stream`; the library's streams join the capture through events). Returns -2
 * if any entry is invalid (nothing enqueued). A failed pivot in any matrix sets
 * the shared info word (which matrix is not recorded).
 */
int bta_factor_selinv_batched(int64_t count, const bta_batch_entry* entries, int nstreams,
                              bta_stream_t stream);

/* ---- Persistent batched form --------------------------------------------- */

/*
 * A plan runs factorization (Algorithm 1), log-det and selected inversion
 * (Algorithm 2, Section 2.2) of `count` independent FP64 BTA matrices of any
 * n, b, a in ONE persistent cooperative kernel launch (not in the paper; the
 * batched form of the same method). Each matrix's work is a graph of
 * operations made of 32 x 32 tile items (the block step's tile Cholesky with
 * its Schur updates, the tip, the inverses L_ii^{-1}, the products G_i, H_i,
 * M_i, X_nn and the backward recurrence). On the device an operation becomes
 * ready when the operations it depends on have completed; the kernel's CTAs
 * take items of ready operations from priority queues (operations of the
 * matrices with the most remaining work first), so no CTA waits for a
 * particular item.
 *
 * Tuning parameters (0 = automatic):
 *   ctas_per_sm    resident CTAs per SM (128 threads each; capped by occupancy)
 *   levels         priority levels, 1..8 (0: 8): an operation's level is the
 *                  share of its matrix's program still ahead of it, relative
 *                  to the longest program; 1 serves operations in ready order
 *   rows_per_item  1 or 2 tile rows per update / product item (tile shape
 *                  32 x 32 or 64 x 32)
 */
typedef struct bta_plan_params {
  int ctas_per_sm;
  int levels;
  int rows_per_item;
  int reserved;
} bta_plan_params;

typedef struct bta_plan_s* bta_plan;

/* Workspace per matrix: L_ii^{-1} [n][b][b], G [n-1][b][b], H [n][a][b],
 * L_nn^{-1} [a][a], pivot reciprocals and per-tile log sums, 256-byte aligned
 * parts. 0 for invalid sizes. */
size_t bta_plan_entry_workspace_bytes(int64_t n, int64_t b, int64_t a);

/*
 * bta_plan_create -- builds the operation graph of `entries` (their pointers are
 * baked into the plan: a plan runs on exactly those buffers) and allocates its
 * device tables (cudaMalloc, on the current device, which must hold the
 * buffers). Entries: prec must be BTA_PREC_FP64; ws of at least
 * bta_plan_entry_workspace_bytes(n, b, a) bytes, 256-byte aligned; logdet_out
 * may be NULL. Size limits per entry: b, a <= 32768, n <= 2^20 and
 * n (ceil(b/32))^2 <= 1.5e9 (the tiles of one product over all blocks). params
 * may be NULL (all automatic). Synchronous. Returns 0 and *out, -1 for count out
 * of [1, 65536], -2 for an invalid entry, -3 for invalid params, -4 for a NULL
 * out, > 0 for a CUDA error.
 */
int bta_plan_create(int64_t count, const bta_batch_entry* entries, const bta_plan_params* params,
                    bta_plan* out);

/*
 * bta_plan_run -- enqueues one run on `stream` (a counter reset and one
 * cooperative launch; capturable in a CUDA graph): every matrix A -> X in
 * place, log det A to its logdet_out. The stream must belong to the plan's
 * device (-1 otherwise). Runs of one plan must not overlap.
 */
int bta_plan_run(bta_plan plan, bta_stream_t stream);

/*
 * bta_plan_status -- synchronizes `stream` and reports the last run: *timed_out
 * = 1 if the kernel gave up waiting for work (no operation completed for
 * seconds; the results are then invalid), and, if info
 * is not NULL, info[k] = 1-based row of matrix k's first non-positive pivot (0:
 * none; LAPACK-style, as bta_get_info).
 */
int bta_plan_status(bta_plan plan, int* timed_out, int64_t* info, bta_stream_t stream);

/* bta_plan_describe -- out[0..nout-1] = grid CTAs, CTAs per SM, priority
 * levels, rows per item, operations, items, algorithmic flops per run,
 * operations ready at the start. */
int bta_plan_describe(bta_plan plan, int64_t* out, int nout);

/* bta_plan_destroy -- frees the plan's device tables (synchronously; no run of
 * the plan may be pending). NULL is a no-op. */
int bta_plan_destroy(bta_plan plan);

/* ---- Partitioned form (the paper's Sections 3.1-3.4 on one device) ------- */

/*
 * bta_factor_selinv_partitioned -- selected inversion (and log-det) of one BTA
 * matrix by the partitioned scheme: the block rows are split into P partitions
 * (top partition lb times a middle one; middle partitions >= 2 blocks), whose
 * interior eliminations run concurrently on library streams (PPOBTAF,
 * Algorithms 3-4: the middle partitions' shifting permutation with its fill-in),
 * the 2P-1-block reduced system of the boundary blocks is factored and inverted
 * (POBTARSSI, Section 3.3), and the partitions' interior blocks of X follow in
 * concurrent backward sweeps (PPOBTASI, Algorithms 5-6). In place: A -> X, the
 * same output as bta_factor followed by bta_selinv; the intermediate factor is of
 * the permuted matrix, so no L is returned. logdet_out (device double, may be
 * NULL) receives log det A. The large products follow bta_set_precision.
 * ws: >= bta_partitioned_workspace_bytes(n, b, a, P, lb) bytes, 256-byte aligned.
 * P is reduced when n is too small for it (P = 1 is the sequential method).
 */
size_t bta_partitioned_workspace_bytes(int64_t n, int64_t b, int64_t a, int64_t P, double lb);
int bta_factor_selinv_partitioned(int64_t n, int64_t b, int64_t a, double* diag, double* lower,
                                  double* arrow, double* tip, int64_t P, double lb,
                                  double* logdet_out, void* ws, size_t ws_bytes,
                                  bta_stream_t stream);

/* ---- Differentiation support ------------------------------------------- */

/*
 * bta_grad_blocks -- gradients of  f = alpha * log det A + beta * x^T A^{-1} x
 * with respect to the stored blocks and to x, given the selected inverse X
 * (bta_selinv output) and y = A^{-1} x (bta_solve output):
 *   df/d diag_i  = alpha X_ii      - beta y_i y_i^T
 *   df/d lower_i = 2 (alpha X_{i+1,i} - beta y_{i+1} y_i^T)
 *   df/d arrow_i = 2 (alpha X_{n,i}   - beta y_n y_i^T)
 *   df/d tip     = alpha X_nn      - beta y_n y_n^T
 *   df/dx        = 2 beta y                    (g_x may be NULL)
 * since d log det A / dA = A^{-1} and d x^T A^{-1} x / dA = -y y^T; each
 * off-diagonal block stands for itself and its transpose (factor 2) and the
 * diagonal blocks take the symmetric convention. Not in the paper: it is what
 * makes the selected inverse the backward of a Gaussian log-likelihood.
 * y, g_x: [N] device vectors; outputs have the layout of the inputs.
 */
int bta_grad_blocks(int64_t n, int64_t b, int64_t a, const double* x_diag, const double* x_lower,
                    const double* x_arrow, const double* x_tip, const double* y, double alpha,
                    double beta, double* g_diag, double* g_lower, double* g_arrow, double* g_tip,
                    double* g_x, bta_stream_t stream);

/* bta_dot -- out_dev = x^T y over N doubles, summed in a fixed order (identical
 * bits on repeat); ws: >= 608 doubles of device scratch. */
int bta_dot(int64_t N, const double* x, const double* y, double* out_dev, void* ws,
            size_t ws_bytes, bta_stream_t stream);

/* ---- Precision of the block products ------------------------------------ */

#define BTA_PREC_FP64 0   /* FP64 DMMA (mma.sync f64) everywhere (default) */
#define BTA_PREC_OZAKI 1  /* large products as FP64 emulated on BF16 tensor cores (tcgen05):
                             7 BF16 digit slices per operand (Ozaki et al. 2012 splitting),
                             exact FP32 accumulation of the leading slice-product groups;
                             about 1e-13 relative error per product for k <= 1024 */
#define BTA_PREC_BF16X3 2 /* mixed precision: the Schur-complement and inverse-recurrence
                             products as split-BF16x3 (hi*hi + hi*lo + lo*hi) with FP32
                             accumulation on tcgen05; POTRF, the triangular inverses and
                             products, the tip and log-det stay FP64 */

/*
 * bta_set_precision -- selects how bta_factor and bta_selinv run their large
 * block products (blocks of at least 64 x 64 with k >= 64; smaller ones always
 * use FP64). Process-wide; set it before querying bta_workspace_bytes (the
 * tensor-core modes need more scratch) and not while calls are in flight.
 * Returns 0, or -1 for an unknown mode. Neither mode is part of the paper, whose
 * computation is all FP64 (Section 5.2).
 */
int bta_set_precision(int prec);
int bta_get_precision(void);

/*
 * bta_gemm -- C = alpha op(A) op(B) + beta C on one device, FP64 in and out,
 * computed in precision `prec` (BTA_PREC_*). op(X) = X or X^T (trans != 0);
 * row-major, M x N output. The dense block product every step of the method is
 * built from, exported for direct use and testing. BTA_PREC_FP64 needs no
 * workspace; the tensor-core modes need bta_gemm_workspace_bytes(prec, M, N, K)
 * bytes of 256-byte aligned device scratch.
 */
size_t bta_gemm_workspace_bytes(int prec, int64_t M, int64_t N, int64_t K);
int bta_gemm(int prec, int64_t M, int64_t N, int64_t K, double alpha, const double* A,
             int64_t lda, int transA, const double* B, int64_t ldb, int transB, double beta,
             double* C, int64_t ldc, void* ws, size_t ws_bytes, bta_stream_t stream);

/*
 * bta_tc_status -- reads and clears the timeout flag of the library's bounded
 * waits (the tcgen05 pipelines' mbarriers, the cooperative factor step's grid
 * barrier and flags): 1 if any wait gave up since the last read (its results are
 * then not valid), else 0. Synchronous.
 */
int bta_tc_status(int* timed_out);

/*
 * bta_factor_selinv_all -- the per-matrix sequence on device buffers in one
 * call: bta_factor, bta_logdet (into logdet_out, one device double), bta_solve
 * of rhs (nrhs right-hand sides, 0: none; in place) and bta_selinv (A -> X in
 * place), with the same results as those four calls in a row. The solve runs on
 * a library stream concurrently with the part of the selected inversion's
 * prologue that only reads the factor (L_ii^{-1}, G_i, H_i); the selected
 * inversion waits for it before writing into the factor's blocks. ws: device
 * scratch of at least bta_all_workspace_bytes(n, b, a, nrhs) bytes, 256-byte
 * aligned. Asynchronous on `stream`; calls must not overlap (they share the
 * library's side streams and events). Returns 0, -k for invalid argument k, or a
 * CUDA error code; pivot failure goes to the info word as in bta_factor.
 */
size_t bta_all_workspace_bytes(int64_t n, int64_t b, int64_t a, int64_t nrhs);
int bta_factor_selinv_all(int64_t n, int64_t b, int64_t a, double* diag, double* lower,
                          double* arrow, double* tip, double* rhs, int64_t nrhs, double* logdet_out,
                          void* ws, size_t ws_bytes, bta_stream_t stream);

/*
 * bta_factor_selinv_host -- the whole per-matrix sequence from host memory:
 * factor (Algorithm 1), log det, a solve with nrhs right-hand sides (0: none)
 * and the selected inversion (Algorithm 2), with the inputs copied in and X,
 * the solution and log det copied back inside the call. The copies overlap the
 * block sweeps: input blocks go up in chunks on a copy stream ahead of the
 * factorization (step i waits only for blocks i and i+1), the solution as soon
 * as the solve is done, and X chunk by chunk as the backward sweep finishes it.
 * Layouts are those of bta_factor / bta_solve / bta_selinv; h_* inputs and x_*
 * outputs are host buffers (pinned for the copies to overlap), h_logdet one host
 * double. The host inputs are not modified. ws: device scratch of at least
 * bta_host_pipeline_workspace_bytes(n, b, a, nrhs) bytes, 256-byte aligned; it
 * holds the device copy of the pattern. Asynchronous on `stream` like the other
 * entry points: outputs are valid once the stream has reached this point; the
 * host buffers must stay valid until then. Calls must not overlap (they share
 * the library's copy streams and events). Precision: bta_set_precision.
 * Returns 0, -k for invalid argument k, or a CUDA error code; pivot failure goes
 * to the info word as in bta_factor.
 */
size_t bta_host_pipeline_workspace_bytes(int64_t n, int64_t b, int64_t a, int64_t nrhs);
int bta_factor_selinv_host(int64_t n, int64_t b, int64_t a, const double* h_diag,
                           const double* h_lower, const double* h_arrow, const double* h_tip,
                           const double* h_rhs, int64_t nrhs, double* x_diag, double* x_lower,
                           double* x_arrow, double* x_tip, double* x_sol, double* h_logdet,
                           void* ws, size_t ws_bytes, bta_stream_t stream);

/*
 * bta_wait_selftest -- exercises the timeout path of the library's bounded
 * waits: one CTA waits, with a limit of `polls` polls (1 <= polls <= 2^20), on a
 * device flag that nothing raises, gives up, records the timeout, and returns.
 * *timed_out then receives bta_tc_status's reading (1 when the path works).
 * Synchronous; allocates and frees 4 bytes of device memory. Not part of the
 * method: it lets a test check failure reporting without faulting the GPU.
 * Returns -1 for polls out of range, -2 for a null timed_out.
 */
int bta_wait_selftest(int64_t polls, int* timed_out);

/* ---- Measurement support (not part of the method) ----------------------- */

/* Kernel ids for bta_timing_read. */
#define BTA_KERNEL_GEMM 0       /* DMMA tile GEMM (Schur updates, TRMM, selinv chain) */
#define BTA_KERNEL_POTRF_TILE 1 /* diagonal-tile Cholesky */
#define BTA_KERNEL_TRSM_PANEL 2 /* panel triangular solve inside POTRF */
#define BTA_KERNEL_TILE_INV 3   /* diagonal-tile inverse inside TRTRI */
#define BTA_KERNEL_ZERO_UPPER 4
#define BTA_KERNEL_MIRROR 5
#define BTA_KERNEL_LOGDET 6
#define BTA_KERNEL_TRSV 7
#define BTA_KERNEL_GEMV 8
#define BTA_KERNEL_ARROW 9
#define BTA_KERNEL_PROBE 10
#define BTA_KERNEL_GEMM_TC 11  /* tcgen05 BF16-slice GEMM (OZAKI / BF16X3 modes); flops recorded
                                  as the FP64 product it stands for (2 M N K, lower half for
                                  lower-only outputs) */
#define BTA_KERNEL_TC_SPLIT 12 /* FP64 -> BF16 slice splitting */
#define BTA_KERNEL_TC_FINAL 13 /* int64 accumulator -> FP64 output */
#define BTA_KERNEL_FACTOR_STEP 14 /* one fused block step of the FP64 factorization */
#define BTA_KERNEL_PERSISTENT 15  /* one run of a persistent batched plan (bta_plan_run) */

/*
 * bta_timing_enable -- on != 0: from now on every kernel launch of the library
 * is bracketed by CUDA events on its stream and tagged with its algorithmic
 * FP64 flop count; previous records are dropped. on == 0 stops recording. Off by
 * default. Host-side cost per launch; meant for measurement runs only.
 */
int bta_timing_enable(int on);

/*
 * bta_timing_read -- waits for the recorded launches of kernel `kernel_id`
 * (BTA_KERNEL_*) and returns their summed device time (ms), summed algorithmic
 * flops and launch count.
 */
int bta_timing_read(int kernel_id, double* total_ms, double* flops, int64_t* launches);

/*
 * bta_probe_fp64_peak -- enqueues a DMMA (mma.sync m8n8k4 f64) throughput
 * kernel on every SM of the current device; *flops receives its flop count
 * (host, at enqueue). Time it with events on `stream` to measure the FP64
 * tensor peak that bounds this library's kernels. out_dev: one device double
 * (written only in a case that cannot occur; keeps the loop live).
 */
int bta_probe_fp64_peak(double* out_dev, int64_t iters, double* flops, bta_stream_t stream);

/* Library version (major * 10000 + minor * 100 + patch). */
int bta_version(void);

#ifdef __cplusplus
}
#endif

#endif /* BTA_H_ */
