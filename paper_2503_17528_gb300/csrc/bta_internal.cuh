// Internal interfaces between the C-ABI layer (bta_api.cu) and the FP64 kernels
// (kernels_f64.cu). Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

namespace bta {

// A launch parameter computed once per device (SM counts, occupancy, function
// attributes). Thread-safe: callers racing on a device's first use may each
// compute it, with the same result; 0 marks "not computed yet", so `compute`
// must return a nonzero value. `compute` runs with that device current.
constexpr int kMaxDevices = 64;
struct PerDevice {
  std::atomic<long long> v[kMaxDevices];
};
template <class F>
inline long long per_device(PerDevice& c, F compute) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return compute();
  long long x = c.v[dev].load(std::memory_order_acquire);
  if (x) return x;
  x = compute();
  c.v[dev].store(x, std::memory_order_release);
  return x;
}

constexpr int T = 32;  // edge of every FP64 tile

enum { OP_N = 0, OP_T = 1 };
// Structure of op(X) for a GEMM operand; lets a tile skip the k-range that is
// known to be zero (triangular factors and inverses).
enum { TRI_NONE = 0, TRI_LOWER = 1, TRI_UPPER = 2 };

// One product term alpha * op(A) * op(B) with op(A): M x K, op(B): K x N.
struct GemmTerm {
  const double* A;
  const double* B;
  int64_t lda, ldb;  // row strides (elements) of the stored A and B
  int64_t sA1, sB1;  // strides per unit of batch index z1
  int64_t sA2, sB2;  // strides per unit of batch index z2
  int K;
  int opA, opB, triA, triB;
  double alpha;
};

// C = beta * C + sum_t alpha_t op(A_t) op(B_t) over a 2-D batch (z1, z2).
constexpr int kMaxTerms = 4;
struct GemmArgs {
  GemmTerm t[kMaxTerms];
  int nterms;
  double* C;
  int64_t ldc, sC1, sC2;
  int M, N;
  double beta;  // C is read only if beta != 0
  int lowerC;   // 1: only output tiles with tile_row >= tile_col are computed
  int nb1, nb2;
};

inline GemmTerm term(const double* A, int64_t lda, int opA, int triA,
                     const double* B, int64_t ldb, int opB, int triB, int K,
                     double alpha) {
  GemmTerm t{};
  t.A = A; t.B = B; t.lda = lda; t.ldb = ldb; t.K = K;
  t.opA = opA; t.opB = opB; t.triA = triA; t.triB = triB; t.alpha = alpha;
  return t;
}

cudaError_t gemm_f64(const GemmArgs& g, cudaStream_t s);
// Algorithmic flops of a GEMM call (2 per structurally non-zero multiply-add over
// the outputs it defines, all batch entries); host-side, for the timing records.
double gemm_alg_flops(const GemmArgs& g);

// Dense block kernels (all FP64, row-major, leading dimension ld; `count`
// blocks at stride `sb` elements; square blocks of order `nrow`).
// Lower Cholesky in place; zeroes the strict upper triangle. info_row0 is the
// 1-based global row of the first row of block 0, info_rstride the increase
// per block.
cudaError_t potrf_blocks(double* A, int64_t ld, int64_t sb, int count, int nrow,
                         long long info_row0, long long info_rstride,
                         cudaStream_t s);
// Largest tile counts of the fused factor step (b, a <= 32768): tiles per block
// order and extended rows (two blocks plus the arrowhead).
constexpr int kStepMaxTiles = 1024;
constexpr int kStepMaxExtTiles = 3 * 1024;
// Scratch of the cooperative factor-step kernel, 256-byte aligned: one flag word
// per extended tile row and one counter per factor column, then 32 pivot
// reciprocals per diagonal tile.
constexpr size_t kStepFlagBytes = 16384;
constexpr size_t kCoopScratch = kStepFlagBytes + (size_t)kStepMaxTiles * 32 * sizeof(double);
static_assert((kStepMaxExtTiles + kStepMaxTiles) * sizeof(int) <= kStepFlagBytes, "step scratch");
// One block step of the factorization in one cooperative launch: L_ii, L_{i+1,i}
// and L_{n,i} in place, and (schur != 0) the Schur updates of A_{i+1,i+1},
// A_{n,i+1} and the tip (lower tiles). next == 0 for the last block (Lw, D1, Ar1
// unused); a == 0: no arrowhead; schur == 0: D1, Ar1 and tip are unused.
// scratch: kCoopScratch bytes, 256-byte aligned. ld (0: b) is the row stride of
// D0, Lw and D1, so a diagonal sub-block of a larger matrix can be factored in
// place; the arrow blocks keep rows of b.
cudaError_t factor_step_coop(double* D0, double* Lw, double* D1, double* Ar0, double* Ar1,
                             double* tip, int b, int a, int next, long long info_row0,
                             void* scratch, cudaStream_t s, int schur = 1, int64_t ld = 0);
// Reads and clears the timeout flag of the cooperative kernels' grid barriers.
cudaError_t wait_error_read_reset(int* out);
// Enqueues one CTA that waits on *flag_dev (never raised) for `polls` polls.
cudaError_t wait_selftest(const int* flag_dev, unsigned polls, cudaStream_t s);

// Inverse of lower-triangular blocks: Linv (separate buffer, same layout) =
// L^{-1}, strict upper triangle zero. The doubling products go through `hook`
// when given (it may run them on the tensor cores), else the FP64 kernels.
typedef cudaError_t (*GemmHook)(const GemmArgs& g, void* ctx, cudaStream_t s);
cudaError_t trtri_blocks(const double* L, int64_t ldl, int64_t sl, double* Linv,
                         int64_t ldi, int64_t si, int count, int nrow,
                         cudaStream_t s, GemmHook hook = nullptr, void* ctx = nullptr);
// Copy the lower triangle onto the upper one (symmetrize) for `count` blocks.
cudaError_t mirror_lower(double* A, int64_t ld, int64_t sb, int count, int nrow,
                         cudaStream_t s);

// log det from factor blocks: out = 2 * (sum log diag(L_ii) + sum log diag(L_nn)).
cudaError_t logdet_f64(const double* diag, int64_t n, int64_t b,
                       const double* tip, int64_t a, double* partial,
                       double* out, cudaStream_t s);

// Per-block log sums (partial[i] = sum_k log diag(block i); the tip last if a > 0).
cudaError_t logdet_partials(const double* diag, int64_t n, int64_t b, const double* tip, int64_t a,
                            double* partial, cudaStream_t s);
// out = 2 * (sum p1 + sum p2), fixed order.
cudaError_t logdet_combine(const double* p1, int64_t n1, const double* p2, int64_t n2, double* out,
                           cudaStream_t s);
// y += alpha x over n doubles.
cudaError_t axpy_f64(int64_t n, double alpha, const double* x, double* y, cudaStream_t s);

// Solve pieces (rhs row-major [rows][R]).
// x <- L^{-1} x (trans: L^{-T} x) by one thread-block cluster (tile substitution;
// used for the arrow tip).
cudaError_t trsv_lower(const double* L, int64_t ld, int nrow, double* x,
                       int64_t ldx, int R, bool trans, cudaStream_t s);
// x[M][R] = beta * xin + alpha * op(A) * y[K][R], op(A) is M x K; xin defaults
// to x (x += alpha op(A) y for beta = 1). triA = TRI_LOWER: the stored A is lower
// triangular and its zero part is not read.
cudaError_t gemv_multi(const double* A, int64_t lda, int opA, int M, int K,
                       const double* y, int64_t ldy, double* x, int64_t ldx,
                       int R, double alpha, cudaStream_t s, double beta = 1.0,
                       const double* xin = nullptr, int triA = TRI_NONE);
// r_n[a][R] -= sum_i arrow[i] (a x b) * y_i (b x R), y_i = rhs block i.
cudaError_t arrow_gather(const double* arrow, int64_t n, int64_t b, int64_t a,
                         const double* rhs, int R, double* partial,
                         int nchunks, double* rn, cudaStream_t s);
// y_i -= arrow[i]^T * x_n for all i.
cudaError_t arrow_scatter(const double* arrow, int64_t n, int64_t b, int64_t a,
                          const double* xn, int R, double* rhs, cudaStream_t s);
int arrow_chunks(int64_t n);

// Gradients of alpha log det A + beta x^T A^{-1} x (y = A^{-1} x): blocks
// G = alpha X - beta y y^T (off-diagonal blocks doubled); gx = 2 beta y (optional).
cudaError_t grad_blocks(int64_t n, int64_t b, int64_t a, const double* Xd, const double* Xl,
                        const double* Xa, const double* Xt, const double* y, double alpha,
                        double beta, double* Gd, double* Gl, double* Ga, double* Gt, double* gx,
                        cudaStream_t s);
constexpr int kDotCtas = 608;
// out = x^T y (deterministic order); partial: kDotCtas doubles.
cudaError_t dot_f64(int64_t N, const double* x, const double* y, double* partial, double* out,
                    cudaStream_t s);

// DMMA peak probe; *flops receives the launch's flop count.
cudaError_t fp64_probe(double* out, long long iters, double* flops, cudaStream_t s);

// Per-device info word (first failed pivot, LAPACK-style 1-based global row).
cudaError_t info_reset(cudaStream_t s);
cudaError_t info_read_reset(cudaStream_t s, long long* out);

}  // namespace bta
