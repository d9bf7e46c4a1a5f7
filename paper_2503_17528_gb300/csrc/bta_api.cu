// C ABI of the BTA library (declared in include/bta.h): argument checks,
// workspace layout and the launch sequences of factor, selinv, solve, logdet.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "../../include/bta.h"
#include "bta_internal.cuh"
#include "kernels_tc.cuh"

using namespace bta;

namespace {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }
inline bool misaligned(const void* p) { return ((uintptr_t)p & 7u) != 0; }

#define BTA_TRY(expr)                                   \
  do {                                                  \
    cudaError_t e_ = (expr);                            \
    if (e_ != cudaSuccess) return (int)e_;              \
  } while (0)

// Workspace carving: consecutive 256-byte aligned regions.
struct Carver {
  char* base;
  size_t off = 0;
  explicit Carver(void* p) : base((char*)p) {}
  double* take(size_t count) {
    double* p = base ? (double*)(base + off) : nullptr;
    off += align_up(count * sizeof(double));
    return p;
  }
};

struct FactorWs { double *Linv, *W, *Wa; void* coop; void* tc; size_t tc_bytes; };
struct SelinvWs { double *Linv, *G, *H, *LtInv; void* tc; size_t tc_bytes; };

extern int g_prec;
size_t tc_bytes_for(int64_t b, int64_t a, int64_t batch, int prec);
struct SolveWs { double* partial; double* dinv; double* tmp; };
struct LogdetWs { double* partial; };

size_t factor_ws(int64_t n, int64_t b, int64_t a, void* p, FactorWs* o, int prec) {
  (void)n;
  Carver c(p);
  FactorWs w;
  w.Linv = c.take((size_t)(b * b));
  w.W = c.take((size_t)(b * b));
  w.Wa = c.take((size_t)(a * b + 1));
  w.coop = (void*)c.take(kCoopScratch / sizeof(double));
  w.tc_bytes = tc_bytes_for(b, a, 1, prec);
  w.tc = w.tc_bytes ? (void*)c.take(w.tc_bytes / sizeof(double) + 1) : nullptr;
  if (o) *o = w;
  return c.off;
}

size_t selinv_ws(int64_t n, int64_t b, int64_t a, void* p, SelinvWs* o, int prec) {
  Carver c(p);
  SelinvWs w;
  w.Linv = c.take((size_t)(n * b * b));
  w.G = c.take((size_t)((n - 1) * b * b + 1));
  w.H = c.take((size_t)(n * a * b + 1));
  w.LtInv = c.take((size_t)(a * a + 1));
  w.tc_bytes = tc_bytes_for(b, a, n, prec);
  w.tc = w.tc_bytes ? (void*)c.take(w.tc_bytes / sizeof(double) + 1) : nullptr;
  if (o) *o = w;
  return c.off;
}

// Order of the diagonal sub-blocks of L_ii that the solve inverts: b itself up
// to 256, else 256 (ceil(b / 256) sub-blocks, the last one ragged).
inline int64_t solve_sub(int64_t b) { return b < 256 ? b : 256; }

// with_inverses: space for the inverses of the diagonal sub-blocks (the
// standalone solve forms them; the one-call forms use the selected inversion's
// L_ii^{-1} instead).
size_t solve_ws(int64_t n, int64_t b, int64_t a, int64_t R, void* p, SolveWs* o,
                bool with_inverses = true) {
  Carver c(p);
  SolveWs w;
  const int64_t ds = solve_sub(b), nsb = (b + ds - 1) / ds;
  w.partial = c.take((size_t)(arrow_chunks(n) * a * R + 1));
  w.dinv = with_inverses ? c.take((size_t)(n * nsb * ds * ds)) : nullptr;
  w.tmp = c.take((size_t)(b * R));
  if (o) *o = w;
  return c.off;
}

size_t logdet_ws(int64_t n, void* p, LogdetWs* o) {
  Carver c(p);
  LogdetWs w;
  w.partial = c.take((size_t)(n + 1));
  if (o) *o = w;
  return c.off;
}

// Shared checks; argument positions follow the C signatures (1-based).
int check_sizes(int64_t n, int64_t b, int64_t a) {
  if (n < 1 || n > (1 << 24)) return -1;
  if (b < 1 || b > 32768) return -2;
  if (a < 0 || a > 32768) return -3;
  return 0;
}

int check_blocks(int64_t n, int64_t a, const double* diag, const double* lower,
                 const double* arrow, const double* tip) {
  if (!diag || misaligned(diag)) return -4;
  if (n > 1 && (!lower || misaligned(lower))) return -5;
  if (a > 0 && (!arrow || misaligned(arrow))) return -6;
  if (a > 0 && (!tip || misaligned(tip))) return -7;
  return 0;
}

GemmArgs one_term(const GemmTerm& t, double* C, int64_t ldc, int M, int N, double beta,
                  int lowerC) {
  GemmArgs g{};
  g.t[0] = t;
  g.nterms = 1;
  g.C = C;
  g.ldc = ldc;
  g.M = M;
  g.N = N;
  g.beta = beta;
  g.lowerC = lowerC;
  g.nb1 = 1;
  g.nb2 = 1;
  return g;
}

// Precision of the large block products (process-wide; see bta_set_precision).
int g_prec = BTA_PREC_FP64;

// Classes of GEMM call sites, to route them by precision mode.
enum { CLS_SCHUR = 0, CLS_TRSM = 1, CLS_SELINV = 2 };

int tc_mode_of(int prec) { return prec == BTA_PREC_OZAKI ? TC_OZ : (prec == BTA_PREC_BF16X3 ? TC_X3 : 0); }

bool routes_to_tc(int prec, int cls) {
  if (prec == BTA_PREC_OZAKI) return true;
  if (prec == BTA_PREC_BF16X3) return cls == CLS_SCHUR || cls == CLS_SELINV;
  return false;
}


struct TcWs {
  void* p = nullptr;
  size_t bytes = 0;
};

// Runs a (one- or two-term) GEMM. In a tensor-core precision mode an eligible
// product goes to gemm_tc (two terms concatenated along k there); otherwise the
// FP64 DMMA kernels run it. *used_tc (optional) tells which; reuse_b: op(B) is
// the one the previous gemm_tc call on tw split (see gemm_tc).
cudaError_t gemm_run(const GemmArgs& g, int cls, const TcWs& tw, int prec, cudaStream_t s,
                     bool* used_tc = nullptr, bool reuse_b = false) {
  if (used_tc) *used_tc = false;
  if (prec == BTA_PREC_FP64 || !routes_to_tc(prec, cls) || !tw.p) return gemm_f64(g, s);
  int kmax = 0, ksum = 0;
  for (int i = 0; i < g.nterms; ++i) {
    kmax = g.t[i].K > kmax ? g.t[i].K : kmax;
    ksum += g.t[i].K;
  }
  // The tensor-core path costs three launches and a splitting pass; it pays for
  // products of at least 2^25 multiply-adds (a 512^3 block product).
  // A product with few rows (the arrowhead's a) pays for the tensor cores only
  // when the split of its large op(B) is already in the workspace.
  const double macs = (double)g.M * g.N * ksum * g.nb1 * g.nb2;
  const bool large = g.M >= 64 && macs >= 33554432.0;
  const bool skinny_reuse = reuse_b && g.nb1 * g.nb2 == 1;
  if (g.N >= 64 && kmax >= 64 && (large || skinny_reuse)) {
    if (used_tc) *used_tc = true;
    return gemm_tc(g, tc_mode_of(prec), tw.p, tw.bytes, s, reuse_b);
  }
  return gemm_f64(g, s);
}

// TRTRI's doubling products, routed like the TRSM substitution they serve.
struct HookCtx {
  TcWs tw;
  int prec;
};
cudaError_t trtri_hook(const GemmArgs& g, void* ctx, cudaStream_t s) {
  return gemm_run(g, CLS_TRSM, ((HookCtx*)ctx)->tw, ((HookCtx*)ctx)->prec, s);
}

// Blocks of at least this order are factored by the cooperative step kernel (one
// matrix at a time); smaller ones, and matrices of a batch running on concurrent
// streams, use the panel-by-panel launches with TRTRI + products for the TRSMs.
constexpr int64_t kCoopMinB = 128;
// In the tensor-core modes, blocks up to this order solve their panels in FP64
// inside the step kernel (n=365, b=1024: Ozaki factor 907 ms against 998 ms with
// TRTRI + tensor-core TRMM). Larger ones do so only where the TRSM products would
// run in FP64 anyway (BF16x3; n=256, b=2048: 3.45 s against 4.66 s); with Ozaki
// they take the inverse + tensor-core product, whose cost grows slower than the
// FP64 solve's b^3 (n=256, b=2048: 2.07 s against 3.64 s).
#ifndef BTA_HYBRID_MAX_B
#define BTA_HYBRID_MAX_B 1024
#endif
constexpr int64_t kHybridMaxB = BTA_HYBRID_MAX_B;

// L_ii = POTRF(A_ii) and Linv = L_ii^{-1} (row stride b) for a block whose
// triangular solves go to the tensor cores (Ozaki, b > kHybridMaxB), by halves
// (h = the first half's order, a multiple of the tile):
//   L11 = POTRF(A11), L11^{-1};  L21 = A21 L11^{-T};  A22 -= L21 L21^T;
//   L22 = POTRF(A22), L22^{-1};  (L^{-1})21 = -L22^{-1} (L21 L11^{-1}).
// The two POTRFs run on the FP64 step kernel in place (a quarter of the FP64
// work of one POTRF of order b); the products run on the tensor cores.
int potrf_trtri_halves(double* Di, int64_t b, int64_t info_row0, const FactorWs& w, const TcWs& tw,
                       int prec, cudaStream_t s) {
  const int64_t h = (b / 2) / T * T, m = b - h;
  double* A11 = Di;
  double* A21 = Di + h * b;
  double* A22 = Di + h * b + h;
  double* I11 = w.Linv;
  double* I21 = w.Linv + h * b;
  double* I22 = w.Linv + h * b + h;
  HookCtx hc{tw, prec};
  BTA_TRY(factor_step_coop(A11, nullptr, nullptr, nullptr, nullptr, nullptr, (int)h, 0, 0, info_row0,
                           w.coop, s, 1, b));
  BTA_TRY(trtri_blocks(A11, b, b * b, I11, b, b * b, 1, (int)h, s, trtri_hook, &hc));
  // L21 = A21 L11^{-T} (via W), then A22 -= L21 L21^T (lower tiles)
  BTA_TRY(gemm_run(one_term(term(A21, b, OP_N, TRI_NONE, I11, b, OP_T, TRI_UPPER, (int)h, 1.0), w.W, b,
                            (int)m, (int)h, 0.0, 0), CLS_TRSM, tw, prec, s));
  BTA_TRY(cudaMemcpy2DAsync(A21, b * sizeof(double), w.W, b * sizeof(double), h * sizeof(double), m,
                            cudaMemcpyDeviceToDevice, s));
  BTA_TRY(gemm_run(one_term(term(A21, b, OP_N, TRI_NONE, A21, b, OP_T, TRI_NONE, (int)h, -1.0), A22, b,
                            (int)m, (int)m, 1.0, 1), CLS_SCHUR, tw, prec, s));
  BTA_TRY(factor_step_coop(A22, nullptr, nullptr, nullptr, nullptr, nullptr, (int)m, 0, 0, info_row0 + h,
                           w.coop, s, 1, b));
  BTA_TRY(trtri_blocks(A22, b, b * b, I22, b, b * b, 1, (int)m, s, trtri_hook, &hc));
  // (L^{-1})21 = -L22^{-1} (L21 L11^{-1})
  BTA_TRY(gemm_run(one_term(term(A21, b, OP_N, TRI_NONE, I11, b, OP_N, TRI_LOWER, (int)h, 1.0), w.W, b,
                            (int)m, (int)h, 0.0, 0), CLS_TRSM, tw, prec, s));
  BTA_TRY(gemm_run(one_term(term(I22, b, OP_N, TRI_LOWER, w.W, b, OP_N, TRI_NONE, (int)m, -1.0), I21, b,
                            (int)m, (int)h, 0.0, 0), CLS_TRSM, tw, prec, s));
  // strict upper triangles: L_ii and L_ii^{-1} are lower triangular
  BTA_TRY(cudaMemset2DAsync(Di + h, b * sizeof(double), 0, m * sizeof(double), h, s));
  BTA_TRY(cudaMemset2DAsync(w.Linv + h, b * sizeof(double), 0, m * sizeof(double), h, s));
  return 0;
}

int factor_impl(int64_t n, int64_t b, int64_t a, double* diag, double* lower, double* arrow,
                double* tip, const FactorWs& w, int prec, cudaStream_t s, bool coop = true) {
  const int B = (int)b, Aa = (int)a;
  const int64_t bb = b * b;
  TcWs tw;
  tw.p = w.tc;
  tw.bytes = w.tc_bytes;
  if (coop && b >= kCoopMinB && prec == BTA_PREC_FP64) {
    // One fused launch per block step: tile Cholesky of the block column with
    // the Schur updates of the next block, its arrow block and the tip.
    for (int64_t i = 0; i < n; ++i) {
      const bool nx = i + 1 < n;
      BTA_TRY(factor_step_coop(diag + i * bb, nx ? lower + i * bb : nullptr,
                               nx ? diag + (i + 1) * bb : nullptr, a > 0 ? arrow + i * a * b : nullptr,
                               (a > 0 && nx) ? arrow + (i + 1) * a * b : nullptr, a > 0 ? tip : nullptr,
                               B, Aa, nx ? 1 : 0, i * b, w.coop, s));
    }
    if (a > 0) BTA_TRY(potrf_blocks(tip, a, a * a, 1, Aa, n * b, 0, s));
    return 0;
  }
  if (coop && b >= kCoopMinB && (b <= kHybridMaxB || !routes_to_tc(prec, CLS_TRSM))) {
    // Tensor-core modes: the step kernel factors the block column (POTRF and the
    // panel solves of L_{i+1,i}, L_{n,i} in FP64); the Schur products go through
    // gemm_run (tensor cores for the large ones).
    for (int64_t i = 0; i < n; ++i) {
      const bool nx = i + 1 < n;
      double* Di = diag + i * bb;
      double* Li = nx ? lower + i * bb : nullptr;
      double* Ai = a > 0 ? arrow + i * a * b : nullptr;
      BTA_TRY(factor_step_coop(Di, Li, nullptr, Ai, nullptr, nullptr, B, Aa, nx ? 1 : 0, i * b,
                               w.coop, s, /*schur=*/0));
      bool split_L = false;  // the SYRK's split of L_{i+1,i} is in the workspace
      if (nx)  // A_{i+1,i+1} -= L_{i+1,i} L_{i+1,i}^T  (lower tiles)
        BTA_TRY(gemm_run(one_term(term(Li, b, OP_N, TRI_NONE, Li, b, OP_T, TRI_NONE, B, -1.0),
                                  Di + bb, b, B, B, 1.0, 1), CLS_SCHUR, tw, prec, s, &split_L));
      if (a > 0) {
        if (nx)  // A_{n,i+1} -= L_{n,i} L_{i+1,i}^T
          BTA_TRY(gemm_run(one_term(term(Ai, b, OP_N, TRI_NONE, Li, b, OP_T, TRI_NONE, B, -1.0),
                                    Ai + a * b, b, Aa, B, 1.0, 0), CLS_SCHUR, tw, prec, s, nullptr,
                           split_L));
        // A_{n,n} -= L_{n,i} L_{n,i}^T
        BTA_TRY(gemm_run(one_term(term(Ai, b, OP_N, TRI_NONE, Ai, b, OP_T, TRI_NONE, B, -1.0),
                                  tip, a, Aa, Aa, 1.0, 1), CLS_SCHUR, tw, prec, s));
      }
    }
    if (a > 0) BTA_TRY(potrf_blocks(tip, a, a * a, 1, Aa, n * b, 0, s));
    return 0;
  }
  for (int64_t i = 0; i < n; ++i) {
    double* Di = diag + i * bb;
    HookCtx hc{tw, prec};
    if (coop && b >= 2 * kCoopMinB && routes_to_tc(prec, CLS_TRSM)) {
      const int rc = potrf_trtri_halves(Di, b, i * b, w, tw, prec, s);
      if (rc) return rc;
    } else {
      if (coop && b >= kCoopMinB)  // the step kernel on A_ii alone: one cooperative POTRF
        BTA_TRY(factor_step_coop(Di, nullptr, nullptr, nullptr, nullptr, nullptr, B, 0, 0, i * b,
                                 w.coop, s));
      else
        BTA_TRY(potrf_blocks(Di, b, bb, 1, B, i * b, 0, s));
      BTA_TRY(trtri_blocks(Di, b, bb, w.Linv, b, bb, 1, B, s, trtri_hook, &hc));
    }
    // The two TRSMs share op(B) = L_ii^{-T}, and the arrow's Schur product shares
    // the SYRK's L_{i+1,i}: on the tensor cores each pair splits it once.
    double* Li = i + 1 < n ? lower + i * bb : nullptr;
    double* Ai = a > 0 ? arrow + i * a * b : nullptr;
    bool split_inv = false, split_L = false;
    if (Li)  // L_{i+1,i} = A_{i+1,i} L_ii^{-T}
      BTA_TRY(gemm_run(one_term(term(Li, b, OP_N, TRI_NONE, w.Linv, b, OP_T, TRI_UPPER, B, 1.0),
                                w.W, b, B, B, 0.0, 0), CLS_TRSM, tw, prec, s, &split_inv));
    if (Ai) {  // L_{n,i} = A_{n,i} L_ii^{-T}
      BTA_TRY(gemm_run(one_term(term(Ai, b, OP_N, TRI_NONE, w.Linv, b, OP_T, TRI_UPPER, B, 1.0),
                                w.Wa, b, Aa, B, 0.0, 0), CLS_TRSM, tw, prec, s, nullptr, split_inv));
      BTA_TRY(cudaMemcpyAsync(Ai, w.Wa, a * b * sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    if (Li) {
      BTA_TRY(cudaMemcpyAsync(Li, w.W, bb * sizeof(double), cudaMemcpyDeviceToDevice, s));
      // A_{i+1,i+1} -= L_{i+1,i} L_{i+1,i}^T  (lower tiles)
      BTA_TRY(gemm_run(one_term(term(Li, b, OP_N, TRI_NONE, Li, b, OP_T, TRI_NONE, B, -1.0),
                                Di + bb, b, B, B, 1.0, 1), CLS_SCHUR, tw, prec, s, &split_L));
      if (Ai)  // A_{n,i+1} -= L_{n,i} L_{i+1,i}^T
        BTA_TRY(gemm_run(one_term(term(Ai, b, OP_N, TRI_NONE, Li, b, OP_T, TRI_NONE, B, -1.0),
                                  Ai + a * b, b, Aa, B, 1.0, 0), CLS_SCHUR, tw, prec, s, nullptr, split_L));
    }
    if (Ai)  // A_{n,n} -= L_{n,i} L_{n,i}^T
      BTA_TRY(gemm_run(one_term(term(Ai, b, OP_N, TRI_NONE, Ai, b, OP_T, TRI_NONE, B, -1.0),
                                tip, a, Aa, Aa, 1.0, 1), CLS_SCHUR, tw, prec, s));
  }
  if (a > 0) BTA_TRY(potrf_blocks(tip, a, a * a, 1, Aa, n * b, 0, s));
  return 0;
}

// Called after backward step i of the selected inversion, once diag[i],
// lower[i] and arrow[i] hold their final X blocks (enqueue-time hook).
typedef cudaError_t (*StepHook)(int64_t i, void* ctx);

// on_linv (called with i = -1) runs as soon as every L_ii^{-1} is in w.Linv (it
// stays there until the call returns). before_write (i = -1) runs after M_i has
// been written into diag and before the first write into the tip, lower or arrow
// blocks (X_nn, then the backward sweep): work that reads the factor's lower,
// arrow and tip blocks and the inverses, but not diag, may run on another stream
// between the two.
int selinv_impl(int64_t n, int64_t b, int64_t a, double* diag, double* lower, double* arrow,
                double* tip, const SelinvWs& w, int prec, cudaStream_t s,
                StepHook after = nullptr, void* after_ctx = nullptr,
                StepHook before_write = nullptr, void* bw_ctx = nullptr,
                StepHook on_linv = nullptr, void* ol_ctx = nullptr) {
  const int B = (int)b, Aa = (int)a;
  const int64_t bb = b * b, ab = a * b;
  TcWs tw;
  tw.p = w.tc;
  tw.bytes = w.tc_bytes;
  // Prologue, independent over i: L_ii^{-1}, G_i, H_i, M_i; then X_nn.
  HookCtx hc{tw, prec};
  BTA_TRY(trtri_blocks(diag, b, bb, w.Linv, b, bb, (int)n, B, s, trtri_hook, &hc));
  if (on_linv) BTA_TRY(on_linv(-1, ol_ctx));
  if (n > 1) {
    GemmArgs g = one_term(term(lower, b, OP_N, TRI_NONE, w.Linv, b, OP_N, TRI_LOWER, B, 1.0),
                          w.G, b, B, B, 0.0, 0);
    g.t[0].sA1 = bb; g.t[0].sB1 = bb; g.sC1 = bb; g.nb1 = (int)(n - 1);
    BTA_TRY(gemm_run(g, CLS_SELINV, tw, prec, s));
  }
  if (a > 0) {
    GemmArgs g = one_term(term(arrow, b, OP_N, TRI_NONE, w.Linv, b, OP_N, TRI_LOWER, B, 1.0),
                          w.H, b, Aa, B, 0.0, 0);
    g.t[0].sA1 = ab; g.t[0].sB1 = bb; g.sC1 = ab; g.nb1 = (int)n;
    BTA_TRY(gemm_run(g, CLS_SELINV, tw, prec, s));
  }
  {
    GemmArgs g = one_term(term(w.Linv, b, OP_T, TRI_UPPER, w.Linv, b, OP_N, TRI_LOWER, B, 1.0),
                          diag, b, B, B, 0.0, 1);
    g.t[0].sA1 = bb; g.t[0].sB1 = bb; g.sC1 = bb; g.nb1 = (int)n;
    BTA_TRY(gemm_run(g, CLS_SELINV, tw, prec, s));
  }
  if (before_write) BTA_TRY(before_write(-1, bw_ctx));
  if (a > 0) {
    BTA_TRY(trtri_blocks(tip, a, a * a, w.LtInv, a, a * a, 1, Aa, s));
    BTA_TRY(gemm_run(one_term(term(w.LtInv, a, OP_T, TRI_UPPER, w.LtInv, a, OP_N, TRI_LOWER, Aa,
                                   1.0),
                              tip, a, Aa, Aa, 0.0, 0), CLS_SELINV, tw, prec, s));
  }
  // Backward sweep.
  for (int64_t i = n - 1; i >= 0; --i) {
    double* Di = diag + i * bb;
    const double* Gi = w.G + i * bb;
    const double* Hi = w.H + i * ab;
    // X_{i+1,i} and X_ii share op(B) = [G_i; H_i]: on the tensor cores the second
    // product reuses the first one's split of it.
    bool b_split = false;
    if (i + 1 < n) {
      // X_{i+1,i} = -X_{i+1,i+1} G_i - X_{n,i+1}^T H_i
      GemmArgs g = one_term(term(Di + bb, b, OP_N, TRI_NONE, Gi, b, OP_N, TRI_NONE, B, -1.0),
                            lower + i * bb, b, B, B, 0.0, 0);
      if (a > 0) {
        g.t[1] = term(arrow + (i + 1) * ab, b, OP_T, TRI_NONE, Hi, b, OP_N, TRI_NONE, Aa, -1.0);
        g.nterms = 2;
      }
      BTA_TRY(gemm_run(g, CLS_SELINV, tw, prec, s, &b_split));
    }
    if (a > 0) {
      // X_{n,i} = -X_{n,i+1} G_i - X_nn H_i (terms in the order of op(B) = [G_i; H_i],
      // whose split it reuses on the tensor cores)
      GemmArgs g = one_term(term(tip, a, OP_N, TRI_NONE, Hi, b, OP_N, TRI_NONE, Aa, -1.0),
                            arrow + i * ab, b, Aa, B, 0.0, 0);
      if (i + 1 < n) {
        g.t[1] = g.t[0];
        g.t[0] = term(arrow + (i + 1) * ab, b, OP_N, TRI_NONE, Gi, b, OP_N, TRI_NONE, B, -1.0);
        g.nterms = 2;
      }
      BTA_TRY(gemm_run(g, CLS_SELINV, tw, prec, s, nullptr, b_split));
    }
    // X_ii = M_i - X_{i+1,i}^T G_i - X_{n,i}^T H_i  (lower tiles, then mirrored)
    GemmArgs g{};
    g.C = Di; g.ldc = b; g.M = B; g.N = B; g.beta = 1.0; g.lowerC = 1; g.nb1 = 1; g.nb2 = 1;
    if (i + 1 < n)
      g.t[g.nterms++] = term(lower + i * bb, b, OP_T, TRI_NONE, Gi, b, OP_N, TRI_NONE, B, -1.0);
    if (a > 0)
      g.t[g.nterms++] = term(arrow + i * ab, b, OP_T, TRI_NONE, Hi, b, OP_N, TRI_NONE, Aa, -1.0);
    if (g.nterms) BTA_TRY(gemm_run(g, CLS_SELINV, tw, prec, s, nullptr, b_split));
    BTA_TRY(mirror_lower(Di, b, bb, 1, B, s));
    if (after) BTA_TRY(after(i, after_ctx));
  }
  return 0;
}

// Standalone solve (block forward / backward substitution over the pattern).
// Inside a block the triangular solve is blocked by the diagonal sub-blocks of
// order ds = min(b, 256): their inverses D_ij are formed first (one batched
// TRTRI per sub-block column), then each sub-step is two matrix-vector products
// that spread over the whole GPU: y_j = D_ij t_j and, right-looking, the rows
// below (forward) or above (backward) take the update from y_j. A block step
// thus has ceil(b / 256) dependent sub-steps instead of one per 32-row tile.
int solve_impl(int64_t n, int64_t b, int64_t a, const double* diag, const double* lower,
               const double* arrow, const double* tip, double* rhs, int64_t R,
               const SolveWs& w, cudaStream_t s) {
  const int B = (int)b, Rr = (int)R;
  const int64_t bb = b * b, bR = b * R;
  const int64_t ds = solve_sub(b), nsb = (b + ds - 1) / ds, dss = ds * ds;
  double* rn = rhs + n * bR;
  for (int64_t j = 0; j < nsb; ++j) {
    const int64_t o = j * ds, sz = std::min(ds, b - o);
    BTA_TRY(trtri_blocks(diag + o * (b + 1), b, bb, w.dinv + j * dss, ds, nsb * dss, (int)n, (int)sz, s));
  }
  for (int64_t i = 0; i < n; ++i) {
    const double* Li = diag + i * bb;
    const double* Di = w.dinv + i * nsb * dss;
    double* yi = rhs + i * bR;
    // t = r_i - L_{i,i-1} y_{i-1}
    if (i > 0)
      BTA_TRY(gemv_multi(lower + (i - 1) * bb, b, OP_N, B, B, rhs + (i - 1) * bR, R, w.tmp, R, Rr, -1.0, s,
                         1.0, yi));
    else
      BTA_TRY(cudaMemcpyAsync(w.tmp, yi, bR * sizeof(double), cudaMemcpyDeviceToDevice, s));
    for (int64_t j = 0; j < nsb; ++j) {
      const int64_t o = j * ds, sz = std::min(ds, b - o);
      BTA_TRY(gemv_multi(Di + j * dss, ds, OP_N, (int)sz, (int)sz, w.tmp + o * R, R, yi + o * R, R, Rr, 1.0, s,
                         0.0, nullptr, TRI_LOWER));
      if (o + sz < b)  // t(o+sz:) -= L_ii(o+sz:, o:o+sz) y_i(o:o+sz)
        BTA_TRY(gemv_multi(Li + (o + sz) * b + o, b, OP_N, (int)(b - o - sz), (int)sz, yi + o * R, R,
                           w.tmp + (o + sz) * R, R, Rr, -1.0, s));
    }
  }
  if (a > 0) {
    BTA_TRY(arrow_gather(arrow, n, b, a, rhs, Rr, w.partial, arrow_chunks(n), rn, s));
    BTA_TRY(trsv_lower(tip, a, (int)a, rn, R, Rr, false, s));
    BTA_TRY(trsv_lower(tip, a, (int)a, rn, R, Rr, true, s));
    BTA_TRY(arrow_scatter(arrow, n, b, a, rn, Rr, rhs, s));
  }
  for (int64_t i = n - 1; i >= 0; --i) {
    const double* Li = diag + i * bb;
    const double* Di = w.dinv + i * nsb * dss;
    double* xi = rhs + i * bR;
    // t = y_i - L_{i+1,i}^T x_{i+1} (the arrow term is already subtracted)
    if (i + 1 < n)
      BTA_TRY(gemv_multi(lower + i * bb, b, OP_T, B, B, rhs + (i + 1) * bR, R, w.tmp, R, Rr, -1.0, s, 1.0,
                         xi));
    else
      BTA_TRY(cudaMemcpyAsync(w.tmp, xi, bR * sizeof(double), cudaMemcpyDeviceToDevice, s));
    for (int64_t j = nsb - 1; j >= 0; --j) {
      const int64_t o = j * ds, sz = std::min(ds, b - o);
      BTA_TRY(gemv_multi(Di + j * dss, ds, OP_T, (int)sz, (int)sz, w.tmp + o * R, R, xi + o * R, R, Rr, 1.0, s,
                         0.0, nullptr, TRI_LOWER));
      if (o > 0)  // t(:o) -= L_ii(o:o+sz, :o)^T x_i(o:o+sz)
        BTA_TRY(gemv_multi(Li + o * b, b, OP_T, (int)o, (int)sz, xi + o * R, R, w.tmp, R, Rr, -1.0, s));
    }
  }
  return 0;
}

// The solve with the block inverses Linv_i = L_ii^{-1} at hand (formed by the
// selected inversion's prologue): every block step is two bandwidth-bound
// products instead of a chain of triangular tile solves, and L_ii itself is not
// read. Forward: y_i = Linv_i (r_i - L_{i,i-1} y_{i-1}); y_n = L_nn^{-1}(r_n -
// sum_i L_{n,i} y_i). Backward: x_n = L_nn^{-T} y_n; x_i = Linv_i^T (y_i -
// L_{i+1,i}^T x_{i+1} - L_{n,i}^T x_n). Reads lower, arrow, tip (L_nn) and Linv.
int solve_inv_impl(int64_t n, int64_t b, int64_t a, const double* lower, const double* arrow,
                   const double* tip, const double* Linv, double* rhs, int64_t R, const SolveWs& w,
                   cudaStream_t s) {
  const int B = (int)b, Rr = (int)R;
  const int64_t bb = b * b, bR = b * R;
  double* rn = rhs + n * bR;
  for (int64_t i = 0; i < n; ++i) {
    // tmp = r_i - L_{i,i-1} y_{i-1}; y_i = Linv_i tmp
    if (i > 0)
      BTA_TRY(gemv_multi(lower + (i - 1) * bb, b, OP_N, B, B, rhs + (i - 1) * bR, R, w.tmp, R, Rr, -1.0,
                         s, 1.0, rhs + i * bR));
    else
      BTA_TRY(cudaMemcpyAsync(w.tmp, rhs, bR * sizeof(double), cudaMemcpyDeviceToDevice, s));
    BTA_TRY(gemv_multi(Linv + i * bb, b, OP_N, B, B, w.tmp, R, rhs + i * bR, R, Rr, 1.0, s, 0.0,
                       nullptr, TRI_LOWER));
  }
  if (a > 0) {
    BTA_TRY(arrow_gather(arrow, n, b, a, rhs, Rr, w.partial, arrow_chunks(n), rn, s));
    BTA_TRY(trsv_lower(tip, a, (int)a, rn, R, Rr, false, s));
    BTA_TRY(trsv_lower(tip, a, (int)a, rn, R, Rr, true, s));
    BTA_TRY(arrow_scatter(arrow, n, b, a, rn, Rr, rhs, s));
  }
  for (int64_t i = n - 1; i >= 0; --i) {
    // tmp = y_i - L_{i+1,i}^T x_{i+1} (the arrow term is already subtracted); x_i = Linv_i^T tmp
    if (i + 1 < n)
      BTA_TRY(gemv_multi(lower + i * bb, b, OP_T, B, B, rhs + (i + 1) * bR, R, w.tmp, R, Rr, -1.0, s,
                         1.0, rhs + i * bR));
    else
      BTA_TRY(cudaMemcpyAsync(w.tmp, rhs + i * bR, bR * sizeof(double), cudaMemcpyDeviceToDevice, s));
    BTA_TRY(gemv_multi(Linv + i * bb, b, OP_T, B, B, w.tmp, R, rhs + i * bR, R, Rr, 1.0, s, 0.0,
                       nullptr, TRI_LOWER));
  }
  return 0;
}

// Runs `body(ws)` on a stream-ordered temporary workspace of `bytes`.
template <class F>
int with_async_ws(size_t bytes, cudaStream_t s, F body) {
  void* p = nullptr;
  if (bytes) BTA_TRY(cudaMallocAsync(&p, bytes, s));
  const int rc = body(p);
  if (p) {
    cudaError_t e = cudaFreeAsync(p, s);
    if (rc == 0 && e != cudaSuccess) return (int)e;
  }
  return rc;
}

size_t tc_bytes_for(int64_t b, int64_t a, int64_t batch, int prec) {
  const int mode = tc_mode_of(prec);
  if (!mode || b < 64) return 0;
  const int m = (int)(a > b ? a : b);  // the widest product: b x b, or a x b / a x a blocks
  const int k = (int)(((b + 31) / 32 + (a + 31) / 32) * 32);  // two terms concatenated along k
  return tc_workspace_bytes(mode, m, m, k > m ? k : m, (int)(batch < 1 ? 1 : batch));
}

// Side streams (and fork/join events) for batched calls, created once per device.
struct StreamPool {
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> join;
  cudaEvent_t fork = nullptr;
};
std::mutex g_pool_mu;
StreamPool g_pools[64];

cudaError_t pool_for(int k, StreamPool** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_pool_mu);
  StreamPool& p = g_pools[dev];
  if (!p.fork) {
    e = cudaEventCreateWithFlags(&p.fork, cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
  }
  while ((int)p.streams.size() < k) {
    cudaStream_t st;
    cudaEvent_t ev;
    e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
    p.streams.push_back(st);
    p.join.push_back(ev);
  }
  *out = &p;
  return cudaSuccess;
}

size_t batch_entry_ws(int64_t n, int64_t b, int64_t a, int prec) {
  const size_t f = factor_ws(n, b, a, nullptr, nullptr, prec);
  const size_t s = selinv_ws(n, b, a, nullptr, nullptr, prec);
  const size_t l = logdet_ws(n, nullptr, nullptr);
  return std::max(f, std::max(s, l));
}

double entry_flops(int64_t n, int64_t b, int64_t a) {
  const double B = (double)b, A = (double)a;
  return (double)n * (7.0 * B * B * B + 6.0 * A * B * B);
}


// ---------------------------------------------------------------------------
// Partitioned factorization and selected inversion on one device (the paper's
// Sections 3.1-3.4). The block rows are split into P contiguous partitions: a
// top one and P-1 middle ones. Eliminating the interior blocks of every
// partition is a Schur complement onto the boundary blocks (the top partition's
// last block, each middle partition's first and last block) and the tip, and the
// partitions' eliminations are independent, so each runs on its own stream. In
// a middle partition the first block s is ordered after the interior (the
// paper's shifting permutation, never materialized): eliminating interior block
// i couples s with i+1, a fill-in block carried as the coupling F = A~_{i+1,s}
// and the factor column L_{s,i} (stored per interior block). The boundary blocks
// form a BTA matrix with 2P-1 diagonal blocks (the reduced system), factored and
// inverted as usual. Each partition's interior blocks of X then follow from
// X L = L^{-T} on the permuted factor:
//   X_{i+1,i} = -X_{i+1,i+1} G_i - X_{i+1,s} Gs_i - X_{n,i+1}^T H_i
//   X_{i,s}   = -G_i^T X_{i+1,s} - Gs_i^T X_{s,s} - H_i^T X_{n,s}
//   X_{n,i}   = -X_{n,i+1} G_i - X_{n,s} Gs_i - X_nn H_i
//   X_{i,i}   =  M_i - X_{i+1,i}^T G_i - X_{i,s} Gs_i - X_{n,i}^T H_i
// with G_i = L_{i+1,i} L_ii^{-1}, Gs_i = L_{s,i} L_ii^{-1}, H_i = L_{n,i} L_ii^{-1},
// M_i = L_ii^{-T} L_ii^{-1} (the Gs terms vanish in the top partition).
// ---------------------------------------------------------------------------
constexpr int kMaxParts = 64;

struct PartPlan {
  int P = 0;
  int64_t s[kMaxParts], e[kMaxParts];
};

// Sizes: the top partition is `lb` times a middle one (the paper's load-balancing
// ratio; middle partitions carry the fill-in work), middle partitions >= 2 blocks.
PartPlan plan_partitions(int64_t n, int P, double lb) {
  PartPlan p;
  if (P < 1) P = 1;
  while (P > 1 && (double)n < lb + 2.0 * (P - 1)) --P;
  if (P == 1) {
    p.P = 1; p.s[0] = 0; p.e[0] = n;
    return p;
  }
  int64_t m = (int64_t)((double)n / (lb + (P - 1)));
  if (m < 2) m = 2;
  int64_t top = n - m * (P - 1);
  if (top < 1) { top = 1; m = (n - 1) / (P - 1); }
  p.P = P;
  p.s[0] = 0; p.e[0] = top;
  int64_t at = top;
  for (int j = 1; j < P; ++j) {
    const int64_t len = (j == P - 1) ? n - at : m;
    p.s[j] = at; p.e[j] = at + len;
    at += len;
  }
  return p;
}

struct PartWs {
  double *W, *Wa, *Ft, *LinvF, *U, *Ls, *Li, *G, *Gs, *H;
  void* tc;
  size_t tc_bytes;
};

struct PartLayout {
  PartPlan plan;
  PartWs part[kMaxParts];
  double *rd, *rl, *ra, *rt, *ldp, *rldp;
  FactorWs rf;
  SelinvWs rs;
  int64_t nr;
};

size_t part_layout(int64_t n, int64_t b, int64_t a, int P, double lb, int prec, void* base,
                   PartLayout* out) {
  Carver c(base);
  PartLayout L;
  L.plan = plan_partitions(n, P, lb);
  const int64_t bb = b * b;
  for (int j = 0; j < L.plan.P; ++j) {
    const int64_t nj = L.plan.e[j] - L.plan.s[j];
    PartWs& w = L.part[j];
    w.W = c.take(bb);
    w.Wa = c.take(a * b + 1);
    w.Ft = c.take(bb);
    w.LinvF = c.take(bb);
    w.U = c.take(a * a + 1);
    w.Ls = c.take(j ? nj * bb : 1);
    w.Li = c.take(nj * bb);
    w.G = c.take(nj * bb);
    w.Gs = c.take(j ? nj * bb : 1);
    w.H = c.take(nj * a * b + 1);
    w.tc_bytes = tc_bytes_for(b, a, nj, prec);
    w.tc = w.tc_bytes ? (void*)c.take(w.tc_bytes / sizeof(double) + 1) : nullptr;
  }
  L.nr = 2 * L.plan.P - 1;
  L.rd = c.take(L.nr * bb);
  L.rl = c.take((L.nr - 1) * bb + 1);
  L.ra = c.take(L.nr * a * b + 1);
  L.rt = c.take(a * a + 1);
  L.ldp = c.take(n + 1);
  L.rldp = c.take(L.nr + 2);
  const size_t fsz = factor_ws(L.nr, b, a, base ? (char*)base + c.off : nullptr, &L.rf, prec);
  c.off += align_up(fsz);
  const size_t ssz = selinv_ws(L.nr, b, a, base ? (char*)base + c.off : nullptr, &L.rs, prec);
  c.off += align_up(ssz);
  if (out) *out = L;
  return c.off;
}

// One interior elimination step of block i in partition storage: L_ii, L_{i+1,i},
// L_{n,i}, the Schur updates of block i+1 and of the arrow, and the tip part into U.
int part_eliminate(int64_t i, int64_t b, int64_t a, double* diag, double* lower, double* arrow,
                   const PartWs& w, int prec, cudaStream_t s) {
  const int B = (int)b, Aa = (int)a;
  const int64_t bb = b * b;
  TcWs tw;
  tw.p = w.tc;
  tw.bytes = w.tc_bytes;
  double* Di = diag + i * bb;
  BTA_TRY(potrf_blocks(Di, b, bb, 1, B, i * b, 0, s));
  HookCtx hc{tw, prec};
  BTA_TRY(trtri_blocks(Di, b, bb, w.LinvF, b, bb, 1, B, s, trtri_hook, &hc));
  double* Li = lower + i * bb;
  BTA_TRY(gemm_run(one_term(term(Li, b, OP_N, TRI_NONE, w.LinvF, b, OP_T, TRI_UPPER, B, 1.0), w.W, b,
                            B, B, 0.0, 0), CLS_TRSM, tw, prec, s));
  BTA_TRY(cudaMemcpyAsync(Li, w.W, bb * sizeof(double), cudaMemcpyDeviceToDevice, s));
  BTA_TRY(gemm_run(one_term(term(Li, b, OP_N, TRI_NONE, Li, b, OP_T, TRI_NONE, B, -1.0), Di + bb, b,
                            B, B, 1.0, 1), CLS_SCHUR, tw, prec, s));
  if (a > 0) {
    double* Ai = arrow + i * a * b;
    BTA_TRY(gemm_run(one_term(term(Ai, b, OP_N, TRI_NONE, w.LinvF, b, OP_T, TRI_UPPER, B, 1.0), w.Wa,
                              b, Aa, B, 0.0, 0), CLS_TRSM, tw, prec, s));
    BTA_TRY(cudaMemcpyAsync(Ai, w.Wa, a * b * sizeof(double), cudaMemcpyDeviceToDevice, s));
    BTA_TRY(gemm_run(one_term(term(Ai, b, OP_N, TRI_NONE, Li, b, OP_T, TRI_NONE, B, -1.0), Ai + a * b,
                              b, Aa, B, 1.0, 0), CLS_SCHUR, tw, prec, s));
    BTA_TRY(gemm_run(one_term(term(Ai, b, OP_N, TRI_NONE, Ai, b, OP_T, TRI_NONE, B, -1.0), w.U, a, Aa,
                              Aa, 1.0, 1), CLS_SCHUR, tw, prec, s));
  }
  return 0;
}

int part_factor(int j, const PartLayout& L, int64_t b, int64_t a, double* diag, double* lower,
                double* arrow, int prec, cudaStream_t s) {
  const PartWs& w = L.part[j];
  const int64_t st = L.plan.s[j], en = L.plan.e[j], bb = b * b;
  const int B = (int)b, Aa = (int)a;
  TcWs tw;
  tw.p = w.tc;
  tw.bytes = w.tc_bytes;
  if (a > 0) BTA_TRY(cudaMemsetAsync(w.U, 0, a * a * sizeof(double), s));
  if (j == 0) {
    for (int64_t i = st; i < en - 1; ++i) {
      int rc = part_eliminate(i, b, a, diag, lower, arrow, w, prec, s);
      if (rc) return rc;
    }
    if (en - 1 > st) BTA_TRY(logdet_partials(diag + st * bb, en - 1 - st, b, nullptr, 0, L.ldp + st, s));
    return 0;
  }
  // Middle partition: the coupling (first interior, s) is A_{s+1,s}.
  BTA_TRY(cudaMemcpyAsync(w.Ft, lower + st * bb, bb * sizeof(double), cudaMemcpyDeviceToDevice, s));
  double* Ds = diag + st * bb;
  double* As = arrow + st * a * b;
  for (int64_t i = st + 1; i < en - 1; ++i) {
    int rc = part_eliminate(i, b, a, diag, lower, arrow, w, prec, s);
    if (rc) return rc;
    // (part_eliminate left L_ii^{-1} in LinvF)
    double* Lsi = w.Ls + (i - st - 1) * bb;
    double* Lo = lower + i * bb;
    // L_{s,i} = F^T L_ii^{-T}
    BTA_TRY(gemm_run(one_term(term(w.Ft, b, OP_T, TRI_NONE, w.LinvF, b, OP_T, TRI_UPPER, B, 1.0), Lsi,
                              b, B, B, 0.0, 0), CLS_TRSM, tw, prec, s));
    // A_ss -= L_{s,i} L_{s,i}^T ; F <- -L_{i+1,i} L_{s,i}^T ; A_{n,s} -= L_{n,i} L_{s,i}^T
    BTA_TRY(gemm_run(one_term(term(Lsi, b, OP_N, TRI_NONE, Lsi, b, OP_T, TRI_NONE, B, -1.0), Ds, b, B,
                              B, 1.0, 1), CLS_SCHUR, tw, prec, s));
    BTA_TRY(gemm_run(one_term(term(Lo, b, OP_N, TRI_NONE, Lsi, b, OP_T, TRI_NONE, B, -1.0), w.Ft, b, B,
                              B, 0.0, 0), CLS_SCHUR, tw, prec, s));
    if (a > 0)
      BTA_TRY(gemm_run(one_term(term(arrow + i * a * b, b, OP_N, TRI_NONE, Lsi, b, OP_T, TRI_NONE, B,
                                     -1.0), As, b, Aa, B, 1.0, 0), CLS_SCHUR, tw, prec, s));
  }
  if (en - 1 > st + 1)
    BTA_TRY(logdet_partials(diag + (st + 1) * bb, en - 2 - st, b, nullptr, 0, L.ldp + st + 1, s));
  return 0;
}

int part_sweep(int j, const PartLayout& L, int64_t b, int64_t a, double* diag, double* lower,
               double* arrow, const double* tip, int prec, cudaStream_t s) {
  const PartWs& w = L.part[j];
  const int64_t st = L.plan.s[j], en = L.plan.e[j], bb = b * b, ab = a * b;
  const int B = (int)b, Aa = (int)a;
  const int64_t i0 = j == 0 ? st : st + 1, i1 = en - 1, m = i1 - i0;
  TcWs tw;
  tw.p = w.tc;
  tw.bytes = w.tc_bytes;
  if (m > 0) {
    HookCtx hc{tw, prec};
    BTA_TRY(trtri_blocks(diag + i0 * bb, b, bb, w.Li, b, bb, (int)m, B, s, trtri_hook, &hc));
    GemmArgs g = one_term(term(lower + i0 * bb, b, OP_N, TRI_NONE, w.Li, b, OP_N, TRI_LOWER, B, 1.0),
                          w.G, b, B, B, 0.0, 0);
    g.t[0].sA1 = bb; g.t[0].sB1 = bb; g.sC1 = bb; g.nb1 = (int)m;
    BTA_TRY(gemm_run(g, CLS_SELINV, tw, prec, s));
    if (j > 0) {
      GemmArgs gs = one_term(term(w.Ls, b, OP_N, TRI_NONE, w.Li, b, OP_N, TRI_LOWER, B, 1.0), w.Gs, b,
                             B, B, 0.0, 0);
      gs.t[0].sA1 = bb; gs.t[0].sB1 = bb; gs.sC1 = bb; gs.nb1 = (int)m;
      BTA_TRY(gemm_run(gs, CLS_SELINV, tw, prec, s));
    }
    if (a > 0) {
      GemmArgs gh = one_term(term(arrow + i0 * ab, b, OP_N, TRI_NONE, w.Li, b, OP_N, TRI_LOWER, B,
                                  1.0), w.H, b, Aa, B, 0.0, 0);
      gh.t[0].sA1 = ab; gh.t[0].sB1 = bb; gh.sC1 = ab; gh.nb1 = (int)m;
      BTA_TRY(gemm_run(gh, CLS_SELINV, tw, prec, s));
    }
    GemmArgs gm = one_term(term(w.Li, b, OP_T, TRI_UPPER, w.Li, b, OP_N, TRI_LOWER, B, 1.0),
                           diag + i0 * bb, b, B, B, 0.0, 1);
    gm.t[0].sA1 = bb; gm.t[0].sB1 = bb; gm.sC1 = bb; gm.nb1 = (int)m;
    BTA_TRY(gemm_run(gm, CLS_SELINV, tw, prec, s));
  }
  double* Ds = diag + st * bb;   // X_ss (middle partitions)
  double* As = arrow + st * ab;  // X_{n,s}
  for (int64_t i = i1 - 1; i >= i0; --i) {
    const int64_t k = i - i0;
    const double* Gk = w.G + k * bb;
    const double* Gsk = w.Gs + k * bb;
    const double* Hk = w.H + k * ab;
    double* Di = diag + i * bb;
    // X_{i+1,i}
    GemmArgs g1 = one_term(term(Di + bb, b, OP_N, TRI_NONE, Gk, b, OP_N, TRI_NONE, B, -1.0),
                           lower + i * bb, b, B, B, 0.0, 0);
    if (j > 0) g1.t[g1.nterms++] = term(w.Ft, b, OP_N, TRI_NONE, Gsk, b, OP_N, TRI_NONE, B, -1.0);
    if (a > 0) g1.t[g1.nterms++] = term(arrow + (i + 1) * ab, b, OP_T, TRI_NONE, Hk, b, OP_N, TRI_NONE, Aa, -1.0);
    BTA_TRY(gemm_run(g1, CLS_SELINV, tw, prec, s));
    // X_{i,s} (middle) into W
    if (j > 0) {
      GemmArgs g2 = one_term(term(Gk, b, OP_T, TRI_NONE, w.Ft, b, OP_N, TRI_NONE, B, -1.0), w.W, b, B,
                             B, 0.0, 0);
      g2.t[g2.nterms++] = term(Gsk, b, OP_T, TRI_NONE, Ds, b, OP_N, TRI_NONE, B, -1.0);
      if (a > 0) g2.t[g2.nterms++] = term(Hk, b, OP_T, TRI_NONE, As, b, OP_N, TRI_NONE, Aa, -1.0);
      BTA_TRY(gemm_run(g2, CLS_SELINV, tw, prec, s));
    }
    // X_{n,i}
    if (a > 0) {
      GemmArgs g3 = one_term(term(tip, a, OP_N, TRI_NONE, Hk, b, OP_N, TRI_NONE, Aa, -1.0),
                             arrow + i * ab, b, Aa, B, 0.0, 0);
      g3.t[g3.nterms++] = term(arrow + (i + 1) * ab, b, OP_N, TRI_NONE, Gk, b, OP_N, TRI_NONE, B, -1.0);
      if (j > 0) g3.t[g3.nterms++] = term(As, b, OP_N, TRI_NONE, Gsk, b, OP_N, TRI_NONE, B, -1.0);
      BTA_TRY(gemm_run(g3, CLS_SELINV, tw, prec, s));
    }
    // X_ii (lower tiles, then mirrored)
    GemmArgs g4{};
    g4.C = Di; g4.ldc = b; g4.M = B; g4.N = B; g4.beta = 1.0; g4.lowerC = 1; g4.nb1 = 1; g4.nb2 = 1;
    g4.t[g4.nterms++] = term(lower + i * bb, b, OP_T, TRI_NONE, Gk, b, OP_N, TRI_NONE, B, -1.0);
    if (j > 0) g4.t[g4.nterms++] = term(w.W, b, OP_N, TRI_NONE, Gsk, b, OP_N, TRI_NONE, B, -1.0);
    if (a > 0) g4.t[g4.nterms++] = term(arrow + i * ab, b, OP_T, TRI_NONE, Hk, b, OP_N, TRI_NONE, Aa, -1.0);
    BTA_TRY(gemm_run(g4, CLS_SELINV, tw, prec, s));
    BTA_TRY(mirror_lower(Di, b, bb, 1, B, s));
    if (j > 0) BTA_TRY(cudaMemcpyAsync(w.Ft, w.W, bb * sizeof(double), cudaMemcpyDeviceToDevice, s));
  }
  if (j > 0) BTA_TRY(cudaMemcpyAsync(lower + st * bb, w.Ft, bb * sizeof(double), cudaMemcpyDeviceToDevice, s));
  return 0;
}

int partitioned_impl(int64_t n, int64_t b, int64_t a, double* diag, double* lower, double* arrow,
                     double* tip, double* logdet_out, const PartLayout& L, int prec, cudaStream_t s0) {
  const PartPlan& pl = L.plan;
  const int P = pl.P;
  const int64_t bb = b * b, ab = a * b;
  StreamPool* pool = nullptr;
  BTA_TRY(pool_for(P, &pool));
  BTA_TRY(cudaMemsetAsync(L.ldp, 0, (n + 1) * sizeof(double), s0));
  auto fork = [&]() -> int {
    BTA_TRY(cudaEventRecord(pool->fork, s0));
    for (int j = 0; j < P; ++j) BTA_TRY(cudaStreamWaitEvent(pool->streams[j], pool->fork, 0));
    return 0;
  };
  auto join = [&]() -> int {
    for (int j = 0; j < P; ++j) {
      BTA_TRY(cudaEventRecord(pool->join[j], pool->streams[j]));
      BTA_TRY(cudaStreamWaitEvent(s0, pool->join[j], 0));
    }
    return 0;
  };
  int rc = fork();
  if (rc) return rc;
  for (int j = 0; j < P; ++j) {
    rc = part_factor(j, L, b, a, diag, lower, arrow, prec, pool->streams[j]);
    if (rc) return rc;
  }
  rc = join();
  if (rc) return rc;
  // Reduced system: [last_0, first_1, last_1, ..., first_{P-1}, last_{P-1}].
  int64_t idx[2 * kMaxParts];
  int64_t nr = 0;
  idx[nr++] = pl.e[0] - 1;
  for (int j = 1; j < P; ++j) {
    idx[nr++] = pl.s[j];
    idx[nr++] = pl.e[j] - 1;
  }
  const cudaMemcpyKind dd = cudaMemcpyDeviceToDevice;
  for (int64_t k = 0; k < nr; ++k) {
    BTA_TRY(cudaMemcpyAsync(L.rd + k * bb, diag + idx[k] * bb, bb * 8, dd, s0));
    if (a > 0) BTA_TRY(cudaMemcpyAsync(L.ra + k * ab, arrow + idx[k] * ab, ab * 8, dd, s0));
  }
  for (int j = 1; j < P; ++j) {
    BTA_TRY(cudaMemcpyAsync(L.rl + (2 * j - 2) * bb, lower + (pl.s[j] - 1) * bb, bb * 8, dd, s0));
    BTA_TRY(cudaMemcpyAsync(L.rl + (2 * j - 1) * bb, L.part[j].Ft, bb * 8, dd, s0));
  }
  if (a > 0) {
    BTA_TRY(cudaMemcpyAsync(L.rt, tip, a * a * 8, dd, s0));
    for (int j = 0; j < P; ++j) BTA_TRY(axpy_f64(a * a, 1.0, L.part[j].U, L.rt, s0));
  }
  rc = factor_impl(nr, b, a, L.rd, L.rl, L.ra, L.rt, L.rf, prec, s0);
  if (rc) return rc;
  BTA_TRY(logdet_partials(L.rd, nr, b, L.rt, a, L.rldp, s0));
  if (logdet_out) BTA_TRY(logdet_combine(L.ldp, n, L.rldp, nr + (a > 0 ? 1 : 0), logdet_out, s0));
  rc = selinv_impl(nr, b, a, L.rd, L.rl, L.ra, L.rt, L.rs, prec, s0);
  if (rc) return rc;
  for (int64_t k = 0; k < nr; ++k) {
    BTA_TRY(cudaMemcpyAsync(diag + idx[k] * bb, L.rd + k * bb, bb * 8, dd, s0));
    if (a > 0) BTA_TRY(cudaMemcpyAsync(arrow + idx[k] * ab, L.ra + k * ab, ab * 8, dd, s0));
  }
  for (int j = 1; j < P; ++j) {
    BTA_TRY(cudaMemcpyAsync(lower + (pl.s[j] - 1) * bb, L.rl + (2 * j - 2) * bb, bb * 8, dd, s0));
    BTA_TRY(cudaMemcpyAsync(L.part[j].Ft, L.rl + (2 * j - 1) * bb, bb * 8, dd, s0));
  }
  if (a > 0) BTA_TRY(cudaMemcpyAsync(tip, L.rt, a * a * 8, dd, s0));
  rc = fork();
  if (rc) return rc;
  for (int j = 0; j < P; ++j) {
    rc = part_sweep(j, L, b, a, diag, lower, arrow, tip, prec, pool->streams[j]);
    if (rc) return rc;
  }
  return join();
}

}  // namespace

// ---------------------------------------------------------------------------
// The whole per-matrix sequence in one call: factor, log det, solve, selinv.
// The solve only reads the factor, and so does the part of the selected
// inversion's prologue that forms L_ii^{-1}, G_i and H_i: the solve runs on a
// side stream concurrently with them, and the selected inversion waits for it
// before its first write into the factor's blocks. From host memory (host mode)
// the pattern is also streamed in by chunks of blocks ahead of the factor sweep
// and X streamed back behind the backward sweep.
// ---------------------------------------------------------------------------
struct PipeWs {
  double *diag, *lower, *arrow, *tip, *rhs, *ld;  // device copies (host mode)
  FactorWs fw;
  SelinvWs sw;
  SolveWs vw;
  LogdetWs lw;
};

size_t pipe_ws(int64_t n, int64_t b, int64_t a, int64_t R, bool host, void* p, PipeWs* o, int prec) {
  Carver c(p);
  PipeWs w{};
  if (host) {
    w.diag = c.take((size_t)(n * b * b));
    w.lower = c.take((size_t)((n - 1) * b * b + 1));
    w.arrow = c.take((size_t)(n * a * b + 1));
    w.tip = c.take((size_t)(a * a + 1));
    w.rhs = c.take((size_t)((n * b + a) * (R > 0 ? R : 1)));
    w.ld = c.take(1);
  }
  // factor, log det and selinv run one after another on the caller's stream and
  // share one scratch region; the solve, concurrent with selinv, has its own.
  char* sub = p ? (char*)p + c.off : nullptr;
  size_t region = factor_ws(n, b, a, sub, &w.fw, prec);
  region = std::max(region, selinv_ws(n, b, a, sub, &w.sw, prec));
  region = std::max(region, logdet_ws(n, sub, &w.lw));
  c.off += align_up(region);
  if (R > 0) {
    const size_t vsz = solve_ws(n, b, a, R, p ? (char*)p + c.off : nullptr, &w.vw, false);
    c.off += align_up(vsz);
  }
  if (o) *o = w;
  return c.off;
}

std::mutex g_ev_mu;
std::vector<cudaEvent_t> g_events[64];

cudaError_t events_for(size_t k, cudaEvent_t** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_ev_mu);
  std::vector<cudaEvent_t>& v = g_events[dev];
  while (v.size() < k) {
    cudaEvent_t ev;
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
    v.push_back(ev);
  }
  *out = v.data();
  return cudaSuccess;
}

struct PipeCtx {
  int64_t n, b, a, C;
  double *diag, *lower, *arrow;  // device blocks
  double *xd, *xl, *xa;          // host outputs (host mode)
  cudaStream_t s, cout;
  cudaEvent_t* evout;
  cudaEvent_t ev_solved;
  bool host, solving;
  // the solve (R > 0), started once the prologue has formed L_ii^{-1}
  double *tip, *rhs, *x_host;
  int64_t R;
  const SolveWs* vw;
  const double* linv;
  cudaStream_t cs;
  cudaEvent_t ev_linv;
};

// Blocks [i, i + C) are final: copy them back on the copy-out stream.
cudaError_t pipe_after_step(int64_t i, void* ctx) {
  PipeCtx& h = *(PipeCtx*)ctx;
  if (!h.host || i % h.C) return cudaSuccess;
  const int64_t bb = h.b * h.b, ab = h.a * h.b, i1 = std::min(h.n, i + h.C);
  cudaEvent_t ev = h.evout[i / h.C];
  cudaError_t e = cudaEventRecord(ev, h.s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(h.cout, ev, 0);
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(h.xd + i * bb, h.diag + i * bb, (i1 - i) * bb * sizeof(double),
                      cudaMemcpyDeviceToHost, h.cout);
  const int64_t l1 = std::min(h.n - 1, i1);
  if (e == cudaSuccess && l1 > i)
    e = cudaMemcpyAsync(h.xl + i * bb, h.lower + i * bb, (l1 - i) * bb * sizeof(double),
                        cudaMemcpyDeviceToHost, h.cout);
  if (e == cudaSuccess && h.a > 0)
    e = cudaMemcpyAsync(h.xa + i * ab, h.arrow + i * ab, (i1 - i) * ab * sizeof(double),
                        cudaMemcpyDeviceToHost, h.cout);
  return e;
}

// The selected inversion's first write into the blocks the solve reads (tip,
// lower, arrow): the solve must be done.
cudaError_t pipe_before_write(int64_t, void* ctx) {
  PipeCtx& h = *(PipeCtx*)ctx;
  return h.solving ? cudaStreamWaitEvent(h.s, h.ev_solved, 0) : cudaSuccess;
}

// Every L_ii^{-1} is formed: the solve runs on the side stream, beside the rest
// of the prologue, and the solution goes back to the host once it is done.
cudaError_t pipe_solve(int64_t, void* ctx) {
  PipeCtx& h = *(PipeCtx*)ctx;
  if (!h.solving) return cudaSuccess;
  cudaError_t e = cudaEventRecord(h.ev_linv, h.s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(h.cs, h.ev_linv, 0);
  if (e != cudaSuccess) return e;
  const int rc = solve_inv_impl(h.n, h.b, h.a, h.lower, h.arrow, h.tip, h.linv, h.rhs, h.R, *h.vw, h.cs);
  if (rc) return rc > 0 ? (cudaError_t)rc : cudaErrorInvalidValue;
  e = cudaEventRecord(h.ev_solved, h.cs);
  if (e != cudaSuccess) return e;
  if (h.host) {
    e = cudaStreamWaitEvent(h.cout, h.ev_solved, 0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(h.x_host, h.rhs, (h.n * h.b + h.a) * h.R * sizeof(double), cudaMemcpyDeviceToHost,
                          h.cout);
  }
  return e;
}

// Host mode: h* are host inputs, x* host outputs, the blocks live in w's device
// copies. Device mode: d* are the caller's device blocks (in place) and rhs its
// device right-hand sides; ld_dev receives log det.
struct PipeArgs {
  bool host;
  const double *hd, *hl, *ha, *ht, *hr;  // host inputs
  double *xd, *xl, *xa, *xt, *x, *hld;   // host outputs
  double *dd, *dl, *da, *dt, *dr, *ld_dev;  // device blocks (device mode)
};

int pipeline_impl(int64_t n, int64_t b, int64_t a, int64_t R, const PipeArgs& io, const PipeWs& w,
                  int prec, cudaStream_t s) {
  const int64_t bb = b * b, ab = a * b;
  double* diag = io.host ? w.diag : io.dd;
  double* lower = io.host ? w.lower : io.dl;
  double* arrow = io.host ? w.arrow : io.da;
  double* tip = io.host ? w.tip : io.dt;
  double* rhs = io.host ? w.rhs : io.dr;
  double* ld = io.host ? w.ld : io.ld_dev;
  // Chunks of about 32 MB of input (at least one block).
  const int64_t per_block = (2 * bb + ab) * (int64_t)sizeof(double);
  const int64_t C = std::max<int64_t>(1, std::min<int64_t>(n, (32ll << 20) / per_block));
  const int64_t nch = io.host ? (n + C - 1) / C : 0;
  StreamPool* pool = nullptr;
  BTA_TRY(pool_for(3, &pool));
  cudaStream_t cin = pool->streams[0], cout = pool->streams[1], cs = pool->streams[2];
  cudaEvent_t* ev = nullptr;
  BTA_TRY(events_for((size_t)(2 * nch + 4), &ev));
  cudaEvent_t ev_start = ev[0], ev_factored = ev[1], ev_solved = ev[2], ev_done = ev[3];
  cudaEvent_t* evin = ev + 4;
  cudaEvent_t* evout = ev + 4 + nch;
  if (io.host) {
    // The copy streams start after the caller's earlier work on s. Inputs: tip
    // and right-hand sides first, then the blocks chunk by chunk.
    BTA_TRY(cudaEventRecord(ev_start, s));
    BTA_TRY(cudaStreamWaitEvent(cin, ev_start, 0));
    BTA_TRY(cudaStreamWaitEvent(cout, ev_start, 0));
    if (a > 0)
      BTA_TRY(cudaMemcpyAsync(tip, io.ht, a * a * sizeof(double), cudaMemcpyHostToDevice, cin));
    if (R > 0)
      BTA_TRY(cudaMemcpyAsync(rhs, io.hr, (n * b + a) * R * sizeof(double), cudaMemcpyHostToDevice,
                              cin));
    for (int64_t c = 0; c < nch; ++c) {
      const int64_t i0 = c * C, i1 = std::min(n, i0 + C), l1 = std::min(n - 1, i1);
      BTA_TRY(cudaMemcpyAsync(diag + i0 * bb, io.hd + i0 * bb, (i1 - i0) * bb * sizeof(double),
                              cudaMemcpyHostToDevice, cin));
      if (l1 > i0)
        BTA_TRY(cudaMemcpyAsync(lower + i0 * bb, io.hl + i0 * bb, (l1 - i0) * bb * sizeof(double),
                                cudaMemcpyHostToDevice, cin));
      if (a > 0)
        BTA_TRY(cudaMemcpyAsync(arrow + i0 * ab, io.ha + i0 * ab, (i1 - i0) * ab * sizeof(double),
                                cudaMemcpyHostToDevice, cin));
      BTA_TRY(cudaEventRecord(evin[c], cin));
    }
  }
  // Factor: step i needs blocks i and i+1 on the device.
  int64_t waited = -1;
  auto wait_block = [&](int64_t i) -> cudaError_t {
    if (!io.host) return cudaSuccess;
    const int64_t c = std::min(i, n - 1) / C;
    while (waited < c) {
      ++waited;
      cudaError_t e = cudaStreamWaitEvent(s, evin[waited], 0);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  };
  if (b >= kCoopMinB && prec == BTA_PREC_FP64) {
    for (int64_t i = 0; i < n; ++i) {
      const bool nx = i + 1 < n;
      BTA_TRY(wait_block(i + 1));
      BTA_TRY(factor_step_coop(diag + i * bb, nx ? lower + i * bb : nullptr,
                               nx ? diag + (i + 1) * bb : nullptr, a > 0 ? arrow + i * ab : nullptr,
                               (a > 0 && nx) ? arrow + (i + 1) * ab : nullptr, a > 0 ? tip : nullptr,
                               (int)b, (int)a, nx ? 1 : 0, i * b, w.fw.coop, s));
    }
    if (a > 0) BTA_TRY(potrf_blocks(tip, a, a * a, 1, (int)a, n * b, 0, s));
  } else {
    BTA_TRY(wait_block(n - 1));
    const int rc = factor_impl(n, b, a, diag, lower, arrow, tip, w.fw, prec, s);
    if (rc) return rc;
  }
  BTA_TRY(logdet_f64(diag, n, b, tip, a, w.lw.partial, ld, s));
  if (io.host) BTA_TRY(cudaMemcpyAsync(io.hld, ld, sizeof(double), cudaMemcpyDeviceToHost, s));
  PipeCtx hp{n, b, a, C, diag, lower, arrow, io.xd, io.xl, io.xa, s, cout, evout, ev_solved,
             io.host, R > 0, tip, rhs, io.x, R, &w.vw, w.sw.Linv, cs, ev_factored};
  {
    const int rc = selinv_impl(n, b, a, diag, lower, arrow, tip, w.sw, prec, s, pipe_after_step, &hp,
                               pipe_before_write, &hp, pipe_solve, &hp);
    if (rc) return rc;
  }
  if (io.host) {
    if (a > 0)  // X_nn is final since the prologue; it follows chunk 0's event
      BTA_TRY(cudaMemcpyAsync(io.xt, tip, a * a * sizeof(double), cudaMemcpyDeviceToHost, cout));
    BTA_TRY(cudaEventRecord(ev_done, cout));
    BTA_TRY(cudaStreamWaitEvent(s, ev_done, 0));
  }
  return 0;
}

extern "C" {

int bta_version(void) { return 100; }

size_t bta_workspace_bytes(int op, int64_t n, int64_t b, int64_t a, int64_t nrhs) {
  if (check_sizes(n, b, a)) return 0;
  switch (op) {
    case BTA_OP_FACTOR: return factor_ws(n, b, a, nullptr, nullptr, g_prec);
    case BTA_OP_SELINV: return selinv_ws(n, b, a, nullptr, nullptr, g_prec);
    case BTA_OP_SOLVE:
      if (nrhs < 1 || nrhs > 64) return 0;
      return solve_ws(n, b, a, nrhs, nullptr, nullptr);
    case BTA_OP_LOGDET: return logdet_ws(n, nullptr, nullptr);
    default: return 0;
  }
}

int bta_factor_ws(int64_t n, int64_t b, int64_t a, double* diag, double* lower, double* arrow,
                  double* tip, void* ws, size_t ws_bytes, bta_stream_t stream) {
  int rc = check_sizes(n, b, a);
  if (!rc) rc = check_blocks(n, a, diag, lower, arrow, tip);
  if (rc) return rc;
  FactorWs w;
  const int prec = g_prec;
  const size_t need = factor_ws(n, b, a, ws, &w, prec);
  if (!ws || ((uintptr_t)ws % kAlign)) return -8;
  if (ws_bytes < need) return -9;
  return factor_impl(n, b, a, diag, lower, arrow, tip, w, prec, (cudaStream_t)stream);
}

int bta_factor(int64_t n, int64_t b, int64_t a, double* diag, double* lower, double* arrow,
               double* tip, bta_stream_t stream) {
  int rc = check_sizes(n, b, a);
  if (!rc) rc = check_blocks(n, a, diag, lower, arrow, tip);
  if (rc) return rc;
  const size_t need = factor_ws(n, b, a, nullptr, nullptr, g_prec);
  return with_async_ws(need, (cudaStream_t)stream, [&](void* p) {
    return bta_factor_ws(n, b, a, diag, lower, arrow, tip, p, need, stream);
  });
}

int bta_selinv_ws(int64_t n, int64_t b, int64_t a, double* diag, double* lower, double* arrow,
                  double* tip, void* ws, size_t ws_bytes, bta_stream_t stream) {
  int rc = check_sizes(n, b, a);
  if (!rc) rc = check_blocks(n, a, diag, lower, arrow, tip);
  if (rc) return rc;
  SelinvWs w;
  const int prec = g_prec;
  const size_t need = selinv_ws(n, b, a, ws, &w, prec);
  if (!ws || ((uintptr_t)ws % kAlign)) return -8;
  if (ws_bytes < need) return -9;
  return selinv_impl(n, b, a, diag, lower, arrow, tip, w, prec, (cudaStream_t)stream);
}

int bta_selinv(int64_t n, int64_t b, int64_t a, double* diag, double* lower, double* arrow,
               double* tip, bta_stream_t stream) {
  int rc = check_sizes(n, b, a);
  if (!rc) rc = check_blocks(n, a, diag, lower, arrow, tip);
  if (rc) return rc;
  const size_t need = selinv_ws(n, b, a, nullptr, nullptr, g_prec);
  return with_async_ws(need, (cudaStream_t)stream, [&](void* p) {
    return bta_selinv_ws(n, b, a, diag, lower, arrow, tip, p, need, stream);
  });
}

int bta_solve_ws(int64_t n, int64_t b, int64_t a, const double* diag, const double* lower,
                 const double* arrow, const double* tip, double* rhs, int64_t nrhs, void* ws,
                 size_t ws_bytes, bta_stream_t stream) {
  int rc = check_sizes(n, b, a);
  if (!rc) rc = check_blocks(n, a, diag, lower, arrow, tip);
  if (rc) return rc;
  if (!rhs || misaligned(rhs)) return -8;
  if (nrhs < 1 || nrhs > 64) return -9;
  SolveWs w;
  const size_t need = solve_ws(n, b, a, nrhs, ws, &w);
  if (!ws || ((uintptr_t)ws % kAlign)) return -10;
  if (ws_bytes < need) return -11;
  return solve_impl(n, b, a, diag, lower, arrow, tip, rhs, nrhs, w, (cudaStream_t)stream);
}

int bta_solve(int64_t n, int64_t b, int64_t a, const double* diag, const double* lower,
              const double* arrow, const double* tip, double* rhs, int64_t nrhs,
              bta_stream_t stream) {
  int rc = check_sizes(n, b, a);
  if (!rc) rc = check_blocks(n, a, diag, lower, arrow, tip);
  if (rc) return rc;
  if (!rhs || misaligned(rhs)) return -8;
  if (nrhs < 1 || nrhs > 64) return -9;
  const size_t need = solve_ws(n, b, a, nrhs, nullptr, nullptr);
  return with_async_ws(need, (cudaStream_t)stream, [&](void* p) {
    return bta_solve_ws(n, b, a, diag, lower, arrow, tip, rhs, nrhs, p, need, stream);
  });
}

int bta_logdet_ws(int64_t n, int64_t b, int64_t a, const double* diag, const double* tip,
                  double* out_dev, void* ws, size_t ws_bytes, bta_stream_t stream) {
  int rc = check_sizes(n, b, a);
  if (rc) return rc;
  if (!diag || misaligned(diag)) return -4;
  if (a > 0 && (!tip || misaligned(tip))) return -5;
  if (!out_dev || misaligned(out_dev)) return -6;
  LogdetWs w;
  const size_t need = logdet_ws(n, ws, &w);
  if (!ws || ((uintptr_t)ws % kAlign)) return -7;
  if (ws_bytes < need) return -8;
  BTA_TRY(logdet_f64(diag, n, b, tip, a, w.partial, out_dev, (cudaStream_t)stream));
  return 0;
}

int bta_logdet(int64_t n, int64_t b, int64_t a, const double* diag, const double* tip,
               double* out_dev, bta_stream_t stream) {
  int rc = check_sizes(n, b, a);
  if (rc) return rc;
  if (!diag || misaligned(diag)) return -4;
  if (a > 0 && (!tip || misaligned(tip))) return -5;
  if (!out_dev || misaligned(out_dev)) return -6;
  const size_t need = logdet_ws(n, nullptr, nullptr);
  return with_async_ws(need, (cudaStream_t)stream, [&](void* p) {
    return bta_logdet_ws(n, b, a, diag, tip, out_dev, p, need, stream);
  });
}

size_t bta_batch_workspace_bytes(int64_t n, int64_t b, int64_t a, int prec) {
  if (check_sizes(n, b, a)) return 0;
  if (prec != BTA_PREC_FP64 && prec != BTA_PREC_OZAKI && prec != BTA_PREC_BF16X3) return 0;
  return batch_entry_ws(n, b, a, prec);
}

int bta_factor_selinv_batched(int64_t count, const bta_batch_entry* entries, int nstreams,
                              bta_stream_t stream) {
  if (count < 1 || count > (1 << 20)) return -1;
  if (!entries) return -2;
  if (nstreams < 1 || nstreams > 64) return -3;
  for (int64_t k = 0; k < count; ++k) {
    const bta_batch_entry& e = entries[k];
    if (check_sizes(e.n, e.b, e.a) || check_blocks(e.n, e.a, e.diag, e.lower, e.arrow, e.tip))
      return -2;
    if (e.prec != BTA_PREC_FP64 && e.prec != BTA_PREC_OZAKI && e.prec != BTA_PREC_BF16X3) return -2;
    if (!e.ws || ((uintptr_t)e.ws % kAlign) || e.ws_bytes < batch_entry_ws(e.n, e.b, e.a, e.prec))
      return -2;
    if (e.logdet_out && misaligned(e.logdet_out)) return -2;
  }
  const cudaStream_t s0 = (cudaStream_t)stream;
  const int ns = (int)std::min<int64_t>(nstreams, count);
  StreamPool* pool = nullptr;
  BTA_TRY(pool_for(ns, &pool));
  // Largest first, each matrix to the stream with the least work so far.
  std::vector<int64_t> order(count);
  for (int64_t k = 0; k < count; ++k) order[k] = k;
  std::sort(order.begin(), order.end(), [&](int64_t x, int64_t y) {
    return entry_flops(entries[x].n, entries[x].b, entries[x].a) >
           entry_flops(entries[y].n, entries[y].b, entries[y].a);
  });
  std::vector<double> load(ns, 0.0);
  BTA_TRY(cudaEventRecord(pool->fork, s0));
  for (int i = 0; i < ns; ++i) BTA_TRY(cudaStreamWaitEvent(pool->streams[i], pool->fork, 0));
  for (int64_t k : order) {
    const bta_batch_entry& e = entries[k];
    const int j = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    load[j] += entry_flops(e.n, e.b, e.a);
    cudaStream_t st = pool->streams[j];
    FactorWs fw;
    factor_ws(e.n, e.b, e.a, e.ws, &fw, e.prec);
    int rc = factor_impl(e.n, e.b, e.a, e.diag, e.lower, e.arrow, e.tip, fw, e.prec, st, false);
    if (rc) return rc;
    if (e.logdet_out) {
      LogdetWs lw;
      logdet_ws(e.n, e.ws, &lw);
      BTA_TRY(logdet_f64(e.diag, e.n, e.b, e.tip, e.a, lw.partial, e.logdet_out, st));
    }
    SelinvWs sw;
    selinv_ws(e.n, e.b, e.a, e.ws, &sw, e.prec);
    rc = selinv_impl(e.n, e.b, e.a, e.diag, e.lower, e.arrow, e.tip, sw, e.prec, st);
    if (rc) return rc;
  }
  for (int i = 0; i < ns; ++i) {
    BTA_TRY(cudaEventRecord(pool->join[i], pool->streams[i]));
    BTA_TRY(cudaStreamWaitEvent(s0, pool->join[i], 0));
  }
  return 0;
}

size_t bta_partitioned_workspace_bytes(int64_t n, int64_t b, int64_t a, int64_t P, double lb) {
  if (check_sizes(n, b, a) || P < 1 || P > kMaxParts || !(lb > 0.0)) return 0;
  return part_layout(n, b, a, (int)P, lb, g_prec, nullptr, nullptr);
}

int bta_factor_selinv_partitioned(int64_t n, int64_t b, int64_t a, double* diag, double* lower,
                                  double* arrow, double* tip, int64_t P, double lb,
                                  double* logdet_out, void* ws, size_t ws_bytes,
                                  bta_stream_t stream) {
  int rc = check_sizes(n, b, a);
  if (!rc) rc = check_blocks(n, a, diag, lower, arrow, tip);
  if (rc) return rc;
  if (P < 1 || P > kMaxParts) return -8;
  if (!(lb > 0.0)) return -9;
  if (logdet_out && misaligned(logdet_out)) return -10;
  const int prec = g_prec;
  PartLayout L;
  const size_t need = part_layout(n, b, a, (int)P, lb, prec, ws, &L);
  if (!ws || ((uintptr_t)ws % kAlign)) return -11;
  if (ws_bytes < need) return -12;
  return partitioned_impl(n, b, a, diag, lower, arrow, tip, logdet_out, L, prec, (cudaStream_t)stream);
}

size_t bta_host_pipeline_workspace_bytes(int64_t n, int64_t b, int64_t a, int64_t nrhs) {
  if (check_sizes(n, b, a) || nrhs < 0 || nrhs > 64) return 0;
  return pipe_ws(n, b, a, nrhs, true, nullptr, nullptr, g_prec);
}

int bta_factor_selinv_host(int64_t n, int64_t b, int64_t a, const double* h_diag,
                           const double* h_lower, const double* h_arrow, const double* h_tip,
                           const double* h_rhs, int64_t nrhs, double* x_diag, double* x_lower,
                           double* x_arrow, double* x_tip, double* x_sol, double* h_logdet,
                           void* ws, size_t ws_bytes, bta_stream_t stream) {
  int rc = check_sizes(n, b, a);
  if (rc) return rc;
  if (!h_diag || misaligned(h_diag)) return -4;
  if (n > 1 && (!h_lower || misaligned(h_lower))) return -5;
  if (a > 0 && (!h_arrow || misaligned(h_arrow))) return -6;
  if (a > 0 && (!h_tip || misaligned(h_tip))) return -7;
  if (nrhs < 0 || nrhs > 64) return -9;
  if (nrhs > 0 && (!h_rhs || misaligned(h_rhs))) return -8;
  if (!x_diag || misaligned(x_diag)) return -10;
  if (n > 1 && (!x_lower || misaligned(x_lower))) return -11;
  if (a > 0 && (!x_arrow || misaligned(x_arrow))) return -12;
  if (a > 0 && (!x_tip || misaligned(x_tip))) return -13;
  if (nrhs > 0 && (!x_sol || misaligned(x_sol))) return -14;
  if (!h_logdet || misaligned(h_logdet)) return -15;
  PipeWs w;
  const int prec = g_prec;
  const size_t need = pipe_ws(n, b, a, nrhs, true, ws, &w, prec);
  if (!ws || ((uintptr_t)ws % kAlign)) return -16;
  if (ws_bytes < need) return -17;
  PipeArgs io{};
  io.host = true;
  io.hd = h_diag; io.hl = h_lower; io.ha = h_arrow; io.ht = h_tip; io.hr = h_rhs;
  io.xd = x_diag; io.xl = x_lower; io.xa = x_arrow; io.xt = x_tip; io.x = x_sol; io.hld = h_logdet;
  return pipeline_impl(n, b, a, nrhs, io, w, prec, (cudaStream_t)stream);
}

size_t bta_all_workspace_bytes(int64_t n, int64_t b, int64_t a, int64_t nrhs) {
  if (check_sizes(n, b, a) || nrhs < 0 || nrhs > 64) return 0;
  return pipe_ws(n, b, a, nrhs, false, nullptr, nullptr, g_prec);
}

int bta_factor_selinv_all(int64_t n, int64_t b, int64_t a, double* diag, double* lower,
                          double* arrow, double* tip, double* rhs, int64_t nrhs, double* logdet_out,
                          void* ws, size_t ws_bytes, bta_stream_t stream) {
  int rc = check_sizes(n, b, a);
  if (!rc) rc = check_blocks(n, a, diag, lower, arrow, tip);
  if (rc) return rc;
  if (nrhs < 0 || nrhs > 64) return -9;
  if (nrhs > 0 && (!rhs || misaligned(rhs))) return -8;
  if (!logdet_out || misaligned(logdet_out)) return -10;
  PipeWs w;
  const int prec = g_prec;
  const size_t need = pipe_ws(n, b, a, nrhs, false, ws, &w, prec);
  if (!ws || ((uintptr_t)ws % kAlign)) return -11;
  if (ws_bytes < need) return -12;
  PipeArgs io{};
  io.host = false;
  io.dd = diag; io.dl = lower; io.da = arrow; io.dt = tip; io.dr = rhs; io.ld_dev = logdet_out;
  return pipeline_impl(n, b, a, nrhs, io, w, prec, (cudaStream_t)stream);
}

int bta_probe_fp64_peak(double* out_dev, int64_t iters, double* flops,
                        bta_stream_t stream) {
  if (!out_dev) return -1;
  if (iters < 1) return -2;
  if (!flops) return -3;
  BTA_TRY(fp64_probe(out_dev, iters, flops, (cudaStream_t)stream));
  return 0;
}

int bta_grad_blocks(int64_t n, int64_t b, int64_t a, const double* x_diag, const double* x_lower,
                    const double* x_arrow, const double* x_tip, const double* y, double alpha,
                    double beta, double* g_diag, double* g_lower, double* g_arrow, double* g_tip,
                    double* g_x, bta_stream_t stream) {
  int rc = check_sizes(n, b, a);
  if (rc) return rc;
  if (!x_diag || misaligned(x_diag)) return -4;
  if (n > 1 && (!x_lower || misaligned(x_lower))) return -5;
  if (a > 0 && (!x_arrow || misaligned(x_arrow))) return -6;
  if (a > 0 && (!x_tip || misaligned(x_tip))) return -7;
  if (!y || misaligned(y)) return -8;
  if (!g_diag || misaligned(g_diag)) return -11;
  if (n > 1 && (!g_lower || misaligned(g_lower))) return -12;
  if (a > 0 && (!g_arrow || misaligned(g_arrow))) return -13;
  if (a > 0 && (!g_tip || misaligned(g_tip))) return -14;
  if (g_x && misaligned(g_x)) return -15;
  BTA_TRY(grad_blocks(n, b, a, x_diag, x_lower, x_arrow, x_tip, y, alpha, beta, g_diag, g_lower,
                      g_arrow, g_tip, g_x, (cudaStream_t)stream));
  return 0;
}

int bta_dot(int64_t N, const double* x, const double* y, double* out_dev, void* ws,
            size_t ws_bytes, bta_stream_t stream) {
  if (N < 1) return -1;
  if (!x || misaligned(x)) return -2;
  if (!y || misaligned(y)) return -3;
  if (!out_dev || misaligned(out_dev)) return -4;
  if (!ws || misaligned(ws)) return -5;
  if (ws_bytes < (size_t)kDotCtas * sizeof(double)) return -6;
  BTA_TRY(dot_f64(N, x, y, (double*)ws, out_dev, (cudaStream_t)stream));
  return 0;
}

int bta_set_precision(int prec) {
  if (prec != BTA_PREC_FP64 && prec != BTA_PREC_OZAKI && prec != BTA_PREC_BF16X3) return -1;
  g_prec = prec;
  return 0;
}

int bta_get_precision(void) { return g_prec; }

size_t bta_gemm_workspace_bytes(int prec, int64_t M, int64_t N, int64_t K) {
  const int mode = tc_mode_of(prec);
  if (!mode || M < 1 || N < 1 || K < 1 || M > (1 << 30) || N > (1 << 30)) return 0;
  if (K > 16384) return 0;
  return tc_workspace_bytes(mode, (int)M, (int)N, (int)K, 1);
}

int bta_gemm(int prec, int64_t M, int64_t N, int64_t K, double alpha, const double* A, int64_t lda,
             int transA, const double* B, int64_t ldb, int transB, double beta, double* C,
             int64_t ldc, void* ws, size_t ws_bytes, bta_stream_t stream) {
  if (prec != BTA_PREC_FP64 && prec != BTA_PREC_OZAKI && prec != BTA_PREC_BF16X3) return -1;
  if (M < 1 || M > (1 << 30)) return -2;
  if (N < 1 || N > (1 << 30)) return -3;
  if (K < 1 || K > (1 << 30)) return -4;
  if (!A || misaligned(A)) return -6;
  if (lda < (transA ? M : K)) return -7;
  if (!B || misaligned(B)) return -9;
  if (ldb < (transB ? K : N)) return -10;
  if (!C || misaligned(C)) return -13;
  if (ldc < N) return -14;
  GemmArgs g = one_term(term(A, lda, transA ? OP_T : OP_N, TRI_NONE, B, ldb, transB ? OP_T : OP_N,
                             TRI_NONE, (int)K, alpha),
                        C, ldc, (int)M, (int)N, beta, 0);
  const int mode = tc_mode_of(prec);
  if (!mode) {
    BTA_TRY(gemm_f64(g, (cudaStream_t)stream));
    return 0;
  }
  if (!ws || ((uintptr_t)ws % kAlign)) return -15;
  if (K > 16384) return -4;
  if (ws_bytes < tc_workspace_bytes(mode, (int)M, (int)N, (int)K, 1)) return -16;
  BTA_TRY(gemm_tc(g, mode, ws, ws_bytes, (cudaStream_t)stream));
  return 0;
}

int bta_wait_selftest(int64_t polls, int* timed_out) {
  if (!timed_out) return -2;
  if (polls < 1 || polls > (1 << 20)) return -1;
  int* flag = nullptr;
  BTA_TRY(cudaMalloc(&flag, sizeof(int)));
  cudaError_t e = cudaMemset(flag, 0, sizeof(int));
  if (e == cudaSuccess) e = wait_selftest(flag, (unsigned)polls, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  cudaFree(flag);
  if (e != cudaSuccess) return (int)e;
  return bta_tc_status(timed_out);
}

int bta_tc_status(int* timed_out) {
  if (!timed_out) return -1;
  int a = 0, b = 0;
  BTA_TRY(tc_error_read_reset(&a));
  BTA_TRY(wait_error_read_reset(&b));
  *timed_out = (a || b) ? 1 : 0;
  return 0;
}

int bta_get_info(bta_stream_t stream, int64_t* info) {
  if (!info) return -2;
  long long v = 0;
  BTA_TRY(info_read_reset((cudaStream_t)stream, &v));
  *info = (int64_t)v;
  return 0;
}

}  // extern "C"
