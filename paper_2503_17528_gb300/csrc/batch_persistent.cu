// Persistent batched form: factorization (Algorithm 1), log-determinant and
// selected inversion (Algorithm 2) of many independent BTA matrices of uneven
// n, b, a in ONE cooperative launch (FP64).
//
// Work is described on the host as a list of operations per matrix, each a set
// of independent 32 x 32 tile items:
//   factor, per block step i and tile column k of block i (a right-looking tile
//   Cholesky of the block column [A_ii; A_{i+1,i}; A_{n,i}] whose trailing
//   updates reach A_{i+1,i+1}, A_{n,i+1} and the tip, as in the single-matrix
//   step kernel):
//     POTRF(k)   factor the diagonal tile (k, k)            1 item
//     PANEL(k)   solve the tiles below it, X L_kk^T = A      one item per tile
//     UPDATE(k)  A(r, c) -= L(r, k) L(c, k)^T, k < c <= r   R tiles of a column per item
//   then the tip's own tile Cholesky, and the log-determinant (per-tile log sums
//   written by POTRF, summed in a fixed order);
//   selected inversion: the inverses L_ii^{-1} of all blocks at once (diagonal
//   tile inverses, then one row of tiles at a time), the products
//   G_i = L_{i+1,i} L_ii^{-1}, H_i = L_{n,i} L_ii^{-1}, M_i = L_ii^{-T} L_ii^{-1}
//   (every i at once), X_nn, and the backward recurrence for i = n-1 .. 0:
//     X_{i+1,i} = -X_{i+1,i+1} G_i - X_{n,i+1}^T H_i
//     X_{n,i}   = -X_{n,i+1} G_i - X_nn H_i
//     X_ii      =  M_i - X_{i+1,i}^T G_i - X_{n,i}^T H_i   (lower tiles, mirrored)
// An operation depends on at most four earlier operations of the same matrix.
//
// Scheduling is dynamic, on the device. An operation is ready once all the
// operations it depends on have completed; ready operations wait in FIFO queues
// by priority level: an operation's level is set by the number of operations
// after it in its matrix's program relative to the longest program, so the
// matrices with the most remaining work are served first (critical-path order).
// Every CTA repeatedly takes the next item of the first ready operation that
// still has items (highest level first), runs it and counts it done; the CTA
// that completes an operation counts one more finished dependency in each of its
// successors and appends those that become ready to their queue. No CTA waits
// for a particular item: a CTA that finds every queue empty polls until an
// operation completes, so the kernel cannot deadlock, and it ends when every
// operation has completed. The poll is bounded: after many polls with no
// operation completing anywhere it sets the plan's error word and the CTAs
// return. At the start the first operation of every matrix is ready. Data
// written by one item and read by another is read through L2 (ld.global.cg):
// items of the same tile can run on different SMs, whose L1 caches are not
// coherent. The tuning parameters are the CTAs per SM, R (tile rows per item)
// and the number of priority levels (1: plain ready order).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "bta.h"
#include "bta_internal.cuh"
#include "f64_device.cuh"
#include "timing.cuh"

namespace bta {
namespace {

enum PKind { PK_POTRF = 0, PK_PANEL, PK_UPDATE, PK_GEMM, PK_TINV, PK_TRTRI, PK_LOGDET };

// One block step of the factorization (or, with a = 0 and next = 0, the tip's
// own factorization). Extended tile rows: the nt tiles of block i, the nt tiles
// of block i+1 (next), then the na arrow tiles; E of them, Ecol columns.
struct PStep {
  double *D0, *Lw, *D1, *Ar0, *Ar1, *tip;
  int64_t ld;  // row stride of D0, Lw, D1 (the arrow blocks have rows of b, the tip rows of a)
  int b, a, nt, na, next, E, Ecol, mat;
  long long row0;  // 1-based global row of D0's first row, minus one
  double* rdv;     // [nt][T] 1 / L_jj of each factored diagonal tile
  double* ldpart;  // [nt] sum of log L_jj of each diagonal tile
};

struct PTerm {
  const double* A;
  const double* B;
  int64_t lda, ldb, sA, sB;  // row strides; strides per batch entry
  int K, opA, opB, triA, triB;
  double alpha;
};

// C = beta C + sum_t alpha_t op(A_t) op(B_t) over nb batch entries. lowerC: only
// tiles with tile row >= tile column (M == N); mirror: each such tile is also
// written transposed above the diagonal (an exactly symmetric result).
struct PGemm {
  PTerm t[2];
  double* C;
  int64_t ldc, sC;
  int nterms, M, N, nb, lowerC, mirror, R, groupsM, tilesN;
  double beta;
};

// Lower-triangular blocks L (nb of order m, stride s, row stride ld) -> Li.
struct PTrtri {
  const double* L;
  double* Li;
  int64_t ld, s;
  int m, nt, nb;
};

struct POp {
  int kind, nitems, arg, k;
  int ndeps;              // operations that must complete before this one is ready
  int succ_off, nsucc;    // the operations that depend on this one: succ[succ_off ..]
  int prio;               // queue 0..kQueues-1 (taken in that order)
};

struct PMat {
  const double* ldpart;
  double* logdet_out;
  int nparts;
};

// Counters of a run (zeroed, then seeded with the initially ready operations).
// hdr: [0] error word, [1] completed operations, then per queue q [2 + 2q] head
// and [3 + 2q] reserved slots. A queue entry is op + 1 (0: reserved, not written
// yet); every operation enters a queue once, so each queue has nops slots.
// Queue q holds the operations whose matrix has, after them, a remaining chain
// of dependent operations in the q-th eighth of the longest one, longest first
// (critical-path order); the queues are taken in that order.
struct PDev {
  const POp* ops;
  const int* succ;
  const PStep* steps;
  const PGemm* gemms;
  const PTrtri* trtris;
  const PMat* mats;
  int nops;
  int* hdr;
  int* taken;      // [nops] items taken
  int* done;       // [nops] items completed
  int* sat;        // [nops] dependencies completed
  int* queue;      // [kQueues][nops]: queue q at queue + q * nops
  unsigned long long* info;  // [matrices] first failed pivot row
  unsigned max_polls;
};

constexpr int kPThreads = 128;
constexpr int kPMaxR = 2;
constexpr int kCounterHeader = 64;  // ints of the run header (2 + 2 kQueues used)
constexpr int kQueues = 8;

template <int MAXR>
struct PSmem {
  double A[MAXR < 2 ? 2 : MAXR][T][T + 1];  // op(A) chunks, [m][k]; scratch tiles
  double B[T][T + 1];          // op(B) chunk stored transposed, [n][k]
  double rd[T];
  double red[kPThreads];
  int op, item;
};

__device__ __forceinline__ double ldcg(const double* p) { return __ldcg(p); }

__device__ __forceinline__ int ext_group(const PStep& p, int r, int& lr) {
  if (r < p.nt) {
    lr = r;
    return 0;
  }
  r -= p.nt;
  if (p.next) {
    if (r < p.nt) {
      lr = r;
      return 1;
    }
    r -= p.nt;
  }
  lr = r;
  return 2;
}

__device__ __forceinline__ int ext_rows(const PStep& p, int r) {
  int lr;
  const int g = ext_group(p, r, lr);
  return min(T, (g == 2 ? p.a : p.b) - T * lr);
}

// Tile (r, c), r >= c, of the extended lower triangle and its row stride.
__device__ __forceinline__ double* ext_tile(const PStep& p, int r, int c, int64_t& ld) {
  int lr, lc;
  const int gr = ext_group(p, r, lr), gc = ext_group(p, c, lc);
  if (gc == 2) {
    ld = p.a;
    return p.tip + (int64_t)(T * lr) * p.a + T * lc;
  }
  if (gr == 2) {
    ld = p.b;
    return (gc == 0 ? p.Ar0 : p.Ar1) + (int64_t)(T * lr) * p.b + T * lc;
  }
  ld = p.ld;
  double* base = gc == 0 ? (gr == 0 ? p.D0 : p.Lw) : p.D1;
  return base + (int64_t)(T * lr) * p.ld + T * lc;
}

// acc += A (rows wm.., [m][k]) * Bt^T (cols wn.., [n][k]) over the first kl of a
// 32-deep chunk (entries past kl are zero in shared memory).
__device__ __forceinline__ void mma_chunk(double (&acc)[2][2][2], const double (*A)[T + 1],
                                          const double (*Bt)[T + 1], int kl) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gq = lane >> 2, tq = lane & 3, wm = (warp >> 1) * 16, wn = (warp & 1) * 16;
#pragma unroll
  for (int ks = 0; ks < T; ks += 4) {
    if (ks >= kl) break;
    const double a0 = A[wm + gq][ks + tq], a1 = A[wm + 8 + gq][ks + tq];
    const double b0 = Bt[wn + gq][ks + tq], b1 = Bt[wn + 8 + gq][ks + tq];
    dmma_8x8x4(acc[0][0], a0, b0);
    dmma_8x8x4(acc[0][1], a0, b1);
    dmma_8x8x4(acc[1][0], a1, b0);
    dmma_8x8x4(acc[1][1], a1, b1);
  }
}

__device__ __forceinline__ void zero_acc(double (&acc)[2][2][2]) {
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) acc[i][j][0] = acc[i][j][1] = 0.0;
}

// Element of the accumulator fragment: row wm + mi*8 + gq, column wn + ni*8 + 2 tq + j.
#define P_FRAG_LOOP(BODY)                                                             \
  {                                                                                   \
    const int lane_ = threadIdx.x & 31, warp_ = threadIdx.x >> 5;                     \
    const int gq_ = lane_ >> 2, tq_ = lane_ & 3;                                      \
    const int wm_ = (warp_ >> 1) * 16, wn_ = (warp_ & 1) * 16;                        \
    _Pragma("unroll") for (int mi = 0; mi < 2; ++mi)                                  \
      _Pragma("unroll") for (int ni = 0; ni < 2; ++ni)                                \
        _Pragma("unroll") for (int jj = 0; jj < 2; ++jj) {                            \
          const int fr = wm_ + mi * 8 + gq_, fc = wn_ + ni * 8 + 2 * tq_ + jj;        \
          BODY                                                                        \
        }                                                                             \
  }

// ---- items ------------------------------------------------------------------

template <int MAXR>
__device__ void item_potrf(const PDev& d, const PStep& p, int k, PSmem<MAXR>& sm) {
  double(*S)[T + 1] = sm.A[0];
  const int tid = threadIdx.x, tb = min(T, p.b - k * T);
  double* Dk = p.D0 + (int64_t)(k * T) * p.ld + k * T;
  for (int e = tid; e < T * T; e += kPThreads) {
    const int i = e / T, j = e % T;
    S[i][j] = (i < tb && j <= i) ? ldcg(Dk + (int64_t)i * p.ld + j) : 0.0;
  }
  __syncthreads();
  coop_factor(S, sm.rd, tb, p.row0 + (long long)k * T, d.info + p.mat);
  for (int e = tid; e < T * T; e += kPThreads) {
    const int i = e / T, j = e % T;
    if (i < tb && j < tb) Dk[(int64_t)i * p.ld + j] = S[i][j];
  }
  if (tid < T) p.rdv[k * T + tid] = sm.rd[tid];
  if (tid < 32) {  // per-tile log sum, fixed reduction order
    double v = tid < tb ? log(S[tid][tid]) : 0.0;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (tid == 0) p.ldpart[k] = v;
  }
}

template <int MAXR>
__device__ void item_panel(const PStep& p, int k, int r, PSmem<MAXR>& sm) {
  double(*S)[T + 1] = sm.A[0];
  double(*Lt)[T + 1] = sm.A[1];
  const int tid = threadIdx.x, tb = min(T, p.b - k * T), rows = ext_rows(p, r);
  const double* Dk = p.D0 + (int64_t)(k * T) * p.ld + k * T;
  int64_t ldx;
  double* X = ext_tile(p, r, k, ldx);
  for (int e = tid; e < T * T; e += kPThreads) {
    const int i = e / T, j = e % T;
    Lt[i][j] = (i < tb && j <= i) ? ldcg(Dk + (int64_t)i * p.ld + j) : 0.0;
    S[i][j] = (i < rows && j < tb) ? ldcg(X + (int64_t)i * ldx + j) : 0.0;
  }
  if (tid < T) sm.rd[tid] = ldcg(p.rdv + k * T + tid);
  __syncthreads();
  panel_solve(S, Lt, sm.rd, rows, tb);
  for (int e = tid; e < rows * tb; e += kPThreads) {
    const int i = e / tb, j = e % tb;
    X[(int64_t)i * ldx + j] = S[i][j];
  }
}

template <int MAXR>
__device__ void item_update(const PStep& p, int k, int item, int R, PSmem<MAXR>& sm) {
  // Column-major over (c, group of R rows), c = k+1 .. Ecol-1, rows c .. E-1.
  int c = k + 1;
  for (;;) {
    if (c >= p.Ecol) return;  // past the op's items (cannot happen for a valid item)
    const int cnt = (p.E - c + R - 1) / R;
    if (item < cnt) break;
    item -= cnt;
    ++c;
  }
  const int r0 = c + item * R, nr = min(R, p.E - r0);
  const int tid = threadIdx.x, tbk = min(T, p.b - k * T), cb = ext_rows(p, c);
  int64_t ldq;
  const double* Lc = ext_tile(p, c, k, ldq);
  for (int e = tid; e < T * T; e += kPThreads) {
    const int i = e / T, j = e % T;
    sm.B[i][j] = (i < cb && j < tbk) ? ldcg(Lc + (int64_t)i * ldq + j) : 0.0;
  }
  for (int q = 0; q < nr; ++q) {
    const int rb = ext_rows(p, r0 + q);
    int64_t ldr;
    const double* Lr = ext_tile(p, r0 + q, k, ldr);
    for (int e = tid; e < T * T; e += kPThreads) {
      const int i = e / T, j = e % T;
      sm.A[q][i][j] = (i < rb && j < tbk) ? ldcg(Lr + (int64_t)i * ldr + j) : 0.0;
    }
  }
  __syncthreads();
  for (int q = 0; q < nr; ++q) {
    double acc[2][2][2];
    zero_acc(acc);
    mma_chunk(acc, sm.A[q], sm.B, tbk);
    const int rb = ext_rows(p, r0 + q);
    int64_t ldc;
    double* C = ext_tile(p, r0 + q, c, ldc);
    P_FRAG_LOOP(if (fr < rb && fc < cb) {
      double* pc = C + (int64_t)fr * ldc + fc;
      *pc = ldcg(pc) - acc[mi][ni][jj];
    })
  }
}

template <int MAXR>
__device__ void item_gemm(const PGemm& g, int item, PSmem<MAXR>& sm) {
  const int tid = threadIdx.x;
  const int tilesM = (g.M + T - 1) / T;
  int z, tm, tn, nr;
  if (g.lowerC) {
    const int per = tilesM * (tilesM + 1) / 2;
    z = item / per;
    const int t = item % per;
    tm = tri_row(t);
    tn = t - tm * (tm + 1) / 2;
    nr = 1;
  } else {
    const int per = g.groupsM * g.tilesN;
    z = item / per;
    const int t = item % per;
    tn = t % g.tilesN;
    tm = (t / g.tilesN) * g.R;
    nr = min(g.R, tilesM - tm);
  }
  const int m0 = tm * T, n0 = tn * T;
  double acc[MAXR][2][2][2];
#pragma unroll
  for (int q = 0; q < MAXR; ++q) zero_acc(acc[q]);
  // The k-chunks of every term, in order; each chunk's operands are fetched into
  // registers one chunk ahead (ld.global.cg), so the loads of chunk c+1 are in
  // flight while chunk c's DMMAs run.
  // k range of term ti (structural zeros of triangular operands skipped; nr == 1
  // whenever op(A) is triangular).
  auto krange = [&](int ti, int& kb, int& ke) {
    const PTerm& t = g.t[ti];
    kb = 0;
    ke = t.K;
    if (t.triA == TRI_LOWER) ke = min(ke, m0 + T);
    if (t.triA == TRI_UPPER) kb = max(kb, m0);
    if (t.triB == TRI_LOWER) kb = max(kb, n0);
    if (t.triB == TRI_UPPER) ke = min(ke, n0 + T);
  };
  int kb0 = 0, ke0 = 0, kb1 = 0, ke1 = 0;
  if (g.nterms > 0) krange(0, kb0, ke0);
  if (g.nterms > 1) krange(1, kb1, ke1);
  const int nch0 = ke0 > kb0 ? (ke0 - kb0 + T - 1) / T : 0;
  const int nch1 = ke1 > kb1 ? (ke1 - kb1 + T - 1) / T : 0;
  const int total = nch0 + nch1;
  constexpr int PER = T * T / kPThreads;  // elements of a 32 x 32 chunk per thread
  double ra[MAXR][PER], rb[PER];
  auto fetch = [&](int ci) {
    const int ti = ci < nch0 ? 0 : 1;
    const PTerm& t = g.t[ti];
    const int k0 = ti ? kb1 + (ci - nch0) * T : kb0 + ci * T, kl = min(T, (ti ? ke1 : ke0) - k0);
    const double* A = t.A + (int64_t)z * t.sA;
    const double* B = t.B + (int64_t)z * t.sB;
#pragma unroll
    for (int x = 0; x < PER; ++x) {
      const int e = tid + x * kPThreads;
      if (t.opB == OP_N) {
        const int kk = e / T, jj = e % T;
        rb[x] = (kk < kl && n0 + jj < g.N) ? ldcg(B + (int64_t)(k0 + kk) * t.ldb + n0 + jj) : 0.0;
      } else {
        const int jj = e / T, kk = e % T;
        rb[x] = (kk < kl && n0 + jj < g.N) ? ldcg(B + (int64_t)(n0 + jj) * t.ldb + k0 + kk) : 0.0;
      }
    }
#pragma unroll
    for (int q = 0; q < MAXR; ++q) {
      if (q >= nr) break;
      const int mq = m0 + q * T;
#pragma unroll
      for (int x = 0; x < PER; ++x) {
        const int e = tid + x * kPThreads;
        if (t.opA == OP_N) {
          const int ii = e / T, kk = e % T;
          ra[q][x] = (kk < kl && mq + ii < g.M) ? ldcg(A + (int64_t)(mq + ii) * t.lda + k0 + kk) : 0.0;
        } else {
          const int kk = e / T, ii = e % T;
          ra[q][x] = (kk < kl && mq + ii < g.M) ? ldcg(A + (int64_t)(k0 + kk) * t.lda + mq + ii) : 0.0;
        }
      }
    }
  };
  if (total > 0) fetch(0);
  for (int ci = 0; ci < total; ++ci) {
    const int ti = ci < nch0 ? 0 : 1;
    const PTerm& t = g.t[ti];
    const int k0 = ti ? kb1 + (ci - nch0) * T : kb0 + ci * T, kl = min(T, (ti ? ke1 : ke0) - k0);
#pragma unroll
    for (int x = 0; x < PER; ++x) {
      const int e = tid + x * kPThreads;
      if (t.opB == OP_N) sm.B[e % T][e / T] = rb[x];
      else sm.B[e / T][e % T] = rb[x];
    }
#pragma unroll
    for (int q = 0; q < MAXR; ++q) {
      if (q >= nr) break;
#pragma unroll
      for (int x = 0; x < PER; ++x) {
        const int e = tid + x * kPThreads;
        if (t.opA == OP_N) sm.A[q][e / T][e % T] = scale_by(ra[q][x], t.alpha);
        else sm.A[q][e % T][e / T] = scale_by(ra[q][x], t.alpha);
      }
    }
    __syncthreads();
    if (ci + 1 < total) fetch(ci + 1);
#pragma unroll
    for (int q = 0; q < MAXR; ++q)
      if (q < nr) mma_chunk(acc[q], sm.A[q], sm.B, kl);
    __syncthreads();
  }
  double* C = g.C + (int64_t)z * g.sC;
  if (!g.mirror) {
#pragma unroll
    for (int q = 0; q < MAXR; ++q) {
      if (q >= nr) break;
      const int mq = m0 + q * T;
      P_FRAG_LOOP(if (mq + fr < g.M && n0 + fc < g.N) {
        double* pc = C + (int64_t)(mq + fr) * g.ldc + n0 + fc;
        double v = acc[q][mi][ni][jj];
        if (g.beta != 0.0) v += g.beta * ldcg(pc);
        *pc = v;
      })
    }
    return;
  }
  // Mirrored lower tile: stage it, then write it and its transpose.
  double(*S)[T + 1] = sm.A[0];
  P_FRAG_LOOP({
    double v = acc[0][mi][ni][jj];
    if (g.beta != 0.0 && m0 + fr < g.M && n0 + fc < g.N) v += g.beta * ldcg(C + (int64_t)(m0 + fr) * g.ldc + n0 + fc);
    S[fr][fc] = v;
  })
  __syncthreads();
  for (int e = tid; e < T * T; e += kPThreads) {
    const int i = e / T, j = e % T;
    if (m0 + i < g.M && n0 + j < g.N && (tm != tn || j <= i)) C[(int64_t)(m0 + i) * g.ldc + n0 + j] = S[i][j];
  }
  for (int e = tid; e < T * T; e += kPThreads) {
    const int j = e / T, i = e % T;  // row n0 + j, column m0 + i of the upper part
    if (m0 + i < g.M && n0 + j < g.N && (tm != tn || j < i)) C[(int64_t)(n0 + j) * g.ldc + m0 + i] = S[i][j];
  }
}

// Inverse of diagonal tile c of block z.
template <int MAXR>
__device__ void item_tinv(const PTrtri& t, int item, PSmem<MAXR>& sm) {
  double(*Ls)[T + 1] = sm.A[0];
  double(*X)[T + 1] = sm.A[1];
  const int tid = threadIdx.x, z = item / t.nt, c = item % t.nt, tb = min(T, t.m - c * T);
  const double* Lb = t.L + (int64_t)z * t.s + (int64_t)(c * T) * t.ld + c * T;
  double* Xb = t.Li + (int64_t)z * t.s + (int64_t)(c * T) * t.ld + c * T;
  for (int e = tid; e < T * T; e += kPThreads) {
    const int i = e / T, j = e % T;
    Ls[i][j] = (i < tb && j <= i) ? ldcg(Lb + (int64_t)i * t.ld + j) : 0.0;
    X[i][j] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  if (tid < tb) sm.rd[tid] = 1.0 / Ls[tid][tid];
  __syncthreads();
  // Forward substitution on L X = I, one row of X at a time.
  for (int j = 0; j < tb; ++j) {
    for (int c2 = tid; c2 <= j; c2 += kPThreads) X[j][c2] *= sm.rd[j];
    __syncthreads();
    const int rows = tb - j - 1, cols = j + 1;
    for (int e = tid; e < rows * cols; e += kPThreads) {
      const int i = j + 1 + e / cols, c2 = e % cols;
      X[i][c2] -= Ls[i][j] * X[j][c2];
    }
    __syncthreads();
  }
  for (int e = tid; e < tb * tb; e += kPThreads) {
    const int i = e / tb, j = e % tb;
    Xb[(int64_t)i * t.ld + j] = (j <= i) ? X[i][j] : 0.0;
  }
}

// Tile (r, c), c < r, of L^{-1} for block z:
//   Li(r, c) = -Li(r, r) * sum_{k=c}^{r-1} L(r, k) Li(k, c)
// (rows < r of Li and its diagonal tiles are final).
template <int MAXR>
__device__ void item_trtri(const PTrtri& t, int r, int item, PSmem<MAXR>& sm) {
  const int tid = threadIdx.x, z = item / r, c = item % r, rr = min(T, t.m - r * T);
  const double* L = t.L + (int64_t)z * t.s;
  double* Li = t.Li + (int64_t)z * t.s;
  double acc[2][2][2];
  zero_acc(acc);
  for (int k = c; k < r; ++k) {
    for (int e = tid; e < T * T; e += kPThreads) {
      const int i = e / T, kk = e % T;
      sm.A[0][i][kk] = i < rr ? ldcg(L + (int64_t)(r * T + i) * t.ld + k * T + kk) : 0.0;
    }
    for (int e = tid; e < T * T; e += kPThreads) {
      const int kk = e / T, j = e % T;
      sm.B[j][kk] = ldcg(Li + (int64_t)(k * T + kk) * t.ld + c * T + j);
    }
    __syncthreads();
    mma_chunk(acc, sm.A[0], sm.B, T);
    __syncthreads();
  }
  // W = acc (rr x T) becomes op(B) of the second product, stored [n][k].
  P_FRAG_LOOP(sm.B[fc][fr] = acc[mi][ni][jj];)
  for (int e = tid; e < T * T; e += kPThreads) {
    const int i = e / T, kk = e % T;
    sm.A[0][i][kk] = (i < rr && kk <= i) ? ldcg(Li + (int64_t)(r * T + i) * t.ld + r * T + kk) : 0.0;
  }
  __syncthreads();
  zero_acc(acc);
  mma_chunk(acc, sm.A[0], sm.B, rr);
  P_FRAG_LOOP(if (fr < rr) Li[(int64_t)(r * T + fr) * t.ld + c * T + fc] = -acc[mi][ni][jj];)
}

template <int MAXR>
__device__ void item_logdet(const PMat& m, PSmem<MAXR>& sm) {
  const int tid = threadIdx.x, per = (m.nparts + kPThreads - 1) / kPThreads;
  double v = 0.0;
  for (int q = tid * per; q < min(m.nparts, (tid + 1) * per); ++q) v += ldcg(m.ldpart + q);
  sm.red[tid] = v;
  __syncthreads();
  if (tid == 0) {
    double s = 0.0;
    for (int q = 0; q < kPThreads; ++q) s += sm.red[q];
    if (m.logdet_out) *m.logdet_out = 2.0 * s;
  }
}

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;\n" ::"l"(p), "r"(v) : "memory");
}

// Thread 0: the next ready item, the priority queue first; -1 when every
// operation has completed (or a wait ran out). An idle CTA polls; it gives up
// (error word) only after max_polls polls in which no operation completed.
__device__ __forceinline__ int take_item(const PDev& d, int& item) {
  unsigned idle = 0;
  int seen = -1;
  for (;;) {
    // Heads and tails of all queues in one round of independent loads; then the
    // first queue that is not empty.
    int hd[kQueues], tl[kQueues];
#pragma unroll
    for (int q = 0; q < kQueues; ++q) {
      hd[q] = __ldcv(d.hdr + 2 + 2 * q);
      tl[q] = __ldcv(d.hdr + 3 + 2 * q);
    }
    __threadfence();
#pragma unroll
    for (int q = 0; q < kQueues; ++q) {
      if (hd[q] >= tl[q]) continue;
      int* qh = d.hdr + 2 + 2 * q;
      for (;;) {
        const int h = ld_acquire(qh);
        if (h >= ld_acquire(qh + 1)) break;  // empty
        const int v = ld_acquire(d.queue + q * d.nops + h);
        if (v == 0) break;  // reserved, being written: poll again
        const int o = v - 1;
        const int t = atomicAdd(d.taken + o, 1);
        if (t < __ldg(&d.ops[o].nitems)) {
          item = t;
          return o;
        }
        atomicCAS(qh, h, h + 1);  // exhausted: move the head on
      }
    }
    const int completed = ld_acquire(d.hdr + 1);
    if (completed >= d.nops || ld_acquire(d.hdr) != 0) return -1;
    if (completed != seen) {
      seen = completed;
      idle = 0;
    } else if (++idle > d.max_polls) {
      atomicExch(d.hdr, 1);
      return -1;
    }
    __nanosleep(128);
  }
}

// Thread 0, after this CTA's item of operation o is written: count it; the CTA
// that completes the operation releases its successors into the queues.
__device__ __forceinline__ void finish_item(const PDev& d, int o) {
  __threadfence();
  const POp& op = d.ops[o];
  if (atomicAdd(d.done + o, 1) != __ldg(&op.nitems) - 1) return;
  __threadfence();
  const int so = __ldg(&op.succ_off), ns = __ldg(&op.nsucc);
  for (int q = 0; q < ns; ++q) {
    const int sidx = __ldg(d.succ + so + q);
    const POp& sop = d.ops[sidx];
    if (atomicAdd(d.sat + sidx, 1) == __ldg(&sop.ndeps) - 1) {
      const int pq = __ldg(&sop.prio);
      const int slot = atomicAdd(d.hdr + 3 + 2 * pq, 1);
      st_release(d.queue + pq * d.nops + slot, sidx + 1);
    }
  }
  atomicAdd(d.hdr + 1, 1);
}

// MINB: CTAs per SM the register budget is sized for; MAXR: largest R.
template <int MINB, int MAXR>
__global__ void __launch_bounds__(kPThreads, MINB) persistent_kernel(PDev d) {
  __shared__ PSmem<MAXR> sm;
  const int tid = threadIdx.x;
  for (;;) {
    if (tid == 0) {
      int it = 0;
      sm.op = take_item(d, it);
      sm.item = it;
    }
    __syncthreads();
    const int o = sm.op, it = sm.item;
    if (o < 0) break;
    const POp op = d.ops[o];
    switch (op.kind) {
      case PK_POTRF: item_potrf(d, d.steps[op.arg], op.k, sm); break;
      case PK_PANEL: item_panel(d.steps[op.arg], op.k, op.k + 1 + it, sm); break;
      case PK_UPDATE: item_update(d.steps[op.arg], op.k >> 4, it, op.k & 15, sm); break;
      case PK_GEMM: item_gemm(d.gemms[op.arg], it, sm); break;
      case PK_TINV: item_tinv(d.trtris[op.arg], it, sm); break;
      case PK_TRTRI: item_trtri(d.trtris[op.arg], op.k, it, sm); break;
      case PK_LOGDET: item_logdet(d.mats[op.arg], sm); break;
      default: break;
    }
    __syncthreads();
    if (tid == 0) finish_item(d, o);
  }
}

// ---- host: plan construction ------------------------------------------------

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct EntryWs {
  double *Linv, *G, *H, *LtInv, *rdv, *ldpart;
};

size_t entry_ws(int64_t n, int64_t b, int64_t a, void* base, EntryWs* o) {
  const int64_t nt = (b + T - 1) / T, na = (a + T - 1) / T;
  const size_t parts[6] = {(size_t)(n * b * b), (size_t)((n - 1) * b * b), (size_t)(n * a * b),
                           (size_t)(a * a), (size_t)(std::max(nt, na) * T), (size_t)(n * nt + na)};
  size_t off = 0;
  double* ptr[6];
  for (int q = 0; q < 6; ++q) {
    ptr[q] = base ? (double*)((char*)base + off) : nullptr;
    off += align256(std::max<size_t>(parts[q], 1) * sizeof(double));
  }
  if (o) *o = EntryWs{ptr[0], ptr[1], ptr[2], ptr[3], ptr[4], ptr[5]};
  return off;
}

struct HOp {
  POp op;
  int dep[4];  // local indices of the operations this one depends on (-1: none)
  int local;   // position in the matrix's program
};

struct Builder {
  std::vector<PStep> steps;
  std::vector<PGemm> gemms;
  std::vector<PTrtri> trtris;
  std::vector<PMat> mats;
  int R = 1;

  // Appends an op; deps are local indices into `ops` (-1: none).
  static int add(std::vector<HOp>& ops, int kind, int nitems, int arg, int k, int d0 = -1,
                 int d1 = -1, int d2 = -1, int d3 = -1) {
    HOp h{};
    h.op.kind = kind;
    h.op.nitems = nitems;
    h.op.arg = arg;
    h.op.k = k;
    h.dep[0] = d0; h.dep[1] = d1; h.dep[2] = d2; h.dep[3] = d3;
    h.local = (int)ops.size();
    ops.push_back(h);
    return h.local;
  }

  int gemm_items(PGemm& g) {
    const int tm = (g.M + T - 1) / T;
    g.tilesN = (g.N + T - 1) / T;
    bool tri = g.lowerC;
    for (int q = 0; q < g.nterms; ++q) tri = tri || g.t[q].triA != TRI_NONE;
    g.R = tri ? 1 : R;
    g.groupsM = (tm + g.R - 1) / g.R;
    return g.lowerC ? g.nb * tm * (tm + 1) / 2 : g.nb * g.groupsM * g.tilesN;
  }

  int add_gemm(std::vector<HOp>& ops, PGemm g, int d0, int d1 = -1, int d2 = -1, int d3 = -1) {
    const int items = gemm_items(g);
    gemms.push_back(g);
    return add(ops, PK_GEMM, items, (int)gemms.size() - 1, 0, d0, d1, d2, d3);
  }

  // Tile Cholesky ops of one step, chained after `prev`; returns the last op.
  int add_step(std::vector<HOp>& ops, const PStep& p, int prev) {
    steps.push_back(p);
    const int s = (int)steps.size() - 1;
    for (int k = 0; k < p.nt; ++k) {
      prev = add(ops, PK_POTRF, 1, s, k, prev);
      if (p.E - k - 1 > 0) prev = add(ops, PK_PANEL, p.E - k - 1, s, k, prev);
      int items = 0;
      for (int c = k + 1; c < p.Ecol; ++c) items += (p.E - c + R - 1) / R;
      if (items > 0) prev = add(ops, PK_UPDATE, items, s, (k << 4) | R, prev);
    }
    return prev;
  }

  PTerm term(const double* A, int64_t lda, int64_t sA, int opA, int triA, const double* B,
             int64_t ldb, int64_t sB, int opB, int triB, int K, double alpha) {
    PTerm t{};
    t.A = A; t.B = B; t.lda = lda; t.ldb = ldb; t.sA = sA; t.sB = sB;
    t.K = K; t.opA = opA; t.opB = opB; t.triA = triA; t.triB = triB; t.alpha = alpha;
    return t;
  }

  static PGemm gemm(double* C, int64_t ldc, int64_t sC, int M, int N, int nb, double beta,
                    int lowerC, int mirror) {
    PGemm g{};
    g.C = C; g.ldc = ldc; g.sC = sC; g.M = M; g.N = N; g.nb = nb; g.beta = beta;
    g.lowerC = lowerC; g.mirror = mirror;
    return g;
  }

  // The whole program of one matrix.
  void add_matrix(int mi, const bta_batch_entry& e, std::vector<HOp>& ops) {
    const int64_t n = e.n, b = e.b, a = e.a, bb = b * b, ab = a * b;
    const int B = (int)b, Aa = (int)a, nt = (int)((b + T - 1) / T), na = (int)((a + T - 1) / T);
    EntryWs w;
    entry_ws(n, b, a, e.ws, &w);
    // Factorization.
    int prev = -1;
    for (int64_t i = 0; i < n; ++i) {
      PStep p{};
      p.D0 = e.diag + i * bb;
      p.next = i + 1 < n;
      p.Lw = p.next ? e.lower + i * bb : nullptr;
      p.D1 = p.next ? e.diag + (i + 1) * bb : nullptr;
      p.Ar0 = a ? e.arrow + i * ab : nullptr;
      p.Ar1 = (a && p.next) ? e.arrow + (i + 1) * ab : nullptr;
      p.tip = a ? e.tip : nullptr;
      p.ld = b; p.b = B; p.a = Aa; p.nt = nt; p.na = na;
      p.E = nt * (1 + p.next) + na;
      p.Ecol = p.E;
      p.mat = mi;
      p.row0 = i * b;
      p.rdv = w.rdv;
      p.ldpart = w.ldpart + i * nt;
      prev = add_step(ops, p, prev);
    }
    if (a > 0) {
      PStep p{};
      p.D0 = e.tip; p.ld = a; p.b = Aa; p.a = 0; p.nt = na; p.na = 0; p.next = 0;
      p.E = na; p.Ecol = na; p.mat = mi; p.row0 = n * b; p.rdv = w.rdv;
      p.ldpart = w.ldpart + n * nt;
      prev = add_step(ops, p, prev);
    }
    const int fac = prev;
    mats.push_back(PMat{w.ldpart, e.logdet_out, (int)(n * nt + na)});
    add(ops, PK_LOGDET, 1, (int)mats.size() - 1, 0, fac);
    // L_ii^{-1} of every block.
    trtris.push_back(PTrtri{e.diag, w.Linv, b, bb, B, nt, (int)n});
    const int tb = (int)trtris.size() - 1;
    int tr = add(ops, PK_TINV, (int)n * nt, tb, 0, fac);
    for (int r = 1; r < nt; ++r) tr = add(ops, PK_TRTRI, (int)n * r, tb, r, tr);
    int opG = -1, opH = -1;
    if (n > 1) {
      PGemm g = gemm(w.G, b, bb, B, B, (int)(n - 1), 0.0, 0, 0);
      g.t[0] = term(e.lower, b, bb, OP_N, TRI_NONE, w.Linv, b, bb, OP_N, TRI_LOWER, B, 1.0);
      g.nterms = 1;
      opG = add_gemm(ops, g, tr);
    }
    if (a > 0) {
      PGemm g = gemm(w.H, b, ab, Aa, B, (int)n, 0.0, 0, 0);
      g.t[0] = term(e.arrow, b, ab, OP_N, TRI_NONE, w.Linv, b, bb, OP_N, TRI_LOWER, B, 1.0);
      g.nterms = 1;
      opH = add_gemm(ops, g, tr);
    }
    PGemm gm = gemm(e.diag, b, bb, B, B, (int)n, 0.0, 1, 0);
    gm.t[0] = term(w.Linv, b, bb, OP_T, TRI_UPPER, w.Linv, b, bb, OP_N, TRI_LOWER, B, 1.0);
    gm.nterms = 1;
    const int opM = add_gemm(ops, gm, tr);
    int opXnn = -1;
    if (a > 0) {
      trtris.push_back(PTrtri{e.tip, w.LtInv, a, a * a, Aa, na, 1});
      const int tt = (int)trtris.size() - 1;
      int t2 = add(ops, PK_TINV, na, tt, 0, fac);
      for (int r = 1; r < na; ++r) t2 = add(ops, PK_TRTRI, r, tt, r, t2);
      PGemm g = gemm(e.tip, a, 0, Aa, Aa, 1, 0.0, 1, 1);
      g.t[0] = term(w.LtInv, a, 0, OP_T, TRI_UPPER, w.LtInv, a, 0, OP_N, TRI_LOWER, Aa, 1.0);
      g.nterms = 1;
      opXnn = add_gemm(ops, g, t2);
    }
    // Backward recurrence.
    int xd_next = -1, xa_next = opXnn;
    for (int64_t i = n - 1; i >= 0; --i) {
      const double* Gi = w.G + i * bb;
      const double* Hi = w.H + i * ab;
      int opXL = -1, opXA = -1;
      if (i + 1 < n) {
        PGemm g = gemm(e.lower + i * bb, b, 0, B, B, 1, 0.0, 0, 0);
        g.t[0] = term(e.diag + (i + 1) * bb, b, 0, OP_N, TRI_NONE, Gi, b, 0, OP_N, TRI_NONE, B, -1.0);
        g.nterms = 1;
        if (a > 0) {
          g.t[1] = term(e.arrow + (i + 1) * ab, b, 0, OP_T, TRI_NONE, Hi, b, 0, OP_N, TRI_NONE, Aa, -1.0);
          g.nterms = 2;
        }
        opXL = add_gemm(ops, g, xd_next, opG, opH);
      }
      if (a > 0) {
        PGemm g = gemm(e.arrow + i * ab, b, 0, Aa, B, 1, 0.0, 0, 0);
        if (i + 1 < n)
          g.t[g.nterms++] = term(e.arrow + (i + 1) * ab, b, 0, OP_N, TRI_NONE, Gi, b, 0, OP_N, TRI_NONE, B, -1.0);
        g.t[g.nterms++] = term(e.tip, a, 0, OP_N, TRI_NONE, Hi, b, 0, OP_N, TRI_NONE, Aa, -1.0);
        opXA = add_gemm(ops, g, xa_next, opG, opH);
      }
      PGemm g = gemm(e.diag + i * bb, b, 0, B, B, 1, 1.0, 1, 1);
      if (i + 1 < n)
        g.t[g.nterms++] = term(e.lower + i * bb, b, 0, OP_T, TRI_NONE, Gi, b, 0, OP_N, TRI_NONE, B, -1.0);
      if (a > 0)
        g.t[g.nterms++] = term(e.arrow + i * ab, b, 0, OP_T, TRI_NONE, Hi, b, 0, OP_N, TRI_NONE, Aa, -1.0);
      xd_next = add_gemm(ops, g, opXL, opXA, opM);
      xa_next = opXA;
    }
  }
};

}  // namespace


typedef void (*PKernel)(PDev);

// Two builds of the kernel, both with the register budget of 4 CTAs per SM (the
// operands of the next k-chunk are held in registers): items of one tile row,
// or of up to two.
static PKernel pick_kernel(int R) {
  return R > 1 ? (PKernel)persistent_kernel<4, 2> : (PKernel)persistent_kernel<4, 1>;
}

static cudaError_t plan_occupancy(PKernel k, int* per_sm, int* sms) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, (const void*)k, kPThreads, 0);
}

}  // namespace bta

using namespace bta;

// The plan object behind the opaque bta_plan handle.
struct bta_plan_s {
  int device = -1;
  int count = 0;
  int grid = 0, levels = 0, R = 1, ctas_per_sm = 0;
  int nops = 0, ninit = 0;
  long long nitems = 0;
  double flops = 0.0;
  void* desc = nullptr;      // descriptor tables and the seed image of the counters
  void* counters = nullptr;  // header, taken, done, sat, two queues, info
  size_t counter_bytes = 0;
  const int* seed_hdr = nullptr;    // device: header values of a fresh run
  const int* seed_queue[kQueues] = {};  // device: initially ready operations
  int seed_len[kQueues] = {};
  const void* kernel = nullptr;
  PDev d{};
};

extern "C" {

size_t bta_plan_entry_workspace_bytes(int64_t n, int64_t b, int64_t a) {
  if (n < 1 || b < 1 || a < 0 || b > 32768 || a > 32768) return 0;
  return entry_ws(n, b, a, nullptr, nullptr);
}

int bta_plan_create(int64_t count, const bta_batch_entry* entries, const bta_plan_params* params,
                    bta_plan* out) {
  if (count < 1 || count > (1 << 16)) return -1;
  if (!entries) return -2;
  if (!out) return -4;
  *out = nullptr;
  bta_plan_params prm{};
  if (params) prm = *params;
  if (prm.ctas_per_sm < 0 || prm.ctas_per_sm > 16 || prm.levels < 0 || prm.levels > kQueues ||
      prm.rows_per_item < 0 || prm.rows_per_item > kPMaxR)
    return -3;
  for (int64_t k = 0; k < count; ++k) {
    const bta_batch_entry& e = entries[k];
    if (e.n < 1 || e.b < 1 || e.a < 0 || e.b > 32768 || e.a > 32768) return -2;
    // Item indices are ints: the largest operation (a product over all blocks,
    // n (b/32)^2 tiles) must stay well below 2^31.
    const double nt = (double)((e.b + T - 1) / T);
    if (e.n > (1 << 20) || (double)e.n * nt * nt > 1.5e9) return -2;
    if (!e.diag || (e.n > 1 && !e.lower) || (e.a > 0 && (!e.arrow || !e.tip))) return -2;
    if (e.prec != BTA_PREC_FP64) return -2;
    if (!e.ws || ((uintptr_t)e.ws % 256) || e.ws_bytes < entry_ws(e.n, e.b, e.a, nullptr, nullptr))
      return -2;
    if (e.logdet_out && ((uintptr_t)e.logdet_out % 8)) return -2;
  }
  const int R = prm.rows_per_item ? prm.rows_per_item : 1;
  const int levels = prm.levels ? prm.levels : kQueues;
  const PKernel kern = pick_kernel(R);
  int per_sm = 0, sms = 0;
  cudaError_t ce = plan_occupancy(kern, &per_sm, &sms);
  if (ce != cudaSuccess) return (int)ce;
  if (per_sm < 1 || sms < 1) return (int)cudaErrorInvalidConfiguration;
  // Four CTAs per SM by default: enough warps to keep the FP64 pipe busy, while
  // more resident CTAs than ready items only add idle polling (measured on the
  // 64-matrix batch: 2.76 s at 4 per SM, 3.12 s at 8, 3.07 s at 2).
  const int occ = std::min(prm.ctas_per_sm ? prm.ctas_per_sm : 4, per_sm);
  const int G = occ * sms;
  // Matrices largest first: their operations come first in the tables and their
  // first operations first in the initial queue.
  std::vector<double> fl(count);
  double flops = 0.0;
  for (int64_t k = 0; k < count; ++k) {
    const double B = (double)entries[k].b, A = (double)entries[k].a, n = (double)entries[k].n;
    fl[k] = n * B * B * B / 3 + (n - 1) * 2 * B * B * B + n * A * B * B + (n - 1) * 2 * A * B * B +
            n * A * A * B + A * A * A / 3 + 2 * A * A * A / 3 + n * 2 * B * B * B / 3 +
            (n - 1) * 4 * B * B * B + n * (2 * A * B * B + 2 * A * A * B) + (n - 1) * 4 * A * B * B;
    flops += fl[k];
  }
  std::vector<int64_t> order(count);
  for (int64_t k = 0; k < count; ++k) order[k] = k;
  std::stable_sort(order.begin(), order.end(), [&](int64_t x, int64_t y) { return fl[x] > fl[y]; });
  // Critical-path priority: an operation's queue is set by the number of
  // operations after it in its matrix's program (a chain, apart from the
  // prologue's independent products), relative to the longest program. Matrices
  // with the most remaining work are served first; otherwise their chains, slowed
  // by the other matrices' items, end the run alone.
  Builder bld;
  bld.R = R;
  std::vector<POp> ops;
  std::vector<std::vector<int>> succ;
  std::vector<int> init[kQueues];
  long long nitems = 0;
  std::vector<std::vector<HOp>> progs(count);
  size_t longest = 1;
  for (int64_t m : order) {
    bld.add_matrix((int)m, entries[m], progs[m]);
    longest = std::max(longest, progs[m].size());
  }
  for (int64_t m : order) {
    const std::vector<HOp>& prog = progs[m];
    const int base = (int)ops.size();
    if ((size_t)base + prog.size() > (size_t)0x3fffffff) return -1;
    succ.resize(base + prog.size());
    for (const HOp& h : prog) {
      POp o = h.op;
      int deps[4], nd = 0;
      for (int j = 0; j < 4; ++j) {
        const int dl = h.dep[j];
        if (dl < 0) continue;
        if (dl >= h.local) return (int)cudaErrorInvalidValue;  // must be an earlier operation
        bool dup = false;
        for (int q = 0; q < nd; ++q) dup = dup || deps[q] == dl;
        if (!dup) deps[nd++] = dl;
      }
      o.ndeps = nd;
      const double rem = (double)(prog.size() - h.local) / (double)longest;  // in (0, 1]
      o.prio = std::min(levels - 1, std::max(0, (int)((1.0 - rem) * levels)));
      const int gi = base + h.local;
      for (int q = 0; q < nd; ++q) succ[base + deps[q]].push_back(gi);
      if (nd == 0) init[o.prio].push_back(gi);
      nitems += o.nitems;
      ops.push_back(o);
    }
  }
  std::vector<int> succ_flat;
  for (size_t q = 0; q < ops.size(); ++q) {
    ops[q].succ_off = (int)succ_flat.size();
    ops[q].nsucc = (int)succ[q].size();
    succ_flat.insert(succ_flat.end(), succ[q].begin(), succ[q].end());
  }
  const int nops = (int)ops.size();
  // Seed image of a run: header (queue tails = initially ready counts) and the
  // initial queue entries (op + 1).
  std::vector<int> seed_hdr(kCounterHeader, 0);
  std::vector<int> seed_q[kQueues];
  for (int q = 0; q < kQueues; ++q) {
    seed_hdr[3 + 2 * q] = (int)init[q].size();
    for (int v : init[q]) seed_q[q].push_back(v + 1);
  }

  bta_plan_s* P = new (std::nothrow) bta_plan_s;
  if (!P) return (int)cudaErrorMemoryAllocation;
  cudaGetDevice(&P->device);
  P->count = (int)count;
  P->grid = G;
  P->levels = levels;
  P->R = R;
  P->kernel = (const void*)kern;
  P->ctas_per_sm = occ;
  P->nops = nops;
  P->ninit = 0;
  for (int q = 0; q < kQueues; ++q) P->ninit += (int)init[q].size();
  P->nitems = nitems;
  P->flops = flops;
  struct Part {
    const void* src;
    size_t bytes;
  };
  const Part parts[] = {{ops.data(), ops.size() * sizeof(POp)},
                        {succ_flat.data(), succ_flat.size() * sizeof(int)},
                        {bld.steps.data(), bld.steps.size() * sizeof(PStep)},
                        {bld.gemms.data(), bld.gemms.size() * sizeof(PGemm)},
                        {bld.trtris.data(), bld.trtris.size() * sizeof(PTrtri)},
                        {bld.mats.data(), bld.mats.size() * sizeof(PMat)},
                        {seed_hdr.data(), seed_hdr.size() * sizeof(int)},
                        {seed_q[0].data(), seed_q[0].size() * sizeof(int)},
                        {seed_q[1].data(), seed_q[1].size() * sizeof(int)},
                        {seed_q[2].data(), seed_q[2].size() * sizeof(int)},
                        {seed_q[3].data(), seed_q[3].size() * sizeof(int)},
                        {seed_q[4].data(), seed_q[4].size() * sizeof(int)},
                        {seed_q[5].data(), seed_q[5].size() * sizeof(int)},
                        {seed_q[6].data(), seed_q[6].size() * sizeof(int)},
                        {seed_q[7].data(), seed_q[7].size() * sizeof(int)}};
  constexpr int kParts = sizeof(parts) / sizeof(parts[0]);
  size_t total = 0, at[kParts];
  for (int q = 0; q < kParts; ++q) {
    at[q] = total;
    total += align256(parts[q].bytes + 1);
  }
  const size_t n_int = (size_t)nops;
  P->counter_bytes = align256((kCounterHeader + (3 + kQueues) * n_int) * sizeof(int)) +
                     align256(count * sizeof(unsigned long long));
  ce = cudaMalloc(&P->desc, total);
  if (ce == cudaSuccess) ce = cudaMalloc(&P->counters, P->counter_bytes);
  if (ce == cudaSuccess) {
    std::vector<char> host(total, 0);
    for (int q = 0; q < kParts; ++q)
      if (parts[q].bytes) memcpy(host.data() + at[q], parts[q].src, parts[q].bytes);
    ce = cudaMemcpy(P->desc, host.data(), total, cudaMemcpyHostToDevice);
  }
  if (ce != cudaSuccess) {
    if (P->desc) cudaFree(P->desc);
    if (P->counters) cudaFree(P->counters);
    delete P;
    return (int)ce;
  }
  char* D = (char*)P->desc;
  P->d.ops = (const POp*)(D + at[0]);
  P->d.succ = (const int*)(D + at[1]);
  P->d.steps = (const PStep*)(D + at[2]);
  P->d.gemms = (const PGemm*)(D + at[3]);
  P->d.trtris = (const PTrtri*)(D + at[4]);
  P->d.mats = (const PMat*)(D + at[5]);
  P->seed_hdr = (const int*)(D + at[6]);
  for (int q = 0; q < kQueues; ++q) {
    P->seed_queue[q] = (const int*)(D + at[7 + q]);
    P->seed_len[q] = (int)seed_q[q].size();
  }
  int* c = (int*)P->counters;
  P->d.nops = nops;
  P->d.hdr = c;
  P->d.taken = c + kCounterHeader;
  P->d.done = P->d.taken + n_int;
  P->d.sat = P->d.done + n_int;
  P->d.queue = P->d.sat + n_int;
  P->d.info = (unsigned long long*)((char*)P->counters +
                                    align256((kCounterHeader + (3 + kQueues) * n_int) * sizeof(int)));
  P->d.max_polls = 1u << 22;  // polls (128 ns sleeps) without any operation completing
  *out = P;
  return 0;
}

static inline size_t n_ops(const bta_plan_s* P) { return (size_t)P->nops; }

int bta_plan_run(bta_plan plan, bta_stream_t stream) {
  bta_plan_s* P = plan;
  if (!P) return -1;
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return (int)e;
  if (dev != P->device) return -1;
  const cudaStream_t s = (cudaStream_t)stream;
  e = cudaMemsetAsync(P->counters, 0, P->counter_bytes, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(P->d.hdr, P->seed_hdr, kCounterHeader * sizeof(int), cudaMemcpyDeviceToDevice, s);
  for (int q = 0; q < kQueues && e == cudaSuccess; ++q)
    if (P->seed_len[q])
      e = cudaMemcpyAsync(P->d.queue + q * n_ops(P), P->seed_queue[q], P->seed_len[q] * sizeof(int),
                          cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return (int)e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)P->grid);
  cfg.blockDim = dim3(kPThreads);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  TimedLaunch tl(K_PERSISTENT, timing_on() ? P->flops : 0.0, s);
  void* args[] = {&P->d};
  e = cudaLaunchKernelExC(&cfg, P->kernel, args);
  return e == cudaSuccess ? 0 : (int)e;
}

int bta_plan_status(bta_plan plan, int* timed_out, int64_t* info, bta_stream_t stream) {
  bta_plan_s* P = plan;
  if (!P) return -1;
  const cudaStream_t s = (cudaStream_t)stream;
  int err = 0;
  cudaError_t e = cudaMemcpyAsync(&err, P->d.hdr, sizeof(int), cudaMemcpyDeviceToHost, s);
  std::vector<unsigned long long> inf(P->count, 0);
  if (e == cudaSuccess && info)
    e = cudaMemcpyAsync(inf.data(), P->d.info, P->count * sizeof(unsigned long long),
                        cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return (int)e;
  if (timed_out) *timed_out = err;
  if (info)
    for (int k = 0; k < P->count; ++k) info[k] = (int64_t)inf[k];
  return 0;
}

int bta_plan_describe(bta_plan plan, int64_t* out, int nout) {
  bta_plan_s* P = plan;
  if (!P) return -1;
  if (!out || nout < 1) return -2;
  const int64_t v[8] = {P->grid, P->ctas_per_sm, P->levels, P->R, P->nops, P->nitems,
                        (int64_t)P->flops, P->ninit};
  for (int q = 0; q < nout && q < 8; ++q) out[q] = v[q];
  return 0;
}

int bta_plan_destroy(bta_plan plan) {
  bta_plan_s* P = plan;
  if (!P) return 0;
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != P->device) cudaSetDevice(P->device);
  cudaError_t e = cudaFree(P->desc);
  cudaError_t e2 = cudaFree(P->counters);
  if (cur != P->device && cur >= 0) cudaSetDevice(cur);
  delete P;
  return e != cudaSuccess ? (int)e : (e2 != cudaSuccess ? (int)e2 : 0);
}

}  // extern "C"
