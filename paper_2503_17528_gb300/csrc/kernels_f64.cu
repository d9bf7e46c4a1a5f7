// FP64 kernels of the BTA path for sm_103a.
//
// On this part the FP64 pipe (DMMA and DFMA alike) is the bound: HBM and
// shared-memory traffic of these kernels are two orders of magnitude below
// their limits. So every kernel is written to keep the FP64 pipe of all SMs
// busy: dense contractions go through warp-level DMMA (mma.sync m8n8k4 f64) on
// 32x32 output tiles, many small CTAs are resident per SM, and triangular
// operands skip the k-range that is known to be zero.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <stdint.h>

#include "bta_internal.cuh"
#include "f64_device.cuh"
#include "timing.cuh"

namespace bta {

// ---------------------------------------------------------------------------
// Per-device info word: 1-based global row of the first non-positive pivot.
// ---------------------------------------------------------------------------
__device__ unsigned long long g_info;

cudaError_t info_reset(cudaStream_t s) {
  static const unsigned long long zero = 0;
  return cudaMemcpyToSymbolAsync(g_info, &zero, sizeof(zero), 0,
                                 cudaMemcpyHostToDevice, s);
}

cudaError_t info_read_reset(cudaStream_t s, long long* out) {
  unsigned long long v = 0;
  cudaError_t e = cudaMemcpyFromSymbolAsync(&v, g_info, sizeof(v), 0,
                                            cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return e;
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e;
  *out = (long long)v;
  return info_reset(s);
}

// ---------------------------------------------------------------------------
// DMMA tile GEMM: C = beta*C + sum_t alpha_t op(A_t) op(B_t).
// 128 threads, one 32x32 output tile per CTA, each warp a 16x16 quadrant made
// of 2x2 m8n8k4 fragments. Operands are staged through shared memory in 32-deep
// k-chunks; ragged edges are zero-filled.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.aligned;\n" ::: "memory");
  asm volatile("barrier.cluster.wait.aligned;\n" ::: "memory");
}

// Load of a double from the shared memory of CTA `rank` of this cluster, at the
// address that `local` has in this CTA.
__device__ __forceinline__ double ld_dsmem(const double* local, unsigned rank) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(local);
  unsigned ra;
  double v;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(ra) : "r"(a), "r"(rank));
  asm volatile("ld.shared::cluster.f64 %0, [%1];\n" : "=d"(v) : "r"(ra) : "memory");
  return v;
}

// ksplit > 1: the CTAs of a cluster of ksplit share one output tile and split
// its k-chunks (concatenated over the terms) into contiguous ranges; rank 0 adds
// the partial tiles in rank order from distributed shared memory (the result is
// deterministic for a given ksplit) and writes C.
__global__ void __launch_bounds__(128) gemm_f64_kernel(GemmArgs g, int ksplit) {
  __shared__ double As[T][T + 1];  // [m][k]
  __shared__ double Bs[T][T + 1];  // [k][n]
  const int tilesN = (g.N + T - 1) / T;
  const int tilesM = (g.M + T - 1) / T;
  // Tile order: lower-only outputs of a square C enumerate just the lower
  // tiles; triangular operands put the tiles with the longest k-range first
  // (largest-first keeps the tail of the launch short).
  const bool tri_enum = g.lowerC && g.M == g.N;
  const long long per_batch = tri_enum ? (long long)tilesM * (tilesM + 1) / 2
                                       : (long long)tilesM * tilesN;
  long long bid = blockIdx.x;
  unsigned part = 0;
  if (ksplit > 1) {
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(part));
    bid /= ksplit;
  }
  const long long tidx = bid % per_batch;
  bid /= per_batch;
  int tm, tn;
  if (tri_enum) {
    int r = (int)((sqrt(8.0 * (double)tidx + 1.0) - 1.0) * 0.5);
    while ((long long)(r + 1) * (r + 2) / 2 <= tidx) ++r;
    while ((long long)r * (r + 1) / 2 > tidx) --r;
    tm = r;
    tn = (int)(tidx - (long long)r * (r + 1) / 2);
  } else {
    tn = (int)(tidx % tilesN);
    tm = (int)(tidx / tilesN);
    if (g.t[0].triB == TRI_UPPER) tn = tilesN - 1 - tn;
    if (g.t[0].triA == TRI_LOWER) tm = tilesM - 1 - tm;
  }
  const int z1 = (int)(bid % g.nb1);
  const int z2 = (int)(bid / g.nb1);
  if (g.lowerC && tn > tm) return;
  const int m0 = tm * T, n0 = tn * T;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int gq = lane >> 2, tq = lane & 3;
  const int wm = (warp >> 1) * 16, wn = (warp & 1) * 16;

  double acc[2][2][2];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) acc[i][j][0] = acc[i][j][1] = 0.0;

  auto krange = [&](const GemmTerm& t, int& kb, int& ke) {
    kb = 0;
    ke = t.K;
    if (t.triA == TRI_LOWER) ke = min(ke, m0 + T);
    if (t.triA == TRI_UPPER) kb = max(kb, m0);
    if (t.triB == TRI_LOWER) kb = max(kb, n0);
    if (t.triB == TRI_UPPER) ke = min(ke, n0 + T);
  };
  int c_lo = 0, c_hi = 0x7fffffff, cidx = 0;
  if (ksplit > 1) {
    int nch = 0;
    for (int ti = 0; ti < g.nterms; ++ti) {
      int kb, ke;
      krange(g.t[ti], kb, ke);
      if (ke > kb) nch += (ke - kb + T - 1) / T;
    }
    c_lo = (int)((long long)part * nch / ksplit);
    c_hi = (int)((long long)(part + 1) * nch / ksplit);
  }
  for (int ti = 0; ti < g.nterms; ++ti) {
    const GemmTerm& t = g.t[ti];
    const double* A = t.A + (int64_t)z1 * t.sA1 + (int64_t)z2 * t.sA2;
    const double* B = t.B + (int64_t)z1 * t.sB1 + (int64_t)z2 * t.sB2;
    int kb, ke;
    krange(t, kb, ke);
    for (int k0 = kb; k0 < ke; k0 += T, ++cidx) {
      if (cidx < c_lo || cidx >= c_hi) continue;  // uniform over the CTA
      for (int e = tid; e < T * T; e += 128) {
        int i, kk;
        double v = 0.0;
        if (t.opA == OP_N) {
          i = e / T; kk = e % T;
          const int gi = m0 + i, gk = k0 + kk;
          if (gi < g.M && gk < ke) v = A[(int64_t)gi * t.lda + gk];
        } else {
          kk = e / T; i = e % T;
          const int gi = m0 + i, gk = k0 + kk;
          if (gi < g.M && gk < ke) v = A[(int64_t)gk * t.lda + gi];
        }
        As[i][kk] = scale_by(v, t.alpha);
      }
      for (int e = tid; e < T * T; e += 128) {
        int kk, j;
        double v = 0.0;
        if (t.opB == OP_N) {
          kk = e / T; j = e % T;
          const int gk = k0 + kk, gj = n0 + j;
          if (gk < ke && gj < g.N) v = B[(int64_t)gk * t.ldb + gj];
        } else {
          j = e / T; kk = e % T;
          const int gk = k0 + kk, gj = n0 + j;
          if (gk < ke && gj < g.N) v = B[(int64_t)gj * t.ldb + gk];
        }
        Bs[kk][j] = v;
      }
      __syncthreads();
      const int kl = min(T, ke - k0);  // a ragged last chunk stops at its last 4-wide k-step
#pragma unroll
      for (int ks = 0; ks < T; ks += 4) {
        if (ks >= kl) break;
        const double a0 = As[wm + gq][ks + tq];
        const double a1 = As[wm + 8 + gq][ks + tq];
        const double b0 = Bs[ks + tq][wn + gq];
        const double b1 = Bs[ks + tq][wn + 8 + gq];
        dmma_8x8x4(acc[0][0], a0, b0);
        dmma_8x8x4(acc[0][1], a0, b1);
        dmma_8x8x4(acc[1][0], a1, b0);
        dmma_8x8x4(acc[1][1], a1, b1);
      }
      __syncthreads();
    }
  }

  if (ksplit > 1) {
    double* red = &As[0][0];  // 8 partial sums per thread
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int h = 0; h < 2; ++h) red[((i * 2 + j) * 2 + h) * 128 + tid] = acc[i][j][h];
    cluster_sync_all();
    if (part == 0) {
      for (int q = 1; q < ksplit; ++q)
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
          for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int h = 0; h < 2; ++h)
              acc[i][j][h] += ld_dsmem(red + ((i * 2 + j) * 2 + h) * 128 + tid, (unsigned)q);
    }
    cluster_sync_all();  // the partial tiles stay readable until rank 0 is done
    if (part != 0) return;
  }

  double* C = g.C + (int64_t)z1 * g.sC1 + (int64_t)z2 * g.sC2;
#pragma unroll
  for (int mi = 0; mi < 2; ++mi)
#pragma unroll
    for (int ni = 0; ni < 2; ++ni)
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int r = m0 + wm + mi * 8 + gq;
        const int c = n0 + wn + ni * 8 + 2 * tq + j;
        if (r < g.M && c < g.N) {
          double* p = C + (int64_t)r * g.ldc + c;
          double v = acc[mi][ni][j];
          if (g.beta != 0.0) v += g.beta * *p;
          *p = v;
        }
      }
}

// Algorithmic flops of one launch: 2 per multiply-add whose operands are not
// structurally zero, over the output elements the call defines (all of C, or
// its lower triangle for lowerC). Host-side, only evaluated when timing is on.
double gemm_alg_flops(const GemmArgs& g) {
  double total = 0.0;
  for (int ti = 0; ti < g.nterms; ++ti) {
    const GemmTerm& t = g.t[ti];
    double cnt = 0.0;
    if (t.triA == TRI_NONE && t.triB == TRI_NONE) {
      double outs = 0.0;
      if (g.lowerC)
        for (int i = 0; i < g.M; ++i) outs += (double)min(i + 1, g.N);
      else
        outs = (double)g.M * g.N;
      cnt = outs * t.K;
    } else {
      for (int i = 0; i < g.M; ++i) {
        const int jn = g.lowerC ? min(i + 1, g.N) : g.N;
        for (int j = 0; j < jn; ++j) {
          int kb = 0, ke = t.K;
          if (t.triA == TRI_LOWER) ke = min(ke, i + 1);
          if (t.triA == TRI_UPPER) kb = max(kb, i);
          if (t.triB == TRI_LOWER) kb = max(kb, j);
          if (t.triB == TRI_UPPER) ke = min(ke, j + 1);
          if (ke > kb) cnt += ke - kb;
        }
      }
    }
    total += 2.0 * cnt;
  }
  return total * g.nb1 * g.nb2;
}

// Skinny products (M <= 32 rows, the arrowhead blocks): one CTA per 8-column
// strip of C and batch entry, 8 warps splitting k; each warp runs m8n8k4 DMMA
// on row groups of 8 straight from global memory (operands are reused through
// L1/L2), and the warps' partial sums are added in a fixed order in shared memory.
constexpr int kSkinnyMaxM = 32;

__global__ void __launch_bounds__(256) gemm_skinny_kernel(GemmArgs g) {
  __shared__ double red[8][kSkinnyMaxM / 8][64];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int gq = lane >> 2, tq = lane & 3;
  const int tilesN = (g.N + 7) / 8;
  long long bid = blockIdx.x;
  const int tn = (int)(bid % tilesN);
  bid /= tilesN;
  const int z1 = (int)(bid % g.nb1), z2 = (int)(bid / g.nb1);
  const int n0 = tn * 8;
  const int mg = (g.M + 7) / 8;  // row groups of 8
  double acc[kSkinnyMaxM / 8][2];
#pragma unroll
  for (int r = 0; r < kSkinnyMaxM / 8; ++r) acc[r][0] = acc[r][1] = 0.0;
  for (int ti = 0; ti < g.nterms; ++ti) {
    const GemmTerm& t = g.t[ti];
    const double* A = t.A + (int64_t)z1 * t.sA1 + (int64_t)z2 * t.sA2;
    const double* B = t.B + (int64_t)z1 * t.sB1 + (int64_t)z2 * t.sB2;
    int kb = 0, ke = t.K;
    if (t.triB == TRI_LOWER) kb = max(kb, n0);
    if (t.triB == TRI_UPPER) ke = min(ke, n0 + 8);
    // k split across the 8 warps in 4-wide steps
    const int steps = (ke - kb + 3) / 4;
    const int per = (steps + 7) / 8;
    const int s0 = w * per, s1 = min(steps, s0 + per);
    const int col = n0 + gq;
    for (int st = s0; st < s1; ++st) {
      const int k = kb + st * 4 + tq;
      double bv = 0.0;
      if (k < ke && col < g.N)
        bv = t.opB == OP_N ? B[(int64_t)k * t.ldb + col] : B[(int64_t)col * t.ldb + k];
#pragma unroll
      for (int r = 0; r < kSkinnyMaxM / 8; ++r) {
        if (r >= mg) break;
        const int row = r * 8 + gq;
        double av = 0.0;
        const bool in = row < g.M && k < ke;
        if (in) av = t.opA == OP_N ? A[(int64_t)row * t.lda + k] : A[(int64_t)k * t.lda + row];
        if (in && t.triA == TRI_LOWER && k > row) av = 0.0;
        if (in && t.triA == TRI_UPPER && k < row) av = 0.0;
        dmma_8x8x4(acc[r], scale_by(av, t.alpha), bv);
      }
    }
  }
#pragma unroll
  for (int r = 0; r < kSkinnyMaxM / 8; ++r) {
    red[w][r][lane * 2] = acc[r][0];
    red[w][r][lane * 2 + 1] = acc[r][1];
  }
  __syncthreads();
  double* C = g.C + (int64_t)z1 * g.sC1 + (int64_t)z2 * g.sC2;
  for (int e = tid; e < mg * 64; e += 256) {
    const int r = e / 64, q = e % 64;  // q = lane*2 + j -> row r*8 + lane/4, col n0 + 2*(lane%4) + j
    const int ln = q / 2, j = q % 2;
    const int row = r * 8 + (ln >> 2), c = n0 + 2 * (ln & 3) + j;
    if (row >= g.M || c >= g.N) continue;
    if (g.lowerC && c > row) continue;
    double v = 0.0;
    for (int ww = 0; ww < 8; ++ww) v += red[ww][r][q];
    double* p = C + (int64_t)row * g.ldc + c;
    if (g.beta != 0.0) v += g.beta * *p;
    *p = v;
  }
}

// Split of each output tile's k-chunks over a cluster: launches that fill less
// than a wave of CTA slots leave the SMs unevenly loaded (every resident CTA
// shares its SM's FP64 pipe), so the split is chosen to even out the CTAs per SM
// (mean over max CTAs per SM) while staying within one wave and keeping at least
// 4 chunks per part. (Splitting past a wave measured slower: 1024 tiles of a
// 1024 x 1024 x 1032 product took 2.21 ms split 4-way against 2.17 ms unsplit.)
static PerDevice g_gemm_shape;

static int gemm_ksplit(long long ctas, int kchunks) {
  const long long packed = per_device(g_gemm_shape, [] {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gemm_f64_kernel, 128, 0);
    return (long long)std::max(sms, 1) * 4096 + std::max(per_sm, 1);
  });
  const int sms = (int)(packed / 4096), per_sm = (int)(packed % 4096);
  const long long slots = (long long)sms * per_sm;
  if (ctas >= slots) return 1;
  auto eff = [&](long long n) {
    const double per = (double)n / sms;
    return per / std::ceil(per);
  };
  int best = 1;
  double be = eff(ctas);
  for (int k = 2; k <= 4; k *= 2) {
    if (kchunks / k < 4 || ctas * k > slots) break;
    const double e = eff(ctas * k);
    if (e > be + 0.01) {
      be = e;
      best = k;
    }
  }
  return best;
}

cudaError_t gemm_f64(const GemmArgs& g, cudaStream_t s) {
  if (g.M <= 0 || g.N <= 0 || g.nb1 <= 0 || g.nb2 <= 0) return cudaSuccess;
  if (g.M <= kSkinnyMaxM && g.N >= 64) {
    const long long grid = (long long)((g.N + 7) / 8) * g.nb1 * g.nb2;
    if (grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    TimedLaunch tl(K_GEMM, timing_on() ? gemm_alg_flops(g) : 0.0, s);
    gemm_skinny_kernel<<<(unsigned)grid, 256, 0, s>>>(g);
    return cudaGetLastError();
  }
  const long long tm = (g.M + T - 1) / T, tn = (g.N + T - 1) / T;
  const long long tiles = (g.lowerC && g.M == g.N) ? tm * (tm + 1) / 2 : tm * tn;
  const long long grid = tiles * g.nb1 * g.nb2;
  int kch = 0;
  for (int i = 0; i < g.nterms; ++i) kch += (g.t[i].K + T - 1) / T;
  const int ks = gemm_ksplit(grid, kch);
  if (grid * ks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  TimedLaunch tl(K_GEMM, timing_on() ? gemm_alg_flops(g) : 0.0, s);
  if (ks == 1) {
    gemm_f64_kernel<<<(unsigned)grid, 128, 0, s>>>(g, 1);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(grid * ks));
  cfg.blockDim = dim3(128);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = ks;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, gemm_f64_kernel, g, ks);
}

// ---------------------------------------------------------------------------
// POTRF of one diagonal tile; TRSM of the tiles below it; zeroing; mirroring.
// ---------------------------------------------------------------------------

// One right-looking step k of a blocked Cholesky in two launches: the diagonal
// tile (k, k) is factored and written back (recording a failed pivot), then the
// tiles below it are solved against the written factor, X L_kk^T = A(r, k).
// (A single launch in which the row tiles re-factor the diagonal tile while one
// CTA writes it back is a race: CTAs of a launch need not run at the same time,
// and a late one would read the factored tile.)
__global__ void __launch_bounds__(256) potrf_tile_kernel(double* A, int64_t ld, int64_t sb,
                                                         int nrow, int k, long long row0,
                                                         long long rstride) {
  __shared__ double S[T][T + 1];
  __shared__ double rd[T];
  double* Ab = A + (int64_t)blockIdx.y * sb;
  const int o = k * T, tb = min(T, nrow - o), tid = threadIdx.x;
  for (int e = tid; e < T * T; e += blockDim.x) {
    const int i = e / T, j = e % T;
    S[i][j] = (i < tb && j <= i) ? Ab[(int64_t)(o + i) * ld + o + j] : 0.0;
  }
  __syncthreads();
  coop_factor(S, rd, tb, row0 + (long long)blockIdx.y * rstride + o, &g_info);
  for (int e = tid; e < tb * tb; e += blockDim.x) {
    const int i = e / tb, j = e % tb;
    Ab[(int64_t)(o + i) * ld + o + j] = S[i][j];
  }
}

// Row tiles r = k + 1 + blockIdx.x of step k: X = A(r, k) L_kk^{-T}.
__global__ void __launch_bounds__(256) trsm_panel_kernel(double* A, int64_t ld, int64_t sb,
                                                         int nrow, int k) {
  __shared__ double Lt[T][T + 1];
  __shared__ double X[T][T + 1];
  __shared__ double rd[T];
  double* Ab = A + (int64_t)blockIdx.y * sb;
  const int o = k * T, tb = min(T, nrow - o), tid = threadIdx.x;
  const int r0 = o + T * (blockIdx.x + 1), rows = min(T, nrow - r0);
  for (int e = tid; e < T * T; e += blockDim.x) {
    const int i = e / T, j = e % T;
    Lt[i][j] = (i < tb && j <= i) ? Ab[(int64_t)(o + i) * ld + o + j] : 0.0;
    X[i][j] = (i < rows && j < tb) ? Ab[(int64_t)(r0 + i) * ld + o + j] : 0.0;
  }
  __syncthreads();
  if (tid < tb) rd[tid] = 1.0 / Lt[tid][tid];
  __syncthreads();
  panel_solve(X, Lt, rd, rows, tb);
  for (int e = tid; e < rows * tb; e += blockDim.x) {
    const int i = e / tb, j = e % tb;
    Ab[(int64_t)(r0 + i) * ld + o + j] = X[i][j];
  }
}
// Strict upper triangle -> 0 (tiles with tc >= tr).
__global__ void zero_upper_kernel(double* A, int64_t ld, int64_t sb, int nrow) {
  const int nt = (nrow + T - 1) / T;
  const int tr = blockIdx.x / nt, tc = blockIdx.x % nt;
  if (tc < tr) return;
  double* Ab = A + (int64_t)blockIdx.y * sb;
  for (int e = threadIdx.x; e < T * T; e += blockDim.x) {
    const int i = tr * T + e / T, j = tc * T + e % T;
    if (i < nrow && j < nrow && j > i) Ab[(int64_t)i * ld + j] = 0.0;
  }
}

// A[j][i] = A[i][j] for i > j (tiles with tr >= tc; tile (tr,tc) written to (tc,tr)).
__global__ void mirror_kernel(double* A, int64_t ld, int64_t sb, int nrow) {
  __shared__ double S[T][T + 1];
  const int nt = (nrow + T - 1) / T;
  const int tr = blockIdx.x / nt, tc = blockIdx.x % nt;
  if (tc > tr) return;
  double* Ab = A + (int64_t)blockIdx.y * sb;
  for (int e = threadIdx.x; e < T * T; e += blockDim.x) {
    const int i = e / T, j = e % T, gi = tr * T + i, gj = tc * T + j;
    S[i][j] = (gi < nrow && gj < nrow) ? Ab[(int64_t)gi * ld + gj] : 0.0;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < T * T; e += blockDim.x) {
    const int j = e / T, i = e % T;  // write row tc*T+j, column tr*T+i
    const int gi = tr * T + i, gj = tc * T + j;
    if (gi < nrow && gj < nrow && gi > gj) Ab[(int64_t)gj * ld + gi] = S[i][j];
  }
}

// Inverse of one diagonal tile (order tb <= T) of a lower-triangular block:
// Lb points at the tile's (0,0); the inverse goes to Xb (leading dimension ldx),
// zero above the diagonal.
__device__ __forceinline__ void tile_inv_body(const double* Lb, int64_t ldl, double* Xb,
                                              int64_t ldx, int tb) {
  __shared__ double Ls[T][T + 1];
  __shared__ double X[T][T + 1];
  __shared__ double rd[T];
  const int tid = threadIdx.x;
  for (int e = tid; e < T * T; e += blockDim.x) {
    const int i = e / T, j = e % T;
    Ls[i][j] = (i < tb && j <= i) ? Lb[(int64_t)i * ldl + j] : 0.0;
    X[i][j] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  if (tid < tb) rd[tid] = 1.0 / Ls[tid][tid];
  __syncthreads();
  // Forward substitution on L X = I, row j of X at a time (columns <= j only).
  for (int j = 0; j < tb; ++j) {
    for (int c = tid; c <= j; c += blockDim.x) X[j][c] *= rd[j];
    __syncthreads();
    const int rows = tb - j - 1, cols = j + 1;
    for (int e = tid; e < rows * cols; e += blockDim.x) {
      const int i = j + 1 + e / cols, c = e % cols;
      X[i][c] -= Ls[i][j] * X[j][c];
    }
    __syncthreads();
  }
  for (int e = tid; e < tb * tb; e += blockDim.x) {
    const int i = e / tb, j = e % tb;
    Xb[(int64_t)i * ldx + j] = (j <= i) ? X[i][j] : 0.0;
  }
}

// Inverse of each diagonal tile of lower-triangular blocks into the same
// positions of Linv (grid: tiles x blocks).
__global__ void __launch_bounds__(256) tile_inv_kernel(const double* L, int64_t ldl, int64_t sl,
                                                       double* Li, int64_t ldi, int64_t si,
                                                       int nrow) {
  const int o = blockIdx.x * T, tb = min(T, nrow - o);
  tile_inv_body(L + (int64_t)blockIdx.y * sl + (int64_t)o * ldl + o, ldl,
                Li + (int64_t)blockIdx.y * si + (int64_t)o * ldi + o, ldi, tb);
}

static inline unsigned ceil_div(long long a, long long b) { return (unsigned)((a + b - 1) / b); }

// ---------------------------------------------------------------------------
// Cooperative-launch building blocks. A wait that exceeds its poll limit
// records the timeout and lets the CTA go on, so a kernel always ends (the
// caller reads the flag with bta_tc_status).
// ---------------------------------------------------------------------------
__device__ int g_wait_error;

// ---------------------------------------------------------------------------
// One block step i of the factorization (Algorithm 1) in one cooperative
// launch. The block column [A_ii; A_{i+1,i}; A_{n,i}] is factored as a
// right-looking tile Cholesky whose trailing updates also reach the blocks
// that step i's Schur complement modifies:
//   A_{i+1,i+1} -= L_{i+1,i} L_{i+1,i}^T,  A_{n,i+1} -= L_{n,i} L_{i+1,i}^T,
//   A_nn -= L_{n,i} L_{n,i}^T.
// Tiles are indexed over the "extended" rows: the tiles of block i, then those
// of block i+1, then the arrow rows (E in all); the columns are those of block
// i (nt, factored here) and, with the Schur updates on, those of block i+1 and
// the tip (updated only). Operations on a tile (r, c):
//   U(r, c, k)  tile (r, c) -= L(r, k) L(c, k)^T, for every factor column k < c;
//   F(r, c)     (c < nt, after every U) tile (c, c) -> its Cholesky factor, or
//               tile (r, c), r > c -> the panel solve X L(c, c)^T = A(r, c).
// This covers the POTRF of A_ii, the TRSMs of L_{i+1,i} and L_{n,i} (panel
// solves, no inverse of L_ii) and the three Schur products (the U's in the
// columns of block i+1 and of the tip).
//
// Scheduling is dataflow, without grid barriers. Tile (r, c) always belongs to
// CTA u(r, c) mod G, u being the tile's column-major index in the lower
// triangle, so every update of a tile runs on one CTA in program order. The
// only waits are on finalized tiles: pdone[r] counts the finalized columns of
// tile row r (tile (r, c) is final once pdone[r] > c). Each CTA walks phases
//   1(k) = U(., k+1, k) then F(., k+1);  2(k) = U(., k+2, k);  3(k) = U(., c >= k+3, k)
// in the order 1(k), 2(k), 1(k+1), 3(k), 2(k+1), 1(k+2), 3(k+1), ... (phase
// numbers 3k, 3k+2 and 3k+4), taking its own tiles of each phase in column-major
// order. Column k+2 is thus finalized before the bulk of step k: a two-step
// look-ahead. Every wait is on a tile of an earlier phase, or (the panel solves
// of F(., k+1)) on the diagonal tile (k+1, k+1), which its owner takes first in
// the same phase and which waits on earlier phases only; so the schedule cannot
// deadlock while all CTAs are resident (cooperative launch). Every wait is
// bounded and reports through bta_tc_status. The bulk phase 3(k) is one
// contiguous range of u, so its tiles split evenly over the CTAs.
// ---------------------------------------------------------------------------
constexpr int kStepThreads = 256;
// Resident CTAs per SM of the step kernel (its register budget and grid size):
// 60 registers, no spills; 4 per SM factored n=32, b=2048, a=16 in 648 ms
// against 651 ms at 3 and 660 ms at 2 (bit-identical results).
#ifndef BTA_STEP_CTAS_PER_SM
#define BTA_STEP_CTAS_PER_SM 4
#endif
constexpr int kStepCtasPerSm = BTA_STEP_CTAS_PER_SM;

struct StepArgs {
  double* D0;   // A_ii (b x b): L_ii on return, strict upper triangle zeroed
  double* Lw;   // A_{i+1,i} (b x b): L_{i+1,i}; unused when next == 0
  double* D1;   // A_{i+1,i+1} (b x b): lower tiles updated
  double* Ar0;  // A_{n,i} (a x b): L_{n,i}
  double* Ar1;  // A_{n,i+1} (a x b): updated; unused when next == 0
  double* tip;  // A_nn (a x a): lower tiles updated
  int b, a, nt, na, next;
  int64_t ld;      // leading dimension of D0, Lw and D1 (b for whole blocks)
  int schur;       // 0: only block i's columns (no updates of D1, Ar1, tip)
  long long row0;  // 1-based global row of block i's first row, minus one
  int* pdone;      // [E]: finalized columns of each extended tile row (zeroed per launch)
  int* colcnt;     // [nt]: finalized tiles of each factor column (zeroed per launch)
  double* rdv;     // [nt][T]: 1 / L_jj of each factored diagonal tile
};

// Group of an extended tile row (0: block i, 1: block i+1, 2: arrow) and its
// tile index inside the group.
__device__ __forceinline__ int ext_group(const StepArgs& p, int r, int& lr) {
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

__device__ __forceinline__ int ext_rows(const StepArgs& p, int r) {
  int lr;
  const int g = ext_group(p, r, lr);
  return min(T, (g == 2 ? p.a : p.b) - T * lr);
}

// Address and leading dimension of tile (r, c), r >= c, of the extended lower
// triangle (arrow rows have rows of b, the tip rows of a, the rest rows of ld).
__device__ __forceinline__ double* ext_tile(const StepArgs& p, int r, int c, int64_t& ld) {
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

// Bounded wait until *flag >= v (a flag another CTA of the same cooperative
// launch raises); after max_polls polls the error word is set and the CTA goes
// on. Once any wait has timed out, later waits give up at once, so a launch that
// lost a dependency still ends within about one timeout.
__device__ __forceinline__ void wait_flag_ge(const int* flag, int v,
                                             unsigned max_polls = 1u << 22) {
  if (threadIdx.x == 0) {
    unsigned polls = 0;
    while (atomicAdd((int*)flag, 0) < v) {
      if (++polls > max_polls || *(volatile int*)&g_wait_error) {
        atomicExch(&g_wait_error, 1);
        break;
      }
      __nanosleep(32);
    }
    __threadfence();
  }
  __syncthreads();
}

// Bounded wait until flag_a >= va and flag_b >= vb (same rules as wait_flag_ge).
__device__ __forceinline__ void wait_flags_ge(const int* fa, int va, const int* fb, int vb) {
  if (threadIdx.x == 0) {
    unsigned polls = 0;
    while (atomicAdd((int*)fa, 0) < va || atomicAdd((int*)fb, 0) < vb) {
      if (++polls > (1u << 22) || *(volatile int*)&g_wait_error) {
        atomicExch(&g_wait_error, 1);
        break;
      }
      __nanosleep(32);
    }
    __threadfence();
  }
  __syncthreads();
}

// Publishes *flag = v after this CTA's preceding global writes (call after a
// __syncthreads that follows them).
__device__ __forceinline__ void raise_flag(int* flag, int v) {
  if (threadIdx.x == 0) {
    __threadfence();
    atomicExch(flag, v);
  }
}

// 8-byte asynchronous global -> shared copy (zero-fill when !pred).
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem, bool pred) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(sa), "l"(gmem), "r"(pred ? 8 : 0));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

__global__ void __launch_bounds__(kStepThreads, kStepCtasPerSm) factor_step_kernel(StepArgs p) {
  __shared__ double Pb[2][T][T + 1];  // L(r, k), double-buffered
  __shared__ double Qb[2][T][T + 1];  // L(c, k)
  __shared__ double rd[T];
  // Finalizations run outside the pipelined bulk phase, when buffer 1 is idle:
  // S (a diagonal tile being factored, or a panel tile being solved) and Lt (the
  // diagonal factor a panel tile is solved with) live there.
  double(*const S)[T + 1] = Pb[1];
  double(*const Lt)[T + 1] = Qb[1];
  const int tid = threadIdx.x, G = gridDim.x, bid = blockIdx.x;
  const int lane = tid & 31, warp = tid >> 5, gq = lane >> 2, tq = lane & 3;
  const int wm = (warp >> 1) * 8, wn = (warp & 1) * 16;  // this warp's 8 x 16 part of a tile
  const int nt = p.nt, E = nt * (1 + p.next) + p.na, Ecol = p.schur ? E : nt;
  const int64_t b = p.ld;  // row stride of A_ii

  // The strict upper tiles of A_ii belong to no operation: zero them now (upper
  // tile u = (tr, tc), tc > tr, enumerated row by row).
  for (int u = bid; u < nt * (nt - 1) / 2; u += G) {
    int tr = 0, rem = u;
    while (rem >= nt - 1 - tr) rem -= nt - 1 - tr++;
    const int tc = tr + 1 + rem;
    const int rows = min(T, p.b - tr * T), cols = min(T, p.b - tc * T);
    double* Z = p.D0 + (int64_t)(tr * T) * b + tc * T;
    for (int e = tid; e < T * T; e += blockDim.x)
      if (e / T < rows && e % T < cols) Z[(int64_t)(e / T) * b + e % T] = 0.0;
  }

  // Column-major index of the first tile of column c (rows c .. E-1).
  auto off = [&](int c) -> long long { return (long long)c * E - (long long)c * (c - 1) / 2; };

  // U(r, c, k): tile (r, c) -= L(r, k) L(c, k)^T, in two parts: issue the
  // copies of the two panel tiles into buffer bf (one commit group), then, once
  // they have landed, the DMMA update of C in place.
  auto issue = [&](int r, int c, int k, int bf) {
    const int tbk = min(T, p.b - k * T);
    const int rb = ext_rows(p, r), cb = ext_rows(p, c);
    int64_t ldr, ldq;
    const double* Lr = ext_tile(p, r, k, ldr);
    const double* Lc = ext_tile(p, c, k, ldq);
    for (int e = tid; e < T * T; e += blockDim.x) {
      const int i = e / T, j = e % T;
      const bool pr = i < rb && j < tbk, pc = i < cb && j < tbk;
      cp_async8(&Pb[bf][i][j], pr ? Lr + (int64_t)i * ldr + j : Lr, pr);
      cp_async8(&Qb[bf][i][j], pc ? Lc + (int64_t)i * ldq + j : Lc, pc);
    }
    cp_async_commit();
  };
  auto compute = [&](int r, int c, int bf) {
    const int rb = ext_rows(p, r), cb = ext_rows(p, c);
    int64_t ldc;
    double* C = ext_tile(p, r, c, ldc);
    const int row = wm + gq;
    if (wm < rb && wn < cb) {  // warp-uniform
      double cold[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
      double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
#pragma unroll
      for (int ni = 0; ni < 2; ++ni)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const int col = wn + ni * 8 + 2 * tq + j;
          if (row < rb && col < cb) cold[ni][j] = C[(int64_t)row * ldc + col];
        }
#pragma unroll
      for (int ks = 0; ks < T; ks += 4) {
        const double av = Pb[bf][row][ks + tq];
        dmma_8x8x4(acc[0], av, Qb[bf][wn + gq][ks + tq]);
        dmma_8x8x4(acc[1], av, Qb[bf][wn + 8 + gq][ks + tq]);
      }
#pragma unroll
      for (int ni = 0; ni < 2; ++ni)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const int col = wn + ni * 8 + 2 * tq + j;
          if (row < rb && col < cb) C[(int64_t)row * ldc + col] = cold[ni][j] - acc[ni][j];
        }
    }
  };
  // One update with its own waits (the look-ahead columns).
  auto update = [&](int r, int c, int k) {
    wait_flags_ge(p.pdone + r, k + 1, p.pdone + c, k + 1);
    issue(r, c, k, 0);
    cp_async_wait<0>();
    __syncthreads();
    compute(r, c, 0);
    __syncthreads();  // the buffer is consumed
  };

  // F(r, c): factor the diagonal tile (r == c) or solve the panel tile (r > c).
  auto finalize = [&](int r, int c) {
    const int tb = min(T, p.b - c * T);
    if (r == c) {
      double* Dc = p.D0 + (int64_t)(c * T) * b + c * T;
      for (int e = tid; e < T * T; e += blockDim.x) {
        const int i = e / T, j = e % T;
        S[i][j] = (i < tb && j <= i) ? Dc[(int64_t)i * b + j] : 0.0;
      }
      __syncthreads();
      coop_factor(S, rd, tb, p.row0 + (long long)c * T, &g_info);
      for (int e = tid; e < T * T; e += blockDim.x) {
        const int i = e / T, j = e % T;
        if (i < tb && j < tb) Dc[(int64_t)i * b + j] = S[i][j];
      }
      if (tid < T) p.rdv[(int64_t)c * T + tid] = rd[tid];
      __syncthreads();
      raise_flag(p.pdone + c, c + 1);
      if (tid == 0) atomicAdd(p.colcnt + c, 1);
      return;
    }
    wait_flag_ge(p.pdone + c, c + 1);  // the diagonal tile (c, c) is factored
    const int rows = ext_rows(p, r);
    int64_t ldx;
    double* X = ext_tile(p, r, c, ldx);
    const double* Dc = p.D0 + (int64_t)(c * T) * b + c * T;
    for (int e = tid; e < T * T; e += blockDim.x) {
      const int i = e / T, j = e % T;
      Lt[i][j] = (i < tb && j <= i) ? __ldcg(Dc + (int64_t)i * b + j) : 0.0;
      S[i][j] = (i < rows && j < tb) ? X[(int64_t)i * ldx + j] : 0.0;
    }
    if (tid < T) rd[tid] = __ldcg(p.rdv + (int64_t)c * T + tid);
    __syncthreads();
    panel_solve(S, Lt, rd, rows, tb);
    for (int e = tid; e < rows * tb; e += blockDim.x) {
      const int i = e / tb, j = e % tb;
      X[(int64_t)i * ldx + j] = S[i][j];
    }
    __syncthreads();
    raise_flag(p.pdone + r, c + 1);
    if (tid == 0) atomicAdd(p.colcnt + c, 1);
  };

  // This CTA's tiles of column c in rows [c, E), in order.
  auto column = [&](int c, int k, bool fin) {
    const long long lo = off(c), hi = lo + (E - c);
    for (long long u = lo + ((bid - lo % G) % G + G) % G; u < hi; u += G) {
      const int r = c + (int)(u - lo);
      if (k >= 0) update(r, c, k);
      if (fin) finalize(r, c);
    }
  };

  for (int ph = -3; ph <= 3 * (nt - 1) + 4; ++ph) {
    const int m3 = ((ph % 3) + 3) % 3;
    if (m3 == 0) {  // 1(k): column k+1 at step k, then its finalization
      const int k = ph / 3;  // exact: ph is a multiple of 3
      const int c = k + 1;
      if (k >= nt || c >= Ecol) continue;
      column(c, k, c < nt);
    } else if (m3 == 2) {  // 2(k): column k+2 at step k
      const int k = (ph - 2) / 3;
      const int c = k + 2;
      if (ph < 2 || k >= nt || c >= Ecol) continue;
      column(c, k, false);
    } else {  // 3(k): columns k+3 .. Ecol-1 at step k
      const int k = (ph - 4) / 3;
      if (ph < 4 || k >= nt || k + 3 >= Ecol) continue;
      const long long lo = off(k + 3), hi = off(Ecol);
      long long u = lo + ((bid - lo % G) % G + G) % G;
      if (u >= hi) continue;
      // Every tile of this phase reads column k only: wait once for all of it.
      wait_flag_ge(p.colcnt + k, E - k);
      int c = k + 3;
      while (off(c + 1) <= u) ++c;
      int r = c + (int)(u - off(c)), bf = 0;
      issue(r, c, k, 0);
      for (;;) {
        const long long un = u + G;
        int cn = c, rn = 0;
        if (un < hi) {
          while (off(cn + 1) <= un) ++cn;
          rn = cn + (int)(un - off(cn));
          issue(rn, cn, k, bf ^ 1);  // in flight during this update
          cp_async_wait<1>();
        } else {
          cp_async_wait<0>();
        }
        __syncthreads();
        compute(r, c, bf);
        __syncthreads();  // buffer bf is consumed
        if (un >= hi) break;
        u = un;
        c = cn;
        r = rn;
        bf ^= 1;
      }
    }
  }
}

static PerDevice g_step_grid;

// Cooperative grid of the step kernel on the current device (at most 2 CTAs per
// SM, as many as are co-resident; -1 if none can be).
static int step_grid() {
  return (int)per_device(g_step_grid, [] {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, factor_step_kernel, kStepThreads, 0);
    // Several CTAs per SM: one CTA's loads, stores and barriers overlap the
    // others' DMMA work on the SM's FP64 pipe.
    const int g = std::min(per, kStepCtasPerSm) * sms;
    return (long long)(g > 0 ? g : -1);
  });
}

// Algorithmic flops of one step: POTRF b^3/3, the (b [+ b] + a)-row panel solve
// (b^2 per row), and (schur != 0) the Schur products on the lower triangles they
// update; without them the launch does only the POTRF and the panel solves.
static double step_flops(double b, double a, int next, int schur) {
  double f = b * b * b / 3.0 + (next ? b : 0.0) * b * b + a * b * b;
  if (!schur) return f;
  if (next) f += b * (b + 1) * b + 2.0 * a * b * b;
  f += a * (a + 1) * b;
  return f;
}

cudaError_t factor_step_coop(double* D0, double* Lw, double* D1, double* Ar0, double* Ar1,
                             double* tip, int b, int a, int next, long long info_row0,
                             void* scratch, cudaStream_t s, int schur, int64_t ld) {
  StepArgs p;
  p.D0 = D0; p.Lw = Lw; p.D1 = D1; p.Ar0 = Ar0; p.Ar1 = Ar1; p.tip = tip;
  p.b = b; p.a = a; p.nt = (b + T - 1) / T; p.na = (a + T - 1) / T; p.next = next ? 1 : 0;
  p.ld = ld > 0 ? ld : b;
  if (p.ld < b) return cudaErrorInvalidValue;
  p.schur = schur ? 1 : 0;
  p.row0 = info_row0;
  p.pdone = (int*)scratch;
  p.colcnt = p.pdone + kStepMaxExtTiles;
  p.rdv = (double*)((char*)scratch + kStepFlagBytes);
  if (p.nt > kStepMaxTiles || 2 * p.nt + p.na > kStepMaxExtTiles) return cudaErrorInvalidValue;
  if (b < 1 || a < 0 || (next && !Lw) || (a > 0 && !Ar0) ||
      (schur && ((next && (!D1 || (a > 0 && !Ar1))) || (a > 0 && !tip))))
    return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(scratch, 0, kStepFlagBytes, s);
  if (e != cudaSuccess) return e;
  const int G = step_grid();
  if (G < 2) return cudaErrorInvalidConfiguration;
  void* args[] = {&p};
  TimedLaunch tl(K_FACTOR_STEP, timing_on() ? step_flops(b, a, p.next, p.schur) : 0.0, s);
  return cudaLaunchCooperativeKernel((void*)factor_step_kernel, dim3(G), dim3(kStepThreads), args,
                                     0, s);
}

// Self-test of the bounded wait: one CTA waits on a flag that nothing raises,
// with a poll limit of `polls`, so the wait gives up and records the timeout.
__global__ void wait_selftest_kernel(const int* flag, unsigned polls) {
  wait_flag_ge(flag, 1, polls);
}

cudaError_t wait_selftest(const int* flag_dev, unsigned polls, cudaStream_t s) {
  wait_selftest_kernel<<<1, 64, 0, s>>>(flag_dev, polls);
  return cudaGetLastError();
}

cudaError_t wait_error_read_reset(int* out) {
  int v = 0;
  cudaError_t e = cudaMemcpyFromSymbol(&v, g_wait_error, sizeof(int));
  if (e != cudaSuccess) return e;
  *out = v;
  const int zero = 0;
  return cudaMemcpyToSymbol(g_wait_error, &zero, sizeof(int));
}



cudaError_t potrf_blocks(double* A, int64_t ld, int64_t sb, int count, int nrow,
                         long long info_row0, long long info_rstride, cudaStream_t s) {
  if (count <= 0 || nrow <= 0) return cudaSuccess;
  const int nt = (nrow + T - 1) / T;
  for (int c0 = 0; c0 < count; c0 += 65535) {
    const int cnt = min(65535, count - c0);
    double* Ac = A + (int64_t)c0 * sb;
    const long long r0 = info_row0 + (long long)c0 * info_rstride;
    for (int k = 0; k < nt; ++k) {
      {
        TimedLaunch tl(K_POTRF_TILE, 0.0, s);
        potrf_tile_kernel<<<dim3(1, cnt), 256, 0, s>>>(Ac, ld, sb, nrow, k, r0, info_rstride);
      }
      if (k + 1 < nt) {
        TimedLaunch tl(K_TRSM_PANEL, 0.0, s);
        trsm_panel_kernel<<<dim3(nt - k - 1, cnt), 256, 0, s>>>(Ac, ld, sb, nrow, k);
      }
      if (k + 1 < nt) {
        const int o = (k + 1) * T, m = nrow - o;
        GemmArgs g{};
        g.t[0] = term(Ac + (int64_t)o * ld + k * T, ld, OP_N, TRI_NONE,
                      Ac + (int64_t)o * ld + k * T, ld, OP_T, TRI_NONE, T, -1.0);
        g.t[0].sA1 = sb; g.t[0].sB1 = sb;
        g.nterms = 1;
        g.C = Ac + (int64_t)o * ld + o; g.ldc = ld; g.sC1 = sb;
        g.M = m; g.N = m; g.beta = 1.0; g.lowerC = 1; g.nb1 = cnt; g.nb2 = 1;
        cudaError_t e = gemm_f64(g, s);
        if (e != cudaSuccess) return e;
      }
    }
    {
      TimedLaunch tl(K_ZERO_UPPER, 0.0, s);
      zero_upper_kernel<<<dim3(nt * nt, cnt), 256, 0, s>>>(Ac, ld, sb, nrow);
    }
  }
  return cudaGetLastError();
}

cudaError_t trtri_blocks(const double* L, int64_t ldl, int64_t sl, double* Li, int64_t ldi,
                         int64_t si, int count, int nrow, cudaStream_t s, GemmHook hook,
                         void* ctx) {
  if (count <= 0 || nrow <= 0) return cudaSuccess;
  const int nt = (nrow + T - 1) / T;
  for (int c0 = 0; c0 < count; c0 += 65535) {
    const int cnt = min(65535, count - c0);
    const double* Lc = L + (int64_t)c0 * sl;
    double* Xc = Li + (int64_t)c0 * si;
    {
      TimedLaunch tl(K_TILE_INV, 0.0, s);
      tile_inv_kernel<<<dim3(nt, cnt), 256, 0, s>>>(Lc, ldl, sl, Xc, ldi, si, nrow);
    }
    // Doubling: [X11 0; X21 X22] with X21 = -X22 (L21 X11); the product
    // (L21 X11)^T is parked in the (still unused) strict upper part.
    for (int sz = T; sz < nrow; sz *= 2) {
      const int full = nrow / (2 * sz);
      const int tail_o = full * 2 * sz;
      const int tail = (tail_o + sz < nrow) ? nrow - tail_o - sz : 0;
      for (int part = 0; part < 2; ++part) {
        const int pairs = part == 0 ? full : (tail ? 1 : 0);
        if (!pairs) continue;
        const int o = part == 0 ? 0 : tail_o;
        const int s2 = part == 0 ? sz : tail;
        const int64_t pstride_l = (int64_t)2 * sz * (ldl + 1);
        const int64_t pstride_i = (int64_t)2 * sz * (ldi + 1);
        // Tmp^T (sz x s2) = X11^T (sz x sz, upper) * L21^T (sz x s2)
        GemmArgs g1{};
        g1.t[0] = term(Xc + (int64_t)o * ldi + o, ldi, OP_T, TRI_UPPER,
                       Lc + (int64_t)(o + sz) * ldl + o, ldl, OP_T, TRI_NONE, sz, 1.0);
        g1.t[0].sA1 = pstride_i; g1.t[0].sB1 = pstride_l;
        g1.t[0].sA2 = si; g1.t[0].sB2 = sl;
        g1.nterms = 1;
        g1.C = Xc + (int64_t)o * ldi + o + sz; g1.ldc = ldi; g1.sC1 = pstride_i; g1.sC2 = si;
        g1.M = sz; g1.N = s2; g1.beta = 0.0; g1.lowerC = 0; g1.nb1 = pairs; g1.nb2 = cnt;
        cudaError_t e = hook ? hook(g1, ctx, s) : gemm_f64(g1, s);
        if (e != cudaSuccess) return e;
        // X21 (s2 x sz) = -X22 (s2 x s2, lower) * Tmp (s2 x sz)
        GemmArgs g2{};
        g2.t[0] = term(Xc + (int64_t)(o + sz) * ldi + o + sz, ldi, OP_N, TRI_LOWER,
                       Xc + (int64_t)o * ldi + o + sz, ldi, OP_T, TRI_NONE, s2, -1.0);
        g2.t[0].sA1 = pstride_i; g2.t[0].sB1 = pstride_i;
        g2.t[0].sA2 = si; g2.t[0].sB2 = si;
        g2.nterms = 1;
        g2.C = Xc + (int64_t)(o + sz) * ldi + o; g2.ldc = ldi; g2.sC1 = pstride_i; g2.sC2 = si;
        g2.M = s2; g2.N = sz; g2.beta = 0.0; g2.lowerC = 0; g2.nb1 = pairs; g2.nb2 = cnt;
        e = hook ? hook(g2, ctx, s) : gemm_f64(g2, s);
        if (e != cudaSuccess) return e;
      }
    }
    {
      TimedLaunch tl(K_ZERO_UPPER, 0.0, s);
      zero_upper_kernel<<<dim3(nt * nt, cnt), 256, 0, s>>>(Xc, ldi, si, nrow);
    }
  }
  return cudaGetLastError();
}

cudaError_t mirror_lower(double* A, int64_t ld, int64_t sb, int count, int nrow, cudaStream_t s) {
  if (count <= 0 || nrow <= 0) return cudaSuccess;
  const int nt = (nrow + T - 1) / T;
  for (int c0 = 0; c0 < count; c0 += 65535) {
    const int cnt = min(65535, count - c0);
    TimedLaunch tl(K_MIRROR, 0.0, s);
    mirror_kernel<<<dim3(nt * nt, cnt), 256, 0, s>>>(A + (int64_t)c0 * sb, ld, sb, nrow);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// log-determinant: per-block sums in a fixed tree order, then blocks in order.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) logdet_partial_kernel(const double* diag, int64_t n,
                                                             int64_t b, const double* tip,
                                                             int64_t a, double* partial) {
  __shared__ double red[256];
  const int64_t z = blockIdx.x;
  const double* M = z < n ? diag + z * b * b : tip;
  const int64_t m = z < n ? b : a;
  double sum = 0.0;
  for (int64_t k = threadIdx.x; k < m; k += 256) sum += log(M[k * m + k]);
  red[threadIdx.x] = sum;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[z] = red[0];
}

__global__ void logdet_final_kernel(const double* partial, int64_t count, double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int64_t z = 0; z < count; ++z) s += partial[z];
    *out = 2.0 * s;
  }
}

cudaError_t logdet_partials(const double* diag, int64_t n, int64_t b, const double* tip, int64_t a,
                            double* partial, cudaStream_t s) {
  const int64_t count = n + (a > 0 ? 1 : 0);
  if (count <= 0) return cudaSuccess;
  TimedLaunch tl(K_LOGDET, 0.0, s);
  logdet_partial_kernel<<<(unsigned)count, 256, 0, s>>>(diag, n, b, tip, a, partial);
  return cudaGetLastError();
}

// out = 2 * (sum p1[0..n1) + sum p2[0..n2)), in that order.
__global__ void logdet_combine_kernel(const double* p1, int64_t n1, const double* p2, int64_t n2,
                                      double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int64_t z = 0; z < n1; ++z) s += p1[z];
    for (int64_t z = 0; z < n2; ++z) s += p2[z];
    *out = 2.0 * s;
  }
}

cudaError_t logdet_combine(const double* p1, int64_t n1, const double* p2, int64_t n2, double* out,
                           cudaStream_t s) {
  logdet_combine_kernel<<<1, 32, 0, s>>>(p1, n1, p2, n2, out);
  return cudaGetLastError();
}

__global__ void axpy_kernel(int64_t n, double alpha, const double* x, double* y) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    y[e] += alpha * x[e];
}

cudaError_t axpy_f64(int64_t n, double alpha, const double* x, double* y, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  axpy_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 1216), 256, 0, s>>>(n, alpha, x, y);
  return cudaGetLastError();
}

cudaError_t logdet_f64(const double* diag, int64_t n, int64_t b, const double* tip, int64_t a,
                       double* partial, double* out, cudaStream_t s) {
  const int64_t count = n + (a > 0 ? 1 : 0);
  TimedLaunch tl(K_LOGDET, 0.0, s);
  logdet_partial_kernel<<<(unsigned)count, 256, 0, s>>>(diag, n, b, tip, a, partial);
  logdet_final_kernel<<<1, 32, 0, s>>>(partial, count, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Solve pieces.
// ---------------------------------------------------------------------------
// In-place triangular solve L x = r (trans = 0) or L^T x = r (trans = 1) by one
// thread-block cluster. Row tiles are owned round-robin by the cluster's CTAs.
// Step k: the owner of tile k solves it (one warp per right-hand side, lanes =
// rows, shuffles carry x_j down the tile), a cluster barrier (release/acquire)
// publishes it, and every CTA subtracts its contribution from the row tiles it
// owns that are still unsolved. The owner of tile k+1 has applied every update
// to that tile itself, so one barrier per tile step suffices.
constexpr int kTrsvPrefetch = 4;  // row tiles per CTA whose L tiles are prefetched into registers

// L tile element for the update of row tile r by solved tile k: L(r,k) (forward)
// or L(k,r)^T (transposed), as Lk[i][c] with i in tile r, c in tile k.
__device__ __forceinline__ double trsv_tile_el(const double* L, int64_t ld, int trans, int ro, int rb,
                                               int o, int tb, int i, int c) {
  if (i >= rb || c >= tb) return 0.0;
  return trans ? L[(int64_t)(o + c) * ld + ro + i] : L[(int64_t)(ro + i) * ld + o + c];
}

__global__ void __launch_bounds__(256, 1) trsv_cluster_kernel(const double* L, int64_t ld, int nrow,
                                                           double* x, int64_t ldx, int R, int trans) {
  __shared__ double Xk[T][65];
  __shared__ double Lk[T][T + 1];
  __shared__ double Ld[T][T + 1];
  __shared__ double rdiag[T];
  unsigned rank, csize;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(rank));
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(csize));
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nt = (nrow + T - 1) / T;
  for (int step = 0; step < nt; ++step) {
    const int k = trans ? nt - 1 - step : step;
    const int o = k * T, tb = min(T, nrow - o);
    const bool owner = (unsigned)(k % (int)csize) == rank;
    // This CTA's row tiles still to update: r_first + t * csize, t < count.
    int r_first, count;
    if (!trans) {
      r_first = k + 1 + (int)((rank + csize - (unsigned)((k + 1) % (int)csize)) % csize);
      count = r_first < nt ? (nt - 1 - r_first) / (int)csize + 1 : 0;
    } else {
      r_first = (int)rank;
      count = r_first < k ? (k - 1 - r_first) / (int)csize + 1 : 0;
    }
    // Prefetch (independent of x_k) the first kTrsvPrefetch of their L tiles into registers.
    double pre[kTrsvPrefetch][4];
#pragma unroll
    for (int t = 0; t < kTrsvPrefetch; ++t) {
      if (t < count) {
        const int ro = (r_first + t * (int)csize) * T, rb = min(T, nrow - ro);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int e = tid + 256 * q, i = trans ? e % T : e / T, c = trans ? e / T : e % T;
          pre[t][q] = trsv_tile_el(L, ld, trans, ro, rb, o, tb, i, c);
        }
      }
    }
    if (owner) {
      for (int e = tid; e < T * T; e += blockDim.x) {
        const int i = e / T, c = e % T;
        Ld[i][c] = (i < tb && c <= i) ? L[(int64_t)(o + i) * ld + o + c] : 0.0;
      }
      __syncthreads();
      if (tid < tb) rdiag[tid] = 1.0 / Ld[tid][tid];
      __syncthreads();
      for (int q = warp; q < R; q += 8) {
        double xi = lane < tb ? x[(int64_t)(o + lane) * ldx + q] : 0.0;
        if (!trans) {
          for (int j = 0; j < tb; ++j) {
            const double xj = __shfl_sync(0xffffffffu, xi, j) * rdiag[j];
            if (lane == j) xi = xj;
            else if (lane > j) xi -= Ld[lane][j] * xj;
          }
        } else {
          for (int j = tb - 1; j >= 0; --j) {
            const double xj = __shfl_sync(0xffffffffu, xi, j) * rdiag[j];
            if (lane == j) xi = xj;
            else if (lane < j) xi -= Ld[j][lane] * xj;
          }
        }
        if (lane < tb) x[(int64_t)(o + lane) * ldx + q] = xi;
      }
    }
    cluster_sync_all();
    for (int e = tid; e < tb * R; e += blockDim.x) Xk[e / R][e % R] = x[(int64_t)(o + e / R) * ldx + e % R];
#pragma unroll
    for (int t = 0; t < kTrsvPrefetch + 1; ++t) {
      // t < kTrsvPrefetch: one prefetched tile; t == kTrsvPrefetch: every remaining tile, loaded here
      const int tend = t < kTrsvPrefetch ? min(count, t + 1) : count;
      for (int u = t; u < tend; ++u) {
        const int ro = (r_first + u * (int)csize) * T, rb = min(T, nrow - ro);
        __syncthreads();  // Xk written; previous tile's Lk reads done
        if (t < kTrsvPrefetch) {
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int e = tid + 256 * q, i = trans ? e % T : e / T, c = trans ? e / T : e % T;
            Lk[i][c] = pre[t][q];
          }
        } else {
          for (int e = tid; e < T * T; e += blockDim.x) {
            const int i = trans ? e % T : e / T, c = trans ? e / T : e % T;
            Lk[i][c] = trsv_tile_el(L, ld, trans, ro, rb, o, tb, i, c);
          }
        }
        __syncthreads();
        for (int e = tid; e < rb * R; e += blockDim.x) {
          const int i = e / R, q = e % R;
          double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;  // four chains over c
          for (int c = 0; c < tb; c += 4) {
            a0 = fma(Lk[i][c], Xk[c][q], a0);
            if (c + 1 < tb) a1 = fma(Lk[i][c + 1], Xk[c + 1][q], a1);
            if (c + 2 < tb) a2 = fma(Lk[i][c + 2], Xk[c + 2][q], a2);
            if (c + 3 < tb) a3 = fma(Lk[i][c + 3], Xk[c + 3][q], a3);
          }
          x[(int64_t)(ro + i) * ldx + q] -= (a0 + a1) + (a2 + a3);
        }
      }
      if (t < kTrsvPrefetch) continue;
    }
    __syncthreads();
  }
}

static PerDevice g_trsv_cluster;

static int trsv_cluster_size(cudaStream_t s) {
  return (int)per_device(g_trsv_cluster, [s]() -> long long {
  int sz = 16;
  if (cudaFuncSetAttribute(trsv_cluster_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
      cudaSuccess) {
    cudaGetLastError();
    sz = 8;
  }
  if (sz == 16) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(16);
    cfg.blockDim = dim3(256);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 16;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, trsv_cluster_kernel, &cfg) != cudaSuccess ||
        nclusters < 1) {
      cudaGetLastError();
      sz = 8;
    }
  }
  return sz;
  });
}

cudaError_t trsv_lower(const double* L, int64_t ld, int nrow, double* x, int64_t ldx, int R,
                       bool trans, cudaStream_t s) {
  if (nrow <= 0) return cudaSuccess;
  if (R > 64) return cudaErrorInvalidValue;
  const int nt = (nrow + T - 1) / T;
  int csize = trsv_cluster_size(s);
  while (csize > 1 && csize > nt) csize /= 2;
  TimedLaunch tl(K_TRSV, 2.0 * nrow * nrow * R / 2, s);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(csize);
  cfg.blockDim = dim3(256);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = csize;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, trsv_cluster_kernel, L, ld, nrow, x, ldx, R, trans ? 1 : 0);
}

// Waits until the grid this launch depends on has completed and its writes are
// visible (programmatic dependent launch: the launch itself and the scheduling
// of its CTAs overlap the previous kernel's drain). A no-op for a normal launch.
__device__ __forceinline__ void grid_dependency_wait() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

// out[M][R] = beta * xin + alpha * A[M][K] y[K][R]: one warp per row, lanes over
// k, fixed-order shuffle reduction; R is processed 8 columns at a time. tri: A
// is lower triangular (row r reads k <= r only). out may alias xin.
__global__ void __launch_bounds__(256) gemv_n_kernel(const double* A, int64_t lda, int M, int K,
                                                     const double* y, int64_t ldy, double* x,
                                                     int64_t ldx, int R, double alpha, double beta,
                                                     const double* xin, int tri) {
  grid_dependency_wait();
  const int lane = threadIdx.x & 31;
  const int row = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (row >= M) return;
  const int kend = tri ? min(K, row + 1) : K;
  for (int r0 = 0; r0 < R; r0 += 8) {
    const int rc = min(8, R - r0);
    double acc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = 0.0;
    double acc2[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) acc2[q] = 0.0;
    // Two k-steps per pass with separate sums: twice the loads in flight and
    // half the dependent chain; the two sums are added in a fixed order.
    for (int k = lane; k < kend; k += 64) {
      const double av = A[(int64_t)row * lda + k];
      const bool two = k + 32 < kend;
      const double av2 = two ? A[(int64_t)row * lda + k + 32] : 0.0;
#pragma unroll
      for (int q = 0; q < 8; ++q)
        if (q < rc) {
          acc[q] = fma(av, y[(int64_t)k * ldy + r0 + q], acc[q]);
          if (two) acc2[q] = fma(av2, y[(int64_t)(k + 32) * ldy + r0 + q], acc2[q]);
        }
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      double v = acc[q] + acc2[q];
      for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
      acc[q] = v;
    }
    if (lane == 0)
      for (int q = 0; q < rc; ++q) {
        const double base = beta == 0.0 ? 0.0 : beta * xin[(int64_t)row * ldx + r0 + q];
        x[(int64_t)row * ldx + r0 + q] = base + alpha * acc[q];
      }
  }
}

// out[M][R] = beta * xin + alpha * A^T y with A stored K x M: 32 rows per CTA
// (lane = row), 8 warps split k and are summed in a fixed order. tri: A is lower
// triangular (output row m reads k >= m only).
__global__ void __launch_bounds__(256) gemv_t_kernel(const double* A, int64_t lda, int M, int K,
                                                     const double* y, int64_t ldy, double* x,
                                                     int64_t ldx, int R, double alpha, double beta,
                                                     const double* xin, int tri) {
  grid_dependency_wait();
  __shared__ double red[8][32][8];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int row = blockIdx.x * 32 + lane;
  const int kchunk = (K + 7) / 8, kb = w * kchunk, ke = min(K, kb + kchunk);
  const int kb_row = tri ? max(kb, row) : kb;
  for (int r0 = 0; r0 < R; r0 += 8) {
    const int rc = min(8, R - r0);
    double acc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = 0.0;
    if (row < M)
      for (int k = kb_row; k < ke; ++k) {
        const double av = A[(int64_t)k * lda + row];
#pragma unroll
        for (int q = 0; q < 8; ++q)
          if (q < rc) acc[q] += av * y[(int64_t)k * ldy + r0 + q];
      }
#pragma unroll
    for (int q = 0; q < 8; ++q) red[w][lane][q] = acc[q];
    __syncthreads();
    if (w == 0 && row < M) {
      for (int q = 0; q < rc; ++q) {
        double v = 0.0;
        for (int ww = 0; ww < 8; ++ww) v += red[ww][lane][q];
        const double base = beta == 0.0 ? 0.0 : beta * xin[(int64_t)row * ldx + r0 + q];
        x[(int64_t)row * ldx + r0 + q] = base + alpha * v;
      }
    }
    __syncthreads();
  }
}

// out[M][R] = beta * xin + alpha * A^T y (A stored K x M), R <= 8: a cluster of
// kGemvSplit CTAs per 32 output rows splits k; in each CTA 8 warps split its
// k-range (lane = row), the warps' sums are added in a fixed order in shared
// memory, and rank 0 adds the CTAs' sums in rank order from distributed shared
// memory. tri: A is lower triangular (output row m reads k >= m only).
constexpr int kGemvSplit = 4;

__global__ void __launch_bounds__(256) gemv_t_split_kernel(const double* A, int64_t lda, int M, int K,
                                                          const double* y, int64_t ldy, double* x,
                                                          int64_t ldx, int R, double alpha, double beta,
                                                          const double* xin, int tri) {
  grid_dependency_wait();
  __shared__ double red[8][32][8];
  __shared__ double part_sum[32][8];
  unsigned part;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(part));
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int row = (blockIdx.x / kGemvSplit) * 32 + lane;
  // Under a triangular A the k-range of this group of 32 rows starts at its first row.
  const int k0 = tri ? min(K, (blockIdx.x / kGemvSplit) * 32) : 0;
  const int kq = (K - k0 + kGemvSplit - 1) / kGemvSplit, kp0 = k0 + (int)part * kq, kp1 = min(K, kp0 + kq);
  const int kchunk = (kp1 - kp0 + 7) / 8, kb = kp0 + w * kchunk, ke = min(kp1, kb + kchunk);
  const int kb_row = tri ? max(kb, row) : kb;
  double acc[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) acc[q] = 0.0;
  if (row < M)
    for (int k = kb_row; k < ke; ++k) {
      const double av = A[(int64_t)k * lda + row];
#pragma unroll
      for (int q = 0; q < 8; ++q)
        if (q < R) acc[q] = fma(av, y[(int64_t)k * ldy + q], acc[q]);
    }
#pragma unroll
  for (int q = 0; q < 8; ++q) red[w][lane][q] = acc[q];
  __syncthreads();
  if (w == 0) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      double v = 0.0;
      for (int ww = 0; ww < 8; ++ww) v += red[ww][lane][q];
      part_sum[lane][q] = v;
    }
  }
  cluster_sync_all();
  if (part == 0 && w == 0 && row < M) {
    for (int q = 0; q < R; ++q) {
      double v = part_sum[lane][q];
      for (unsigned p = 1; p < kGemvSplit; ++p) v += ld_dsmem(&part_sum[lane][q], p);
      const double base = beta == 0.0 ? 0.0 : beta * xin[(int64_t)row * ldx + q];
      x[(int64_t)row * ldx + q] = base + alpha * v;
    }
  }
  cluster_sync_all();  // the partial sums stay readable until rank 0 is done
}

cudaError_t gemv_multi(const double* A, int64_t lda, int opA, int M, int K, const double* y,
                       int64_t ldy, double* x, int64_t ldx, int R, double alpha, cudaStream_t s,
                       double beta, const double* xin, int triA) {
  if (M <= 0 || R <= 0) return cudaSuccess;
  if (!xin) xin = x;
  const int tri = triA == TRI_LOWER ? 1 : 0;
  TimedLaunch tl(K_GEMV, 2.0 * M * K * R * (tri ? 0.5 : 1.0), s);
  // Programmatic dependent launch: consecutive products of a solve overlap
  // launch latency; each kernel waits for its predecessor before reading.
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(256);
  cfg.stream = s;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (opA == OP_N) {
    cfg.gridDim = dim3(ceil_div(M, 8));
    return cudaLaunchKernelEx(&cfg, gemv_n_kernel, A, lda, M, K, y, ldy, x, ldx, R, alpha, beta, xin, tri);
  }
  if (R <= 8 && K >= 8 * kGemvSplit) {
    cfg.gridDim = dim3(ceil_div(M, 32) * kGemvSplit);
    attr[1].id = cudaLaunchAttributeClusterDimension;
    attr[1].val.clusterDim.x = kGemvSplit;
    attr[1].val.clusterDim.y = 1;
    attr[1].val.clusterDim.z = 1;
    cfg.numAttrs = 2;
    return cudaLaunchKernelEx(&cfg, gemv_t_split_kernel, A, lda, M, K, y, ldy, x, ldx, R, alpha, beta,
                              xin, tri);
  }
  cfg.gridDim = dim3(ceil_div(M, 32));
  return cudaLaunchKernelEx(&cfg, gemv_t_kernel, A, lda, M, K, y, ldy, x, ldx, R, alpha, beta, xin, tri);
}

int arrow_chunks(int64_t n) { return (int)(n < 256 ? n : 256); }

// partial[chunk][p][r] = sum over blocks i of the chunk of arrow[i][p][:] . y_i[:][r]
__global__ void __launch_bounds__(256) arrow_gather_kernel(const double* arrow, int64_t n,
                                                           int64_t b, int64_t a,
                                                           const double* rhs, int R,
                                                           double* partial, int nchunks) {
  __shared__ double red[256];
  const int64_t per = (n + nchunks - 1) / nchunks;
  const int64_t i0 = blockIdx.x * per, i1 = min(n, i0 + per);
  for (int64_t p = 0; p < a; ++p)
    for (int r = 0; r < R; ++r) {
      double sum = 0.0;
      for (int64_t i = i0; i < i1; ++i)
        for (int64_t j = threadIdx.x; j < b; j += 256)
          sum += arrow[(i * a + p) * b + j] * rhs[(i * b + j) * R + r];
      red[threadIdx.x] = sum;
      __syncthreads();
      for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
      }
      if (threadIdx.x == 0) partial[((int64_t)blockIdx.x * a + p) * R + r] = red[0];
      __syncthreads();
    }
}

__global__ void arrow_gather_final_kernel(const double* partial, int nchunks, int64_t a, int R,
                                          double* rn) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= a * R) return;
  double s = 0.0;
  for (int c = 0; c < nchunks; ++c) s += partial[(int64_t)c * a * R + e];
  rn[e] -= s;
}

cudaError_t arrow_gather(const double* arrow, int64_t n, int64_t b, int64_t a, const double* rhs,
                         int R, double* partial, int nchunks, double* rn, cudaStream_t s) {
  if (a <= 0) return cudaSuccess;
  TimedLaunch tl(K_ARROW, 2.0 * n * a * b * R, s);
  arrow_gather_kernel<<<nchunks, 256, 0, s>>>(arrow, n, b, a, rhs, R, partial, nchunks);
  arrow_gather_final_kernel<<<ceil_div(a * R, 128), 128, 0, s>>>(partial, nchunks, a, R, rn);
  return cudaGetLastError();
}

// rhs[i*b + j][r] -= sum_p arrow[i][p][j] * xn[p][r]
__global__ void arrow_scatter_kernel(const double* arrow, int64_t n, int64_t b, int64_t a,
                                     const double* xn, int R, double* rhs) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * b) return;
  const int64_t i = e / b, j = e % b;
  for (int r = 0; r < R; ++r) {
    double acc = 0.0;
    for (int64_t p = 0; p < a; ++p) acc += arrow[(i * a + p) * b + j] * xn[p * R + r];
    rhs[e * R + r] -= acc;
  }
}

cudaError_t arrow_scatter(const double* arrow, int64_t n, int64_t b, int64_t a, const double* xn,
                          int R, double* rhs, cudaStream_t s) {
  if (a <= 0) return cudaSuccess;
  TimedLaunch tl(K_ARROW, 2.0 * n * a * b * R, s);
  arrow_scatter_kernel<<<ceil_div(n * b, 256), 256, 0, s>>>(arrow, n, b, a, xn, R, rhs);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Gradient assembly for alpha log det A + beta x^T A^{-1} x with respect to the
// stored blocks: G = alpha X - beta y y^T on the pattern, doubled on the
// off-diagonal (lower, arrow) blocks, which stand for themselves and their
// transposes; and with respect to x: 2 beta y.
// ---------------------------------------------------------------------------
__global__ void grad_blocks_kernel(int64_t n, int64_t b, int64_t a, const double* Xd,
                                   const double* Xl, const double* Xa, const double* Xt,
                                   const double* y, double alpha, double qbeta, double* Gd,
                                   double* Gl, double* Ga, double* Gt, double* gx) {
  const int64_t nd = n * b * b, nl = (n - 1) * b * b, na = n * a * b, nt = a * a;
  const int64_t total = nd + nl + na + nt;
  const double beta = -qbeta;
  if (gx)
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * b + a;
         e += (int64_t)gridDim.x * blockDim.x)
      gx[e] = 2.0 * qbeta * y[e];
  const double* yn = y + n * b;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    if (e < nd) {
      const int64_t i = e / (b * b), r = (e / b) % b, c = e % b;
      Gd[e] = alpha * Xd[e] + beta * y[i * b + r] * y[i * b + c];
    } else if (e < nd + nl) {
      const int64_t f = e - nd, i = f / (b * b), r = (f / b) % b, c = f % b;
      Gl[f] = 2.0 * (alpha * Xl[f] + beta * y[(i + 1) * b + r] * y[i * b + c]);
    } else if (e < nd + nl + na) {
      const int64_t f = e - nd - nl, i = f / (a * b), r = (f / b) % a, c = f % b;
      Ga[f] = 2.0 * (alpha * Xa[f] + beta * yn[r] * y[i * b + c]);
    } else {
      const int64_t f = e - nd - nl - na, r = f / a, c = f % a;
      Gt[f] = alpha * Xt[f] + beta * yn[r] * yn[c];
    }
  }
}

cudaError_t grad_blocks(int64_t n, int64_t b, int64_t a, const double* Xd, const double* Xl,
                        const double* Xa, const double* Xt, const double* y, double alpha,
                        double beta, double* Gd, double* Gl, double* Ga, double* Gt, double* gx,
                        cudaStream_t s) {
  grad_blocks_kernel<<<1216, 256, 0, s>>>(n, b, a, Xd, Xl, Xa, Xt, y, alpha, beta, Gd, Gl, Ga, Gt,
                                          gx);
  return cudaGetLastError();
}

// Deterministic dot product x^T y (per-CTA tree sums, then CTAs in order).
__global__ void __launch_bounds__(256) dot_partial_kernel(int64_t N, const double* x,
                                                          const double* y, double* partial) {
  __shared__ double red[256];
  double acc = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x; e < N; e += (int64_t)gridDim.x * 256)
    acc = fma(x[e], y[e], acc);
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void ordered_sum_kernel(const double* partial, int count, double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int z = 0; z < count; ++z) s += partial[z];
    *out = s;
  }
}

cudaError_t dot_f64(int64_t N, const double* x, const double* y, double* partial, double* out,
                    cudaStream_t s) {
  dot_partial_kernel<<<kDotCtas, 256, 0, s>>>(N, x, y, partial);
  ordered_sum_kernel<<<1, 32, 0, s>>>(partial, kDotCtas, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// FP64 peak probe: independent DMMA m8n8k4 chains on every SM (the denominator
// of the FP64 roofline, measured on the device that runs the path).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) fp64_probe_kernel(double* out, long long iters) {
  double a = threadIdx.x * 1e-3, b = 0.999;
  double c[4][2];
#pragma unroll
  for (int j = 0; j < 4; ++j) c[j][0] = c[j][1] = 0.0;
  for (long long it = 0; it < iters; ++it) {
#pragma unroll
    for (int j = 0; j < 4; ++j) dmma_8x8x4(c[j], a, b);
  }
  double r = 0.0;
#pragma unroll
  for (int j = 0; j < 4; ++j) r += c[j][0] + c[j][1];
  if (r == 1234.5678) out[0] = r;  // never true; keeps the loop live
}

cudaError_t fp64_probe(double* out, long long iters, double* flops, cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int blocks = 2 * sms, threads = 256;
  *flops = 512.0 * 4.0 * (double)iters * blocks * (threads / 32);
  TimedLaunch tl(K_PROBE, *flops, s);
  fp64_probe_kernel<<<blocks, threads, 0, s>>>(out, iters);
  return cudaGetLastError();
}

}  // namespace bta
