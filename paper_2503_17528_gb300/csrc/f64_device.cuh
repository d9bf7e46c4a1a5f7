// Device helpers shared by the FP64 kernels (kernels_f64.cu) and the persistent
// batched kernel (batch_persistent.cu): DMMA fragment product, pivot reciprocal
// square root, the shared-memory tile Cholesky and the panel solve.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

#include "bta_internal.cuh"

namespace bta {

// D(8x8) += A(8x4) B(4x8) in FP64 on the tensor pipe (m8n8k4, row.col): lane
// (g = lane / 4, t = lane % 4) holds A[g][t], B[t][g] and D[g][2t], D[g][2t+1].
__device__ __forceinline__ void dmma_8x8x4(double (&c)[2], double a, double b) {
  asm volatile(
      "mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, "
      "{%0,%1};\n"
      : "+d"(c[0]), "+d"(c[1])
      : "d"(a), "d"(b));
}

__device__ __forceinline__ double scale_by(double v, double alpha) {
  if (alpha == 1.0) return v;
  if (alpha == -1.0)
    return __longlong_as_double(__double_as_longlong(v) ^ (long long)0x8000000000000000ull);
  return alpha * v;
}

// 1/sqrt(d) for d > 0 by Newton-Raphson on f(y) = 1/y^2 - d (y <- y (3 - d y^2) / 2),
// seeded with the single-precision hardware estimate rsqrtf. Two steps take the
// ~2^-23 seed error below FP64 rounding. Every dependent FP64 instruction is
// expensive on this part, and this chain is about half the length of a
// correctly rounded sqrt followed by a division; the pivot is then d * y.
// A pivot outside the float range (binary exponent beyond +-100, or subnormal)
// is first written d = d' 4^k with d' near 1 (exact power-of-two scaling), the
// iteration runs on d', and y = y' 2^-k: an SPD matrix scaled by any power of
// two factors like the unscaled one. Inf or NaN pivots are not rescaled and
// come out NaN (0 * inf) in the pivot.
__device__ __forceinline__ double rsqrt_newton(double d) {
  const int e = (int)((__double_as_longlong(d) >> 52) & 0x7ff) - 1023;  // -1023: zero/subnormal
  const int k = (e > 100 || e < -100) && e != 1024 ? e / 2 : 0;          // |k| <= 511
  // 2^-2k and 2^-k as bit patterns: biased exponents 1023-2k in [1, 2045], 1023-k in [512, 1534].
  const double ds = k ? d * __longlong_as_double((long long)(1023 - 2 * k) << 52) : d;
  double y = (double)rsqrtf((float)ds);
  const double h = 0.5 * ds;
  y = y * fma(-h * y, y, 1.5);
  y = y * fma(-h * y, y, 1.5);
  return k ? y * __longlong_as_double((long long)(1023 - k) << 52) : y;
}

// Row of the lower-triangular index u (u = row (row + 1) / 2 + col, col <= row).
__device__ __forceinline__ int tri_row(int u) {
  int r = (int)((sqrtf(8.0f * (float)u + 1.0f) - 1.0f) * 0.5f);
  while ((r + 1) * (r + 2) / 2 <= u) ++r;
  while (r * (r + 1) / 2 > u) --r;
  return r;
}

// Pivot of a tile Cholesky: L_jj = d y with y = 1 / sqrt(d). A non-positive
// pivot is recorded in *info (the first one wins: LAPACK-style 1-based row) and
// poisons the rest with NaN.
__device__ __forceinline__ void pivot_of(double d, long long row, unsigned long long* info,
                                         double& Ljj, double& y) {
  if (!(d > 0.0)) {
    atomicCAS(info, 0ull, (unsigned long long)row);
    d = __longlong_as_double(0x7ff8000000000000ll);
  }
  y = rsqrt_newton(d);
  Ljj = d * y;
}

// Shared-memory Cholesky of a tb x tb tile in S (lower part valid); returns with
// S = L (zero above) and rd[j] = 1 / L_jj. Records a failed pivot in *info
// (row_base + 1 is the row of the tile's first pivot). Phase j applies pivot j
// to the trailing triangle from the unscaled column j (S_ic -= S_ij S_cj rd_j^2)
// and scales column j-1, while thread 0 finishes diagonal entry j+1 and computes
// the next pivot: the pivot chain runs one step ahead of the updates, one
// barrier per pivot. Needs more than one warp (the updates run on warps 1 and up).
static __device__ void coop_factor(double (*S)[T + 1], double* rd, int tb, long long row_base,
                                   unsigned long long* info) {
  const int tid = threadIdx.x, nthr = blockDim.x;
  if (tid == 0) {
    double L0, y0;
    pivot_of(S[0][0], row_base + 1, info, L0, y0);
    S[0][0] = L0;
    rd[0] = y0;
  }
  __syncthreads();
  for (int j = 0; j < tb; ++j) {
    const double r = rd[j];
    if (tid == 0) {
      if (j + 1 < tb) {
        const double sj = S[j + 1][j] * r;
        double L1, y1;
        pivot_of(fma(-sj, sj, S[j + 1][j + 1]), row_base + j + 2, info, L1, y1);
        S[j + 1][j + 1] = L1;
        rd[j + 1] = y1;
      }
    } else if (tid >= 32) {
      const double r2 = r * r;
      const int w = tb - j - 1, nel = w * (w + 1) / 2;
      for (int e = tid - 32; e < nel; e += nthr - 32) {
        const int rr = tri_row(e), cc = e - rr * (rr + 1) / 2;
        if (rr == 0) continue;  // (j+1, j+1): thread 0's
        const int i = j + 1 + rr, c = j + 1 + cc;
        S[i][c] = fma(-S[i][j] * S[c][j], r2, S[i][c]);
      }
    }
    if (j > 0) {  // column j-1 is no longer read: scale it
      const double rp = rd[j - 1];
      for (int i = j + tid; i < tb; i += nthr) S[i][j - 1] *= rp;
    }
    __syncthreads();
  }
  for (int e = tid; e < T * T; e += nthr) {
    const int i = e / T, c = e % T;
    if (c > i) S[i][c] = 0.0;
  }
  __syncthreads();
}

// Panel solve in shared memory: X (rows x tb) <- X L^{-T}, L lower in Lt,
// rdv = 1 / diag(L). Needs blockDim.x >= rows.
__device__ __forceinline__ void panel_solve(double (*X)[T + 1], const double (*Lt)[T + 1],
                                            const double* rdv, int rows, int tb) {
  const int tid = threadIdx.x;
  for (int j = 0; j < tb; ++j) {
    if (tid < rows) X[tid][j] *= rdv[j];
    __syncthreads();
    const int w = tb - j - 1;
    for (int e = tid; e < rows * w; e += blockDim.x) {
      const int i = e / w, c = j + 1 + e % w;
      X[i][c] -= X[i][j] * Lt[c][j];
    }
    __syncthreads();
  }
}

}  // namespace bta
