// Tensor-core GEMM for the BTA path on sm_103a: FP64 operands are split into
// BF16 slices and multiplied on the 5th-generation tensor cores (tcgen05,
// kind::f16, FP32 accumulation in TMEM), operands staged by TMA.
//
// Two splittings share one kernel:
//  * OZ (FP64-class): the error-free splitting of Ozaki et al. (2012). Every row
//    of op(A) (column of op(B)) gets a power-of-two scale 2^e with all entries
//    below 2^(e-1); the scaled value is rounded to a 7*s-bit integer Y and cut
//    into s balanced base-128 digits d_1..d_s (|d_1| <= 65, |d_p| <= 64), stored
//    as BF16 values d_p * 2^-7p (exact). Products of digit slices p, q (0-based)
//    are grouped by g = p + q, and pairs with g > s - 1 are dropped (triangular
//    truncation). Each group accumulates in its own FP32 TMEM accumulator over
//    k-units of at most 512: a group holds at most s pairs of digit products
//    |d d'| <= 65 * 64, so every partial sum is an integer multiple of 2^-7(g+2)
//    below 2^24 of them and exact whatever the accumulator's rounding. Each
//    k-unit's groups become one int64 fixed-point value (quantum 2^-49 of the
//    scales; the g = 6 group is rounded to it), and the units of a tile are
//    summed in integers: exact and independent of order. The FP64 output is then
//    assembled from the integer with integer operations (the scales are powers of
//    two), which keeps the epilogue off this part's narrow FP64 pipe.
//  * X3 (mixed precision): x = hi + lo with hi = bf16(x), lo = bf16(x - hi); the
//    products hi*hi (group 0) and hi*lo + lo*hi (group 1) accumulate in FP32 and
//    are added at the end.
//
// Slice p of op(A) against slices q0..q0+c-1 of op(B) is ONE tcgen05.mma with
// N = 64c (c <= 4): the B slices sit one after another in shared memory, and the
// accumulators of groups p+q0 .. p+q0+c-1 sit one after another in TMEM (group g
// at column 64g). Seven digit slices take 10 MMAs per 16-deep k step instead of
// 28, each reading its A slice once for up to 256 output columns.
//
// Tile: 128 x 64 outputs; k-blocks of 32 BF16 (64-byte rows, 64-byte swizzle),
// every slice of A and B for a k-block in one pipeline stage, loaded by two 3-D
// TMA copies (slices as the third dimension). Persistent, warp-specialized CTAs
// (one per SM): warp 8 issues TMA, warp 9 issues tcgen05.mma, warps 0-7 drain the
// accumulators (warp w reads TMEM lanes 32(w%4).. and columns 32(w/4)..). A work
// item is one output tile and a range of its k-units; when every tile holds all
// of its units the result is written directly, otherwise the items add int64
// partial tiles with atomics and a finalize kernel writes C. Every wait is
// bounded: on a timeout the kernel records an error, stops issuing, drains what
// it issued, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>

#include "bta_internal.cuh"
#include "kernels_tc.cuh"
#include "timing.cuh"

namespace bta {
namespace tc {

constexpr int BM = 128, BN = 64, BK = 32;
constexpr int kUnitK = 512;     // k per unit in OZ mode (exactness bound of the digit groups)
constexpr int kFixShift = 49;   // int64 fixed point: value = T * 2^-49 * scales
constexpr int kEpiWarps = 8;
constexpr int kThreads = (kEpiWarps + 2) * 32;  // + TMA warp + MMA warp
constexpr int kTmaWarp = kEpiWarps, kMmaWarp = kEpiWarps + 1;
constexpr uint32_t kSpinLimit = 1u << 22;  // polls of try_wait (each suspends ~us) before giving up
constexpr int kMaxStages = 4;

__device__ int g_tc_error;  // set on a bounded-wait timeout

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ uint32_t mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok;
}

// Bounded wait on an mbarrier phase; false (and the error word set) on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (uint32_t i = 0; i < kSpinLimit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  atomicExch(&g_tc_error, 1);
  return false;
}

// 3-D tiled TMA load (x = k, y = row, z = slice plane) completing on `bar`.
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
      : "memory");
}

// Shared-memory matrix descriptor: K-major tile, rows of 64 bytes, 64-byte
// swizzle, 8-row groups 512 bytes apart (descriptor version 1). Rows continue
// across slice boundaries (each slice is a whole number of 8-row groups), so one
// descriptor can span several consecutive slices.
__device__ __forceinline__ uint64_t sdesc_sw64(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;                     // leading byte offset (unused here)
  d |= (uint64_t)((512u >> 4) & 0x3FFFu) << 32;  // stride byte offset
  d |= (uint64_t)1 << 46;                     // version
  d |= (uint64_t)4 << 61;                     // swizzle 64B
  return d;
}

// Instruction descriptor: BF16 x BF16 -> FP32, both operands K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                          uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
        "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
        "=r"(r[31])
      : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Output addressing of a chunk of a (two-level) batch.
struct COut {
  double* C;
  int64_t ldc, s1, s2;
  int nb1, zbase;
};

__device__ __forceinline__ double* c_base(const COut& c, int zl) {
  const int z = c.zbase + zl;
  return c.C + (int64_t)(z % c.nb1) * c.s1 + (int64_t)(z / c.nb1) * c.s2;
}

// Exact FP32 -> FP64 with integer operations (normal numbers and zeros; the
// rare rest through the conversion instruction).
__device__ __forceinline__ double f32_to_f64(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t e = (u >> 23) & 0xffu;
  if (e == 0u || e == 255u) return (u & 0x7fffffffu) ? (double)f : __longlong_as_double((long long)(u >> 31) << 63);
  const unsigned long long bits = ((unsigned long long)(u >> 31) << 63) |
                                  ((unsigned long long)(e + 896u) << 52) |
                                  ((unsigned long long)(u & 0x7fffffu) << 29);
  return __longlong_as_double((long long)bits);
}

// v * 2^(s - 49), rounded to nearest even, for the int64 accumulator v, with
// integer operations; s is the sum of the power-of-two scales' exponents.
// Results outside the normal range take the FP64 path.
__device__ __forceinline__ double fix_to_f64(long long v, int s) {
  if (v == 0) return 0.0;
  const unsigned long long sign = v < 0 ? 1ull : 0ull;
  unsigned long long m = sign ? 0ull - (unsigned long long)v : (unsigned long long)v;
  int top = 63 - __clzll((long long)m);  // index of the leading one
  if (top > 52) {
    const int sh = top - 52;
    const unsigned long long rem = m & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
    m >>= sh;
    if (rem > half || (rem == half && (m & 1ull))) ++m;
    if (m >> 53) {
      m >>= 1;
      ++top;
    }
  } else {
    m <<= (52 - top);
  }
  const int biased = top - kFixShift + s + 1023;
  if (biased < 1 || biased > 2046) return ldexp((double)v, s - kFixShift);
  return __longlong_as_double((long long)((sign << 63) | ((unsigned long long)biased << 52) |
                                          (m & 0xfffffffffffffull)));
}

// Exponent of a power of two held as a double; returns false for anything else
// (NaN rows, zero scales, non-powers).
__device__ __forceinline__ bool pow2_exponent(double x, int& e) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int be = (int)((b >> 52) & 0x7ff);
  if ((b & 0xfffffffffffffull) || be == 0 || be == 2047 || (b >> 63)) return false;
  e = be - 1023;
  return true;
}

struct TcArgs {
  int M, N;           // logical output size
  int Kc;             // padded k extent of the slices (multiple of BK)
  int unitk;          // k per unit (multiple of BK)
  int nunits;         // units per tile
  int ups;            // units per work item
  int chunks;         // work items per tile (chunks == 1: direct write)
  int tilesN;         // tile columns
  int tiles_z;        // computed tiles per batch entry (lower tiles only if lowerC)
  long long items;    // nb * tiles_z * chunks
  long long* T;       // chunks > 1: [nb][Mpad][Npad] int64 accumulators (zeroed before)
  int s;              // slices per operand
  int gmax;           // largest group index kept (OZ: s - 1; X3: 1)
  int mode;           // TC_OZ or TC_X3
  int Mpad, Npad;     // padded rows of the A / B slice planes
  int nstages;
  int triA, triB;     // structure of op(A), op(B) (TRI_*), global k coordinates
  int lowerC;
  const double* sa;   // [nb][Mpad] row scales of A
  const double* sb;   // [nb][Npad] column scales of B
  COut co;
  double alpha, beta;
};

// Output tiles of a row of tiles (all, or those touching the lower triangle).
__device__ __forceinline__ int tiles_in_row(const TcArgs& g, int tm) {
  if (!g.lowerC) return g.tilesN;
  const int c = (tm * BM + BM - 1) / BN + 1;
  return c < g.tilesN ? c : g.tilesN;
}

// Work item -> batch entry z, tile (tm, tn), units [u0, u1).
__device__ __forceinline__ void decode_item(const TcArgs& g, long long item, int& z, int& tm, int& tn,
                                            int& u0, int& u1) {
  const int c = (int)(item % g.chunks);
  item /= g.chunks;
  int t = (int)(item % g.tiles_z);
  z = (int)(item / g.tiles_z);
  if (!g.lowerC) {
    tm = t / g.tilesN;
    tn = t % g.tilesN;
  } else {
    tm = 0;
    for (int w = tiles_in_row(g, 0); t >= w; w = tiles_in_row(g, ++tm)) t -= w;
    tn = t;
  }
  u0 = c * g.ups;
  u1 = min(g.nunits, u0 + g.ups);
}

// k-block range [kb, kb + nk*BK) of unit u of tile (tm, tn); structural zeros of
// triangular operands are skipped.
__device__ __forceinline__ int unit_kblocks(const TcArgs& g, int tm, int tn, int u, int& kb) {
  const int m0 = tm * BM, n0 = tn * BN;
  int gb = 0, ge = g.Kc;
  if (g.triA == TRI_LOWER) ge = min(ge, m0 + BM);
  if (g.triA == TRI_UPPER) gb = max(gb, m0);
  if (g.triB == TRI_LOWER) gb = max(gb, n0);
  if (g.triB == TRI_UPPER) ge = min(ge, n0 + BN);
  gb = gb / BK * BK;
  kb = max(gb, u * g.unitk);
  const int ke = min(ge, (u + 1) * g.unitk);
  return ke > kb ? (ke - kb + BK - 1) / BK : 0;
}

__global__ void __launch_bounds__(kThreads, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const TcArgs g) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[kMaxStages];
  __shared__ __align__(8) uint64_t empty_bar[kMaxStages];
  __shared__ __align__(8) uint64_t tfull_bar;   // accumulators ready (MMA commit)
  __shared__ __align__(8) uint64_t tempty_bar;  // accumulators drained (kEpiWarps arrivals)
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int s_abort;

  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int S = g.s, NS = g.nstages;
  const uint32_t a_bytes = BM * BK * 2, b_bytes = BN * BK * 2;
  const uint32_t stage_bytes = (uint32_t)S * (a_bytes + b_bytes);

  if (tid == 0) {
    for (int i = 0; i < NS; ++i) {
      mbar_init(&full_bar[i], 1);
      mbar_init(&empty_bar[i], 1);
    }
    mbar_init(&tfull_bar, 1);
    mbar_init(&tempty_bar, kEpiWarps);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;

  if (warp == kTmaWarp) {
    if (lane == 0) {
      // TMA producer: every k-block of every unit of this CTA's items, in order.
      long long it = 0;
      bool ok = true;
      for (long long item = blockIdx.x; item < g.items && ok; item += gridDim.x) {
        int z, tm, tn, u0, u1;
        decode_item(g, item, z, tm, tn, u0, u1);
        for (int u = u0; u < u1 && ok; ++u) {
          int kb;
          const int nk = unit_kblocks(g, tm, tn, u, kb);
          for (int kk = 0; kk < nk; ++kk, ++it) {
            const int st = (int)(it % NS);
            if (it >= NS && !mbar_wait(&empty_bar[st], (uint32_t)((it / NS) - 1) & 1u)) ok = false;
            if (!ok || s_abort) {
              ok = false;
              break;
            }
            mbar_arrive_expect_tx(&full_bar[st], stage_bytes);
            uint8_t* sbase = smem + (size_t)st * stage_bytes;
            const int kx = kb + kk * BK;
            tma_load_3d(sbase, &tmA, &full_bar[st], kx, tm * BM, z * S);
            tma_load_3d(sbase + S * a_bytes, &tmB, &full_bar[st], kx, tn * BN, z * S);
          }
        }
      }
      if (!ok) {
        s_abort = 1;
        // Drain the loads still in flight (at most NS stages) before leaving.
        for (long long j = it > NS ? it - NS : 0; j < it; ++j) mbar_wait(&full_bar[j % NS], (uint32_t)(j / NS) & 1u);
      }
    }
  } else if (warp == kMmaWarp) {
    if (lane == 0) {
      // MMA issuer.
      long long it = 0, tuse = 0;
      bool ok = true;
      for (long long item = blockIdx.x; item < g.items && ok; item += gridDim.x) {
        int z, tm, tn, u0, u1;
        decode_item(g, item, z, tm, tn, u0, u1);
        for (int u = u0; u < u1 && ok; ++u) {
          int kb;
          const int nk = unit_kblocks(g, tm, tn, u, kb);
          if (nk == 0) continue;
          // The epilogue must have drained the previous unit's accumulators.
          if (tuse > 0 && !mbar_wait(&tempty_bar, (uint32_t)(tuse - 1) & 1u)) ok = false;
          if (!ok || s_abort) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          for (int kk = 0; kk < nk; ++kk, ++it) {
            const int st = (int)(it % NS);
            if (!mbar_wait(&full_bar[st], (uint32_t)(it / NS) & 1u) || s_abort) {
              ok = false;
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t sbase = smem_u32(smem + (size_t)st * stage_bytes);
#pragma unroll
            for (int k16 = 0; k16 < BK / 16; ++k16) {
              for (int p = 0; p < S; ++p) {
                const int m = min(S, g.gmax + 1 - p);  // B slices q = 0 .. m-1 meet slice p
                const uint64_t adesc = sdesc_sw64(sbase + p * a_bytes + k16 * 32);
                for (int q0 = 0; q0 < m; q0 += 4) {
                  const int c = min(4, m - q0);
                  const uint32_t acc = (kk > 0 || k16 > 0 || p > 0) ? 1u : 0u;
                  umma_bf16(tmem + (uint32_t)((p + q0) * BN),
                            adesc, sdesc_sw64(sbase + S * a_bytes + q0 * b_bytes + k16 * 32),
                            idesc_bf16_f32(BM, c * BN), acc);
                }
              }
            }
            umma_commit(&empty_bar[st]);
          }
          if (!ok) break;
          umma_commit(&tfull_bar);
          ++tuse;
        }
      }
      if (!ok) {
        // Every MMA this CTA issued completes before its TMEM is freed: one more
        // commit, and a wait for the phase it completes.
        s_abort = 1;
        umma_commit(&tfull_bar);
        mbar_wait(&tfull_bar, (uint32_t)tuse & 1u);
      }
    }
  } else {
    // Epilogue warps: rows m0 + 32 (warp % 4) + lane, columns n0 + 32 (warp / 4) + j.
    const int quarter = warp & 3, half = warp >> 2;
    const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(half * 32);
    long long tuse = 0;
    bool ok = true;
    for (long long item = blockIdx.x; item < g.items && ok; item += gridDim.x) {
      int z, tm, tn, u0, u1;
      decode_item(g, item, z, tm, tn, u0, u1);
      const int row = tm * BM + quarter * 32 + lane;
      const int col0 = tn * BN + half * 32;
      long long acc[32];
      float accf[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        acc[j] = 0;
        accf[j] = 0.f;
      }
      for (int u = u0; u < u1; ++u) {
        int kb;
        if (unit_kblocks(g, tm, tn, u, kb) == 0) continue;
        if (!mbar_wait(&tfull_bar, (uint32_t)tuse & 1u) || s_abort) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (g.mode == TC_OZ) {
          for (int gi = 0; gi <= g.gmax; ++gi) {
            uint32_t r[32];
            tmem_ld32(lane_base + (uint32_t)(gi * BN), r);
            tmem_wait_ld();
            if (gi <= 5) {
              // exact group: v 2^(7(gi+2)) is an integer below 2^24
              const float up = __int_as_float((127 + 7 * (gi + 2)) << 23);
              const int sh = kFixShift - 7 * (gi + 2);
#pragma unroll
              for (int j = 0; j < 32; ++j)
                acc[j] += (long long)__float2int_rn(__uint_as_float(r[j]) * up) << sh;
            } else {
              // the g = 6 group: rounded to the 2^-49 quantum
              const float up = __int_as_float((127 + kFixShift) << 23);
#pragma unroll
              for (int j = 0; j < 32; ++j) acc[j] += (long long)__float2int_rn(__uint_as_float(r[j]) * up);
            }
          }
        } else {
          uint32_t r0[32], r1[32];
          tmem_ld32(lane_base, r0);
          tmem_ld32(lane_base + (uint32_t)BN, r1);
          tmem_wait_ld();
#pragma unroll
          for (int j = 0; j < 32; ++j) accf[j] += __uint_as_float(r0[j]) + __uint_as_float(r1[j]);
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty_bar);
        ++tuse;
      }
      if (!ok) break;
      if (row >= g.M) continue;
      if (g.chunks > 1) {
        long long* Tz = g.T + ((int64_t)z * g.Mpad + row) * g.Npad + col0;
#pragma unroll
        for (int j = 0; j < 32; ++j)
          if (acc[j]) atomicAdd((unsigned long long*)(Tz + j), (unsigned long long)acc[j]);
        continue;
      }
      // Direct write: C = alpha * result + beta * C on the defined elements.
      double* Cz = c_base(g.co, z) + (int64_t)row * g.co.ldc;
      int ea = 0, eb = 0;
      const bool fastA = g.mode == TC_OZ ? pow2_exponent(g.sa[(int64_t)z * g.Mpad + row], ea) : true;
      const bool neg = g.alpha == -1.0;
      const bool unit_alpha = g.alpha == 1.0 || neg;
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int col = col0 + j;
        if (col >= g.N) break;
        double v;
        if (g.mode == TC_OZ) {
          const double sbj = g.sb[(int64_t)z * g.Npad + col];
          if (fastA && pow2_exponent(sbj, eb)) {
            v = fix_to_f64(acc[j], ea + eb);
          } else {
            v = ((double)acc[j] * (1.0 / (double)(1ll << kFixShift))) * g.sa[(int64_t)z * g.Mpad + row] * sbj;
          }
        } else {
          v = f32_to_f64(accf[j]);
        }
        if (unit_alpha) {
          if (neg) v = __longlong_as_double(__double_as_longlong(v) ^ (long long)0x8000000000000000ull);
        } else {
          v *= g.alpha;
        }
        double* p = Cz + col;
        if (g.beta == 1.0) v += *p;
        else if (g.beta != 0.0) v += g.beta * *p;
        *p = v;
      }
    }
    if (!ok) s_abort = 1;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512)
                 : "memory");
  }
}

// ---------------------------------------------------------------------------
// Splitting kernels. The logical operand X is R x Kc (rows reduced over k):
// element (r, k) of batch z is X[z*sz + r*sr + (k0 + k)*sk].
// ---------------------------------------------------------------------------
struct SplitArgs {
  const double* X;      // part base
  int64_t sr, sk;       // element (r, k) of a batch entry at X[r*sr + k*sk]
  int64_t s1, s2;       // batch strides: entry z -> (z % nb1) * s1 + (z / nb1) * s2
  int nb1, zbase;       // flattened batch decomposition; first entry of this chunk
  int R, Kc;            // rows, k extent of this part
  int kout0, Kp;        // first output column of the part, padded row length of the slices
  int Rpad, s, mode, nb;
  int mask;             // structural zeros: 0 none, 1 where k > r, 2 where k < r
  __nv_bfloat16* out;   // [nb][s][Rpad][Kp]
  double* scale;        // [nb][Rpad]
  unsigned long long* rowmax;  // [nb][Rpad], |x| bit patterns, zeroed before the first part
};

__device__ __forceinline__ bool masked(const SplitArgs& a, int r, int k) {
  return (a.mask == 1 && k > r) || (a.mask == 2 && k < r);
}

__device__ __forceinline__ const double* part_base(const SplitArgs& a, int zl) {
  const int z = a.zbase + zl;
  return a.X + (int64_t)(z % a.nb1) * a.s1 + (int64_t)(z / a.nb1) * a.s2;
}

// One operand side (op(A) rows m, or op(B)^T rows n): up to two parts along k.
struct SplitOp {
  SplitArgs part[kMaxTerms];
  int nparts;
};

__device__ __forceinline__ double load_el(const SplitArgs& a, const double* X, int r, int k) {
  return (r < a.R && k < a.Kc && !masked(a, r, k)) ? X[(int64_t)r * a.sr + (int64_t)k * a.sk] : 0.0;
}

// Digits of one value (OZ) with the row's max bit pattern mb; returns the s slice values.
__device__ __forceinline__ void oz_digits(double x, unsigned long long mb, int s, float* dig) {
  const int emax = (int)(mb >> 52);  // biased exponent of the row max
  const long long bits = __double_as_longlong(x);
  const int ex = (int)((bits >> 52) & 0x7ff);
  long long Y = 0;
  if (emax > 0 && emax < 2047 && ex > 0) {
    // |x| = M 2^(ex-1075); row scale 2^e with e = emax - 1021 puts |x| 2^-e below 1/2;
    // Y = round(|x| 2^(7s - e)) = round(M 2^sh), sh <= 7s - 54 < 0.
    const long long M = (bits & 0x000fffffffffffffll) | 0x0010000000000000ll;
    const int e = emax - 1021;
    const int sh = ex - 1075 + 7 * s - e;
    if (sh >= 0) Y = M << sh;
    else if (sh > -64) Y = (M + (1ll << (-sh - 1))) >> (-sh);
    if (bits < 0) Y = -Y;
  }
  // Balanced base-128 digits, least significant first: d_s ... d_2 in [-64, 63], d_1 the rest.
  // (the digits fit in 32 bits: converting from int keeps the 64-bit integer
  // conversion, which issues on this part's narrow FP64 pipe, out of the loop)
  for (int p = s - 1; p >= 1; --p) {
    const long long d = ((Y + 64) & 127) - 64;
    dig[p] = (float)(int)d;
    Y = (Y - d) >> 7;
  }
  dig[0] = (float)(int)Y;
}

// Part of `op` holding concatenated column k (parts start on 32-column boundaries).
__device__ __forceinline__ int part_of(const SplitOp& op, int k) {
  int pi = 0;
  while (pi + 1 < op.nparts && k >= op.part[pi + 1].kout0) ++pi;
  return pi;
}

// Row maxima of |x| over the concatenated k range, both operands in one launch:
// blockIdx.z = 2 * batch entry + side; each CTA reduces 32 rows over a
// kRowmaxSlab-wide slab and merges with atomicMax (FP64 bit patterns order |x|).
constexpr int kRowmaxSlab = 64;
__global__ void __launch_bounds__(256) split_rowmax_kernel(SplitOp sa_op, SplitOp sb_op,
                                                           unsigned long long* rmA,
                                                           unsigned long long* rmB, int nsides) {
  const int side = nsides == 2 ? (int)(blockIdx.z & 1) : 0;
  const int zl = nsides == 2 ? (int)(blockIdx.z >> 1) : (int)blockIdx.z;
  const SplitOp& op = side == 0 ? sa_op : sb_op;
  unsigned long long* rm = side == 0 ? rmA : rmB;
  const SplitArgs& a0 = op.part[0];
  const int r0 = blockIdx.y * 32, k0 = blockIdx.x * kRowmaxSlab;
  if (r0 >= a0.Rpad || k0 >= a0.Kp) return;
  __shared__ unsigned long long red[8][32];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  unsigned long long m = 0;
  for (int pi = 0; pi < op.nparts; ++pi) {
    const SplitArgs& a = op.part[pi];
    const int lo = max(k0, a.kout0), hi = min(k0 + kRowmaxSlab, a.kout0 + a.Kc);
    if (lo >= hi) continue;
    const double* X = part_base(a, zl);
    if (a.sk == 1) {
      for (int rr = w; rr < 32; rr += 8) {
        const int r = r0 + rr;
        unsigned long long mr = 0;
        for (int kc = lo + lane; kc < hi; kc += 32) {
          const unsigned long long v =
              (unsigned long long)__double_as_longlong(load_el(a, X, r, kc - a.kout0)) & 0x7fffffffffffffffull;
          mr = v > mr ? v : mr;
        }
        for (int off = 16; off > 0; off >>= 1) {
          const unsigned long long o = __shfl_xor_sync(0xffffffffu, mr, off);
          mr = o > mr ? o : mr;
        }
        if (lane == 0 && mr) atomicMax(&rm[(int64_t)zl * a0.Rpad + r], mr);
      }
    } else {
      const int r = r0 + lane;
      for (int kc = lo + w; kc < hi; kc += 8) {
        const unsigned long long v =
            (unsigned long long)__double_as_longlong(load_el(a, X, r, kc - a.kout0)) & 0x7fffffffffffffffull;
        m = v > m ? v : m;
      }
    }
  }
  red[w][lane] = m;
  __syncthreads();
  if (w == 0) {
    for (int ww = 1; ww < 8; ++ww) m = red[ww][lane] > m ? red[ww][lane] : m;
    if (m) atomicMax(&rm[(int64_t)zl * a0.Rpad + r0 + lane], m);
  }
}

// Slices of one 32 x 32 tile of the concatenated operand (blockIdx.z = 2 * batch
// entry + side, or the batch entry when only side A is split), plus the row
// scales (first column of tiles) and, for side A, the zeroing of the int64
// accumulator rows.
__global__ void __launch_bounds__(256) split_digits_kernel(SplitOp sa_op, SplitOp sb_op,
                                                           const unsigned long long* rmA,
                                                           const unsigned long long* rmB,
                                                           long long* T, int Tcols, int nsides) {
  const int side = nsides == 2 ? (int)(blockIdx.z & 1) : 0;
  const int zl = nsides == 2 ? (int)(blockIdx.z >> 1) : (int)blockIdx.z;
  const SplitOp& op = side == 0 ? sa_op : sb_op;
  const unsigned long long* rm = side == 0 ? rmA : rmB;
  const SplitArgs& a0 = op.part[0];
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  if (r0 >= a0.Rpad || c0 >= a0.Kp) return;
  __shared__ double tile[32][33];
  __shared__ unsigned long long rmax[32];
  const int tid = threadIdx.x;
  const int pi = part_of(op, c0);
  const SplitArgs& a = op.part[pi];
  const double* X = part_base(a, zl);
  const int kc0 = c0 - a.kout0;  // column within the part
  if (tid < 32) rmax[tid] = a0.mode == TC_OZ ? rm[(int64_t)zl * a0.Rpad + r0 + tid] : 0ull;
  for (int e = tid; e < 1024; e += 256) {
    int i, j;
    if (a.sk == 1) { i = e / 32; j = e % 32; } else { j = e / 32; i = e % 32; }
    tile[i][j] = load_el(a, X, r0 + i, kc0 + j);
  }
  __syncthreads();
  const int64_t plane = (int64_t)a0.Rpad * a0.Kp;
  for (int e = tid; e < 1024; e += 256) {
    const int i = e / 32, j = e % 32;
    __nv_bfloat16* o = a0.out + (((int64_t)zl * a0.s) * a0.Rpad + r0 + i) * a0.Kp + c0 + j;
    const double x = tile[i][j];
    if (a0.mode == TC_X3) {
      const float xf = (float)x;
      const __nv_bfloat16 hi = __float2bfloat16_rn(xf);
      o[0] = hi;
      o[plane] = __float2bfloat16_rn(xf - __bfloat162float(hi));
      continue;
    }
    float dig[8];
    oz_digits(x, rmax[i], a0.s, dig);
    float sc = 1.0f / 128.0f;
    for (int p = 0; p < a0.s; ++p) {
      o[p * plane] = __float2bfloat16_rn(dig[p] * sc);  // exact: |d| <= 65, power-of-two scale
      sc *= 1.0f / 128.0f;
    }
  }
  if (blockIdx.x == 0) {
    if (tid < 32) {
      const int r = r0 + tid;
      double sc = 1.0;
      if (a0.mode == TC_OZ && r < a0.R) {
        const int emax = (int)(rmax[tid] >> 52);
        if (emax == 2047) sc = __longlong_as_double(0x7ff8000000000000ll);  // NaN/Inf row
        else if (emax > 0) sc = ldexp(1.0, emax - 1021);
      }
      a0.scale[(int64_t)zl * a0.Rpad + r] = sc;
    }
    if (side == 0 && T) {
      long long* Tz = T + ((int64_t)zl * a0.Rpad + r0) * Tcols;
      for (int64_t e = tid; e < (int64_t)32 * Tcols; e += 256) Tz[e] = 0;
    }
  }
}


// C = alpha * T 2^-49 sa_i sb_j + beta * C for tiles split over several work
// items (their int64 partial tiles summed in T), on the elements the GEMM defines.
__global__ void __launch_bounds__(256) tc_finalize_kernel(const long long* T, int M, int N, int Mpad,
                                                          int Npad, const double* sa,
                                                          const double* sb, COut co, double alpha,
                                                          double beta, int lowerC) {
  const int zl = blockIdx.y;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)M * N) return;
  const int i = (int)(e / N), j = (int)(e % N);
  if (lowerC && (j / BN) * BN > (i / BM) * BM + BM - 1) return;
  const long long t = T[((int64_t)zl * Mpad + i) * Npad + j];
  const double si = sa[(int64_t)zl * Mpad + i], sj = sb[(int64_t)zl * Npad + j];
  int ea, eb;
  double out;
  if (pow2_exponent(si, ea) && pow2_exponent(sj, eb)) out = fix_to_f64(t, ea + eb);
  else out = ((double)t * (1.0 / (double)(1ll << kFixShift))) * si * sj;
  if (alpha == -1.0) out = __longlong_as_double(__double_as_longlong(out) ^ (long long)0x8000000000000000ull);
  else if (alpha != 1.0) out *= alpha;
  double* p = c_base(co, zl) + (int64_t)i * co.ldc + j;
  if (beta == 1.0) out += *p;
  else if (beta != 0.0) out += beta * *p;
  *p = out;
}

}  // namespace tc

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
using namespace tc;

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static std::atomic<EncodeTiledFn> fn{nullptr};
  EncodeTiledFn f = fn.load();
  if (!f) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess) {
      f = (EncodeTiledFn)p;
      fn.store(f);
    }
  }
  return f;
}

// 3-D map over `planes` slice planes of `rows` x kp BF16 (row-major, kp
// contiguous); one box is BK x box_rows x slices (every slice of one row block
// for one k-block).
static bool make_map(CUtensorMap* m, void* base, uint64_t planes, uint64_t rows, uint64_t kp,
                     int box_rows, int slices) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  const cuuint64_t dims[3] = {kp, rows, planes};
  const cuuint64_t strides[2] = {kp * 2, rows * kp * 2};
  const cuuint32_t box[3] = {(cuuint32_t)BK, (cuuint32_t)box_rows, (cuuint32_t)slices};
  const cuuint32_t estr[3] = {1, 1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

static inline int64_t rup(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

int tc_slices(int mode) { return mode == TC_X3 ? 2 : kOzSlices; }

// Bytes of scratch one chunk of `nb` batch entries needs (k extent K).
// Workspace of one chunk, in this order: op(B)'s slices, scales and row maxima
// (at offsets that depend on N, K and the batch only, so that a later call with
// another M can reuse them), then op(A)'s, then the int64 accumulators.
static size_t tc_side_bytes(int64_t rows_pad, int64_t Kp, int64_t s, int64_t nb) {
  return rup(rows_pad * Kp * s * 2 * nb, 256) + 2 * rup(rows_pad * 8 * nb, 256);
}

static size_t tc_chunk_bytes(int mode, int M, int N, int K, int nb) {
  const int64_t s = tc_slices(mode);
  const int64_t Mp = rup(M, BM), Np = rup(N, BN), Kp = rup(K, BK);
  size_t b = tc_side_bytes(Np, Kp, s, nb) + tc_side_bytes(Mp, Kp, s, nb);
  if (mode == TC_OZ) b += rup(Mp * Np * 8 * nb, 256);  // int64 accumulators (split tiles)
  return b;
}

static int tc_batch_chunk(int M, int N, int K) {
  // Keep one chunk's slice planes and accumulators near 512 MB.
  const int64_t per = (rup(M, BM) + rup(N, BN)) * rup(K, BK) * kOzSlices * 2 + rup(M, BM) * rup(N, BN) * 8;
  int64_t nb = (512ll << 20) / (per > 0 ? per : 1);
  return (int)(nb < 1 ? 1 : (nb > 64 ? 64 : nb));
}

size_t tc_workspace_bytes(int mode, int M, int N, int K, int batch) {
  const int c = tc_batch_chunk(M, N, K);
  return tc_chunk_bytes(mode, M, N, K, batch < c ? batch : c);
}

// One operand part along k: element (r, k) at X[r*sr + k*sk] plus batch offsets.
struct Part {
  const double* X;
  int64_t sr, sk, s1, s2;
  int K;
  int mask;  // see SplitArgs::mask
};

static void fill_op(SplitOp* op, const Part* parts, int np, int nb1, int zbase, int R, int Kp,
                    int Rpad, int s, int mode, int nb, __nv_bfloat16* out, double* scale) {
  op->nparts = np;
  int k0 = 0;
  for (int i = 0; i < np; ++i) {
    SplitArgs& a = op->part[i];
    a = SplitArgs{};
    a.X = parts[i].X; a.sr = parts[i].sr; a.sk = parts[i].sk;
    a.s1 = parts[i].s1; a.s2 = parts[i].s2; a.nb1 = nb1; a.zbase = zbase;
    a.R = R; a.Kc = parts[i].K; a.kout0 = k0; a.Kp = Kp;
    a.Rpad = Rpad; a.s = s; a.mode = mode; a.nb = nb;
    a.out = out; a.scale = scale; a.rowmax = nullptr; a.mask = parts[i].mask;
    k0 += (int)rup(parts[i].K, BK);
  }
}

// Dynamic shared memory limit of the GEMM kernel (set on the kernel) and the SM
// count, per device; -1 if a query failed.
static PerDevice g_tc_dyn_limit, g_tc_sms;

static bool same_part(const Part& x, const Part& y) {
  return x.X == y.X && x.sr == y.sr && x.sk == y.sk && x.s1 == y.s1 && x.s2 == y.s2 && x.K == y.K &&
         x.mask == y.mask;
}

cudaError_t gemm_tc(const GemmArgs& g, int mode, void* ws, size_t ws_bytes, cudaStream_t s,
                    bool reuse_b) {
  if (g.nterms < 1 || g.nterms > kMaxTerms) return cudaErrorInvalidValue;
  // Several terms are one product over the concatenated k range when they share
  // alpha and no operand is triangular; otherwise they run one after the other.
  bool concat = g.nterms > 1;
  for (int i = 0; i < g.nterms && concat; ++i)
    concat = g.t[i].alpha == g.t[0].alpha && g.t[i].triA == TRI_NONE && g.t[i].triB == TRI_NONE;
  if (g.nterms > 1 && !concat) {
    for (int i = 0; i < g.nterms; ++i) {
      GemmArgs gi = g;
      gi.t[0] = g.t[i];
      gi.nterms = 1;
      if (i > 0) gi.beta = 1.0;
      cudaError_t e = gemm_tc(gi, mode, ws, ws_bytes, s, false);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  const int S = tc_slices(mode);
  const int M = g.M, N = g.N;
  if (M <= 0 || N <= 0) return cudaSuccess;
  Part pa[kMaxTerms], pb[kMaxTerms];
  int Kp = 0;
  for (int i = 0; i < g.nterms; ++i) {
    const GemmTerm& t = g.t[i];
    // op(A) element (m, k); op(B)^T element (n, k)
    // Structural zeros are applied while splitting: triangular operands may hold
    // anything in their zero parts. op(A) row m: LOWER -> k > m, UPPER -> k < m;
    // op(B)^T row n: LOWER (zero for k < n), UPPER (zero for k > n).
    const int ma = t.triA == TRI_LOWER ? 1 : (t.triA == TRI_UPPER ? 2 : 0);
    const int mb = t.triB == TRI_LOWER ? 2 : (t.triB == TRI_UPPER ? 1 : 0);
    pa[i] = Part{t.A, t.opA == OP_N ? t.lda : 1, t.opA == OP_N ? 1 : t.lda, t.sA1, t.sA2, t.K, ma};
    pb[i] = Part{t.B, t.opB == OP_N ? 1 : t.ldb, t.opB == OP_N ? t.ldb : 1, t.sB1, t.sB2, t.K, mb};
    Kp += (int)rup(t.K, BK);
  }
  if (Kp <= 0) return cudaSuccess;
  if (Kp > 16384) return cudaErrorInvalidValue;  // int64 accumulator headroom
  const int Mp = (int)rup(M, BM), Np = (int)rup(N, BN);
  const int total = g.nb1 * g.nb2;
  // A product of an operand with its own transpose (a SYRK, L^-T L^-1) splits it
  // once: op(B)^T has the rows, scales and slices of op(A).
  const bool self = g.nterms == 1 && M == N && Mp == Np && same_part(pa[0], pb[0]);
  // Batch entries per pass: as many as the design size and the workspace allow.
  int chunk_nb = tc_batch_chunk(M, N, Kp);
  if (chunk_nb > total) chunk_nb = total;
  while (chunk_nb > 1 && tc_chunk_bytes(mode, M, N, Kp, chunk_nb) > ws_bytes) --chunk_nb;
  if (tc_chunk_bytes(mode, M, N, Kp, chunk_nb) > ws_bytes) return cudaErrorInvalidValue;
  // The caller's previous call left this call's op(B) split in the workspace
  // (op(B)'s part of it sits at the start whatever M is): only valid for one
  // chunk holding the whole batch.
  if (reuse_b && (chunk_nb != total || self)) reuse_b = false;
  const long long dyn_limit = per_device(g_tc_dyn_limit, []() -> long long {
    int dev = 0, optin = 0;
    cudaFuncAttributes fa;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaFuncGetAttributes(&fa, tc_gemm_kernel) != cudaSuccess)
      return -1;
    const long long lim = (long long)optin - (long long)fa.sharedSizeBytes;
    if (lim <= 0 || cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)lim) != cudaSuccess)
      return -1;
    return lim;
  });
  const long long sms = per_device(g_tc_sms, []() -> long long {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1)
      return -1;
    return n;
  });
  if (dyn_limit < 0 || sms < 0) return cudaErrorInvalidConfiguration;
  const uint32_t stage_bytes = (uint32_t)S * (BM + BN) * BK * 2;
  int nstages = (int)((dyn_limit - 1024) / stage_bytes);
  if (nstages > kMaxStages) nstages = kMaxStages;
  if (nstages < 1) return cudaErrorInvalidValue;
  const size_t smem = (size_t)nstages * stage_bytes + 1024;
  const int unitk = mode == TC_OZ ? kUnitK : Kp;
  const int nunits = (Kp + unitk - 1) / unitk;
  const GemmTerm& t0 = g.t[0];
  // Output tiles per batch entry (only those touching the lower triangle for lowerC).
  const int tilesM = Mp / BM, tilesN = Np / BN;
  long long tiles_z = 0;
  for (int tm = 0; tm < tilesM; ++tm) {
    const int c = g.lowerC ? std::min(tilesN, (tm * BM + BM - 1) / BN + 1) : tilesN;
    tiles_z += c;
  }

  for (int c0 = 0; c0 < total; c0 += chunk_nb) {
    const int nb = total - c0 < chunk_nb ? total - c0 : chunk_nb;
    // Work items: whole tiles when they fill every SM at least once; otherwise
    // each tile's units are split over `chunks` items that add int64 partials.
    const long long tiles = tiles_z * nb;
    int chunks = 1;
    if (nunits > 1 && tiles < sms) {
      chunks = (int)std::min<long long>(nunits, (2 * sms + tiles - 1) / tiles);
    }
    const int ups = (nunits + chunks - 1) / chunks;
    chunks = (nunits + ups - 1) / ups;
    char* w = (char*)ws;
    __nv_bfloat16* Bs = (__nv_bfloat16*)w;
    w += rup((int64_t)Np * Kp * S * 2 * nb, 256);
    double* sb = (double*)w;
    w += rup((int64_t)Np * 8 * nb, 256);
    unsigned long long* rmB = (unsigned long long*)w;
    w += rup((int64_t)Np * 8 * nb, 256);
    __nv_bfloat16* As = (__nv_bfloat16*)w;
    w += rup((int64_t)Mp * Kp * S * 2 * nb, 256);
    double* sa = (double*)w;
    w += rup((int64_t)Mp * 8 * nb, 256);
    unsigned long long* rmA = (unsigned long long*)w;
    w += rup((int64_t)Mp * 8 * nb, 256);
    long long* Tacc = (long long*)w;
    // A self-product splits its operand once, into op(B)'s place, and reads op(A)
    // from there too.
    if (self) {
      As = Bs;
      sa = sb;
      rmA = rmB;
    }
    SplitOp opA, opB;
    fill_op(&opA, pa, g.nterms, g.nb1, c0, M, Kp, Mp, S, mode, nb, As, sa);
    fill_op(&opB, pb, g.nterms, g.nb1, c0, N, Kp, Np, S, mode, nb, Bs, sb);
    cudaError_t e;
    {
      TimedLaunch tl(K_TC_SPLIT, 0.0, s);
      const int nsides = (self || reuse_b) ? 1 : 2;
      const int bands = (nsides == 1 ? Mp : (Mp > Np ? Mp : Np)) / 32;
      if (mode == TC_OZ) {
        e = cudaMemsetAsync(rmA, 0, (size_t)Mp * nb * 8, s);
        if (e == cudaSuccess && nsides == 2) e = cudaMemsetAsync(rmB, 0, (size_t)Np * nb * 8, s);
        if (e != cudaSuccess) return e;
        split_rowmax_kernel<<<dim3((Kp + kRowmaxSlab - 1) / kRowmaxSlab, bands, nsides * nb), 256, 0, s>>>(
            opA, opB, rmA, rmB, nsides);
      }
      split_digits_kernel<<<dim3(Kp / 32, bands, nsides * nb), 256, 0, s>>>(
          opA, opB, rmA, rmB, (mode == TC_OZ && chunks > 1) ? Tacc : nullptr, Np, nsides);
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
    CUtensorMap mA, mB;
    if (!make_map(&mA, As, (uint64_t)nb * S, (uint64_t)Mp, (uint64_t)Kp, BM, S) ||
        !make_map(&mB, Bs, (uint64_t)nb * S, (uint64_t)Np, (uint64_t)Kp, BN, S))
      return cudaErrorInvalidValue;
    TcArgs a{};
    a.M = M; a.N = N; a.Kc = Kp; a.unitk = unitk; a.nunits = nunits; a.ups = ups; a.chunks = chunks;
    a.tilesN = tilesN; a.tiles_z = (int)tiles_z; a.items = tiles * chunks;
    a.T = Tacc; a.s = S; a.gmax = mode == TC_OZ ? S - 1 : 1; a.mode = mode;
    a.Mpad = Mp; a.Npad = Np; a.nstages = nstages; a.lowerC = g.lowerC;
    a.triA = g.nterms == 1 ? t0.triA : TRI_NONE;
    a.triB = g.nterms == 1 ? t0.triB : TRI_NONE;
    a.sa = sa; a.sb = sb;
    a.co = COut{g.C, g.ldc, g.sC1, g.sC2, g.nb1, c0};
    a.alpha = t0.alpha; a.beta = g.beta;
    const long long grid = std::min<long long>(a.items, sms);
    {
      // algorithmic flops of this chunk's nb batch entries
      const double fl = timing_on() ? gemm_alg_flops(g) / total * nb : 0.0;
      TimedLaunch tl(K_GEMM_TC, fl, s);
      tc_gemm_kernel<<<(unsigned)grid, kThreads, smem, s>>>(mA, mB, a);
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
    if (mode == TC_OZ && chunks > 1) {
      const int64_t elems = (int64_t)M * N;
      TimedLaunch tl(K_TC_FINAL, 0.0, s);
      tc_finalize_kernel<<<dim3((unsigned)((elems + 255) / 256), nb), 256, 0, s>>>(
          Tacc, M, N, Mp, Np, a.sa, a.sb, a.co, t0.alpha, g.beta, g.lowerC);
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

cudaError_t tc_error_read_reset(int* out) {
  int v = 0;
  cudaError_t e = cudaMemcpyFromSymbol(&v, g_tc_error, sizeof(int));
  if (e != cudaSuccess) return e;
  *out = v;
  const int zero = 0;
  return cudaMemcpyToSymbol(g_tc_error, &zero, sizeof(int));
}

}  // namespace bta
