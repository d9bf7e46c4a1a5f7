// Opt-in per-kernel timing: when enabled, every kernel launch of the library
// is bracketed by CUDA events on its stream, with the launch's algorithmic
// FP64 flop count. Used by the benchmark to measure a kernel's average launch
// duration and achieved rate; off by default and free when off.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace bta {

enum KernelId {
  K_GEMM = 0,
  K_POTRF_TILE,
  K_TRSM_PANEL,
  K_TILE_INV,
  K_ZERO_UPPER,
  K_MIRROR,
  K_LOGDET,
  K_TRSV,
  K_GEMV,
  K_ARROW,
  K_PROBE,
  K_GEMM_TC,
  K_TC_SPLIT,
  K_TC_FINAL,
  K_FACTOR_STEP,
  K_PERSISTENT,
  K_COUNT
};

bool timing_on();
// Returns a slot to close with timing_stop (or -1 when timing is off).
int timing_start(int kid, double flops, cudaStream_t s);
void timing_stop(int slot, cudaStream_t s);

struct TimedLaunch {
  int slot;
  cudaStream_t s;
  TimedLaunch(int kid, double flops, cudaStream_t st) : slot(-1), s(st) {
    if (timing_on()) slot = timing_start(kid, flops, st);
  }
  ~TimedLaunch() {
    if (slot >= 0) timing_stop(slot, s);
  }
};

}  // namespace bta
