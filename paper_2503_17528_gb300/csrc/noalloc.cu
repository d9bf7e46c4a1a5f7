// bta_logdet_noalloc: the log-determinant without any device allocation.
//
// Some callers cannot allocate device memory at the moment they need the
// log-determinant: for example code that runs under a device-memory budget
// owned by a host framework, or latency-critical loops where cudaMalloc and
// cudaFree are not acceptable because they can synchronize the whole device.
// This entry point keeps its scratch (one partial sum per diagonal block, plus
// one for the tip) in a fixed array compiled into the library, so it needs no
// allocation from the caller or from the library.
//
// The array below is a file-scope device variable: every GPU that loads the
// library holds its 512 KiB until the process exits. Host code cannot use its
// name as a device address, so the address is looked up once per device with
// cudaGetSymbolAddress (the first call on each device does that, with that
// device current). All calls on a device share the one array and it keeps the
// last call's contents; each call overwrites every partial it later reads, so
// nothing has to start at zero, but calls that overlap on the GPU (different
// streams, no ordering between them) race on the array. The looked-up address
// is kept for the life of the process: a cudaDeviceReset on a device unloads the
// library's module there, so a process that resets a device must not call this
// entry point on that device afterwards.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/bta.h"
#include "bta_internal.cuh"

namespace {

constexpr int64_t kMaxBlocks = 65536;  // largest n accepted
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_logdet_scratch[kMaxBlocks + 1];

std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_logdet_scratch on device `dev` (looked up once per
// device, with that device current).
cudaError_t scratch_address(int dev, double** out) {
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_logdet_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = (double*)p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" int bta_logdet_noalloc(int64_t n, int64_t b, int64_t a, const double* diag,
                                  const double* tip, double* out_dev, bta_stream_t stream) {
  if (n < 1 || n > kMaxBlocks) return -1;
  if (b < 1 || b > 32768) return -2;
  if (a < 0 || a > 32768) return -3;
  if (!diag || ((uintptr_t)diag & 7u)) return -4;
  if (a > 0 && (!tip || ((uintptr_t)tip & 7u))) return -5;
  if (!out_dev || ((uintptr_t)out_dev & 7u)) return -6;
  // The scratch address is per device: the one the kernel runs on is the
  // stream's, which must be the current device (a kernel cannot be launched
  // into another device's stream).
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return (int)e;
  if (stream) {
    int sdev = -1;
    e = cudaStreamGetDevice((cudaStream_t)stream, &sdev);
    if (e != cudaSuccess) return (int)e;
    if (sdev != dev) return -7;
  }
  double* scratch = nullptr;
  e = scratch_address(dev, &scratch);
  if (e != cudaSuccess) return (int)e;
  e = bta::logdet_f64(diag, n, b, tip, a, scratch, out_dev, (cudaStream_t)stream);
  return e == cudaSuccess ? 0 : (int)e;
}
