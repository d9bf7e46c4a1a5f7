#include <mutex>
#include <vector>

#include "../../include/bta.h"
#include "timing.cuh"

namespace bta {
namespace {

struct Rec {
  cudaEvent_t a, b;
  int kid;
  double flops;
};

std::mutex g_mu;
bool g_on = false;
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;

cudaEvent_t get_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

}  // namespace

bool timing_on() { return g_on; }

int timing_start(int kid, double flops, cudaStream_t s) {
  std::lock_guard<std::mutex> lk(g_mu);
  Rec r{get_event(), get_event(), kid, flops};
  cudaEventRecord(r.a, s);
  g_recs.push_back(r);
  return (int)g_recs.size() - 1;
}

void timing_stop(int slot, cudaStream_t s) {
  std::lock_guard<std::mutex> lk(g_mu);
  cudaEventRecord(g_recs[slot].b, s);
}

}  // namespace bta

using namespace bta;

extern "C" {

int bta_timing_enable(int on) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto& r : g_recs) {
    g_pool.push_back(r.a);
    g_pool.push_back(r.b);
  }
  g_recs.clear();
  g_on = on != 0;
  return 0;
}

int bta_timing_read(int kernel_id, double* total_ms, double* flops, int64_t* launches) {
  if (kernel_id < 0 || kernel_id >= K_COUNT || !total_ms || !flops || !launches) return -1;
  std::lock_guard<std::mutex> lk(g_mu);
  double ms = 0.0, fl = 0.0;
  int64_t cnt = 0;
  for (auto& r : g_recs) {
    if (r.kid != kernel_id) continue;
    cudaError_t e = cudaEventSynchronize(r.b);
    if (e != cudaSuccess) return (int)e;
    float t = 0.f;
    e = cudaEventElapsedTime(&t, r.a, r.b);
    if (e != cudaSuccess) return (int)e;
    ms += t;
    fl += r.flops;
    ++cnt;
  }
  *total_ms = ms;
  *flops = fl;
  *launches = cnt;
  return 0;
}

}  // extern "C"
