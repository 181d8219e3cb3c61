// Launch accounting and optional per-kernel-family CUDA event timing.
#include <atomic>
#include <mutex>
#include <vector>

#include "ps_internal.cuh"

namespace ps {

namespace {
std::atomic<uint64_t> g_launches{0};
std::mutex g_mu;
uint32_t g_mask = 0;
struct Tally {
  std::vector<cudaEvent_t> ev;  // start, stop pairs
  uint64_t launches = 0;
};
Tally g_tally[PS_KID_COUNT_];
std::vector<cudaEvent_t> g_pool;

cudaEvent_t take_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}
}  // namespace

void prof_begin(uint32_t kid, cudaStream_t s) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  if (!(g_mask & (1u << kid))) return;
  std::lock_guard<std::mutex> lk(g_mu);
  cudaEvent_t e = take_event();
  if (!e) return;
  cudaEventRecord(e, s);
  g_tally[kid].ev.push_back(e);
}

void prof_end(uint32_t kid, cudaStream_t s) {
  if (!(g_mask & (1u << kid))) return;
  std::lock_guard<std::mutex> lk(g_mu);
  Tally& t = g_tally[kid];
  if (t.ev.size() % 2 == 0) return;  // the start event was not recorded
  cudaEvent_t e = take_event();
  if (!e) {
    g_pool.push_back(t.ev.back());
    t.ev.pop_back();
    return;
  }
  cudaEventRecord(e, s);
  t.ev.push_back(e);
  t.launches += 1;
}

}  // namespace ps

using namespace ps;

extern "C" {

uint64_t ps_launch_count(void) { return g_launches.load(); }

int ps_prof_enable(uint32_t kid_mask) {
  std::lock_guard<std::mutex> lk(g_mu);
  PS_CUDA(cudaDeviceSynchronize());
  for (auto& t : g_tally) {
    for (cudaEvent_t e : t.ev) g_pool.push_back(e);
    t.ev.clear();
    t.launches = 0;
  }
  g_mask = kid_mask;
  return PS_OK;
}

int ps_prof_read(uint32_t kid, uint64_t* launches, double* total_ms) {
  if (kid == 0 || kid >= PS_KID_COUNT_ || !launches || !total_ms) return fail(PS_ERR_INVALID_ARG, "ps_prof_read");
  std::lock_guard<std::mutex> lk(g_mu);
  const Tally& t = g_tally[kid];
  double ms = 0.0;
  for (size_t i = 0; i + 1 < t.ev.size(); i += 2) {
    PS_CUDA(cudaEventSynchronize(t.ev[i + 1]));
    float x = 0.f;
    PS_CUDA(cudaEventElapsedTime(&x, t.ev[i], t.ev[i + 1]));
    ms += x;
  }
  *launches = t.launches;
  *total_ms = ms;
  return PS_OK;
}

}  // extern "C"
