// Launch tracing for measurement tools (amm_trace_enable / amm_trace_collect).
// When enabled, each kernel launch made by the library is bracketed by two CUDA events
// recorded on the launch's own stream; collect() synchronises on the stop events and sums
// the elapsed time per kernel name.  Disabled (the default) it costs one atomic load per launch.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdio>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "api_internal.h"
#include "trace.h"

namespace amm {

static std::atomic<int> g_trace_on{0};
static std::mutex g_trace_mu;
struct Rec {
  const char* name;
  cudaEvent_t a, b;
  double flops, bytes;
  int slot;  // index into the pinned count slots, -1 if the work is fixed
};
static int32_t* g_slots = nullptr;  // pinned host memory receiving device-side counts
static int g_nslots = 0, g_used = 0;
static std::vector<Rec> g_recs;
static std::vector<cudaEvent_t> g_pool;

static cudaEvent_t take_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

TraceScope::TraceScope(const char* name, cudaStream_t st, double flops, double bytes, const int32_t* dev_count)
    : name_(name), st_(st), flops_(flops), bytes_(bytes), dev_count_(dev_count) {
  if (!g_trace_on.load(std::memory_order_relaxed)) return;
  std::lock_guard<std::mutex> lk(g_trace_mu);
  a_ = take_event();
  cudaEventRecord((cudaEvent_t)a_, st_);
  active_ = true;
}

TraceScope::~TraceScope() {
  if (!active_) return;
  std::lock_guard<std::mutex> lk(g_trace_mu);
  cudaEvent_t b = take_event();
  cudaEventRecord(b, st_);
  int slot = -1;
  if (dev_count_) {
    if (!g_slots) {
      g_nslots = 1 << 16;
      if (cudaMallocHost((void**)&g_slots, sizeof(int32_t) * g_nslots) != cudaSuccess) g_slots = nullptr;
    }
    if (g_slots && g_used < g_nslots) {
      slot = g_used++;
      cudaMemcpyAsync(g_slots + slot, dev_count_, sizeof(int32_t), cudaMemcpyDeviceToHost, st_);
    }
  }
  g_recs.push_back({name_, (cudaEvent_t)a_, b, flops_, bytes_, slot});
}

}  // namespace amm

using namespace amm;

extern "C" amm_status_t amm_trace_enable(int32_t on) {
  g_trace_on.store(on ? 1 : 0);
  return AMM_OK;
}

extern "C" amm_status_t amm_trace_collect(char* host_json, int64_t cap, int64_t* launches) {
  if (!host_json || cap <= 0) return fail(AMM_ERR_INVALID_ARG, "amm_trace_collect: bad buffer");
  std::lock_guard<std::mutex> lk(g_trace_mu);
  struct Agg {
    long n = 0;
    double ms = 0, flops = 0, bytes = 0;
  };
  std::map<std::string, Agg> agg;
  long total = 0;
  if (!g_recs.empty()) {
    cudaError_t e = cudaDeviceSynchronize();  // the count copies ride on the launches' streams
    if (e != cudaSuccess) return cuda_fail(e, "amm_trace_collect");
  }
  for (auto& r : g_recs) {
    cudaError_t e = cudaEventSynchronize(r.b);
    if (e != cudaSuccess) return cuda_fail(e, "amm_trace_collect");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, r.a, r.b);
    auto& v = agg[r.name];
    double mult = 1.0;
    if (r.slot >= 0) mult = (double)g_slots[r.slot];
    v.n += 1;
    v.ms += ms;
    v.flops += r.flops * mult;
    v.bytes += r.bytes;
    ++total;
    g_pool.push_back(r.a);
    g_pool.push_back(r.b);
  }
  g_recs.clear();
  g_used = 0;
  std::string s = "{";
  bool first = true;
  for (auto& kv : agg) {
    char buf[256];
    snprintf(buf, sizeof(buf), "%s\"%s\": [%ld, %.6f, %.6e, %.6e]", first ? "" : ", ", kv.first.c_str(), kv.second.n,
             kv.second.ms, kv.second.flops, kv.second.bytes);
    s += buf;
    first = false;
  }
  s += "}";
  if ((int64_t)s.size() + 1 > cap) return fail(AMM_ERR_INVALID_ARG, "amm_trace_collect: buffer too small");
  memcpy(host_json, s.c_str(), s.size() + 1);
  if (launches) *launches = total;
  return AMM_OK;
}
