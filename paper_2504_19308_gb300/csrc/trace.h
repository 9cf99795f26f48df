// RAII bracket of one kernel launch for amm_trace_collect().
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace amm {
class TraceScope {
 public:
  // flops / bytes: algorithmic work of this launch.  If dev_count is given, flops is per unit
  // and is multiplied by the value *dev_count holds when the launch runs.
  TraceScope(const char* name, cudaStream_t st, double flops = 0.0, double bytes = 0.0,
             const int32_t* dev_count = nullptr);
  ~TraceScope();
  TraceScope(const TraceScope&) = delete;
  TraceScope& operator=(const TraceScope&) = delete;

 private:
  const char* name_;
  cudaStream_t st_;
  void* a_ = nullptr;
  bool active_ = false;
  double flops_ = 0.0, bytes_ = 0.0;
  const int32_t* dev_count_ = nullptr;
};
}  // namespace amm

#define AMM_CAT2(a, b) a##b
#define AMM_CAT(a, b) AMM_CAT2(a, b)
#define AMM_TRACE(name, st) ::amm::TraceScope AMM_CAT(amm_trace_scope_, __LINE__)(name, st)
#define AMM_TRACE_W(name, st, flops, bytes, cnt) \
  ::amm::TraceScope AMM_CAT(amm_trace_scope_, __LINE__)(name, st, flops, bytes, cnt)
