// RAII bracket of one kernel launch for amm_trace_collect().
#pragma once
#include <cuda_runtime.h>

namespace amm {
class TraceScope {
 public:
  TraceScope(const char* name, cudaStream_t st);
  ~TraceScope();
  TraceScope(const TraceScope&) = delete;
  TraceScope& operator=(const TraceScope&) = delete;

 private:
  const char* name_;
  cudaStream_t st_;
  void* a_ = nullptr;
  bool active_ = false;
};
}  // namespace amm

#define AMM_CAT2(a, b) a##b
#define AMM_CAT(a, b) AMM_CAT2(a, b)
#define AMM_TRACE(name, st) ::amm::TraceScope AMM_CAT(amm_trace_scope_, __LINE__)(name, st)
