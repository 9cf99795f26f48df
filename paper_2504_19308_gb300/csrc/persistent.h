// Persistent work-queue executor of a batch's cycle-sparsifier products (batch_persistent.cu).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

namespace amm {

constexpr int PQ_MAX_N = 4096;  // largest n taken (shared memory of the panel tiles: 16 n + 4 k bytes)

// one forward product C = A_s B + dA B_s of square FP32 n x n operands, k cycles per operand
struct PqDesc {
  const float* A;
  const float* B;
  float* C;
  int64_t lda, ldb, ldc, n, k;
};

struct PqPlan;
// method / dtype / shapes that the executor takes (forward products only)
bool pq_eligible(int method, int dtype, int64_t m, int64_t n, int64_t p, bool has_grad);
// Allocates the plan's device buffers and uploads its queue (synchronous; not inside a capture).
cudaError_t pq_build(const std::vector<PqDesc>& items, PqPlan** out);
// Zeroes the counters and launches the executor on st (capturable).
cudaError_t pq_launch(PqPlan* p, cudaStream_t st, uint64_t limit_ns);
// The control block after the launch has completed (the caller synchronises first).
cudaError_t pq_status(PqPlan* p, int32_t* status, int32_t* item, int32_t* stage);
void pq_destroy(PqPlan* p);

}  // namespace amm
