// Kernel-variant autotuner shared by the FFT-based kernels (an implementation choice; the paper has
// no counterpart).  A tuned kernel has a few compiled variants (packed signals and threads per
// CTA) that compute every output with the same operations; the first call of a key with autotuning
// on times each variant on the call's own operands into scratch memory and keeps the fastest for the
// process.  Keys: kernel id << 24 | length << 3 | flags (the kernel's direction / element type).
#pragma once
#include <cuda_runtime.h>

#include "api_internal.h"

namespace amm {

// autotuner table (circulant.cu): -1 = not timed yet; a set entry is also written to the cache
// file named by AMM_TUNE_CACHE, which the first lookup loads
int cd_tune_get(int key);
void cd_tune_set(int key, int variant);

enum TuneKernel : int { TUNE_APPLY = 0, TUNE_RESIDUAL = 1, TUNE_BW_COL = 2, TUNE_BW_ROW = 3 };
constexpr int tune_key(int kernel, int n, int flags) { return (kernel << 24) | (n << 3) | flags; }

// The variant for `key`: the table's entry, else (autotuning off, or the stream being captured into
// a graph) `dflt`, else the fastest of run(0) .. run(nvar - 1) by CUDA events on `st` (one warm-up
// and three timed launches each).  run(v) launches variant v writing scratch outputs only.
template <class RUN>
int tune_pick(int key, int nvar, int dflt, cudaStream_t st, RUN run) {
  const int v = cd_tune_get(key);
  if (v >= 0 && v < nvar) return v;
  if (!amm_autotune_enabled()) return dflt;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return dflt;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float best = 0.f;
  int pick = dflt;
  for (int cand = 0; cand < nvar && e == cudaSuccess; ++cand) {
    e = run(cand);  // warm-up
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    for (int it = 0; it < 3 && e == cudaSuccess; ++it) e = run(cand);
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && (cand == 0 || ms < best)) {
      best = ms;
      pick = cand;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) {
    cudaGetLastError();  // clear a failed candidate; the default runs instead
    return dflt;
  }
  cd_tune_set(key, pick);
  return pick;
}

}  // namespace amm
