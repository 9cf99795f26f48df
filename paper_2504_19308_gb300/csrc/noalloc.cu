// amm_circulant_spectrum_noalloc: the cycle spectrum and component keys of one square matrix,
// computed without allocating any device memory.
//
// Who needs this: callers that must not call cudaMalloc -- code that runs while a CUDA graph is
// being captured by a framework that forbids allocation inside capture, processes whose device
// memory is fully handed to another allocator or pool, and short-lived helper threads of runtimes
// that treat a device allocation as a synchronisation point.  They pass the input and both
// outputs; the only scratch the kernels need (per-CTA partial sums of the keys and the twiddle
// table) lives in the file-scope device array below.
//
// The scratch array occupies AMM_NOALLOC_SCRATCH_BYTES on every GPU that loads this library, for
// the lifetime of the process.  All calls share it, so calls whose kernels overlap on the GPU
// (different streams, or different host threads) race on it; order them on one stream.  Every
// byte a call reads from the array is written earlier by the same call, so nothing has to be
// cleared between calls.
//
// The keys are reduced by the same kernel, in the same order, as in amm_decompose (cd_keys), and
// the square root is taken in FP64 as the selection kernel takes it, so both paths return the same
// doubles and a selection made from these keys equals amm_decompose's, exact ties included.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/amm.h"
#include "api_internal.h"
#include "kernels.h"

namespace {

constexpr int kMaxN = AMM_NOALLOC_MAX_N;
constexpr size_t kTwBytes = sizeof(float2) * kMaxN;
// key partials: (n / J) rows of (n/2 + 1) floats, J = 8 columns per spectrum CTA for n <= 4096
constexpr size_t kPartBytes = sizeof(float) * (size_t)(kMaxN / 8) * (kMaxN / 2 + 1);
// reduced squared keys, t = 0..n/2 (FP64), 256-byte aligned after the partials
constexpr size_t kKey2Off = (kTwBytes + kPartBytes + 255) / 256 * 256;
constexpr size_t kKey2Bytes = sizeof(double) * (kMaxN / 2 + 1);
static_assert(kKey2Off + kKey2Bytes <= AMM_NOALLOC_SCRATCH_BYTES, "scratch too small");

__device__ __align__(256) unsigned char g_noalloc_scratch[AMM_NOALLOC_SCRATCH_BYTES];

// Host copies of the array's device address, one per device, set on the first call made with
// that device current.
std::mutex g_mu;
void* g_addr[64] = {nullptr};

// keys[t] = sqrt(key2[t]) for t <= n/2 (key2 reduced by cd_keys), mirrored to n - t: the values
// the circulant selection kernel writes to a handle's keys.
__global__ void noalloc_sqrt_mirror_kernel(const double* __restrict__ key2, int n, double* __restrict__ keys) {
  const int kh = n / 2 + 1;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < kh; t += gridDim.x * blockDim.x) {
    const double v = sqrt(key2[t]);
    keys[t] = v;
    if (t > 0 && t < n - t) keys[n - t] = v;
  }
}

}  // namespace

extern "C" amm_status_t amm_circulant_spectrum_noalloc(const float* A, int64_t n, int64_t lda, void* R,
                                                       double* keys, void* stream) {
  using namespace amm;
  if (!A || !R || !keys) return fail(AMM_ERR_INVALID_ARG, "amm_circulant_spectrum_noalloc: NULL pointer");
  if (n < 16 || n > kMaxN || (n & (n - 1)) != 0)
    return fail(AMM_ERR_UNSUPPORTED_SIZE,
                "amm_circulant_spectrum_noalloc: n=%lld must be a power of two in [16, %d] (scratch limit)",
                (long long)n, kMaxN);
  if (lda < n) return fail(AMM_ERR_INVALID_ARG, "amm_circulant_spectrum_noalloc: lda=%lld < n", (long long)lda);
  if (((uintptr_t)R & 15) != 0) return fail(AMM_ERR_INVALID_ARG, "amm_circulant_spectrum_noalloc: R not 16-byte aligned");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "amm_circulant_spectrum_noalloc: cudaGetDevice");
  if (dev < 0 || dev >= 64) return fail(AMM_ERR_INVALID_ARG, "amm_circulant_spectrum_noalloc: device %d", dev);
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess) return cuda_fail(e, "amm_circulant_spectrum_noalloc: cudaGetSymbolAddress");
      g_addr[dev] = p;
    }
    base = g_addr[dev];
  }
  cudaStream_t st = (cudaStream_t)stream;
  float2* tw = (float2*)base;
  float* kpart = (float*)((unsigned char*)base + kTwBytes);
  double* key2 = (double*)((unsigned char*)base + kKey2Off);
  const int nn = (int)n;
  const int nparts = nn / cd_cols_per_cta(nn);
  if ((size_t)nparts * (nn / 2 + 1) * sizeof(float) > kPartBytes)
    return fail(AMM_ERR_UNSUPPORTED_SIZE, "amm_circulant_spectrum_noalloc: key partials exceed the scratch");
  if ((e = cd_twiddles(tw, nn, st)) != cudaSuccess) return cuda_fail(e, "noalloc twiddles");
  if ((e = cd_spectrum(nn, A, lda, false, tw, (float2*)R, kpart, st)) != cudaSuccess)
    return cuda_fail(e, "noalloc spectrum");
  if ((e = cd_keys(nn / 2 + 1, kpart, nparts, key2, st)) != cudaSuccess) return cuda_fail(e, "noalloc key reduction");
  noalloc_sqrt_mirror_kernel<<<(nn / 2 + 256) / 256, 256, 0, st>>>(key2, nn, keys);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "noalloc keys");
  return AMM_OK;
}
