// The circulant kernels at lengths n = 3 * 2^a (48 .. 6144), in a translation unit of their own so
// that the two sets of instantiations compile in parallel.  The FFT takes one radix-3 pass before
// its power-of-two passes; every cyclic index is taken mod n.
#include "circulant_kernels.cuh"

namespace amm {

#define AMM_DISPATCH_R3(n, EXPR)                      \
  switch (n) {                                        \
    case 48: { constexpr int NN = 48; EXPR; }         \
    case 96: { constexpr int NN = 96; EXPR; }         \
    case 192: { constexpr int NN = 192; EXPR; }       \
    case 384: { constexpr int NN = 384; EXPR; }       \
    case 768: { constexpr int NN = 768; EXPR; }       \
    case 1536: { constexpr int NN = 1536; EXPR; }     \
    case 3072: { constexpr int NN = 3072; EXPR; }     \
    case 6144: { constexpr int NN = 6144; EXPR; }     \
    default: return cudaErrorInvalidValue;            \
  }

cudaError_t cd_spectrum_r3(int n, const void* A, int64_t lda, bool bf16, const float2* tw, float2* R, float* kpart,
                           cudaStream_t st) {
  AMM_DISPATCH_R3(n, return CdOps<NN>::spectrum(A, lda, bf16, tw, R, kpart, st));
}

cudaError_t cd_eigen_r3(int n, const float2* R, const float2* tw, const int32_t* list, const float* coef,
                        const int32_t* count, int cap, int imag_coef, float2* L, cudaStream_t st) {
  AMM_DISPATCH_R3(n, return CdOps<NN>::eigen(R, tw, list, coef, count, cap, imag_coef, L, st));
}

cudaError_t cd_residual_r3(int n, const float2* R, const float2* tw, const float* g, int mode, const int32_t* dcount,
                           const int32_t* dcount2, float* X, int64_t ldx, int accumulate, cudaStream_t st) {
  AMM_DISPATCH_R3(n, return CdOps<NN>::residual(R, tw, g, mode, dcount, dcount2, X, ldx, accumulate, st));
}

cudaError_t cd_apply_r3(int n, bool row, const void* X, int64_t ldx, bool bf16, int64_t nvec, const float2* tw,
                        const int32_t* list, const float2* Lc, const int32_t* count, const int32_t* gate0,
                        const int32_t* gate1, float* out, int64_t ldo, int accumulate, int rev, cudaStream_t st) {
  AMM_DISPATCH_R3(n, return CdOps<NN>::apply(row, X, ldx, bf16, nvec, tw, list, Lc, count, gate0, gate1, out, ldo,
                                             accumulate, rev, st));
}

}  // namespace amm
