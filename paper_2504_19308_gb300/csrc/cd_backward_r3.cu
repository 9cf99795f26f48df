// The circulant backward kernels at lengths n = 3 * 2^a (48 .. 6144), in a translation unit of
// their own (compiled in parallel with the power-of-two instantiations).
#include "cd_backward_kernels.cuh"

namespace amm {

#define AMM_BW_DISPATCH_R3(n, EXPR)                   \
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

cudaError_t bw_spectrum_r3(int n, bool row, const float* X, int64_t ldx, const float2* tw, float2* Xh,
                           const int32_t* gate0, const int32_t* gate1, cudaStream_t st) {
  AMM_BW_DISPATCH_R3(n, return BwOps<NN>::spectrum(row, X, ldx, tw, Xh, gate0, gate1, st));
}

cudaError_t cd_sddmm_r3(int n, const float2* Xh, const float2* Yh, const int32_t* list, const int32_t* count, int cap,
                        float2* K, const int32_t* gate0, const int32_t* gate1, cudaStream_t st) {
  AMM_BW_DISPATCH_R3(n, return BwOps<NN>::sddmm(Xh, Yh, list, count, cap, K, gate0, gate1, st));
}

cudaError_t cd_rho_r3(int n, const float2* K, const float2* tw, const int32_t* list, const int32_t* count, int cap,
                      float2* RX, const int32_t* gate0, const int32_t* gate1, cudaStream_t st) {
  AMM_BW_DISPATCH_R3(n, return BwOps<NN>::rho(K, tw, list, count, cap, RX, gate0, gate1, st));
}

}  // namespace amm
