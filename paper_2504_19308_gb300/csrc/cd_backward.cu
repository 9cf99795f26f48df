// Backward of the circulant first-order product with the selections frozen (sm_103a).
//
// With S the selection of A (weights w, unpaired coefficients v as in the forward) and G the
// upstream gradient, the gradients of <G, Re M> are (bilinear adjoint of P_S is P_{S-bar}):
//   dA = G B~_w^T + sum_{t in S u S-bar} w_t R_t(G dB_w^T) D^t + sum_{t unpaired} (i v_t) R_t(G V_B^T) D^t
//   dB = A~_w^T G + sum_{s} w_s R_s(dA_w^T G) D^s + sum_{s unpaired} (i v_s) R_s(Y_A^T G) D^s
// where dB_w = B - Re B~, V_B = Im B~, dA_w = A - Re A~, Y_A = Im A~.  The first terms are spectral
// applies with the adjoint coefficient pairing.  A component of a product matrix is an SDDMM on
// spectra: with column spectra Xh = F X, Yh = F Y (DFT along the row index),
//   r_{j,t}(X Y^T) = (1/n^2) sum_p e^{2 pi i p j/n} K_t(p),   K_t(p) = sum_m Xh(p, m) Yh(t - p, m),
// and for X^T Y the same with row spectra stored transposed ([frequency][row]).  Real products
// have Hermitian component spectra, so only t <= n/2 is formed; the dense result comes from the
// inverse cycle transform (cd_residual) with the coefficient w_t or i v_t.
#include <cuda_runtime.h>

#include "cd_backward_kernels.cuh"

namespace amm {

#define AMM_BW_DISPATCH(n, EXPR)                  \
  switch (n) {                                    \
    case 16: { constexpr int NN = 16; EXPR; }     \
    case 32: { constexpr int NN = 32; EXPR; }     \
    case 64: { constexpr int NN = 64; EXPR; }     \
    case 128: { constexpr int NN = 128; EXPR; }   \
    case 256: { constexpr int NN = 256; EXPR; }   \
    case 512: { constexpr int NN = 512; EXPR; }   \
    case 1024: { constexpr int NN = 1024; EXPR; } \
    case 2048: { constexpr int NN = 2048; EXPR; } \
    case 4096: { constexpr int NN = 4096; EXPR; } \
    case 8192: { constexpr int NN = 8192; EXPR; } \
    case 16384: { constexpr int NN = 16384; EXPR; } \
    default: break;                               \
  }

cudaError_t bw_spectrum(int n, bool row, const float* X, int64_t ldx, const float2* tw, float2* Xh, cudaStream_t st,
                        const int32_t* gate0, const int32_t* gate1) {
  AMM_TRACE_W(row ? "bw_row_spectrum" : "bw_col_spectrum", st, 0.0, (double)n * n * 4 + (n / 2 + 1.0) * n * 8,
              nullptr);
  AMM_BW_DISPATCH(n, return BwOps<NN>::spectrum(row, X, ldx, tw, Xh, gate0, gate1, st));
  if (cd_r3_length(n)) return bw_spectrum_r3(n, row, X, ldx, tw, Xh, gate0, gate1, st);
  return bw_spectrum_any(n, row, X, ldx, Xh, gate0, gate1, st);
}

cudaError_t cd_sddmm(int n, const float2* Xh, const float2* Yh, const int32_t* list, const int32_t* count, int cap,
                     float2* K, const int32_t* gate0, const int32_t* gate1, cudaStream_t st) {
  // work per listed component (those with t <= n/2 are formed, about half): n dot products of
  // length n, 8 FLOP per complex MAC
  const bool tiled = n >= 2 * SDT_W && (int64_t)cap * 12 >= n;  // the variant BwOps<N>::sddmm launches
  AMM_TRACE_W(tiled ? "cd_sddmm_tiled" : "cd_sddmm", st, 4.0 * n * (double)n, 0.0, count);
  AMM_BW_DISPATCH(n, return BwOps<NN>::sddmm(Xh, Yh, list, count, cap, K, gate0, gate1, st));
  if (cd_r3_length(n)) return cd_sddmm_r3(n, Xh, Yh, list, count, cap, K, gate0, gate1, st);
  return cd_sddmm_any(n, Xh, Yh, list, count, cap, K, gate0, gate1, st);
}

cudaError_t cd_rho(int n, const float2* K, const float2* tw, const int32_t* list, const int32_t* count, int cap,
                   float2* RX, const int32_t* gate0, const int32_t* gate1, cudaStream_t st) {
  AMM_TRACE("cd_rho", st);
  AMM_BW_DISPATCH(n, return BwOps<NN>::rho(K, tw, list, count, cap, RX, gate0, gate1, st));
  if (cd_r3_length(n)) return cd_rho_r3(n, K, tw, list, count, cap, RX, gate0, gate1, st);
  return cd_rho_any(n, K, list, count, cap, RX, gate0, gate1, st);
}

}  // namespace amm
