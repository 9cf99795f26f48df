// Internal launch interface between the C ABI (api.cu) and the kernel files.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace amm {

// Outputs of the circulant selection kernel (all device pointers).
struct SelectOut {
  double* keys;     // n      T[k] = ||R_A[k]||_2 (mirrored)
  double* norms;    // 3      ||A||_F^2, ||dA||_F^2, relative boundary gap (-1 if forced)
  int32_t* sel;     // k      selection in (key desc, index asc) order
  int32_t* ulist;   // <= 2k  S u S-bar in index order
  float* uw;        // <= 2k  weight w_t in {1/2, 1}
  int32_t* dlist;   // <= 2k  unpaired set {t : exactly one of t, n-t in S}
  float* dv;        // <= 2k  v_t = +-1/2
  float* wfull;     // n      w_t for every t (0 outside S u S-bar)
  float* vfull;     // n      v_t for every t
  int32_t* counts;  // 2      |S u S-bar|, |unpaired|
};

int cd_cols_per_cta(int n);
cudaError_t cd_twiddles(float2* tw, int n, cudaStream_t st);
cudaError_t cd_spectrum(int n, const void* A, int64_t lda, bool bf16, const float2* tw, float2* R, float* kpart,
                        cudaStream_t st);
cudaError_t cd_select(int n, int k, const float* kpart, int nparts, const int32_t* forced, const SelectOut& o,
                      cudaStream_t st);
cudaError_t cd_eigen(int n, const float2* R, const float2* tw, const int32_t* list, const float* coef,
                     const int32_t* count, int cap, int imag_coef, float2* L, cudaStream_t st);
cudaError_t cd_residual(int n, const float2* R, const float2* tw, const float* g, int mode, const int32_t* dcount,
                        float* X, cudaStream_t st);
cudaError_t cd_apply(int n, bool row, const void* X, int64_t ldx, bool bf16, int64_t nvec, const float2* tw,
                     const int32_t* list, const float2* Lc, const int32_t* count, const int32_t* gate0,
                     const int32_t* gate1, float* out, int64_t ldo, int accumulate, cudaStream_t st);

}  // namespace amm
