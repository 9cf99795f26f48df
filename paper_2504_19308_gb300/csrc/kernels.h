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
                      cudaStream_t st, bool mirror = true);
cudaError_t cd_eigen(int n, const float2* R, const float2* tw, const int32_t* list, const float* coef,
                     const int32_t* count, int cap, int imag_coef, float2* L, cudaStream_t st);
cudaError_t cd_residual(int n, const float2* R, const float2* tw, const float* g, int mode, const int32_t* dcount,
                        float* X, cudaStream_t st);
cudaError_t cd_apply(int n, bool row, const void* X, int64_t ldx, bool bf16, int64_t nvec, const float2* tw,
                     const int32_t* list, const float2* Lc, const int32_t* count, const int32_t* gate0,
                     const int32_t* gate1, float* out, int64_t ldo, int accumulate, cudaStream_t st);

// cycle.cu
int cyc_rows_per_part(int n);
cudaError_t cyc_keys(int n, const float* A, int64_t lda, float* part, cudaStream_t st);
cudaError_t cyc_gather(int n, int k, const float* A, int64_t lda, const int32_t* sel, float* cyc,
                       unsigned char* insel, cudaStream_t st);
cudaError_t cyc_apply(int n, const float* A, int64_t lda, const float* B, int64_t ldb, const int32_t* selA, int ka,
                      const float* cycA, const unsigned char* inselA, const int32_t* selB, int kb, const float* cycB,
                      float* C, int64_t ldc, cudaStream_t st);

// fourier.cu
cudaError_t ft_transform(int n, bool row, const float* X, int64_t ldx, int nvec, const float2* tw, float2* T,
                         float2* TT, float* mag, cudaStream_t st);
cudaError_t ft_select(int n, int k, int rows, const float* mag, int32_t* sel, uint32_t* maskT, int mask_words,
                      cudaStream_t st);
cudaError_t ft_product(int n, int m, int p, int k_a, int k_b, const float2* At, const float2* AtT,
                       const int32_t* selA, const uint32_t* maskT, int mask_words, const float2* Bt,
                       const int32_t* selB, float* C, int64_t ldc, cudaStream_t st);

}  // namespace amm
