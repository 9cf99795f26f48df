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
  double* key2;     // n      scratch: reduced squared keys
};

int cd_cols_per_cta(int n);
// lengths of the fused kernels: 3 * 2^a in [48, 6144] (circulant_r3.cu; 2^a in circulant.cu)
inline bool cd_r3_length(int64_t n) {
  return n % 3 == 0 && n >= 48 && n <= 6144 && ((n / 3) & (n / 3 - 1)) == 0;
}
// circulant_any.cu: every other length n in [16, CD_ANY_MAX_N], by chirp-z (Bluestein) DFTs; the
// same steps, outputs and layouts as the fixed-length wrappers below
constexpr int CD_ANY_MAX_N = 4096;
bool cd_any_length_ok(int64_t n);
cudaError_t cd_spectrum_any(int n, const void* A, int64_t lda, bool bf16, float2* R, float* kpart, cudaStream_t st);
cudaError_t cd_eigen_any(int n, const float2* R, const int32_t* list, const float* coef, const int32_t* count,
                         int cap, int imag_coef, float2* L, cudaStream_t st);
cudaError_t cd_residual_any(int n, const float2* R, const float* g, int mode, const int32_t* dcount,
                            const int32_t* dcount2, float* X, int64_t ldx, int accumulate, cudaStream_t st);
cudaError_t cd_apply_any(int n, bool row, const void* X, int64_t ldx, bool bf16, int64_t nvec, const int32_t* list,
                         const float2* Lc, const int32_t* count, const int32_t* gate0, const int32_t* gate1,
                         float* out, int64_t ldo, int accumulate, int rev, cudaStream_t st);
cudaError_t bw_spectrum_any(int n, bool row, const float* X, int64_t ldx, float2* Xh, const int32_t* gate0,
                            const int32_t* gate1, cudaStream_t st);
cudaError_t cd_sddmm_any(int n, const float2* Xh, const float2* Yh, const int32_t* list, const int32_t* count,
                         int cap, float2* K, const int32_t* gate0, const int32_t* gate1, cudaStream_t st);
cudaError_t cd_rho_any(int n, const float2* K, const int32_t* list, const int32_t* count, int cap, float2* RX,
                       const int32_t* gate0, const int32_t* gate1, cudaStream_t st);
cudaError_t cd_twiddles(float2* tw, int n, cudaStream_t st);
cudaError_t cd_spectrum(int n, const void* A, int64_t lda, bool bf16, const float2* tw, float2* R, float* kpart,
                        cudaStream_t st);
// key2[t] = sum over the nparts partial rows of kpart[c][t], t < kh (fixed order, FP64)
cudaError_t cd_keys(int kh, const float* kpart, int nparts, double* key2, cudaStream_t st);
// pair_closed (circulant only): the selection is closed under t -> n - t (S u S-bar), so M is real
cudaError_t cd_select(int n, int k, const float* kpart, int nparts, const int32_t* forced, const SelectOut& o,
                      cudaStream_t st, bool mirror = true, bool pair_closed = false);
cudaError_t cd_eigen(int n, const float2* R, const float2* tw, const int32_t* list, const float* coef,
                     const int32_t* count, int cap, int imag_coef, float2* L, cudaStream_t st);
// inverse cycle transform of a (half) spectrum R with coefficients by mode (0: 1-g, 1: -i g,
// 2: g, 3: +i g); writes or adds X((c+j) mod n, c), leading dimension ldx (0 = n).  Rows of R
// whose coefficient is zero are not read.  Odd modes skip when *dcount == 0; any mode skips
// when dcount2 is given and *dcount2 == 0.
// The inverse cycle transform of the listed components only (list / coef / *count: S u S-bar with w,
// or the unpaired set with v), evaluated term by term without FFTs; mode 0 needs the operand A
// (dtype bf16 or FP32).  Taken for few components (cd_residual_direct_ok(k): 2k small).
bool cd_residual_direct_ok(int64_t k);
cudaError_t cd_residual_direct(int n, const float2* R, const float2* tw, const int32_t* list, const float* coef,
                               const int32_t* count, int mode, const void* A, int64_t lda, bool bf16, float* X,
                               int64_t ldx, int accumulate, const int32_t* dcount, const int32_t* dcount2,
                               cudaStream_t st);
cudaError_t cd_residual(int n, const float2* R, const float2* tw, const float* g, int mode, const int32_t* dcount,
                        float* X, cudaStream_t st, int64_t ldx = 0, int accumulate = 0,
                        const int32_t* dcount2 = nullptr);
// cd_backward.cu
cudaError_t bw_spectrum(int n, bool row, const float* X, int64_t ldx, const float2* tw, float2* Xh, cudaStream_t st,
                        const int32_t* gate0 = nullptr, const int32_t* gate1 = nullptr);
cudaError_t cd_sddmm(int n, const float2* Xh, const float2* Yh, const int32_t* list, const int32_t* count, int cap,
                     float2* K, const int32_t* gate0, const int32_t* gate1, cudaStream_t st);
cudaError_t cd_rho(int n, const float2* K, const float2* tw, const int32_t* list, const int32_t* count, int cap,
                   float2* RX, const int32_t* gate0, const int32_t* gate1, cudaStream_t st);
// rev: coefficient index L((t - p) mod n) if 1, L(p) if 0, -1 = the forward pairing (rev = row)
cudaError_t cd_apply(int n, bool row, const void* X, int64_t ldx, bool bf16, int64_t nvec, const float2* tw,
                     const int32_t* list, const float2* Lc, const int32_t* count, const int32_t* gate0,
                     const int32_t* gate1, float* out, int64_t ldo, int accumulate, cudaStream_t st, int rev = -1);

// cycle.cu
int cyc_rows_per_part(int n);
cudaError_t cyc_keys(int n, const float* A, int64_t lda, float* part, cudaStream_t st);
cudaError_t cyc_gather(int n, int k, const float* A, int64_t lda, const int32_t* sel, float* cyc,
                       unsigned char* insel, cudaStream_t st);
cudaError_t cyc_apply(int n, const float* A, int64_t lda, const float* B, int64_t ldb, const int32_t* selA, int ka,
                      const float* cycA, const unsigned char* inselA, const int32_t* selB, int kb, const float* cycB,
                      float* C, int64_t ldc, cudaStream_t st);

cudaError_t cyc_backward(int n, const float* A, int64_t lda, const float* B, int64_t ldb, const int32_t* selA, int ka,
                         const float* cycA, const unsigned char* inselA, const int32_t* selB, int kb,
                         const float* cycB, const unsigned char* inselB, const float* G, int64_t ldg, float* dA,
                         int64_t ldda, float* dB, int64_t lddb, cudaStream_t st);
// fourier.cu
cudaError_t ft_transform(int n, bool row, const float* X, int64_t ldx, int nvec, const float2* tw, float2* T,
                         float2* TT, float* mag, cudaStream_t st);
cudaError_t ft_select(int n, int k, int rows, const float* mag, int32_t* sel, uint32_t* maskT, int mask_words,
                      cudaStream_t st);
cudaError_t ft_product(int n, int m, int p, int k_a, int k_b, const float2* At, const float2* AtT,
                       const int32_t* selA, const uint32_t* maskT, int mask_words, const float2* Bt,
                       const int32_t* selB, float* C, int64_t ldc, cudaStream_t st);

// ft_backward.cu: dA and/or dB (either may be NULL) of the frozen Fourier-domain product.
struct FtBwArgs {
  int n, m, p, ka, kb;
  const float2* tw;      // e^{-2 pi i j/n}
  const float2* AtT;     // A~^T half spectrum [n/2+1][m]
  const int32_t* selA;   // [m][ka]
  const uint32_t* maskA; // [n][ceil(m/32)]
  const float2* Bt;      // B~ half spectrum [n/2+1][p]
  const int32_t* selB;   // [p][kb]
  const uint32_t* maskB; // [n][ceil(p/32)]
  const float* G;        // upstream gradient m x p
  int64_t ldg;
  float* dA;             // m x n
  int64_t ldda;
  float* dB;             // n x p
  int64_t lddb;
};
cudaError_t ft_backward(const FtBwArgs& a, cudaStream_t st);
// svd.cu: Y (FP32, ldy) = X (BF16, rows x cols, ldx)
cudaError_t widen_bf16(const void* X, int64_t rows, int64_t cols, int64_t ldx, float* Y, int64_t ldy,
                       cudaStream_t st);
// svd.cu: *out = sum of squares of X (FP64 accumulation), stream-ordered
cudaError_t sumsq_f32(const float* X, int64_t rows, int64_t cols, int64_t ld, double* out, cudaStream_t st);
// fourier.cu: out[0] = ||A||_F^2 (Parseval over the half spectrum), out[1] = the kept part
cudaError_t ft_norms(int n, int k, int nvec, const float* mag, const int32_t* sel, double* out, cudaStream_t st);
// svd.cu: Y (cols x rows, ldy) = X^T
cudaError_t transpose_f32(const float* X, int64_t rows, int64_t cols, int64_t ldx, float* Y, int64_t ldy,
                          cudaStream_t st);

// mixed-method pieces (cycle.cu, fourier.cu)
cudaError_t cyc_left_apply(int n, const int32_t* selA, int ka, const float* cycA, const float* X, int64_t ldx,
                           int64_t p, float* C, int64_t ldc, cudaStream_t st);
cudaError_t cyc_right_apply(int n, const int32_t* selB, int kb, const float* cycB, const float* Y, int64_t ldy,
                            int64_t m, float* C, int64_t ldc, cudaStream_t st);
cudaError_t cyc_residual(int n, const float* A, int64_t lda, const unsigned char* insel, float* D, int64_t ldd,
                         cudaStream_t st);
cudaError_t cyc_rt_apply(int n, const float* G, int64_t ldg, const int32_t* selB, int kb, const float* cycB,
                         float* out, int64_t ldo, cudaStream_t st);
cudaError_t cyc_lt_apply(int n, const float* G, int64_t ldg, const int32_t* selA, int ka, const float* cycA,
                         float* out, int64_t ldo, cudaStream_t st);
cudaError_t cyc_diag_project(int n, int len, const float* X, int64_t ldx, const float* Y, int64_t ldy,
                             const int32_t* sel, int k, float* out, int64_t ldo, cudaStream_t st);
cudaError_t ft_dense(int n, const float2* At, const int32_t* sel, int k, int m, const float2* tw, int part,
                     const float* A, int64_t lda, float* D, int64_t ldd, cudaStream_t st);
cudaError_t ft_left_apply(int n, int m, const float2* At, const int32_t* selA, int ka, const float2* tw,
                          const float* X, int64_t ldx, int p, float* C, int64_t ldc, cudaStream_t st);
cudaError_t ft_right_apply(int n, int p, const float2* Bt, const int32_t* selB, int kb, const float2* tw,
                           const float* Y, int64_t ldy, int m, bool imag, float* C, int64_t ldc, cudaStream_t st);
// ft_backward.cu, pieces of the mixed-method backward with a Fourier operand (D = B - Re B_s
// for part 0, Im B_s for part 1; sign_im multiplies the imaginary part Dim of the dense factor)
cudaError_t ft_right_dense(int n, int p, const float2* Bt, const int32_t* selB, int kb, const float2* tw, int part,
                           const float* B, int64_t ldb, float* D, int64_t ldd, cudaStream_t st);
cudaError_t ft_rt_apply_bw(int n, int m, int p, const float2* Bt, const uint32_t* maskB, int kb, const float2* tw,
                           const float* G, int64_t ldg, float* out, int64_t ldo, cudaStream_t st);
cudaError_t ft_lt_apply_bw(int n, int m, int p, const float2* AtT, const uint32_t* maskA, int ka, const float2* tw,
                           const float* G, int64_t ldg, float* out, int64_t ldo, cudaStream_t st);
cudaError_t ft_proj_left(int n, int m, int p, const int32_t* selA, const uint32_t* maskA, int ka, const float2* tw,
                         const float* G, int64_t ldg, const float* Dre, const float* Dim, int sign_im, int64_t ldd,
                         float* out, int64_t ldo, cudaStream_t st);
cudaError_t ft_proj_right(int n, int m, int p, const int32_t* selB, const uint32_t* maskB, int kb,
                          const float2* tw, const float* Dre, const float* Dim, int sign_im, int64_t ldd,
                          const float* G, int64_t ldg, float* out, int64_t ldo, cudaStream_t st);

// umma_gemm.cu: C = alpha A B^T + beta C on tcgen05 tensor cores (A, B K-major);
// tf32 = FP32 inputs with TF32 hi/lo splitting, else BF16 inputs.  err: device flag.
cudaError_t umma_gemm_tn(bool tf32, int M, int N, int K, float alpha, const void* A, int64_t lda, const void* B,
                         int64_t ldb, float beta, float* C, int64_t ldc, int* err, cudaStream_t st);

}  // namespace amm
