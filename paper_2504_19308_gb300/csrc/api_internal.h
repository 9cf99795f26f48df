// Handle layout and helpers shared by the C ABI implementation files.
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/amm.h"
#include "kernels.h"

struct amm_handle {
  // what was decomposed (borrowed pointer, see amm_decompose)
  const void* A = nullptr;
  int64_t rows = 0, cols = 0, lda = 0, k = 0;
  int dtype = AMM_F32, method = AMM_CIRCULANT, role = AMM_LEFT, compute = AMM_F32;
  cudaStream_t stream = nullptr;
  std::vector<void*> owned;  // device buffers released by amm_handle_destroy
  std::vector<size_t> owned_bytes;  // their sizes

  struct Circulant {
    const float2* tw = nullptr;   // twiddle table (process-wide cache, not owned)
    float2* R = nullptr;          // (n/2+1) x n half spectrum
    float* kpart = nullptr;       // per-CTA key partials
    int nparts = 0, cap = 0;      // cap = min(2k, n) rows of Lw / Ld
    amm::SelectOut so{};
    float2* Lw = nullptr;         // w_t L_t for t in S u S-bar
    float2* Ld = nullptr;         // -i v_t L_t for unpaired t
    float* resid = nullptr;       // right operand: dB_w (n x n)
    float* imag = nullptr;        // right operand: Im B~_S (n x n)
  } cd;

  struct Cycle {
    float* kpart = nullptr;       // per row-block partial cycle norms
    int nparts = 0;
    amm::SelectOut so{};
    float* cyc = nullptr;         // k x n, the selected cycles Lambda_t
    unsigned char* insel = nullptr;  // n flags
  } cy;

  struct Fourier {
    const float2* tw = nullptr;
    int n = 0, nvec = 0, mask_words = 0;  // transform length, rows (left) / columns (right)
    float2* T = nullptr;          // left: A~ [m][n/2+1]; right: B~ [n/2+1][p]
    float2* TT = nullptr;         // left: A~^T [n/2+1][m]
    float* mag = nullptr;         // [nvec][n/2+1] |.|^2
    int32_t* sel = nullptr;       // [nvec][k] kept frequencies, ascending
    uint32_t* maskT = nullptr;    // [n][ceil(nvec/32)] kept-entry bits (frequency-major)
  } ft;

  struct Svd {
    float* phi = nullptr;    // cols x k test matrix
    float* Q = nullptr;      // rows x k, orthonormal columns spanning A phi
    float* X = nullptr;      // k x cols, Q^T A
    double* norms = nullptr; // ||A||_F^2, ||X||_F^2
    // K-major copies in the compute type E of the tensor-core GEMMs (FP32 for TF32X3, BF16)
    bool bf16 = false;
    const void* Xe = nullptr;  // rows x cols (the input itself when it already fits)
    int64_t ldxe = 0;
    void *XTe = nullptr, *Qe = nullptr, *QTe = nullptr, *Ze = nullptr, *ZTe = nullptr;
    int* err = nullptr;        // device flag: a bounded wait of a tensor-core kernel gave up
  } svd;

  // rectangular circulant operand in b x b blocks (amm_opts_t.block): every block is a square
  // circulant handle of its own; the ragged edge is read from a zero-padded copy
  struct Blocks {
    int64_t b = 0;                    // block size; 0 = one square decomposition (no blocks)
    int64_t nbr = 0, nbc = 0;         // block rows / columns
    const void* base = nullptr;       // padded operand (or A itself), nbr*b x nbc*b
    int64_t ld = 0;                   // its leading dimension
    std::vector<amm_handle*> sub;     // nbr x nbc, row-major; owned
  } blk;

  void release();
  cudaError_t alloc(void** p, size_t bytes);
  void release_one(void* p);   // one owned buffer, stream-ordered
  int64_t device_bytes() const;  // bytes of the owned buffers (blocks included)
};

namespace amm {
using Handle = ::amm_handle;

amm_status_t fail(amm_status_t s, const char* fmt, ...);
// circulant transform lengths: 2^a in [16, 16384] or 3 * 2^a in [48, 6144]
bool cd_length_ok(int64_t n);      // the circulant method: fixed FFT lengths or any n in [16, 4096]
bool cd_fft_length_ok(int64_t n);  // the fixed lengths 2^a in [16, 16384], 3 * 2^a in [48, 6144]
// circulant.cu: the spectral-apply autotuner's table as text, and its parser (false: malformed)
std::string cd_tune_dump();
bool cd_tune_load(const char* text, bool (*length_ok)(int64_t));
// cycle-sparsifier lengths: multiples of 4 in [16, 8192]
bool cyc_length_ok(int64_t n);
// amm_set_autotune: kernel variants are timed on first use and the fastest kept
bool amm_autotune_enabled();
amm_status_t cuda_fail(cudaError_t e, const char* what);
cudaError_t dev_alloc(void** p, size_t bytes, cudaStream_t st);
void dev_free(void* p, cudaStream_t st);
cudaError_t twiddles(int n, cudaStream_t st, const float2** out);
// The half spectrum of a square circulant handle: its stored R, or (store_spectra = 0) R computed
// again from the borrowed operand into *temp, which the caller releases with dev_free.
cudaError_t cd_spectrum_of(Handle* h, const float2** R, float2** temp, cudaStream_t st);

// svd.cu
amm_status_t decompose_svd(Handle* h, const amm_opts_t* o);
amm_status_t svd_matmul(Handle* a, Handle* b, float* C, int64_t ldc, cudaStream_t st);
amm_status_t svd_backward(Handle* a, Handle* b, const float* G, int64_t ldg, float* dA, int64_t ldda, float* dB,
                          int64_t lddb, cudaStream_t st);
amm_status_t svd_info(Handle* h, amm_info_t* info);
cudaError_t svd_left_apply(Handle* a, const float* X, int64_t ldx, int64_t p, float* C, int64_t ldc, float beta,
                           cudaStream_t st);
cudaError_t svd_right_apply(Handle* b, const float* Y, int64_t ldy, int64_t m, float* C, int64_t ldc, float beta,
                            cudaStream_t st);
cudaError_t svd_residual(Handle* a, float* D, int64_t ldd, cudaStream_t st);
// mixed-method backward pieces: out = G B~^T (m x n); out = A~^T G (n x p); out += Q_A Q_A^T (G D^T);
// out += Q_B Q_B^T (D^T G)
cudaError_t svd_rt_apply(Handle* b, const float* G, int64_t ldg, int64_t m, float* out, int64_t ldo, cudaStream_t st);
cudaError_t svd_lt_apply(Handle* a, const float* G, int64_t ldg, int64_t p, float* out, int64_t ldo, cudaStream_t st);
cudaError_t svd_proj_left(Handle* a, const float* G, int64_t ldg, const float* D, int64_t ldd, int64_t p, float* out,
                          int64_t ldo, cudaStream_t st);
cudaError_t svd_proj_right(Handle* b, const float* D, int64_t ldd, const float* G, int64_t ldg, int64_t m, float* out,
                           int64_t ldo, cudaStream_t st);
amm_status_t mixed_backward(Handle* a, Handle* b, const float* G, int64_t ldg, float* dA, int64_t ldda, float* dB,
                            int64_t lddb, cudaStream_t st);
// api.cu: one square circulant block pair; acc = 1 adds to C / dA / dB instead of overwriting
amm_status_t decompose_circulant(Handle* h, const amm_opts_t* o);
cudaError_t cd_first_order(Handle* a, Handle* b, float* C, int64_t ldc, int acc, cudaStream_t st);
amm_status_t cd_backward(Handle* a, Handle* b, const float* G, int64_t ldg, float* dA, int64_t ldda, int acc_a,
                         float* dB, int64_t lddb, int acc_b, cudaStream_t st);
// blocked.cu
amm_status_t decompose_circulant_blocked(Handle* h, const amm_opts_t* o);
amm_status_t blocked_matmul(Handle* a, Handle* b, float* C, int64_t ldc, cudaStream_t st);
amm_status_t blocked_backward(Handle* a, Handle* b, const float* G, int64_t ldg, float* dA, int64_t ldda, float* dB,
                              int64_t lddb, cudaStream_t st);
amm_status_t blocked_info(Handle* h, amm_info_t* info);
amm_status_t blocked_selection(Handle* h, int32_t* host_idx, int64_t cap, int64_t* count);
// the blockwise pieces of a mixed-method product (C, D padded to whole blocks)
cudaError_t blocked_left_apply(Handle* a, const float* X, int64_t ldx, int64_t p, float* C, int64_t ldc,
                               cudaStream_t st);
cudaError_t blocked_right_apply(Handle* b, const float* Y, int64_t ldy, int64_t m, bool imag, float* C,
                                int64_t ldc, cudaStream_t st);
cudaError_t blocked_residual(Handle* a, bool imag, float* D, int64_t ldd, cudaStream_t st);
// mixed.cu
amm_status_t mixed_matmul(Handle* a, Handle* b, float* C, int64_t ldc, cudaStream_t st);
// D = Re dA (rows x cols, ldd); C += Re M2 - Im(A~) Im(B~) with a2, b2 decompositions of Re dA, Re dB
amm_status_t handle_residual(Handle* h, float* D, int64_t ldd, cudaStream_t st);
amm_status_t refine_product(Handle* a, Handle* b, Handle* a2, Handle* b2, float* C, int64_t ldc, cudaStream_t st);

amm_status_t svd_get_sketch(Handle* h, float* host_phi, int64_t cap);
}  // namespace amm
