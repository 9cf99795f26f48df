// First-order product of two operands truncated by DIFFERENT methods (the paper allows the two
// decompositions to differ; Section 1 and Section 5).  With A~ from A's method and B~ from B's,
//
//   Re M = Re(A~ B + dA B~) = Re(A~) B + (A - Re A~) Re(B~) + Im(A~) Im(B~)
//
// (dA = A - A~, Im dA = -Im A~, A and B real).  Each term is one operand's truncation applied to
// a dense real matrix from the left or the right, so the product needs, per method, a left
// apply, a right apply, the dense real residual and, for the methods whose truncation can be
// complex (circulant with a split conjugate pair, the Fourier sparsifier), the dense imaginary
// part and the right apply of Im(B~).  SVD and cycle truncations are real: the last term then
// vanishes and is skipped.
//
// A circulant operand taken in square blocks (amm_opts_t.block) is evaluated on its zero-padded
// blocks: the product is formed on the padded shape (the other operand padded with zeros along
// the shared dimension, which leaves its truncation zero there as well) and cropped.
#include <cuda_runtime.h>

#include <vector>

#include "api_internal.h"
#include "kernels.h"
#include "trace.h"

namespace amm {

static bool can_be_complex(const Handle* h) {
  return h->method == AMM_CIRCULANT || h->method == AMM_SPARSE_FOURIER;
}

// C = Re(A~) X for X (n x p)
static cudaError_t left_apply(Handle* a, const float* X, int64_t ldx, int64_t p, float* C, int64_t ldc,
                              cudaStream_t st) {
  const int n = (int)a->cols;
  if (a->blk.b) return blocked_left_apply(a, X, ldx, p, C, ldc, st);
  switch (a->method) {
    case AMM_SVD:
      return svd_left_apply(a, X, ldx, p, C, ldc, 0.f, st);
    case AMM_CIRCULANT:
      return cd_apply(n, false, X, ldx, false, p, a->cd.tw, a->cd.so.ulist, a->cd.Lw, a->cd.so.counts, nullptr,
                      nullptr, C, ldc, 0, st);
    case AMM_SPARSE_CYCLE:
      return cyc_left_apply(n, a->cy.so.sel, (int)a->k, a->cy.cyc, X, ldx, p, C, ldc, st);
    case AMM_SPARSE_FOURIER:
      return ft_left_apply(n, (int)a->rows, a->ft.T, a->ft.sel, (int)a->k, a->ft.tw, X, ldx, (int)p, C, ldc, st);
  }
  return cudaErrorInvalidValue;
}

// C += Y Re(B~) for Y (m x n)
static cudaError_t right_apply(Handle* b, const float* Y, int64_t ldy, int64_t m, float* C, int64_t ldc,
                               cudaStream_t st) {
  const int n = (int)b->rows;
  if (b->blk.b) return blocked_right_apply(b, Y, ldy, m, false, C, ldc, st);
  switch (b->method) {
    case AMM_SVD:
      return svd_right_apply(b, Y, ldy, m, C, ldc, 1.f, st);
    case AMM_CIRCULANT:
      return cd_apply(n, true, Y, ldy, false, m, b->cd.tw, b->cd.so.ulist, b->cd.Lw, b->cd.so.counts, nullptr,
                      nullptr, C, ldc, 1, st);
    case AMM_SPARSE_CYCLE:
      return cyc_right_apply(n, b->cy.so.sel, (int)b->k, b->cy.cyc, Y, ldy, m, C, ldc, st);
    case AMM_SPARSE_FOURIER:
      return ft_right_apply(n, (int)b->cols, b->ft.T, b->ft.sel, (int)b->k, b->ft.tw, Y, ldy, (int)m, false, C, ldc,
                            st);
  }
  return cudaErrorInvalidValue;
}

// C += Y Im(B~) for Y (m x n); circulant: the unpaired coefficients -i v_s L_s, skipped on the
// device when B's selection has no unpaired component
static cudaError_t right_apply_imag(Handle* b, const float* Y, int64_t ldy, int64_t m, float* C, int64_t ldc,
                                    cudaStream_t st) {
  const int n = (int)b->rows;
  if (b->blk.b) return blocked_right_apply(b, Y, ldy, m, true, C, ldc, st);
  if (b->method == AMM_CIRCULANT)
    return cd_apply(n, true, Y, ldy, false, m, b->cd.tw, b->cd.so.dlist, b->cd.Ld, b->cd.so.counts + 1,
                    b->cd.so.counts + 1, b->cd.so.counts + 1, C, ldc, 1, st);
  if (b->method == AMM_SPARSE_FOURIER)
    return ft_right_apply(n, (int)b->cols, b->ft.T, b->ft.sel, (int)b->k, b->ft.tw, Y, ldy, (int)m, true, C, ldc, st);
  return cudaErrorInvalidValue;
}

// D = A - Re(A~), m x n
static cudaError_t residual(Handle* a, float* D, int64_t ldd, cudaStream_t st) {
  const int n = (int)a->cols;
  if (a->blk.b) return blocked_residual(a, false, D, ldd, st);
  switch (a->method) {
    case AMM_SVD:
      return svd_residual(a, D, ldd, st);
    case AMM_CIRCULANT: {
      const float2* R = nullptr;
      float2* temp = nullptr;
      cudaError_t e = cd_spectrum_of(a, &R, &temp, st);
      if (e == cudaSuccess) e = cd_residual(n, R, a->cd.tw, a->cd.so.wfull, 0, nullptr, D, st, ldd, 0);
      if (temp) dev_free(temp, st);
      return e;
    }
    case AMM_SPARSE_CYCLE:
      return cyc_residual(n, (const float*)a->A, a->lda, a->cy.insel, D, ldd, st);
    case AMM_SPARSE_FOURIER:
      return ft_dense(n, a->ft.T, a->ft.sel, (int)a->k, (int)a->rows, a->ft.tw, 0, (const float*)a->A, a->lda, D, ldd,
                      st);
  }
  return cudaErrorInvalidValue;
}

// D = Im(A~), m x n (zero for a circulant selection without unpaired components)
static cudaError_t imag_part(Handle* a, float* D, int64_t ldd, cudaStream_t st) {
  const int n = (int)a->cols;
  if (a->blk.b) return blocked_residual(a, true, D, ldd, st);
  if (a->method == AMM_CIRCULANT) {
    cudaError_t e = cudaMemset2DAsync(D, sizeof(float) * ldd, 0, sizeof(float) * n, n, st);
    if (e != cudaSuccess) return e;
    const float2* R = nullptr;
    float2* temp = nullptr;
    e = cd_spectrum_of(a, &R, &temp, st);
    if (e == cudaSuccess) e = cd_residual(n, R, a->cd.tw, a->cd.so.vfull, 1, a->cd.so.counts + 1, D, st, ldd, 0);
    if (temp) dev_free(temp, st);
    return e;
  }
  if (a->method == AMM_SPARSE_FOURIER)
    return ft_dense(n, a->ft.T, a->ft.sel, (int)a->k, (int)a->rows, a->ft.tw, 1, nullptr, 0, D, ldd, st);
  return cudaErrorInvalidValue;
}

amm_status_t mixed_matmul(Handle* a, Handle* b, float* C, int64_t ldc, cudaStream_t st) {
  const int64_t m = a->rows, n = a->cols, p = b->cols;
  if (a->dtype != AMM_F32 || b->dtype != AMM_F32)
    return fail(AMM_ERR_NOT_IMPLEMENTED, "mixed methods: BF16 operands are not built (use FP32 inputs)");
  // padded shape: whole blocks of a blocked circulant operand (at most one side is circulant)
  const int64_t mp = a->blk.b ? a->blk.nbr * a->blk.b : m;
  const int64_t np = a->blk.b ? a->blk.nbc * a->blk.b : b->blk.b ? b->blk.nbr * b->blk.b : n;
  const int64_t pp = b->blk.b ? b->blk.nbc * b->blk.b : p;
  std::vector<void*> tmp;
  cudaError_t e = cudaSuccess;
  auto al = [&](size_t elems) -> float* {
    void* q = nullptr;
    if (e == cudaSuccess) e = dev_alloc(&q, sizeof(float) * elems, st);
    if (q) tmp.push_back(q);
    return (float*)q;
  };
  // dense B with np rows: the blocked operand's padded copy, or B padded with zero rows
  const float* X = (const float*)(b->blk.b ? b->blk.base : b->A);
  int64_t ldx = b->blk.b ? b->blk.ld : b->lda;
  if (np != n && !b->blk.b) {
    float* t = al((size_t)np * p);
    if (e == cudaSuccess) e = cudaMemsetAsync(t, 0, sizeof(float) * (size_t)np * p, st);
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(t, sizeof(float) * p, X, sizeof(float) * ldx, sizeof(float) * p, n,
                            cudaMemcpyDeviceToDevice, st);
    X = t;
    ldx = p;
  }
  const bool crop = mp != m || pp != p;
  float* Cp = crop ? al((size_t)mp * pp) : C;
  const int64_t ldcp = crop ? pp : ldc;
  float* D = al((size_t)mp * np);
  // a residual of an unblocked operand covers m x n; the padding columns of D stay zero
  if (e == cudaSuccess && np != n && !a->blk.b) e = cudaMemsetAsync(D, 0, sizeof(float) * (size_t)mp * np, st);
  // C = Re(A~) B
  if (e == cudaSuccess) e = left_apply(a, X, ldx, pp, Cp, ldcp, st);
  // C += (A - Re A~) Re(B~)
  if (e == cudaSuccess) e = residual(a, D, np, st);
  if (e == cudaSuccess) e = right_apply(b, D, np, mp, Cp, ldcp, st);
  // C += Im(A~) Im(B~)
  if (e == cudaSuccess && can_be_complex(a) && can_be_complex(b)) {
    e = imag_part(a, D, np, st);
    if (e == cudaSuccess) e = right_apply_imag(b, D, np, mp, Cp, ldcp, st);
  }
  if (e == cudaSuccess && crop)
    e = cudaMemcpy2DAsync(C, sizeof(float) * ldc, Cp, sizeof(float) * ldcp, sizeof(float) * p, m,
                          cudaMemcpyDeviceToDevice, st);
  for (void* q : tmp) dev_free(q, st);
  if (e != cudaSuccess) return cuda_fail(e, "mixed-method product");
  return AMM_OK;
}

// ---------------------------------------------------------------------------- backward
// Gradients of <G, Re M> with the projectors frozen, each operand by its own method:
//   dA = Re(G B~^T) + Re P_A'(G dB^T),   dB = Re(A~^T G) + Re P_B'(dA^T G),
// P' the bilinear adjoint of the operand's projector (circulant: the mirrored components S-bar,
// whose real part on a real matrix is the w-weighted projection; SVD Q Q^T; cycles the kept cycles).
// dA, dB above are the residuals of the other operand, dB = Re dB - i Im B~ (Im B~ = 0 for SVD and
// cycles), and every projector is linear over the complex numbers, so
//   Re P_A'(G dB^T) = Re P_A'(G (Re dB)^T) + Im P_A'(G (Im B~)^T)
// (and likewise for dB).  The imaginary term is non-zero only when both truncations can be complex
// (a circulant with a split conjugate pair and a Fourier sparsifier).  Built for all pairs of the
// SVD, circulant, cycle and Fourier methods on square operands (m = n = p): the circulant
// projections run as SDDMMs on spectra of length n (the imaginary term over the unpaired
// components, gated on the device), the cycle projections as selected-diagonal dot products, the
// Fourier ones as sampled products on the transforms of the dense factor.

namespace {

struct Buf {
  cudaStream_t st;
  std::vector<void*> v;
  cudaError_t e = cudaSuccess;
  explicit Buf(cudaStream_t s) : st(s) {}
  template <typename T>
  T* get(size_t cnt) {
    void* q = nullptr;
    if (e == cudaSuccess) e = dev_alloc(&q, sizeof(T) * cnt, st);
    if (q) v.push_back(q);
    return (T*)q;
  }
  ~Buf() {
    for (void* q : v) dev_free(q, st);
  }
};

// out += Re P_{S-bar}(Z) (unpaired = false) or out -= Im P_S(Z) (unpaired = true: the unpaired
// components t with weight v_t, skipped on the device when there are none) for the circulant handle
// h and Z = X Y^T (row = false) or X^T Y (row = true), X and Y n x n: component spectra from the
// SDDMM on column / row spectra.  For real Z, P_{S-bar}(Z) = conj P_S(Z), so the second form is
// Re(-i P_{S-bar}(Z)).
cudaError_t cd_project_product(Handle* h, bool row, const float* X, int64_t ldx, const float* Y, int64_t ldy,
                               float* out, int64_t ldo, cudaStream_t st, bool unpaired = false) {
  const int n = (int)h->rows;
  const size_t kh = (size_t)n / 2 + 1;
  auto& c = h->cd;
  Buf b(st);
  float2* X1 = b.get<float2>(kh * n);
  float2* X2 = b.get<float2>(kh * n);
  float2* RX = b.get<float2>(kh * n);
  float2* K = b.get<float2>((size_t)c.cap * n);
  const int32_t* list = unpaired ? c.so.dlist : c.so.ulist;
  const int32_t* count = unpaired ? c.so.counts + 1 : c.so.counts;
  // the gated kernels read both gates whenever the first is given: pass the unpaired count twice
  const int32_t* gate = unpaired ? c.so.counts + 1 : nullptr;
  if (b.e == cudaSuccess) b.e = bw_spectrum(n, row, X, ldx, c.tw, X1, st, gate, gate);
  if (b.e == cudaSuccess) b.e = bw_spectrum(n, row, Y, ldy, c.tw, X2, st, gate, gate);
  if (b.e == cudaSuccess) b.e = cd_sddmm(n, X1, X2, list, count, c.cap, K, gate, gate, st);
  if (b.e == cudaSuccess) b.e = cd_rho(n, K, c.tw, list, count, c.cap, RX, gate, gate, st);
  if (b.e == cudaSuccess)
    b.e = unpaired ? cd_residual(n, RX, c.tw, c.so.vfull, 3, count, out, st, ldo, 1)
                   : cd_residual(n, RX, c.tw, c.so.wfull, 2, nullptr, out, st, ldo, 1);
  return b.e;
}

bool aligned16(const float* p, int64_t ld) { return ((uintptr_t)p & 15) == 0 && (ld & 3) == 0; }

// D = B - Re(B~) / Im(B~) of the right operand b, n x p (a right Fourier handle holds column
// transforms; the other methods' truncations do not depend on the side)
cudaError_t right_dense(Handle* b, bool imag, float* D, int64_t ldd, cudaStream_t st) {
  if (b->method == AMM_SPARSE_FOURIER)
    return ft_right_dense(b->ft.n, (int)b->cols, b->ft.T, b->ft.sel, (int)b->k, b->ft.tw, imag ? 1 : 0,
                          (const float*)b->A, b->lda, D, ldd, st);
  return imag ? imag_part(b, D, ldd, st) : residual(b, D, ldd, st);
}

}  // namespace

amm_status_t mixed_backward_blocked(Handle* a, Handle* b, const float* G, int64_t ldg, float* dA, int64_t ldda,
                                    float* dB, int64_t lddb, cudaStream_t st);

amm_status_t mixed_backward(Handle* a, Handle* b, const float* G, int64_t ldg, float* dA, int64_t ldda, float* dB,
                            int64_t lddb, cudaStream_t st) {
  const int64_t m = a->rows, n = a->cols, p = b->cols;
  if (a->blk.b || b->blk.b) return mixed_backward_blocked(a, b, G, ldg, dA, ldda, dB, lddb, st);
  if (m != n || p != n)
    return fail(AMM_ERR_UNSUPPORTED_SIZE, "backward of a mixed-method product needs square operands (%lldx%lld, "
                "%lldx%lld)", (long long)m, (long long)n, (long long)n, (long long)p);
  if (a->dtype != AMM_F32 || b->dtype != AMM_F32)
    return fail(AMM_ERR_NOT_IMPLEMENTED, "mixed methods: BF16 operands are not built (use FP32 inputs)");
  const int nn = (int)n;
  Buf buf(st);
  // the imaginary parts enter only when both truncations can be complex
  const bool cplx = can_be_complex(a) && can_be_complex(b);
  float* DA = dB ? buf.get<float>((size_t)nn * nn) : nullptr;  // Re dA = A - Re A~
  float* DB = dA ? buf.get<float>((size_t)nn * nn) : nullptr;  // Re dB = B - Re B~
  float* IA = dB && cplx ? buf.get<float>((size_t)nn * nn) : nullptr;  // Im A~
  float* IB = dA && cplx ? buf.get<float>((size_t)nn * nn) : nullptr;  // Im B~
  cudaError_t e = buf.e;
  if (e == cudaSuccess && DA) e = residual(a, DA, nn, st);
  if (e == cudaSuccess && DB) e = right_dense(b, false, DB, nn, st);
  if (e == cudaSuccess && IA) e = imag_part(a, IA, nn, st);
  if (e == cudaSuccess && IB) e = right_dense(b, true, IB, nn, st);
  // an aligned copy of G for the cycle projections (float4 rows)
  const float* Ga = G;
  int64_t ldga = ldg;
  if (e == cudaSuccess && (a->method == AMM_SPARSE_CYCLE || b->method == AMM_SPARSE_CYCLE) && !aligned16(G, ldg)) {
    float* t = buf.get<float>((size_t)nn * nn);
    e = buf.e;
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(t, sizeof(float) * nn, G, sizeof(float) * ldg, sizeof(float) * nn, nn,
                            cudaMemcpyDeviceToDevice, st);
    Ga = t;
    ldga = nn;
  }
  if (dA && e == cudaSuccess) {
    // Re(G B~^T)
    switch (b->method) {
      case AMM_SVD: e = svd_rt_apply(b, G, ldg, nn, dA, ldda, st); break;
      case AMM_CIRCULANT:
        e = cd_apply(nn, true, G, ldg, false, nn, b->cd.tw, b->cd.so.ulist, b->cd.Lw, b->cd.so.counts, nullptr,
                     nullptr, dA, ldda, 0, st, 0);
        break;
      case AMM_SPARSE_FOURIER:
        e = ft_rt_apply_bw(nn, nn, nn, b->ft.T, b->ft.maskT, (int)b->k, b->ft.tw, G, ldg, dA, ldda, st);
        break;
      default: e = cyc_rt_apply(nn, G, ldg, b->cy.so.sel, (int)b->k, b->cy.cyc, dA, ldda, st); break;
    }
    // + Re P_A'(G dB^T) = Re P_A'(G (Re dB)^T) + Im P_A'(G (Im B~)^T)
    if (e == cudaSuccess) {
      switch (a->method) {
        case AMM_SVD: e = svd_proj_left(a, G, ldg, DB, nn, nn, dA, ldda, st); break;
        case AMM_CIRCULANT:
          e = cd_project_product(a, false, G, ldg, DB, nn, dA, ldda, st);
          if (e == cudaSuccess && IB) e = cd_project_product(a, false, G, ldg, IB, nn, dA, ldda, st, true);
          break;
        case AMM_SPARSE_FOURIER:
          e = ft_proj_left(nn, nn, nn, a->ft.sel, a->ft.maskT, (int)a->k, a->ft.tw, G, ldg, DB, IB, -1, nn, dA, ldda,
                           st);
          break;
        default: e = cyc_diag_project(nn, nn, Ga, ldga, DB, nn, a->cy.so.sel, (int)a->k, dA, ldda, st); break;
      }
    }
  }
  if (dB && e == cudaSuccess) {
    // Re(A~^T G)
    switch (a->method) {
      case AMM_SVD: e = svd_lt_apply(a, G, ldg, nn, dB, lddb, st); break;
      case AMM_CIRCULANT:
        e = cd_apply(nn, false, G, ldg, false, nn, a->cd.tw, a->cd.so.ulist, a->cd.Lw, a->cd.so.counts, nullptr,
                     nullptr, dB, lddb, 0, st, 1);
        break;
      case AMM_SPARSE_FOURIER:
        e = ft_lt_apply_bw(nn, nn, nn, a->ft.TT, a->ft.maskT, (int)a->k, a->ft.tw, G, ldg, dB, lddb, st);
        break;
      default: e = cyc_lt_apply(nn, G, ldg, a->cy.so.sel, (int)a->k, a->cy.cyc, dB, lddb, st); break;
    }
    // + Re P_B'(dA^T G) = Re P_B'((Re dA)^T G) + Im P_B'((Im A~)^T G)
    if (e == cudaSuccess) {
      switch (b->method) {
        case AMM_SVD: e = svd_proj_right(b, DA, nn, G, ldg, nn, dB, lddb, st); break;
        case AMM_CIRCULANT:
          e = cd_project_product(b, true, DA, nn, G, ldg, dB, lddb, st);
          if (e == cudaSuccess && IA) e = cd_project_product(b, true, IA, nn, G, ldg, dB, lddb, st, true);
          break;
        case AMM_SPARSE_FOURIER:
          e = ft_proj_right(nn, nn, nn, b->ft.sel, b->ft.maskT, (int)b->k, b->ft.tw, DA, IA, -1, nn, G, ldg, dB, lddb,
                            st);
          break;
        default: {
          // (dA^T G)((l + s), l) = <dA^T(l + s, :), G^T(l, :)>
          float* DAT = buf.get<float>((size_t)nn * nn);
          float* GT = buf.get<float>((size_t)nn * nn);
          e = buf.e;
          if (e == cudaSuccess) e = transpose_f32(DA, nn, nn, nn, DAT, nn, st);
          if (e == cudaSuccess) e = transpose_f32(G, nn, nn, ldg, GT, nn, st);
          if (e == cudaSuccess) e = cyc_diag_project(nn, nn, DAT, nn, GT, nn, b->cy.so.sel, (int)b->k, dB, lddb, st);
        }
      }
    }
  }
  if (e != cudaSuccess) return cuda_fail(e, "mixed-method backward");
  return AMM_OK;
}

// ---------------------------------------------------------------------------- refinement
// Section 2.5: when Re M is not accurate enough, the residue product is approximated by the same
// first-order approach and added.  For real A, B,
//   Re(dA dB) = Re dA Re dB - Im dA Im dB = Re dA Re dB - Im(A~) Im(B~),
// the first term by the first-order product of decompositions of Re dA and Re dB (handles a2, b2,
// made by the caller from amm_handle_residual), the second exactly (non-zero only when both
// truncations can be complex).

namespace {

// C += T - U (U may be NULL), rows x cols
__global__ void __launch_bounds__(256) add_diff_kernel(float* __restrict__ C, int64_t ldc, const float* __restrict__ T,
                                                       int64_t ldt, const float* __restrict__ U, int64_t ldu,
                                                       int64_t rows, int64_t cols) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= rows * cols) return;
  const int64_t r = e / cols, c = e - r * cols;
  float v = T[r * ldt + c];
  if (U != nullptr) v -= U[r * ldu + c];
  C[r * ldc + c] += v;
}

amm_status_t refinable(const Handle* h, const char* what) {
  if (h->dtype != AMM_F32)
    return fail(AMM_ERR_NOT_IMPLEMENTED, "%s: BF16 operands are not built (use FP32 inputs)", what);
  if (h->blk.b) return fail(AMM_ERR_NOT_IMPLEMENTED, "%s: circulant blocks are not built", what);
  return AMM_OK;
}

}  // namespace

amm_status_t handle_residual(Handle* h, float* D, int64_t ldd, cudaStream_t st) {
  amm_status_t s = refinable(h, "amm_handle_residual");
  if (s != AMM_OK) return s;
  const int64_t m = h->rows, n = h->cols;
  Buf buf(st);
  float* T = buf.get<float>((size_t)m * n);  // the pieces write a dense m x n scratch, copied out
  cudaError_t e = buf.e;
  if (e == cudaSuccess) e = h->role == AMM_LEFT ? residual(h, T, n, st) : right_dense(h, false, T, n, st);
  if (e == cudaSuccess)
    e = cudaMemcpy2DAsync(D, sizeof(float) * ldd, T, sizeof(float) * n, sizeof(float) * n, m,
                          cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e, "amm_handle_residual");
  return AMM_OK;
}

amm_status_t refine_product(Handle* a, Handle* b, Handle* a2, Handle* b2, float* C, int64_t ldc, cudaStream_t st) {
  amm_status_t s;
  if ((s = refinable(a, "amm_refine_product")) != AMM_OK || (s = refinable(b, "amm_refine_product")) != AMM_OK)
    return s;
  const int64_t m = a->rows, n = a->cols, p = b->cols;
  const bool im = can_be_complex(a) && can_be_complex(b);
  Buf buf(st);
  float* T = buf.get<float>((size_t)m * p);
  float* U = im ? buf.get<float>((size_t)m * p) : nullptr;
  float* I = im ? buf.get<float>((size_t)m * n) : nullptr;
  if (buf.e != cudaSuccess) return cuda_fail(buf.e, "amm_refine_product: scratch");
  // T = Re M2, the first-order product of the residues' decompositions
  if ((s = amm_approx_matmul(a2, b2, T, p, st)) != AMM_OK) return s;
  cudaError_t e = cudaSuccess;
  if (im) {  // U = Im(A~) Im(B~)
    e = cudaMemsetAsync(U, 0, sizeof(float) * (size_t)m * p, st);
    if (e == cudaSuccess) e = imag_part(a, I, n, st);
    if (e == cudaSuccess) e = right_apply_imag(b, I, n, m, U, p, st);
  }
  if (e == cudaSuccess) {
    AMM_TRACE_W("refine_add", st, 0.0, 4.0 * (double)m * p * (im ? 4 : 3), nullptr);
    const int64_t total = m * p;
    add_diff_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(C, ldc, T, p, U, p, m, p);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return cuda_fail(e, "amm_refine_product");
  return AMM_OK;
}

// ---------------------------------------------------------------------------- backward with blocks
// One operand a blockwise circulant truncation (b x b blocks of its zero-padded copy), the other
// truncated by another method.  As in the product, M is formed on the padded shape and cropped,
// so with G_p = G padded with zeros and the unblocked operand padded with zeros along the inner
// dimension (its truncation and residual are zero there):
//   dA = crop Re[G_p B~_p^T + P_A'(G_p dB_p^T)],   dB = crop Re[A~_p^T G_p + P_B'(dA_p^T G_p)].
// The blocked operand's terms run block by block on the square kernels with every inner sum cut
// into b-wide pieces (block IJ of G_p dB_p^T is sum_L G_IL dB_JL^T); the other operand's terms are
// its pieces of the unblocked mixed backward on the cropped factors (dA_p^T G_p cropped to n x p
// is dA^T G over the first m rows, the padded rows of G_p being zero).  Im B~ (Im A~) enters the
// blocked projection only beside a Fourier operand, whose truncation is complex; the SVD and cycle
// projectors are real, so their imaginary terms vanish.
amm_status_t mixed_backward_blocked(Handle* a, Handle* b, const float* G, int64_t ldg, float* dA, int64_t ldda,
                                    float* dB, int64_t lddb, cudaStream_t st) {
  const int64_t m = a->rows, n = a->cols, p = b->cols;
  const bool left = a->blk.b != 0;  // the blocked circulant is A (else B)
  Handle* c = left ? a : b;
  Handle* o = left ? b : a;
  if (a->dtype != AMM_F32 || b->dtype != AMM_F32)
    return fail(AMM_ERR_NOT_IMPLEMENTED, "mixed methods: BF16 operands are not built (use FP32 inputs)");
  if (o->method == AMM_SPARSE_CYCLE && (m != n || n != p))
    return fail(AMM_ERR_UNSUPPORTED_SIZE, "backward of a blocked circulant x cycle product needs square operands "
                "(%lldx%lld, %lldx%lld)", (long long)m, (long long)n, (long long)n, (long long)p);
  const int64_t bs = c->blk.b;
  const int bsi = (int)bs;
  const int64_t mq = (m + bs - 1) / bs * bs, nq = (n + bs - 1) / bs * bs, pq = (p + bs - 1) / bs * bs;
  auto sub = [&](int64_t i, int64_t j) { return (Handle*)c->blk.sub[(size_t)(i * c->blk.nbc + j)]; };
  const bool cplx = o->method == AMM_SPARSE_FOURIER;
  Buf buf(st);
#define STEP(x) \
  if (buf.e == cudaSuccess) buf.e = (x)
  auto zeros = [&](int64_t r, int64_t cols) {
    float* q = buf.get<float>((size_t)(r * cols));
    STEP(cudaMemsetAsync(q, 0, sizeof(float) * (size_t)(r * cols), st));
    return q;
  };
  auto put = [&](float* dst, int64_t ldd, const float* src, int64_t lds, int64_t r, int64_t cols) {
    STEP(cudaMemcpy2DAsync(dst, sizeof(float) * ldd, src, sizeof(float) * lds, sizeof(float) * cols, r,
                           cudaMemcpyDeviceToDevice, st));
  };
  float* Gq = zeros(mq, pq);  // G_p, rows and columns cut into b-wide pieces
  put(Gq, pq, G, ldg, m, p);
  if (left) {
    const int64_t nbr = c->blk.nbr, nbc = c->blk.nbc, nbl = pq / bs;
    if (dA) {
      float* DBq = zeros(nq, pq);                  // Re dB in the n x p corner
      float* IBq = cplx ? zeros(nq, pq) : nullptr;  // Im B~
      float* Dq = zeros(mq, nq);                   // dA on the padded shape
      STEP(right_dense(b, false, DBq, pq, st));
      if (IBq) STEP(right_dense(b, true, IBq, pq, st));
      switch (b->method) {  // Re(G B~^T), the m x n corner
        case AMM_SVD: STEP(svd_rt_apply(b, G, ldg, m, Dq, nq, st)); break;
        case AMM_SPARSE_FOURIER:
          STEP(ft_rt_apply_bw((int)n, (int)m, (int)p, b->ft.T, b->ft.maskT, (int)b->k, b->ft.tw, G, ldg, Dq, nq, st));
          break;
        default: STEP(cyc_rt_apply((int)n, G, ldg, b->cy.so.sel, (int)b->k, b->cy.cyc, Dq, nq, st)); break;
      }
      for (int64_t i = 0; i < nbr; ++i)
        for (int64_t j = 0; j < nbc; ++j)
          for (int64_t l = 0; l < nbl; ++l) {
            const float* Gil = Gq + i * bs * pq + l * bs;
            float* Dij = Dq + i * bs * nq + j * bs;
            STEP(cd_project_product(sub(i, j), false, Gil, pq, DBq + j * bs * pq + l * bs, pq, Dij, nq, st));
            if (IBq)
              STEP(cd_project_product(sub(i, j), false, Gil, pq, IBq + j * bs * pq + l * bs, pq, Dij, nq, st, true));
          }
      put(dA, ldda, Dq, nq, m, n);
    }
    if (dB) {
      float* Eq = zeros(nq, pq);  // Re(A~_p^T G_p), block column j = sum_i A~_ij^T G_i
      for (int64_t j = 0; j < nbc; ++j)
        for (int64_t i = 0; i < nbr; ++i) {
          const Handle* s = sub(i, j);
          STEP(cd_apply(bsi, false, Gq + i * bs * pq, pq, false, pq, s->cd.tw, s->cd.so.ulist, s->cd.Lw,
                        s->cd.so.counts, nullptr, nullptr, Eq + j * bs * pq, pq, i > 0, st, 1));
        }
      put(dB, lddb, Eq, pq, n, p);
      float* DAq = buf.get<float>((size_t)(mq * nq));               // Re dA_p
      float* IAq = cplx ? buf.get<float>((size_t)(mq * nq)) : nullptr;  // Im A~_p
      STEP(blocked_residual(a, false, DAq, nq, st));
      if (IAq) STEP(blocked_residual(a, true, IAq, nq, st));
      switch (b->method) {  // + Re P_B'(dA^T G) over the first m rows and n columns
        case AMM_SVD: STEP(svd_proj_right(b, DAq, nq, G, ldg, m, dB, lddb, st)); break;
        case AMM_SPARSE_FOURIER:
          STEP(ft_proj_right((int)n, (int)m, (int)p, b->ft.sel, b->ft.maskT, (int)b->k, b->ft.tw, DAq, IAq, -1, nq,
                             G, ldg, dB, lddb, st));
          break;
        default: {  // square: the selected diagonals of dA^T G
          float* DAT = buf.get<float>((size_t)(n * n));
          float* GT = buf.get<float>((size_t)(n * n));
          STEP(transpose_f32(DAq, n, n, nq, DAT, n, st));
          STEP(transpose_f32(G, n, n, ldg, GT, n, st));
          STEP(cyc_diag_project((int)n, (int)n, DAT, n, GT, n, b->cy.so.sel, (int)b->k, dB, lddb, st));
        }
      }
    }
  } else {
    const int64_t nbr = c->blk.nbr, nbc = c->blk.nbc, nbi = mq / bs;
    if (dA) {
      float* Dq = zeros(m, nq);  // Re(G_p B~_p^T), block column j = sum_l G_l B~_jl^T
      for (int64_t j = 0; j < nbr; ++j)
        for (int64_t l = 0; l < nbc; ++l) {
          const Handle* s = sub(j, l);
          STEP(cd_apply(bsi, true, Gq + l * bs, pq, false, m, s->cd.tw, s->cd.so.ulist, s->cd.Lw, s->cd.so.counts,
                        nullptr, nullptr, Dq + j * bs, nq, l > 0, st, 0));
        }
      put(dA, ldda, Dq, nq, m, n);
      float* DBq = buf.get<float>((size_t)(nq * pq));               // Re dB_p
      float* IBq = cplx ? buf.get<float>((size_t)(nq * pq)) : nullptr;  // Im B~_p
      STEP(blocked_residual(b, false, DBq, pq, st));
      if (IBq) STEP(blocked_residual(b, true, IBq, pq, st));
      switch (a->method) {  // + Re P_A'(G dB^T) over the first n rows and p columns
        case AMM_SVD: STEP(svd_proj_left(a, G, ldg, DBq, pq, p, dA, ldda, st)); break;
        case AMM_SPARSE_FOURIER:
          STEP(ft_proj_left((int)n, (int)m, (int)p, a->ft.sel, a->ft.maskT, (int)a->k, a->ft.tw, G, ldg, DBq, IBq, -1,
                            pq, dA, ldda, st));
          break;
        default:  // square: the selected diagonals of G dB^T (rows of Gq and DBq are 16-byte aligned)
          STEP(cyc_diag_project((int)n, (int)n, Gq, pq, DBq, pq, a->cy.so.sel, (int)a->k, dA, ldda, st));
          break;
      }
    }
    if (dB) {
      switch (a->method) {  // Re(A~^T G)
        case AMM_SVD: STEP(svd_lt_apply(a, G, ldg, p, dB, lddb, st)); break;
        case AMM_SPARSE_FOURIER:
          STEP(ft_lt_apply_bw((int)n, (int)m, (int)p, a->ft.TT, a->ft.maskT, (int)a->k, a->ft.tw, G, ldg, dB, lddb,
                              st));
          break;
        default: STEP(cyc_lt_apply((int)n, G, ldg, a->cy.so.sel, (int)a->k, a->cy.cyc, dB, lddb, st)); break;
      }
      float* DAq = zeros(mq, nq);                  // Re dA in the m x n corner
      float* IAq = cplx ? zeros(mq, nq) : nullptr;  // Im A~
      STEP(residual(a, DAq, nq, st));
      if (IAq) STEP(imag_part(a, IAq, nq, st));
      float* Eq = zeros(nq, pq);  // Re P_B'(dA_p^T G_p), block jl = sum_i P_jl'(dA_ij^T G_il)
      for (int64_t j = 0; j < nbr; ++j)
        for (int64_t l = 0; l < nbc; ++l)
          for (int64_t i = 0; i < nbi; ++i) {
            const float* Gil = Gq + i * bs * pq + l * bs;
            float* Ejl = Eq + j * bs * pq + l * bs;
            STEP(cd_project_product(sub(j, l), true, DAq + i * bs * nq + j * bs, nq, Gil, pq, Ejl, pq, st));
            if (IAq)
              STEP(cd_project_product(sub(j, l), true, IAq + i * bs * nq + j * bs, nq, Gil, pq, Ejl, pq, st, true));
          }
      if (buf.e == cudaSuccess) {
        add_diff_kernel<<<(unsigned)((n * p + 255) / 256), 256, 0, st>>>(dB, lddb, Eq, pq, nullptr, 0, n, p);
        buf.e = cudaGetLastError();
      }
    }
  }
#undef STEP
  if (buf.e != cudaSuccess) return cuda_fail(buf.e, "mixed-method backward with circulant blocks");
  return AMM_OK;
}

}  // namespace amm
