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
// dA, dB above are the dense real residuals of the other operand.  Built for the SVD, circulant and
// cycle methods on square operands (m = n = p): the circulant projections run as SDDMMs on
// spectra of length n, the cycle projections as selected-diagonal dot products.

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

// out += Re P_{S-bar}(X Y^T) (row = false) or Re P_{S-bar}(X^T Y) (row = true) for the circulant
// handle h, X and Y n x n: component spectra from the SDDMM on column / row spectra
cudaError_t cd_project_product(Handle* h, bool row, const float* X, int64_t ldx, const float* Y, int64_t ldy,
                               float* out, int64_t ldo, cudaStream_t st) {
  const int n = (int)h->rows;
  const size_t kh = (size_t)n / 2 + 1;
  auto& c = h->cd;
  Buf b(st);
  float2* X1 = b.get<float2>(kh * n);
  float2* X2 = b.get<float2>(kh * n);
  float2* RX = b.get<float2>(kh * n);
  float2* K = b.get<float2>((size_t)c.cap * n);
  if (b.e == cudaSuccess) b.e = bw_spectrum(n, row, X, ldx, c.tw, X1, st);
  if (b.e == cudaSuccess) b.e = bw_spectrum(n, row, Y, ldy, c.tw, X2, st);
  if (b.e == cudaSuccess) b.e = cd_sddmm(n, X1, X2, c.so.ulist, c.so.counts, c.cap, K, nullptr, nullptr, st);
  if (b.e == cudaSuccess) b.e = cd_rho(n, K, c.tw, c.so.ulist, c.so.counts, c.cap, RX, nullptr, nullptr, st);
  if (b.e == cudaSuccess) b.e = cd_residual(n, RX, c.tw, c.so.wfull, 2, nullptr, out, st, ldo, 1);
  return b.e;
}

bool aligned16(const float* p, int64_t ld) { return ((uintptr_t)p & 15) == 0 && (ld & 3) == 0; }

}  // namespace

amm_status_t mixed_backward(Handle* a, Handle* b, const float* G, int64_t ldg, float* dA, int64_t ldda, float* dB,
                            int64_t lddb, cudaStream_t st) {
  const int64_t m = a->rows, n = a->cols, p = b->cols;
  if (a->method == AMM_SPARSE_FOURIER || b->method == AMM_SPARSE_FOURIER)
    return fail(AMM_ERR_NOT_IMPLEMENTED, "backward of a mixed-method product with the Fourier sparsifier is not built");
  if (a->blk.b || b->blk.b)
    return fail(AMM_ERR_NOT_IMPLEMENTED, "backward of a mixed-method product with circulant blocks is not built");
  if (m != n || p != n)
    return fail(AMM_ERR_UNSUPPORTED_SIZE, "backward of a mixed-method product needs square operands (%lldx%lld, "
                "%lldx%lld)", (long long)m, (long long)n, (long long)n, (long long)p);
  if (a->dtype != AMM_F32 || b->dtype != AMM_F32)
    return fail(AMM_ERR_NOT_IMPLEMENTED, "mixed methods: BF16 operands are not built (use FP32 inputs)");
  const int nn = (int)n;
  Buf buf(st);
  float* DA = buf.get<float>((size_t)nn * nn);  // Re dA = A - Re A~
  float* DB = buf.get<float>((size_t)nn * nn);
  cudaError_t e = buf.e;
  if (e == cudaSuccess) e = residual(a, DA, nn, st);
  if (e == cudaSuccess) e = residual(b, DB, nn, st);
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
      default: e = cyc_rt_apply(nn, G, ldg, b->cy.so.sel, (int)b->k, b->cy.cyc, dA, ldda, st); break;
    }
    // + Re P_A'(G dB^T)
    if (e == cudaSuccess) {
      switch (a->method) {
        case AMM_SVD: e = svd_proj_left(a, G, ldg, DB, nn, nn, dA, ldda, st); break;
        case AMM_CIRCULANT: e = cd_project_product(a, false, G, ldg, DB, nn, dA, ldda, st); break;
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
      default: e = cyc_lt_apply(nn, G, ldg, a->cy.so.sel, (int)a->k, a->cy.cyc, dB, lddb, st); break;
    }
    // + Re P_B'(dA^T G)
    if (e == cudaSuccess) {
      switch (b->method) {
        case AMM_SVD: e = svd_proj_right(b, DA, nn, G, ldg, nn, dB, lddb, st); break;
        case AMM_CIRCULANT: e = cd_project_product(b, true, DA, nn, G, ldg, dB, lddb, st); break;
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
  if (h->method == AMM_SPARSE_FOURIER && h->role != AMM_LEFT)
    return fail(AMM_ERR_NOT_IMPLEMENTED, "amm_handle_residual: the Fourier sparsifier's right operand is not built");
  const int64_t m = h->rows, n = h->cols;
  Buf buf(st);
  float* T = buf.get<float>((size_t)m * n);  // the pieces write a dense m x n scratch, copied out
  cudaError_t e = buf.e;
  if (e == cudaSuccess) e = residual(h, T, n, st);
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

}  // namespace amm
