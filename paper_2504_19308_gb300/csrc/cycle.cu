// Cycle sparsification (Section 1.2.2 and the sparsified first-order form Eq. (2.4)-(2.5) of
// arXiv 2504.19308) for sm_103a.
//
// A = sum_j C^j Lambda_j with Lambda_j(l) = A((l+j) mod n, l).  The kept part A_s holds the k
// cycles with the largest ||Lambda_j||_2; dA = A - A_s.  Multiplying by one cycle is a row
// shift plus a scaling (~2 n^2 operations), so both first-order terms are k real MACs per
// output entry:
//   (A_s B)(r, c)  = sum_{t in S_A} Lambda^A_t(r - t) B(r - t, c)                 (column panels)
//   (dA B_s)(r, c) = sum_{s in S_B} dA(r, c + s) Lambda^B_s(c),                     (row panels)
//   dA(r, q) = A(r, q) if (r - q) mod n is not in S_A, else 0.
#include <cuda_runtime.h>

#include "api_internal.h"
#include "common.cuh"
#include "cycle_kernels.cuh"
#include "kernels.h"
#include "trace.h"

namespace amm {

__global__ void __launch_bounds__(256) cyc_keys_kernel(const float* __restrict__ A, int64_t lda, int n, int rows_per,
                                                       float* __restrict__ part) {
  cyc_keys_tile(A, lda, n, rows_per, part, blockIdx.x, blockIdx.y);
}

__global__ void cyc_gather_kernel(const float* __restrict__ A, int64_t lda, int n, int k,
                                  const int32_t* __restrict__ sel, float* __restrict__ cyc,
                                  unsigned char* __restrict__ insel) {
  cyc_gather_tile<false>(A, lda, n, sel, cyc, insel, blockIdx.y, blockIdx.x * blockDim.x + threadIdx.x,
                  gridDim.x * blockDim.x, blockIdx.x == 0);
}

template <bool P2>
__global__ void __launch_bounds__(CYC_NT) cyc_apply_col_kernel(const float* __restrict__ B, int64_t ldb, int n,
                                                               const int32_t* __restrict__ sel, int k,
                                                               const float* __restrict__ cyc, float* __restrict__ out,
                                                               int64_t ldo, int ncols) {
  extern __shared__ float4 bp[];  // n x 4 columns, then the k selected cycle indices
  cyc_apply_col_tile<P2, false>(B, ldb, n, sel, k, cyc, out, ldo, ncols, blockIdx.x, bp);
}

template <bool P2>
__global__ void __launch_bounds__(CYC_NT) cyc_apply_row_kernel(const float* __restrict__ A, int64_t lda, int n,
                                                               const unsigned char* __restrict__ inselA,
                                                               const int32_t* __restrict__ selB, int kb,
                                                               const float* __restrict__ cycB, float* __restrict__ out,
                                                               int64_t ldo, int nrows) {
  extern __shared__ float ar[];  // CYC_RW x n, masked dA
  cyc_apply_row_tile<P2, false>(A, lda, n, inselA, selB, kb, cycB, out, ldo, nrows, blockIdx.x, ar);
}

// ============================================================================ backward (selections frozen)
//   dA = G B_s^T + P_{S_A}(G dB^T),   dB = A_s^T G + P_{S_B}(dA^T G)
// (G B_s^T)(r, q) = sum_{s in S_B} G(r, q - s) Lambda^B_s(q - s)           (row panels)
// (A_s^T G)(q, c) = sum_{t in S_A} Lambda^A_t(q) G(q + t, c)               (column panels)
// P_S keeps the cycles t in S: P_{S_A}(G dB^T)((l + t), l) = <G(l + t, :), dB(l, :)>,
// P_{S_B}(dA^T G)((l + s), l) = <dA(:, l + s), G(:, l)>; dA, dB are masked on the fly.

// out(r0..r0+3, q) = sum_u G(r, q - s_u) cycB[u][q - s_u]
template <bool P2>
__global__ void __launch_bounds__(CYC_NT) cyc_bw_row_kernel(const float* __restrict__ G, int64_t ldg, int n,
                                                            const int32_t* __restrict__ selB, int kb,
                                                            const float* __restrict__ cycB, float* __restrict__ out,
                                                            int64_t ldo) {
  extern __shared__ float gr[];  // CYC_RW x n
  const int r0 = blockIdx.x * CYC_RW;
  for (int e = threadIdx.x; e < CYC_RW * n; e += CYC_NT) gr[e] = __ldg(G + (int64_t)(r0 + e / n) * ldg + e % n);
  __syncthreads();
  for (int q = threadIdx.x; q < n; q += CYC_NT) {
    float acc[CYC_RW] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 8
    for (int u = 0; u < kb; ++u) {
      const int l = cwrap<P2>(q - __ldg(selB + u), n);
      const float b = __ldg(cycB + (int64_t)u * n + l);
#pragma unroll
      for (int rr = 0; rr < CYC_RW; ++rr) acc[rr] = fmaf(gr[rr * n + l], b, acc[rr]);
    }
#pragma unroll
    for (int rr = 0; rr < CYC_RW; ++rr) out[(int64_t)(r0 + rr) * ldo + q] = acc[rr];
  }
}

// out(q, c0..c0+3) = sum_u cycA[u][q] G(q + t_u, c)
template <bool P2>
__global__ void __launch_bounds__(CYC_NT) cyc_bw_col_kernel(const float* __restrict__ G, int64_t ldg, int n,
                                                            const int32_t* __restrict__ selA, int ka,
                                                            const float* __restrict__ cycA, float* __restrict__ out,
                                                            int64_t ldo) {
  extern __shared__ float4 gp[];  // n x 4 columns; then the ka selected cycle indices of A
  int* s_sel = reinterpret_cast<int*>(gp + n);
  const int c0 = blockIdx.x * CYC_CW;
  for (int r = threadIdx.x; r < n; r += CYC_NT) {
    const float* src = G + (int64_t)r * ldg + c0;
    gp[r] = make_float4(__ldg(src), __ldg(src + 1), __ldg(src + 2), __ldg(src + 3));
  }
  for (int u = threadIdx.x; u < ka; u += CYC_NT) s_sel[u] = __ldg(selA + u);
  __syncthreads();
  for (int qb = threadIdx.x; qb < n; qb += CYC_NT * CYC_RG) {
    float4 acc[CYC_RG];
#pragma unroll
    for (int i = 0; i < CYC_RG; ++i) acc[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int u = 0; u < ka; ++u) {
      const int t = s_sel[u];
      const float* arow = cycA + (int64_t)u * n;
#pragma unroll
      for (int i = 0; i < CYC_RG; ++i) {
        const int q = qb + i * CYC_NT;
        if (q < n) {
          const float a = __ldg(arow + q);
          const float4 g = gp[cwrap<P2>(q + t, n)];
          acc[i].x = fmaf(a, g.x, acc[i].x);
          acc[i].y = fmaf(a, g.y, acc[i].y);
          acc[i].z = fmaf(a, g.z, acc[i].z);
          acc[i].w = fmaf(a, g.w, acc[i].w);
        }
      }
    }
#pragma unroll
    for (int i = 0; i < CYC_RG; ++i) {
      const int q = qb + i * CYC_NT;
      if (q >= n) continue;
      float* o = out + (int64_t)q * ldo + c0;
      o[0] = acc[i].x;
      o[1] = acc[i].y;
      o[2] = acc[i].z;
      o[3] = acc[i].w;
    }
  }
}

static bool pow2n(int n) { return (n & (n - 1)) == 0; }

// dynamic shared memory of the apply kernels (both index forms), set once
static cudaError_t cyc_attrs() {
  static DeviceOnce once;
  return once([] {
    const int col = 8192 * (int)sizeof(float4) + 8192 * (int)sizeof(int), row = CYC_RW * 8192 * (int)sizeof(float);
    const void* fs[8] = {(const void*)cyc_apply_col_kernel<true>, (const void*)cyc_apply_col_kernel<false>,
                         (const void*)cyc_bw_col_kernel<true>, (const void*)cyc_bw_col_kernel<false>,
                         (const void*)cyc_apply_row_kernel<true>, (const void*)cyc_apply_row_kernel<false>,
                         (const void*)cyc_bw_row_kernel<true>, (const void*)cyc_bw_row_kernel<false>};
    cudaError_t r = cudaSuccess;
    for (int i = 0; i < 8 && r == cudaSuccess; ++i)
      r = cudaFuncSetAttribute(fs[i], cudaFuncAttributeMaxDynamicSharedMemorySize, i < 4 ? col : row);
    return r;
  });
}

// launch KERNEL<P2> with P2 = (n is a power of two)
#define CYC_LAUNCH(KERNEL, GRID, SMEM, ...)                                     \
  do {                                                                          \
    if (pow2n(n)) KERNEL<true><<<(GRID), CYC_NT, (SMEM), st>>>(__VA_ARGS__);    \
    else KERNEL<false><<<(GRID), CYC_NT, (SMEM), st>>>(__VA_ARGS__);            \
  } while (0)

// Selected diagonals of a product: out((l + t) mod n, l) += <X((l + t) mod n, :), Y(l, :)> for
// t = sel[u], every l.  The projection terms of the cycle backward are of this form (the kept
// cycles of G dB^T and of dA^T G, with the masks applied to dense residuals beforehand).  A warp
// takes one l and CYC_DG selected t's: lanes stride the rows in float4s, each float4 of Y(l, :)
// serves CYC_DG products.  The t-groups are the fast grid dimension, so the CTAs in flight share
// their rows Y(l, :) through L2.  Rows 16-byte aligned (n a multiple of 4, ldx, ldy too).
constexpr int CYC_DG = 4;
template <bool P2>
__global__ void __launch_bounds__(256) cyc_diag_dot_kernel(const float* __restrict__ X, int64_t ldx,
                                                           const float* __restrict__ Y, int64_t ldy, int n,
                                                           int len, const int32_t* __restrict__ sel, int k,
                                                           float* __restrict__ out, int64_t ldo) {
  const int g0 = blockIdx.x * CYC_DG;
  const int l = blockIdx.y * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (l >= n) return;  // whole warps
  const int nt = min(CYC_DG, k - g0);
  int r[CYC_DG];
  const float4* xr[CYC_DG];
#pragma unroll
  for (int j = 0; j < CYC_DG; ++j) {
    r[j] = cwrap<P2>(l + __ldg(sel + g0 + (j < nt ? j : 0)), n);
    xr[j] = reinterpret_cast<const float4*>(X + (int64_t)r[j] * ldx);
  }
  const float4* yr = reinterpret_cast<const float4*>(Y + (int64_t)l * ldy);
  float acc[CYC_DG];
#pragma unroll
  for (int j = 0; j < CYC_DG; ++j) acc[j] = 0.f;
#pragma unroll 4
  for (int m4 = lane; m4 < len / 4; m4 += 32) {
    const float4 y = __ldg(yr + m4);
#pragma unroll
    for (int j = 0; j < CYC_DG; ++j) {
      const float4 x = __ldg(xr[j] + m4);
      acc[j] = fmaf(x.x, y.x, acc[j]);
      acc[j] = fmaf(x.y, y.y, acc[j]);
      acc[j] = fmaf(x.z, y.z, acc[j]);
      acc[j] = fmaf(x.w, y.w, acc[j]);
    }
  }
#pragma unroll
  for (int j = 0; j < CYC_DG; ++j)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc[j] += __shfl_xor_sync(0xffffffffu, acc[j], o);
#pragma unroll
  for (int j = 0; j < CYC_DG; ++j)
    if (lane == j && j < nt) out[(int64_t)r[j] * ldo + l] += acc[j];
}

// rows of len entries (a multiple of 4, 16-byte aligned rows)
static cudaError_t diag_dot(const float* X, int64_t ldx, const float* Y, int64_t ldy, int n, int len,
                            const int32_t* sel, int k, float* out, int64_t ldo, const char* name, cudaStream_t st) {
  AMM_TRACE_W(name, st, 2.0 * k * (double)n * len, 4.0 * len * ((double)k + (k + CYC_DG - 1) / CYC_DG) * n, nullptr);
  auto kern = pow2n(n) ? cyc_diag_dot_kernel<true> : cyc_diag_dot_kernel<false>;
  kern<<<dim3((k + CYC_DG - 1) / CYC_DG, (n + 7) / 8), 256, 0, st>>>(X, ldx, Y, ldy, n, len, sel, k, out, ldo);
  return cudaGetLastError();
}

cudaError_t cyc_backward(int n, const float* A, int64_t lda, const float* B, int64_t ldb, const int32_t* selA, int ka,
                         const float* cycA, const unsigned char* inselA, const int32_t* selB, int kb,
                         const float* cycB, const unsigned char* inselB, const float* G, int64_t ldg, float* dA,
                         int64_t ldda, float* dB, int64_t lddb, cudaStream_t st) {
  if (cudaError_t ea = cyc_attrs(); ea != cudaSuccess) return ea;
  // dense scratch: the masked residual of the other operand, and for dB the transposes
  const int64_t nn = (int64_t)n * n;
  float* T = nullptr;
  cudaError_t e = dev_alloc((void**)&T, sizeof(float) * 3 * nn, st);
  if (e != cudaSuccess) return e;
  float *T0 = T, *T1 = T + nn, *T2 = T + 2 * nn;
  auto aligned = [](const float* p, int64_t ld) { return ((uintptr_t)p & 15) == 0 && (ld & 3) == 0; };
  if (dA) {
    {
      AMM_TRACE_W("cyc_bw_row", st, 2.0 * kb * (double)n * n, 8.0 * n * (double)n, nullptr);
      CYC_LAUNCH(cyc_bw_row_kernel, n / CYC_RW, sizeof(float) * CYC_RW * n, G, ldg, n, selB, kb, cycB, dA, ldda);
    }
    e = cudaGetLastError();
    // dA((l + t), l) += <G(l + t, :), dB(l, :)> for t in S_A, dB = B with its kept cycles zeroed
    if (e == cudaSuccess) e = cyc_residual(n, B, ldb, inselB, T0, n, st);
    const float* Gx = G;
    int64_t ldgx = ldg;
    if (e == cudaSuccess && !aligned(G, ldg)) {
      e = cudaMemcpy2DAsync(T1, sizeof(float) * n, G, sizeof(float) * ldg, sizeof(float) * n, n,
                            cudaMemcpyDeviceToDevice, st);
      Gx = T1;
      ldgx = n;
    }
    if (e == cudaSuccess) e = diag_dot(Gx, ldgx, T0, n, n, n, selA, ka, dA, ldda, "cyc_bw_proj_rows", st);
  }
  if (dB && e == cudaSuccess) {
    {
      AMM_TRACE_W("cyc_bw_col", st, 2.0 * ka * (double)n * n, 8.0 * n * (double)n, nullptr);
      CYC_LAUNCH(cyc_bw_col_kernel, n / CYC_CW, sizeof(float4) * n + sizeof(int) * ka, G, ldg, n, selA, ka, cycA, dB,
                 lddb);
    }
    e = cudaGetLastError();
    // dB((l + s), l) += sum_r dA(r, l + s) G(r, l) = <dA^T(l + s, :), G^T(l, :)> for s in S_B
    if (e == cudaSuccess) e = cyc_residual(n, A, lda, inselA, T0, n, st);
    if (e == cudaSuccess) e = transpose_f32(T0, n, n, n, T1, n, st);
    if (e == cudaSuccess) e = transpose_f32(G, n, n, ldg, T2, n, st);
    if (e == cudaSuccess) e = diag_dot(T1, n, T2, n, n, n, selB, kb, dB, lddb, "cyc_bw_proj_cols", st);
  }
  dev_free(T, st);
  return e;
}

// ---------------------------------------------------------------------------- mixed-method backward pieces
// out = G B_s^T (n x n, G n x n)
cudaError_t cyc_rt_apply(int n, const float* G, int64_t ldg, const int32_t* selB, int kb, const float* cycB,
                         float* out, int64_t ldo, cudaStream_t st) {
  if (cudaError_t ea = cyc_attrs(); ea != cudaSuccess) return ea;
  AMM_TRACE_W("cyc_bw_row", st, 2.0 * kb * (double)n * n, 8.0 * n * (double)n, nullptr);
  CYC_LAUNCH(cyc_bw_row_kernel, n / CYC_RW, sizeof(float) * CYC_RW * n, G, ldg, n, selB, kb, cycB, out, ldo);
  return cudaGetLastError();
}
// out = A_s^T G (n x n)
cudaError_t cyc_lt_apply(int n, const float* G, int64_t ldg, const int32_t* selA, int ka, const float* cycA,
                         float* out, int64_t ldo, cudaStream_t st) {
  if (cudaError_t ea = cyc_attrs(); ea != cudaSuccess) return ea;
  AMM_TRACE_W("cyc_bw_col", st, 2.0 * ka * (double)n * n, 8.0 * n * (double)n, nullptr);
  CYC_LAUNCH(cyc_bw_col_kernel, n / CYC_CW, sizeof(float4) * n + sizeof(int) * ka, G, ldg, n, selA, ka, cycA, out,
             ldo);
  return cudaGetLastError();
}
// out((l + t) mod n, l) += <X((l + t) mod n, :), Y(l, :)> for the selected t (rows of len entries,
// 16-byte aligned, len a multiple of 4)
cudaError_t cyc_diag_project(int n, int len, const float* X, int64_t ldx, const float* Y, int64_t ldy,
                             const int32_t* sel, int k, float* out, int64_t ldo, cudaStream_t st) {
  return diag_dot(X, ldx, Y, ldy, n, len, sel, k, out, ldo, "cyc_proj", st);
}

int cyc_rows_per_part(int n) { return n >= 1024 ? 64 : 16; }

cudaError_t cyc_keys(int n, const float* A, int64_t lda, float* part, cudaStream_t st) {
  AMM_TRACE_W("cyc_keys", st, 0.0, (double)n * n * 4, nullptr);
  const int rp = cyc_rows_per_part(n);
  dim3 grid((n + 255) / 256, (n + rp - 1) / rp);
  cyc_keys_kernel<<<grid, 256, 0, st>>>(A, lda, n, rp, part);
  return cudaGetLastError();
}

cudaError_t cyc_gather(int n, int k, const float* A, int64_t lda, const int32_t* sel, float* cyc,
                       unsigned char* insel, cudaStream_t st) {
  AMM_TRACE("cyc_gather", st);
  cudaError_t e = cudaMemsetAsync(insel, 0, n, st);
  if (e != cudaSuccess) return e;
  dim3 grid((n + 255) / 256, k);
  cyc_gather_kernel<<<grid, 256, 0, st>>>(A, lda, n, k, sel, cyc, insel);
  return cudaGetLastError();
}

cudaError_t cyc_apply(int n, const float* A, int64_t lda, const float* B, int64_t ldb, const int32_t* selA, int ka,
                      const float* cycA, const unsigned char* inselA, const int32_t* selB, int kb, const float* cycB,
                      float* C, int64_t ldc, cudaStream_t st) {
  if (cudaError_t ea = cyc_attrs(); ea != cudaSuccess) return ea;
  {
    AMM_TRACE_W("cyc_apply_col", st, 2.0 * ka * (double)n * n, 8.0 * n * (double)n, nullptr);
    CYC_LAUNCH(cyc_apply_col_kernel, (n + CYC_CW - 1) / CYC_CW, sizeof(float4) * n + sizeof(int) * ka, B, ldb, n, selA,
               ka, cycA, C, ldc, n);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  {
    AMM_TRACE_W("cyc_apply_row", st, 2.0 * kb * (double)n * n, 12.0 * n * (double)n, nullptr);
    CYC_LAUNCH(cyc_apply_row_kernel, (n + CYC_RW - 1) / CYC_RW, sizeof(float) * CYC_RW * n, A, lda, n, inselA, selB,
               kb, cycB, C, ldc, n);
  }
  return cudaGetLastError();
}

// ============================================================================ mixed-method pieces
// D = A with the kept cycles zeroed (the dense residual dA = A - A_s)
// D = A with the selected cycles zeroed: row r, four consecutive columns per thread.
__global__ void __launch_bounds__(256) cyc_residual_kernel(const float* __restrict__ A, int64_t lda, int n,
                                                           const unsigned char* __restrict__ insel,
                                                           float* __restrict__ D, int64_t ldd) {
  const int r = blockIdx.y;
  const int c0 = (blockIdx.x * 256 + threadIdx.x) * 4;
  if (c0 >= n) return;
  const float* a = A + (int64_t)r * lda + c0;
  float v[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) v[i] = insel[cwrap<false>(r - c0 - i, n)] ? 0.f : __ldg(a + i);
  float* d = D + (int64_t)r * ldd + c0;
  if ((((uintptr_t)d) & 15) == 0) {
    *reinterpret_cast<float4*>(d) = make_float4(v[0], v[1], v[2], v[3]);
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i) d[i] = v[i];
  }
}

// C = A_s X for X (n x p)
cudaError_t cyc_left_apply(int n, const int32_t* selA, int ka, const float* cycA, const float* X, int64_t ldx,
                           int64_t p, float* C, int64_t ldc, cudaStream_t st) {
  cudaError_t e = cyc_attrs();
  if (e != cudaSuccess) return e;
  AMM_TRACE_W("cyc_apply_col", st, 2.0 * ka * (double)n * p, 8.0 * n * (double)p, nullptr);
  CYC_LAUNCH(cyc_apply_col_kernel, (unsigned)((p + CYC_CW - 1) / CYC_CW), sizeof(float4) * n + sizeof(int) * ka, X,
             ldx, n, selA, ka, cycA, C, ldc, (int)p);
  return cudaGetLastError();
}

// C += Y B_s for Y (m x n)
cudaError_t cyc_right_apply(int n, const int32_t* selB, int kb, const float* cycB, const float* Y, int64_t ldy,
                            int64_t m, float* C, int64_t ldc, cudaStream_t st) {
  cudaError_t e = cyc_attrs();
  if (e != cudaSuccess) return e;
  AMM_TRACE_W("cyc_apply_row", st, 2.0 * kb * (double)n * m, 12.0 * n * (double)m, nullptr);
  CYC_LAUNCH(cyc_apply_row_kernel, (unsigned)((m + CYC_RW - 1) / CYC_RW), sizeof(float) * CYC_RW * n, Y, ldy, n,
             (const unsigned char*)nullptr, selB, kb, cycB, C, ldc, (int)m);
  return cudaGetLastError();
}

cudaError_t cyc_residual(int n, const float* A, int64_t lda, const unsigned char* insel, float* D, int64_t ldd,
                         cudaStream_t st) {
  AMM_TRACE_W("cyc_residual", st, 0.0, 8.0 * n * (double)n, nullptr);
  cyc_residual_kernel<<<dim3((n / 4 + 255) / 256, n), 256, 0, st>>>(A, lda, n, insel, D, ldd);
  return cudaGetLastError();
}

}  // namespace amm
