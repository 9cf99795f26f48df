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

#include "common.cuh"
#include "kernels.h"
#include "trace.h"

namespace amm {

// part[rb][j] = sum over rows r of block rb of A(r, (r - j) mod n)^2 (thread per cycle j:
// a warp reads 32 consecutive columns of one row).
__global__ void __launch_bounds__(256) cyc_keys_kernel(const float* __restrict__ A, int64_t lda, int n, int rows_per,
                                                       float* __restrict__ part) {
  const int j = blockIdx.x * 256 + threadIdx.x;
  if (j >= n) return;
  const int r0 = blockIdx.y * rows_per;
  float s = 0.f;
  for (int r = r0; r < min(n, r0 + rows_per); ++r) {
    const float v = __ldg(A + (int64_t)r * lda + ((r - j) & (n - 1)));
    s = fmaf(v, v, s);
  }
  part[(int64_t)blockIdx.y * n + j] = s;
}

// cyc[u][l] = A((l + t_u) mod n, l) for the k selected cycles; insel[t] = 1 for selected t.
__global__ void cyc_gather_kernel(const float* __restrict__ A, int64_t lda, int n, int k,
                                  const int32_t* __restrict__ sel, float* __restrict__ cyc,
                                  unsigned char* __restrict__ insel) {
  const int u = blockIdx.y;
  const int t = sel[u];
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < n; l += gridDim.x * blockDim.x)
    cyc[(int64_t)u * n + l] = __ldg(A + (int64_t)((l + t) & (n - 1)) * lda + l);
  if (blockIdx.x == 0 && threadIdx.x == 0) insel[t] = 1;
}

constexpr int CYC_CW = 4;    // columns per CTA (A_s B)
constexpr int CYC_RW = 4;    // rows per CTA (dA B_s)
constexpr int CYC_NT = 256;

// out(:, c0..c0+3) = sum_u cyc[u][r - t_u] B(r - t_u, c)
__global__ void __launch_bounds__(CYC_NT) cyc_apply_col_kernel(const float* __restrict__ B, int64_t ldb, int n,
                                                               const int32_t* __restrict__ sel, int k,
                                                               const float* __restrict__ cyc, float* __restrict__ out,
                                                               int64_t ldo, int ncols) {
  extern __shared__ float4 bp[];  // n x 4 columns
  const int c0 = blockIdx.x * CYC_CW;
  for (int r = threadIdx.x; r < n; r += CYC_NT) {
    const float* src = B + (int64_t)r * ldb + c0;
    float4 v;
    v.x = c0 + 0 < ncols ? __ldg(src + 0) : 0.f;
    v.y = c0 + 1 < ncols ? __ldg(src + 1) : 0.f;
    v.z = c0 + 2 < ncols ? __ldg(src + 2) : 0.f;
    v.w = c0 + 3 < ncols ? __ldg(src + 3) : 0.f;
    bp[r] = v;
  }
  __syncthreads();
  for (int r = threadIdx.x; r < n; r += CYC_NT) {
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int u = 0; u < k; ++u) {
      const int l = (r - __ldg(sel + u)) & (n - 1);
      const float a = __ldg(cyc + (int64_t)u * n + l);
      const float4 b = bp[l];
      acc.x = fmaf(a, b.x, acc.x);
      acc.y = fmaf(a, b.y, acc.y);
      acc.z = fmaf(a, b.z, acc.z);
      acc.w = fmaf(a, b.w, acc.w);
    }
    float* o = out + (int64_t)r * ldo + c0;
    if (c0 + 0 < ncols) o[0] = acc.x;
    if (c0 + 1 < ncols) o[1] = acc.y;
    if (c0 + 2 < ncols) o[2] = acc.z;
    if (c0 + 3 < ncols) o[3] = acc.w;
  }
}

// out(r0..r0+3, :) += sum_u dA(r, c + s_u) cycB[u][c]
__global__ void __launch_bounds__(CYC_NT) cyc_apply_row_kernel(const float* __restrict__ A, int64_t lda, int n,
                                                               const unsigned char* __restrict__ inselA,
                                                               const int32_t* __restrict__ selB, int kb,
                                                               const float* __restrict__ cycB, float* __restrict__ out,
                                                               int64_t ldo, int nrows) {
  extern __shared__ float ar[];  // CYC_RW x n, masked dA
  const int r0 = blockIdx.x * CYC_RW;
  for (int e = threadIdx.x; e < CYC_RW * n; e += CYC_NT) {
    const int rr = e / n, q = e % n, r = r0 + rr;
    float v = 0.f;
    if (r < nrows && !inselA[(r - q) & (n - 1)]) v = __ldg(A + (int64_t)r * lda + q);
    ar[e] = v;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < n; c += CYC_NT) {
    float acc[CYC_RW] = {0.f, 0.f, 0.f, 0.f};
    for (int u = 0; u < kb; ++u) {
      const int q = (c + __ldg(selB + u)) & (n - 1);
      const float b = __ldg(cycB + (int64_t)u * n + c);
#pragma unroll
      for (int rr = 0; rr < CYC_RW; ++rr) acc[rr] = fmaf(ar[rr * n + q], b, acc[rr]);
    }
#pragma unroll
    for (int rr = 0; rr < CYC_RW; ++rr)
      if (r0 + rr < nrows) out[(int64_t)(r0 + rr) * ldo + c] += acc[rr];
  }
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
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute((const void*)cyc_apply_col_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         8192 * (int)sizeof(float4));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute((const void*)cyc_apply_row_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               CYC_RW * 8192 * (int)sizeof(float));
    if (e != cudaSuccess) return e;
    attr = true;
  }
  {
    AMM_TRACE_W("cyc_apply_col", st, 2.0 * ka * (double)n * n, 8.0 * n * (double)n, nullptr);
    cyc_apply_col_kernel<<<(n + CYC_CW - 1) / CYC_CW, CYC_NT, sizeof(float4) * n, st>>>(B, ldb, n, selA, ka, cycA, C,
                                                                                         ldc, n);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  {
    AMM_TRACE_W("cyc_apply_row", st, 2.0 * kb * (double)n * n, 12.0 * n * (double)n, nullptr);
    cyc_apply_row_kernel<<<(n + CYC_RW - 1) / CYC_RW, CYC_NT, sizeof(float) * CYC_RW * n, st>>>(
        A, lda, n, inselA, selB, kb, cycB, C, ldc, n);
  }
  return cudaGetLastError();
}

}  // namespace amm
