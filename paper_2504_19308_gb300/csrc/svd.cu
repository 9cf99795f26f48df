// Randomized truncated SVD path (Alg. 1 and Section 2.2 of arXiv 2504.19308) for sm_103a.
//
// Decomposition of one operand X (rows x cols), test matrix phi (cols x k):
//   Y = X phi                      FP32 GEMM
//   Q = orth(Y)                    CholeskyQR2 in FP64 (k x k Gram, Cholesky, triangular apply)
//   Z = Q^T X                      FP32 GEMM            ->  X~ = Q Z = Q Q^T X
// The small SVD of Z that ends Alg. 1 rotates Q and Z by the same k x k factors and does
// not change X~, so the product does not need it.
//
// Product (A m x n left, B n x p right), with A~ = Q_A Z_A and B~ = Q_B Z_B:
//   M = A~ B + (A - A~) B~ = Q_A (Z_A B) + W Z_B,    W = A Q_B - Q_A (Z_A Q_B)
// Backward of <G, M> with Q_A, Q_B frozen:
//   dA = (G Z_B^T) Q_B^T + Q_A [ (Q_A^T G) B^T - ((Q_A^T G) Z_B^T) Q_B^T ]
//   dB = Z_A^T (Q_A^T G) + Q_B (W^T G)
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>

#include "api_internal.h"
#include "common.cuh"
#include "trace.h"

namespace amm {

// ============================================================================ FP32 SIMT GEMM
// C = alpha op(A) op(B) + beta C, op(A) is M x K, op(B) is K x N.  TA: A stored K x M.
// TB: B stored N x K.  128 x 128 x 8 tiles, 256 threads, 8 x 8 outputs per thread.
// With gridDim.z > 1 each z-slice covers a K range and writes its partial tile to ws.
constexpr int GB_M = 128, GB_N = 128, GB_K = 8;

template <bool TA, bool TB, typename TIn>
__global__ void __launch_bounds__(256) sgemm_kernel(int M, int N, int K, float alpha, const TIn* __restrict__ A,
                                                    int64_t lda, const TIn* __restrict__ B, int64_t ldb, float beta,
                                                    float* __restrict__ C, int64_t ldc, int kchunk,
                                                    float* __restrict__ ws) {
  __shared__ __align__(16) float As[2][GB_K][GB_M];
  __shared__ __align__(16) float Bs[2][GB_K][GB_N];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * GB_M, n0 = blockIdx.x * GB_N;
  const int kbeg = blockIdx.z * kchunk;
  const int kend = min(K, kbeg + kchunk);
  auto ldA = [&](int i, int k) -> float {
    if (i >= M || k >= kend) return 0.f;
    const TIn* p = TA ? (A + (int64_t)k * lda + i) : (A + (int64_t)i * lda + k);
    if constexpr (sizeof(TIn) == 2) return __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(p));
    else return __ldg(reinterpret_cast<const float*>(p));
  };
  auto ldB = [&](int k, int j) -> float {
    if (j >= N || k >= kend) return 0.f;
    const TIn* p = TB ? (B + (int64_t)j * ldb + k) : (B + (int64_t)k * ldb + j);
    if constexpr (sizeof(TIn) == 2) return __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(p));
    else return __ldg(reinterpret_cast<const float*>(p));
  };
  // per-thread load coordinates for one 128 x 8 (A) and 8 x 128 (B) tile: 4 elements each
  float ra[4], rb[4];
  auto fetch = [&](int k0) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (TA) { int kk = tid >> 5, ii = (tid & 31) * 4 + q; ra[q] = ldA(m0 + ii, k0 + kk); }
      else { int ii = tid >> 1, kk = (tid & 1) * 4 + q; ra[q] = ldA(m0 + ii, k0 + kk); }
      if (!TB) { int kk = tid >> 5, jj = (tid & 31) * 4 + q; rb[q] = ldB(k0 + kk, n0 + jj); }
      else { int jj = tid >> 1, kk = (tid & 1) * 4 + q; rb[q] = ldB(k0 + kk, n0 + jj); }
    }
  };
  auto stash = [&](int buf) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (TA) As[buf][tid >> 5][(tid & 31) * 4 + q] = ra[q];
      else As[buf][(tid & 1) * 4 + q][tid >> 1] = ra[q];
      if (!TB) Bs[buf][tid >> 5][(tid & 31) * 4 + q] = rb[q];
      else Bs[buf][(tid & 1) * 4 + q][tid >> 1] = rb[q];
    }
  };
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
  int buf = 0;
  if (kbeg < kend) {
    fetch(kbeg);
    stash(0);
  }
  __syncthreads();
  for (int k0 = kbeg; k0 < kend; k0 += GB_K) {
    const bool more = k0 + GB_K < kend;
    if (more) fetch(k0 + GB_K);
#pragma unroll
    for (int kk = 0; kk < GB_K; ++kk) {
      float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 4]);
      float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][64 + ty * 4]);
      float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][kk][tx * 4]);
      float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][kk][64 + tx * 4]);
      float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    if (more) stash(buf ^ 1);
    __syncthreads();
    buf ^= 1;
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int row = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
    if (row >= M) continue;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int col = n0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + (j - 4));
      if (col >= N) continue;
      if (ws) {
        ws[((int64_t)blockIdx.z * M + row) * N + col] = acc[i][j];
      } else {
        float* c = C + (int64_t)row * ldc + col;
        *c = (beta == 0.f) ? alpha * acc[i][j] : fmaf(alpha, acc[i][j], beta * *c);
      }
    }
  }
}

// partial tiles summed in FP64 in a fixed order (deterministic; no error growth across chunks)
__global__ void splitk_reduce_kernel(int M, int N, int splits, const float* __restrict__ ws, float alpha, float beta,
                                     float* __restrict__ C, int64_t ldc) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)M * N) return;
  const int row = (int)(e / N), col = (int)(e % N);
  double s = 0.0;
#pragma unroll 8
  for (int z = 0; z < splits; ++z) s += (double)ws[(int64_t)z * M * N + e];
  float* c = C + (int64_t)row * ldc + col;
  *c = (beta == 0.f) ? (float)(alpha * s) : (float)fma((double)alpha, s, (double)beta * *c);
}

// SM count of the current device, queried once per process (thread-safe static initialisation);
// 152, GB300's count, only if the query fails
static int num_sms() {
  static const int n = [] {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 152;
  }();
  return n;
}

// Host launcher: picks a deterministic split of K when the output has too few tiles.
template <typename TIn>
static cudaError_t sgemm(bool ta, bool tb, int M, int N, int K, float alpha, const TIn* A, int64_t lda, const TIn* B,
                         int64_t ldb, float beta, float* C, int64_t ldc, cudaStream_t st) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  const int tiles = ((M + GB_M - 1) / GB_M) * ((N + GB_N - 1) / GB_N);
  int splits = 1;
  const int target = 2 * num_sms();
  if (tiles < target && K >= 256) splits = std::min((target + tiles - 1) / tiles, std::max(1, K / 128));
  // long FP32 dot products dominate the rounding error of thin GEMMs: keep chunks <= 512 when
  // the output is small enough for the partial tiles to be cheap
  if ((int64_t)M * N <= (int64_t)2 << 20 && K > 512) splits = std::max(splits, (K + 511) / 512);
  splits = std::min(splits, 64);
  int kchunk = (K + splits - 1) / splits;
  kchunk = ((kchunk + GB_K - 1) / GB_K) * GB_K;
  splits = std::max(1, (K + kchunk - 1) / kchunk);
  float* ws = nullptr;
  cudaError_t e;
  if (splits > 1) {
    e = dev_alloc((void**)&ws, sizeof(float) * (size_t)splits * M * N, st);
    if (e != cudaSuccess) return e;
  }
  dim3 grid((N + GB_N - 1) / GB_N, (M + GB_M - 1) / GB_M, splits);
  {
  AMM_TRACE_W("sgemm", st, 2.0 * M * N * (double)K,
              4.0 * ((double)M * K + (double)K * N + (double)M * N * (beta != 0.f ? 2 : 1)), nullptr);
#define AMM_SGEMM_LAUNCH(TA_, TB_) \
  sgemm_kernel<TA_, TB_, TIn><<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, kchunk, ws)
  if (!ta && !tb) AMM_SGEMM_LAUNCH(false, false);
  else if (ta && !tb) AMM_SGEMM_LAUNCH(true, false);
  else if (!ta && tb) AMM_SGEMM_LAUNCH(false, true);
  else AMM_SGEMM_LAUNCH(true, true);
#undef AMM_SGEMM_LAUNCH
  }
  e = cudaGetLastError();
  if (e == cudaSuccess && splits > 1) {
    const int64_t tot = (int64_t)M * N;
    AMM_TRACE("splitk_reduce", st);
    splitk_reduce_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(M, N, splits, ws, alpha, beta, C, ldc);
    e = cudaGetLastError();
  }
  if (ws) dev_free(ws, st);
  return e;
}

// ============================================================================ skinny SIMT GEMMs
// The shapes a 128-row tensor-core tile (or the 128 x 128 SIMT tile above) mostly wastes:
//   short contraction: C = alpha A op(B) + beta C with K <= SK_KMAX and a thin output (M or N at
//     most 64), e.g. Y L^{-T} in CholeskyQR (m x k times k x k) or Q_A (Z_A Q_B) in the product;
//   split contraction: 64 x 64 output tiles with K cut into ranges of at most TK_KPER (shorter when
//     there are too few tiles to fill the GPU twice over), e.g. a tiny
//     output over a long K (Z_A Q_B, k x k over n) or CholeskyQR's m x k by k x k applies for
//     64 < k <= 256.
// A is M x K row-major; B is N x K (BT) or K x N.  FP32 arithmetic: every output of the short
// form is one FMA chain over k in order; the split form keeps one FMA chain per K range (staged
// 64 k at a time) and splitk_reduce_kernel sums the ranges' partials in FP64 in range order.
// Both are deterministic.
constexpr int SK_TM = 32, SK_TN = 64, SK_KMAX = 64;
constexpr int TK_T = 64, TK_C = 64, TK_KPER = 256;

template <typename TIn>
__device__ __forceinline__ float ld_elem(const TIn* p) {
  if constexpr (sizeof(TIn) == 2) return __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(p));
  else return __ldg(reinterpret_cast<const float*>(p));
}

template <bool BT, typename TIn>
__global__ void __launch_bounds__(256) gemm_shortk_kernel(int M, int N, int K, float alpha, const TIn* __restrict__ A,
                                                          int64_t lda, const TIn* __restrict__ B, int64_t ldb,
                                                          float beta, float* __restrict__ C, int64_t ldc) {
  __shared__ float As[SK_TM][SK_KMAX + 1];
  __shared__ float Bs[SK_KMAX][SK_TN + 1];
  const int m0 = blockIdx.y * SK_TM, n0 = blockIdx.x * SK_TN;
  for (int e = threadIdx.x; e < SK_TM * K; e += 256) {  // rows of A along k: coalesced
    const int r = e / K, kk = e % K;
    As[r][kk] = m0 + r < M ? ld_elem(A + (int64_t)(m0 + r) * lda + kk) : 0.f;
  }
  for (int e = threadIdx.x; e < SK_TN * K; e += 256) {
    if (BT) {
      const int j = e / K, kk = e % K;
      Bs[kk][j] = n0 + j < N ? ld_elem(B + (int64_t)(n0 + j) * ldb + kk) : 0.f;
    } else {
      const int kk = e / SK_TN, j = e % SK_TN;
      Bs[kk][j] = n0 + j < N ? ld_elem(B + (int64_t)kk * ldb + n0 + j) : 0.f;
    }
  }
  __syncthreads();
  // thread: column j, rows rb, rb + 4, ..., rb + 28 (a warp shares its rows: broadcast reads of As)
  const int j = threadIdx.x & (SK_TN - 1), rb = threadIdx.x / SK_TN;
  constexpr int RPT = SK_TM / (256 / SK_TN);
  float acc[RPT];
#pragma unroll
  for (int i = 0; i < RPT; ++i) acc[i] = 0.f;
  for (int kk = 0; kk < K; ++kk) {
    const float b = Bs[kk][j];
#pragma unroll
    for (int i = 0; i < RPT; ++i) acc[i] = fmaf(As[rb + 4 * i][kk], b, acc[i]);
  }
  const int col = n0 + j;
  if (col >= N) return;
#pragma unroll
  for (int i = 0; i < RPT; ++i) {
    const int row = m0 + rb + 4 * i;
    if (row >= M) break;
    float* c = C + (int64_t)row * ldc + col;
    *c = (beta == 0.f) ? alpha * acc[i] : fmaf(alpha, acc[i], beta * *c);
  }
}

// ws[z][i][j] = sum over the K range z of A(i, k) op(B)(k, j) for the 64 x 64 output tile
// (blockIdx.y, blockIdx.x); thread: column j, rows rb, rb + 4, ..., rb + 60.
template <bool BT, typename TIn>
__global__ void __launch_bounds__(256) gemm_splitk_kernel(int M, int N, int K, int kper, const TIn* __restrict__ A,
                                                          int64_t lda, const TIn* __restrict__ B, int64_t ldb,
                                                          float* __restrict__ ws) {
  __shared__ float As[TK_T][TK_C + 1];
  __shared__ float Bs[TK_T][TK_C + 1];  // [j][k]
  const int m0 = blockIdx.y * TK_T, n0 = blockIdx.x * TK_T;
  const int kbeg = blockIdx.z * kper, kend = min(K, kbeg + kper);
  const int j = threadIdx.x & (TK_T - 1), rb = threadIdx.x / TK_T;
  constexpr int RPT = TK_T / (256 / TK_T);
  float acc[RPT];
#pragma unroll
  for (int i = 0; i < RPT; ++i) acc[i] = 0.f;
  for (int k0 = kbeg; k0 < kend; k0 += TK_C) {
    const int kn = min(TK_C, kend - k0);
    __syncthreads();  // the previous chunk's reads are done
    for (int e = threadIdx.x; e < TK_T * TK_C; e += 256) {
      const int r = e / TK_C, kk = e % TK_C;
      As[r][kk] = (m0 + r < M && kk < kn) ? ld_elem(A + (int64_t)(m0 + r) * lda + k0 + kk) : 0.f;
    }
    for (int e = threadIdx.x; e < TK_T * TK_C; e += 256) {
      if (BT) {
        const int r = e / TK_C, kk = e % TK_C;
        Bs[r][kk] = (n0 + r < N && kk < kn) ? ld_elem(B + (int64_t)(n0 + r) * ldb + k0 + kk) : 0.f;
      } else {
        const int kk = e / TK_T, r = e % TK_T;
        Bs[r][kk] = (n0 + r < N && kk < kn) ? ld_elem(B + (int64_t)(k0 + kk) * ldb + n0 + r) : 0.f;
      }
    }
    __syncthreads();
    for (int kk = 0; kk < kn; ++kk) {
      const float b = Bs[j][kk];
#pragma unroll
      for (int i = 0; i < RPT; ++i) acc[i] = fmaf(As[rb + 4 * i][kk], b, acc[i]);
    }
  }
  const int col = n0 + j;
  if (col >= N) return;
#pragma unroll
  for (int i = 0; i < RPT; ++i) {
    const int row = m0 + rb + 4 * i;
    if (row >= M) break;
    ws[((int64_t)blockIdx.z * M + row) * N + col] = acc[i];
  }
}

template <typename TIn>
static cudaError_t gemm_splitk(bool bt, int M, int N, int K, float alpha, const TIn* A, int64_t lda, const TIn* B,
                               int64_t ldb, float beta, float* C, int64_t ldc, cudaStream_t st) {
  const int tiles = ((M + TK_T - 1) / TK_T) * ((N + TK_T - 1) / TK_T);
  int kper = TK_KPER;  // a multiple of TK_C
  while (kper > TK_C && (int64_t)tiles * ((K + kper - 1) / kper) < 2 * (int64_t)num_sms()) kper /= 2;
  const int ranges = (K + kper - 1) / kper;
  float* ws = nullptr;
  cudaError_t e = dev_alloc((void**)&ws, sizeof(float) * (size_t)ranges * M * N, st);
  if (e == cudaSuccess) {
    AMM_TRACE_W("gemm_splitk", st, 2.0 * M * N * (double)K, (double)sizeof(TIn) * ((double)M + N) * K, nullptr);
    const dim3 grid((unsigned)((N + TK_T - 1) / TK_T), (unsigned)((M + TK_T - 1) / TK_T), (unsigned)ranges);
    if (bt) gemm_splitk_kernel<true, TIn><<<grid, 256, 0, st>>>(M, N, K, kper, A, lda, B, ldb, ws);
    else gemm_splitk_kernel<false, TIn><<<grid, 256, 0, st>>>(M, N, K, kper, A, lda, B, ldb, ws);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    AMM_TRACE("splitk_reduce", st);
    splitk_reduce_kernel<<<(unsigned)(((int64_t)M * N + 255) / 256), 256, 0, st>>>(M, N, ranges, ws, alpha, beta, C,
                                                                                     ldc);
    e = cudaGetLastError();
  }
  if (ws) dev_free(ws, st);
  return e;
}

// the short form for K <= SK_KMAX with a thin output, the split form for a tiny output (M, N <= 64)
// over a longer K; false when the shape is neither
template <typename TIn>
static bool skinny_gemm(bool bt, int M, int N, int K, float alpha, const TIn* A, int64_t lda, const TIn* B,
                        int64_t ldb, float beta, float* C, int64_t ldc, cudaStream_t st, cudaError_t* err) {
  if (M <= 0 || N <= 0 || K <= 0) return false;
  if (K <= SK_KMAX && (M <= 64 || N <= 64)) {
    AMM_TRACE_W("gemm_shortk", st, 2.0 * M * N * (double)K,
                (double)sizeof(TIn) * ((double)M * K + (double)K * N) + 4.0 * M * N * (beta != 0.f ? 2 : 1), nullptr);
    const dim3 grid((unsigned)((N + SK_TN - 1) / SK_TN), (unsigned)((M + SK_TM - 1) / SK_TM));
    if (bt) gemm_shortk_kernel<true, TIn><<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
    else gemm_shortk_kernel<false, TIn><<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
    *err = cudaGetLastError();
    return true;
  }
  if (M <= TK_T && N <= TK_T) {
    *err = gemm_splitk<TIn>(bt, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, st);
    return true;
  }
  return false;
}

// ============================================================================ compensated Gram (FP32)
// G = X^T X for X (m x k, FP32).  Each thread accumulates its dot products with error-free
// transformations (TwoProduct via fma and TwoSum: Ogita, Rump, Oishi, "Accurate sum and dot
// product", SIAM J. Sci. Comput. 2005, Algorithm Dot2), so a partial is as accurate as if it had
// been computed in twice FP32 precision.  K (= m) is split over grid.z; the partials (hi + lo,
// widened to double) are summed in a fixed order and rounded to FP32.
__global__ void __launch_bounds__(256) gram_dot2_kernel(int k, int m, const float* __restrict__ X, int kchunk,
                                                        double* __restrict__ ws) {
  __shared__ float xi[32][33];
  __shared__ float xj[32][33];
  const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
  const int r0 = blockIdx.z * kchunk, r1 = min(m, r0 + kchunk);
  const int ti = threadIdx.x >> 3, tj = (threadIdx.x & 7) * 4;  // (ti, tj..tj+3)
  float s[4] = {0.f, 0.f, 0.f, 0.f}, c[4] = {0.f, 0.f, 0.f, 0.f};
  for (int rb = r0; rb < r1; rb += 32) {
    for (int e = threadIdx.x; e < 32 * 32; e += 256) {
      const int rr = e >> 5, cc = e & 31, r = rb + rr;
      xi[rr][cc] = (r < r1 && i0 + cc < k) ? X[(int64_t)r * k + i0 + cc] : 0.f;
      xj[rr][cc] = (r < r1 && j0 + cc < k) ? X[(int64_t)r * k + j0 + cc] : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int rr = 0; rr < 32; ++rr) {
      const float a = xi[rr][ti];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        // explicit _rn operations: the compiler must not fuse them into FMAs
        const float b = xj[rr][tj + q];
        const float p = __fmul_rn(a, b);
        const float pe = fmaf(a, b, -p);                  // a*b = p + pe exactly
        const float t = __fadd_rn(s[q], p);
        const float z = __fsub_rn(t, s[q]);
        const float se = __fadd_rn(__fsub_rn(s[q], __fsub_rn(t, z)), __fsub_rn(p, z));  // s + p = t + se
        s[q] = t;
        c[q] = __fadd_rn(c[q], __fadd_rn(pe, se));
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = i0 + ti, j = j0 + tj + q;
    if (i < k && j < k) ws[((int64_t)blockIdx.z * k + i) * k + j] = (double)s[q] + (double)c[q];
  }
}

// G = sum of partials; with ns = 1 the output is -(G - I)/2 (Newton-Schulz correction factor),
// formed from the double sum so that the small entries of G - I keep their accuracy.  The order of
// the additions is fixed for a given split count.  WARP: one warp per entry, lane l summing the
// partials l, l + 32, ... and a fixed shuffle tree adding the lanes (a thin Gram at n = 4096 has
// 128 partials per entry); otherwise one thread per entry (few partials, many entries).
template <bool WARP>
__global__ void __launch_bounds__(256) gram_reduce_kernel(int k, int splits, const double* __restrict__ ws,
                                                          float* __restrict__ G, int ns) {
  const int e = WARP ? blockIdx.x * 8 + (threadIdx.x >> 5) : blockIdx.x * 256 + threadIdx.x;
  const int lane = WARP ? threadIdx.x & 31 : 0;
  if (e >= k * k) return;  // WARP: e is uniform across the warp
  double s = 0.0;
  for (int z = lane; z < splits; z += WARP ? 32 : 1) s += ws[(int64_t)z * k * k + e];
  if (WARP) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  }
  if (lane == 0) {
    if (ns) s = -0.5 * (s - ((e / k) == (e % k) ? 1.0 : 0.0));
    G[e] = (float)s;
  }
}

static cudaError_t gram_dot2(int64_t m, int k, const float* X, float* G, cudaStream_t st, int ns = 0) {
  const int tiles = ((k + 31) / 32) * ((k + 31) / 32);
  int splits = std::max(1, std::min((int)(m / 32), (2 * num_sms() + tiles - 1) / tiles));
  int kchunk = (int)((m + splits - 1) / splits);
  kchunk = ((kchunk + 31) / 32) * 32;
  splits = std::max(1, (int)((m + kchunk - 1) / kchunk));
  double* ws = nullptr;
  cudaError_t e = dev_alloc((void**)&ws, sizeof(double) * (size_t)splits * k * k, st);
  if (e != cudaSuccess) return e;
  {
    AMM_TRACE_W("gram_dot2", st, 2.0 * m * (double)k * k, 4.0 * m * (double)k, nullptr);
    dim3 grid((k + 31) / 32, (k + 31) / 32, splits);
    gram_dot2_kernel<<<grid, 256, 0, st>>>(k, (int)m, X, kchunk, ws);
  }
  e = cudaGetLastError();
  if (e == cudaSuccess) {
    AMM_TRACE("gram_reduce", st);
    if (splits >= 32) gram_reduce_kernel<true><<<(k * k + 7) / 8, 256, 0, st>>>(k, splits, ws, G, ns);
    else gram_reduce_kernel<false><<<(k * k + 255) / 256, 256, 0, st>>>(k, splits, ws, G, ns);
    e = cudaGetLastError();
  }
  dev_free(ws, st);
  return e;
}

// ============================================================================ Cholesky + inverse (FP32, one CTA)
// G (k x k, symmetric positive semi-definite) -> Linv = L^{-1} with G + s I = L L^T,
// s = shift_rel * trace(G).  Blocked in 32 x 32 tiles (k padded to kp, a multiple of 32, with an
// identity block), so that the sequential part runs inside one warp without block barriers:
//   per block column J: warp 0 factors the diagonal tile with shuffles (lane r holds row r); the
//   rows below solve against it (x L_JJ^T = a, a thread per row); all threads update the
//   trailing matrix;
//   inverse: every diagonal tile is inverted by its own warp (lane c holds column c of the
//   inverse), then the tiles at distance d = I - J below the diagonal, for d = 1, 2, ...:
//   T_IJ = sum_{J <= K < I} L_IK Linv_KJ (kept in the unused upper triangle of W), then
//   Linv_IJ = -Linv_II T_IJ.
// Rows have the odd stride kp + 1 (conflict-free column walks).  For kp > CHOL_SMEM_K the same
// arrays live in a global work area of 2 kp (kp + 1) floats.
constexpr int CHOL_SMEM_K = 160;
constexpr int CHOL_T = 512;

// Trailing update of a blocked Cholesky step: W(i, l) -= sum_{c < 32} W(i, j0 + c) W(l, j0 + c) for
// j0 + 32 <= l <= i < kp (idx(i, j) locates element (i, j)).  Each thread takes 4 x 4 blocks of the
// lower triangle, so a pair of loads feeds four FMAs instead of one.
template <class IDX>
AMM_DEV void chol_trailing(float* W, IDX idx, int j0, int kp) {
  const int t0 = j0 + 32, mb = (kp - t0) / 4;
  const int nblk = mb * (mb + 1) / 2;
  for (int b = threadIdx.x; b < nblk; b += CHOL_T) {
    int bi = (int)((sqrtf(8.f * (float)b + 1.f) - 1.f) * 0.5f);  // b -> block (bi, bl), bl <= bi
    while (bi * (bi + 1) / 2 > b) --bi;
    while ((bi + 1) * (bi + 2) / 2 <= b) ++bi;
    const int bl = b - bi * (bi + 1) / 2;
    const int i0 = t0 + 4 * bi, l0 = t0 + 4 * bl;
    float acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[r][q] = 0.f;
#pragma unroll 8
    for (int c = 0; c < 32; ++c) {
      float a[4], bb[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = W[idx(i0 + r, j0 + c)];
#pragma unroll
      for (int q = 0; q < 4; ++q) bb[q] = W[idx(l0 + q, j0 + c)];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[r][q] = fmaf(a[r], bb[q], acc[r][q]);
    }
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (l0 + q <= i0 + r) W[idx(i0 + r, l0 + q)] -= acc[r][q];
  }
}
__host__ __device__ constexpr int chol_kp(int k) { return (k + 31) & ~31; }
__host__ __device__ constexpr size_t chol_floats(int k) { return 2 * (size_t)chol_kp(k) * (chol_kp(k) + 1); }

__global__ void __launch_bounds__(CHOL_T) chol_inv_kernel(int k, const float* __restrict__ G, float shift_rel,
                                                          float* __restrict__ Linv_out, float* __restrict__ gwork) {
  extern __shared__ float sh_dyn[];
  const int kp = chol_kp(k), nb = kp / 32, ldw = kp + 1;
  float* sh = (kp <= CHOL_SMEM_K) ? sh_dyn : gwork;
  float* W = sh;               // kp x kp (stride ldw): G + sI, then L in the lower triangle
  float* Li = sh + kp * ldw;   // kp x kp (stride ldw): L^{-1}, lower triangle
  __shared__ float red[32];
  __shared__ float shift_s;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  float tr = 0.f;
  for (int i = tid; i < k; i += CHOL_T) tr += G[(int64_t)i * k + i];
  for (int o = 16; o > 0; o >>= 1) tr += __shfl_xor_sync(0xffffffffu, tr, o);
  if (lane == 0) red[warp] = tr;
  __syncthreads();
  if (tid == 0) {
    float t = 0.f;
    for (int w = 0; w < CHOL_T / 32; ++w) t += red[w];
    shift_s = fmaxf(shift_rel * t, 1e-30f);
  }
  __syncthreads();
  const float shift = shift_s;
  for (int e = tid; e < kp * kp; e += CHOL_T) {
    const int i = e / kp, j = e - i * kp;
    W[i * ldw + j] = (i < k && j < k) ? G[(int64_t)i * k + j] + (i == j ? shift : 0.f) : (i == j ? 1.f : 0.f);
    Li[i * ldw + j] = 0.f;
  }
  __syncthreads();
  for (int J = 0; J < nb; ++J) {
    const int j0 = 32 * J;
    if (warp == 0) {
      // diagonal tile: right-looking Cholesky, lane r holds row r
      float a[32];
#pragma unroll
      for (int c = 0; c < 32; ++c) a[c] = (c <= lane) ? W[(j0 + lane) * ldw + j0 + c] : 0.f;
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        const float d = sqrtf(fmaxf(__shfl_sync(0xffffffffu, a[c], c), shift));
        const float rd = 1.f / d;
        if (lane == c) a[c] = d;
        else if (lane > c) a[c] *= rd;
        const float lrc = a[c];
#pragma unroll
        for (int l = 0; l < 32; ++l) {  // fixed bounds: the loop nest unrolls and a[] stays in registers
          if (l > c) {
            const float llc = __shfl_sync(0xffffffffu, a[c], l);
            if (lane >= l) a[l] = fmaf(-lrc, llc, a[l]);
          }
        }
      }
#pragma unroll
      for (int c = 0; c < 32; ++c)
        if (c <= lane) W[(j0 + lane) * ldw + j0 + c] = a[c];
    }
    __syncthreads();
    // panel below the tile: x L_JJ^T = a, a thread per row
    for (int i = j0 + 32 + tid; i < kp; i += CHOL_T) {
      float* wr = W + i * ldw + j0;
      float x[32];
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        const float* lc = W + (j0 + c) * ldw + j0;
        float v = wr[c];
#pragma unroll
        for (int l = 0; l < c; ++l) v = fmaf(-x[l], lc[l], v);
        x[c] = v * (1.f / lc[c]);
      }
#pragma unroll
      for (int c = 0; c < 32; ++c) wr[c] = x[c];
    }
    __syncthreads();
    chol_trailing(W, [ldw](int i, int j) { return i * ldw + j; }, j0, kp);  // trailing lower triangle
    __syncthreads();
  }
  // inverse of every diagonal tile: lane c holds column c
  for (int J = warp; J < nb; J += CHOL_T / 32) {
    const int j0 = 32 * J;
    float col[32];
#pragma unroll
    for (int r = 0; r < 32; ++r) {
      const float* lr = W + (j0 + r) * ldw + j0;
      float s = 0.f;
#pragma unroll
      for (int l = 0; l < r; ++l) s = fmaf(lr[l], col[l], s);
      const float di = 1.f / lr[r];
      col[r] = (r < lane) ? 0.f : (r == lane) ? di : -s * di;
    }
#pragma unroll
    for (int r = 0; r < 32; ++r)
      if (r >= lane) Li[(j0 + r) * ldw + j0 + lane] = col[r];
  }
  __syncthreads();
  // tiles below the diagonal, by distance d
  for (int d = 1; d < nb; ++d) {
    const int cnt = (nb - d) * 1024;
    for (int e = tid; e < cnt; e += CHOL_T) {
      const int J = e >> 10, r = (e >> 5) & 31, c = e & 31, I = J + d;
      const float* lrow = W + (32 * I + r) * ldw;
      float s = 0.f;
      for (int q = 32 * J; q < 32 * I; ++q) s = fmaf(lrow[q], Li[q * ldw + 32 * J + c], s);
      W[(32 * J + r) * ldw + 32 * I + c] = s;  // T_IJ in the upper triangle
    }
    __syncthreads();
    for (int e = tid; e < cnt; e += CHOL_T) {
      const int J = e >> 10, r = (e >> 5) & 31, c = e & 31, I = J + d;
      const float* lirow = Li + (32 * I + r) * ldw + 32 * I;
      float s = 0.f;
#pragma unroll 8
      for (int q = 0; q <= r; ++q) s = fmaf(lirow[q], W[(32 * J + q) * ldw + 32 * I + c], s);
      Li[(32 * I + r) * ldw + 32 * J + c] = -s;
    }
    __syncthreads();
  }
  for (int e = tid; e < k * k; e += CHOL_T) {
    const int i = e / k, c = e - i * k;
    Linv_out[e] = (c <= i) ? Li[i * ldw + c] : 0.f;
  }
}

// ============================================================================ Cholesky for 160 < kp <= 256
// The two work arrays of chol_inv_kernel do not fit in shared memory beyond kp = 160, and in
// global memory one CTA waits on every access.  Here the factorisation keeps only the lower
// triangle, packed (row i at i (i + 1) / 2: 132 KB at kp = 256), in one CTA with the same blocked
// steps as above, and writes L to global memory; the inverse is then formed by one CTA per
// 32-column block J by blocked forward substitution, X_I = L_II^{-1} (E_IJ - sum_{J <= K < I} L_IK X_K)
// for I = J, J + 1, ... (E the identity), with its column block X in shared memory.
constexpr int CHOL_PACKED_K = 256;
__host__ __device__ constexpr size_t chol_packed_floats(int kp) { return (size_t)kp * (kp + 1) / 2; }
AMM_DEV int tri(int i) { return i * (i + 1) / 2; }

__global__ void __launch_bounds__(CHOL_T) chol_factor_packed_kernel(int k, const float* __restrict__ G, float shift_rel,
                                                                   float* __restrict__ L) {
  extern __shared__ float W[];  // packed lower triangle of G + sI, then of L
  const int kp = chol_kp(k), nb = kp / 32;
  __shared__ float red[32];
  __shared__ float shift_s;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  float tr = 0.f;
  for (int i = tid; i < k; i += CHOL_T) tr += G[(int64_t)i * k + i];
  for (int o = 16; o > 0; o >>= 1) tr += __shfl_xor_sync(0xffffffffu, tr, o);
  if (lane == 0) red[warp] = tr;
  __syncthreads();
  if (tid == 0) {
    float t = 0.f;
    for (int w = 0; w < CHOL_T / 32; ++w) t += red[w];
    shift_s = fmaxf(shift_rel * t, 1e-30f);
  }
  __syncthreads();
  const float shift = shift_s;
  for (int i = warp; i < kp; i += CHOL_T / 32)
    for (int j = lane; j <= i; j += 32)
      W[tri(i) + j] = (i < k && j < k) ? G[(int64_t)i * k + j] + (i == j ? shift : 0.f) : (i == j ? 1.f : 0.f);
  __syncthreads();
  for (int J = 0; J < nb; ++J) {
    const int j0 = 32 * J;
    if (warp == 0) {  // diagonal tile, lane r holds row j0 + r
      float a[32];
#pragma unroll
      for (int c = 0; c < 32; ++c) a[c] = (c <= lane) ? W[tri(j0 + lane) + j0 + c] : 0.f;
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        const float d = sqrtf(fmaxf(__shfl_sync(0xffffffffu, a[c], c), shift));
        const float rd = 1.f / d;
        if (lane == c) a[c] = d;
        else if (lane > c) a[c] *= rd;
        const float lrc = a[c];
#pragma unroll
        for (int l = 0; l < 32; ++l) {
          if (l > c) {
            const float llc = __shfl_sync(0xffffffffu, a[c], l);
            if (lane >= l) a[l] = fmaf(-lrc, llc, a[l]);
          }
        }
      }
#pragma unroll
      for (int c = 0; c < 32; ++c)
        if (c <= lane) W[tri(j0 + lane) + j0 + c] = a[c];
    }
    __syncthreads();
    for (int i = j0 + 32 + tid; i < kp; i += CHOL_T) {  // panel: x L_JJ^T = a, a thread per row
      float* wr = W + tri(i) + j0;
      float x[32];
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        const float* lc = W + tri(j0 + c) + j0;
        float v = wr[c];
#pragma unroll
        for (int l = 0; l < c; ++l) v = fmaf(-x[l], lc[l], v);
        x[c] = v * (1.f / lc[c]);
      }
#pragma unroll
      for (int c = 0; c < 32; ++c) wr[c] = x[c];
    }
    __syncthreads();
    chol_trailing(W, [](int i, int j) { return tri(i) + j; }, j0, kp);  // trailing lower triangle
    __syncthreads();
  }
  for (int i = warp; i < kp; i += CHOL_T / 32)
    for (int j = lane; j < kp; j += 32) L[(int64_t)i * kp + j] = j <= i ? W[tri(i) + j] : 0.f;
}

// CTA J: columns 32 J .. 32 J + 31 of L^{-1} (kp x kp, L from chol_factor_packed_kernel), written to
// Linv (k x k, row-major, the leading k rows / columns).  256 threads.  For each block row I the
// rows i0 .. i0 + 31 of L, columns j0 .. i0 + 31, are first copied to shared memory (coalesced),
// then T = E_IJ - sum_K L_IK X_K is formed there (a thread takes four consecutive columns of one
// row) and warp 0 solves L_II X_I = T.
constexpr int TRINV_T = 256;
constexpr int TRINV_LDX = 36;                       // X row stride (16-byte rows)
constexpr int TRINV_LDL = CHOL_PACKED_K + 1;        // staged L row stride (odd: conflict-free rows)
constexpr size_t TRINV_SMEM = sizeof(float) * ((size_t)CHOL_PACKED_K * TRINV_LDX + 32 * TRINV_LDL + 32 * 33);
__global__ void __launch_bounds__(TRINV_T) chol_trinv_kernel(int k, const float* __restrict__ L,
                                                            float* __restrict__ Linv) {
  extern __shared__ float sm_trinv[];
  float* X = sm_trinv;                              // rows j0.. of the column block, [i - j0][c]
  float* Lr = X + CHOL_PACKED_K * TRINV_LDX;        // staged block row of L, [r][q - j0]
  float* T = Lr + 32 * TRINV_LDL;                   // right-hand side of the tile solve, [r][c]
  const int kp = chol_kp(k), nb = kp / 32, J = blockIdx.x, j0 = 32 * J;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int I = J; I < nb; ++I) {
    const int i0 = 32 * I, w = i0 + 32 - j0;        // staged width: columns j0 .. i0 + 31
    for (int e = tid; e < 32 * w; e += TRINV_T) {
      const int r = e / w, q = e - r * w;
      Lr[r * TRINV_LDL + q] = __ldg(L + (int64_t)(i0 + r) * kp + j0 + q);
    }
    __syncthreads();
    {
      const int r = tid >> 3, c4 = (tid & 7) * 4;   // row r, columns c4 .. c4 + 3
      float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
      if (I == J) {
        s0 = (r == c4) ? 1.f : 0.f;
        s1 = (r == c4 + 1) ? 1.f : 0.f;
        s2 = (r == c4 + 2) ? 1.f : 0.f;
        s3 = (r == c4 + 3) ? 1.f : 0.f;
      }
      const float* lr = Lr + r * TRINV_LDL;
#pragma unroll 4
      for (int q = 0; q < i0 - j0; ++q) {
        const float a = lr[q];
        const float4 x = *reinterpret_cast<const float4*>(X + q * TRINV_LDX + c4);
        s0 = fmaf(-a, x.x, s0);
        s1 = fmaf(-a, x.y, s1);
        s2 = fmaf(-a, x.z, s2);
        s3 = fmaf(-a, x.w, s3);
      }
      float* t = T + r * 33 + c4;
      t[0] = s0;
      t[1] = s1;
      t[2] = s2;
      t[3] = s3;
    }
    __syncthreads();
    if (warp == 0) {  // L_II X_I = T by forward substitution, lane c holds column c
      const float* lt = Lr + (i0 - j0);             // the diagonal tile L_II: lt[r * TRINV_LDL + l]
      float x[32];
#pragma unroll
      for (int r = 0; r < 32; ++r) {
        float v = T[r * 33 + lane];
#pragma unroll
        for (int l = 0; l < r; ++l) v = fmaf(-lt[r * TRINV_LDL + l], x[l], v);
        x[r] = v / lt[r * TRINV_LDL + r];
      }
#pragma unroll
      for (int r = 0; r < 32; ++r) X[(i0 - j0 + r) * TRINV_LDX + lane] = x[r];
    }
    __syncthreads();
  }
  for (int e = tid; e < k * 32; e += TRINV_T) {
    const int i = e >> 5, c = j0 + (e & 31);
    if (c < k) Linv[(int64_t)i * k + c] = i >= j0 ? X[(i - j0) * TRINV_LDX + (e & 31)] : 0.f;
  }
}

// ============================================================================ Philox sketch
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC 2011) keyed by the seed, counter = element
// group; Box-Muller turns each pair of uniforms into two N(0,1) draws.
AMM_DEV void philox_round(uint32_t& c0, uint32_t& c1, uint32_t& c2, uint32_t& c3, uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  uint32_t hi0 = __umulhi(M0, c0), lo0 = M0 * c0;
  uint32_t hi1 = __umulhi(M1, c2), lo1 = M1 * c2;
  uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
  c0 = n0; c1 = n1; c2 = n2; c3 = n3;
}

__global__ void philox_normal_kernel(float* __restrict__ out, int64_t count, uint64_t seed) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g * 4 >= count) return;
  uint32_t c0 = (uint32_t)g, c1 = (uint32_t)(g >> 32), c2 = 0x5EED0001u, c3 = 0;
  uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    philox_round(c0, c1, c2, c3, k0, k1);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  const uint32_t u[4] = {c0, c1, c2, c3};
  float z[4];
#pragma unroll
  for (int q = 0; q < 4; q += 2) {
    const double u1 = ((double)u[q] + 1.0) * (1.0 / 4294967296.0);  // (0, 1]
    const double u2 = (double)u[q + 1] * (1.0 / 4294967296.0);
    const double r = sqrt(-2.0 * log(u1));
    double s, c;
    sincospi(2.0 * u2, &s, &c);
    z[q] = (float)(r * c);
    z[q + 1] = (float)(r * s);
  }
  for (int q = 0; q < 4; ++q)
    if (g * 4 + q < count) out[g * 4 + q] = z[q];
}

// ============================================================================ norms
template <typename T>
__global__ void sumsq_kernel(const T* __restrict__ X, int64_t rows, int64_t cols, int64_t ld,
                             double* __restrict__ partial) {
  double s = 0.0;
  for (int64_t r = blockIdx.x; r < rows; r += gridDim.x) {
    for (int64_t c = threadIdx.x; c < cols; c += blockDim.x) {
      double v;
      if constexpr (sizeof(T) == 2) v = (double)__bfloat162float(X[r * ld + c]);
      else v = (double)X[r * ld + c];
      s += v * v;
    }
  }
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    partial[blockIdx.x] = t;
  }
}

// one warp; lane l sums p[l], p[l+32], ... then a fixed shuffle tree (deterministic)
__global__ void sum_partials_kernel(const double* __restrict__ p, int n, double* __restrict__ out) {
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += 32) s += p[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (threadIdx.x == 0) *out = s;
}

template <typename T>
static cudaError_t sumsq(const T* X, int64_t rows, int64_t cols, int64_t ld, double* out, cudaStream_t st) {
  const int nb = (int)std::min<int64_t>(rows, 1024);
  double* part = nullptr;
  cudaError_t e = dev_alloc((void**)&part, sizeof(double) * nb, st);
  if (e != cudaSuccess) return e;
  {
    AMM_TRACE("sumsq", st);
    sumsq_kernel<T><<<nb, 256, 0, st>>>(X, rows, cols, ld, part);
  }
  {
    AMM_TRACE("sum_partials", st);
    sum_partials_kernel<<<1, 32, 0, st>>>(part, nb, out);
  }
  e = cudaGetLastError();
  dev_free(part, st);
  return e;
}

// W: global work area of at least chol_floats(k) floats (used when chol_kp(k) > CHOL_SMEM_K; for
// kp <= CHOL_PACKED_K it holds L between the factorisation and the inverse)
static cudaError_t chol_inv(int k, const float* G, float shift_rel, float* W, float* Li, cudaStream_t st) {
  static DeviceOnce once;
  const cudaError_t attr = once([] {
    cudaError_t e = cudaFuncSetAttribute((const void*)chol_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(chol_floats(CHOL_SMEM_K) * sizeof(float)));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute((const void*)chol_factor_packed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)(chol_packed_floats(CHOL_PACKED_K) * sizeof(float)));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute((const void*)chol_trinv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)TRINV_SMEM);
    return e;
  });
  if (attr != cudaSuccess) return attr;
  const int kp = chol_kp(k);
  if (kp > CHOL_SMEM_K && kp <= CHOL_PACKED_K) {
    {
      AMM_TRACE_W("chol_factor", st, (double)k * k * k / 3.0 * 2.0, 0.0, nullptr);
      chol_factor_packed_kernel<<<1, CHOL_T, sizeof(float) * chol_packed_floats(kp), st>>>(k, G, shift_rel, W);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    AMM_TRACE_W("chol_trinv", st, (double)k * k * k / 3.0 * 2.0, 0.0, nullptr);
    chol_trinv_kernel<<<kp / 32, TRINV_T, TRINV_SMEM, st>>>(k, W, Li);
    return cudaGetLastError();
  }
  AMM_TRACE_W("chol_inv", st, (double)k * k * k / 3.0 * 2.0 * 2.0, 0.0, nullptr);
  const size_t sm = chol_kp(k) <= CHOL_SMEM_K ? sizeof(float) * chol_floats(k) : 0;
  chol_inv_kernel<<<1, CHOL_T, sm, st>>>(k, G, shift_rel, Li, W);
  return cudaGetLastError();
}

// ============================================================================ orth(Y): shifted CholeskyQR2 + one Newton-Schulz step
// Y (m x k, FP32) -> Q (m x k, FP32 with orthonormal columns, same span).  Each CholQR pass:
// G = X^T X (compensated FP32), G + sI = L L^T and L^{-1} (FP32, one CTA), X <- X L^{-T} (FP32
// GEMM).  Any invertible triangular factor keeps span(Y), so the passes only improve
// orthogonality: the first pass is shifted (s ~ k u ||G||, Fukaya, Kannan, Nakatsukasa,
// Yamamoto, Yanagisawa, "Shifted Cholesky QR", SIAM J. Sci. Comput. 2020) so that it cannot break
// down on rank-deficient sketches, the second restores orthogonality to the level of the FP32
// Cholesky.  A final Newton-Schulz step X <- X (I - (X^T X - I)/2), with X^T X - I taken from the
// accurate Gram, leaves the span unchanged and brings ||X^T X - I|| down to FP32 rounding.
static cudaError_t orthonormalize(int64_t m, int k, const float* Y, float* Q, cudaStream_t st) {
  float *G = nullptr, *W = nullptr, *Li = nullptr, *Q1 = nullptr, *Q2 = nullptr;
  cudaError_t e = cudaSuccess;
  auto al = [&](float** p, size_t cnt) {
    if (e == cudaSuccess) e = dev_alloc((void**)p, sizeof(float) * cnt, st);
  };
  al(&G, (size_t)k * k);
  al(&W, chol_floats(k));
  al(&Li, (size_t)k * k);
  al(&Q1, (size_t)m * k);
  al(&Q2, (size_t)m * k);
  const float shift1 = std::max(1e-5f, 1e-7f * (float)k);
  const float* src = Y;
  float* dsts[2] = {Q1, Q2};
  for (int pass = 0; pass < 2 && e == cudaSuccess; ++pass) {
    e = gram_dot2(m, k, src, G, st);
    if (e == cudaSuccess) e = chol_inv(k, G, pass == 0 ? shift1 : 1e-7f, W, Li, st);
    if (e == cudaSuccess)
      if (!skinny_gemm<float>(true, (int)m, k, k, 1.f, src, k, Li, k, 0.f, dsts[pass], k, st, &e))  // src Linv^T
        e = gemm_splitk<float>(true, (int)m, k, k, 1.f, src, k, Li, k, 0.f, dsts[pass], k, st);
    src = dsts[pass];
  }
  if (e == cudaSuccess) e = gram_dot2(m, k, Q2, G, st, 1);  // G <- -(Q2^T Q2 - I) / 2
  if (e == cudaSuccess) e = cudaMemcpyAsync(Q, Q2, sizeof(float) * (size_t)m * k, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess && !skinny_gemm<float>(false, (int)m, k, k, 1.f, Q2, k, G, k, 1.f, Q, k, st, &e))
    e = gemm_splitk<float>(false, (int)m, k, k, 1.f, Q2, k, G, k, 1.f, Q, k, st);
  for (float* p : {G, W, Li, Q1, Q2}) dev_free(p, st);
  return e;
}

// ============================================================================ tensor-core path
// Y[c][r] = X[r][c] (cols x rows), 32 x 32 tiles through shared memory, with a type cast.
template <typename TI, typename TO>
__global__ void transpose_cast_kernel(const TI* __restrict__ X, int64_t rows, int64_t cols, int64_t ldx,
                                      TO* __restrict__ Y, int64_t ldy) {
  // 64 x 64 tile through padded shared memory; each thread moves 16 elements each way, so
  // 16 independent loads per thread are in flight
  __shared__ float t[64][65];
  const int64_t r0 = (int64_t)blockIdx.y * 64, c0 = (int64_t)blockIdx.x * 64;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int ri = threadIdx.y + 8 * i, ci = threadIdx.x + 32 * h;
      const int64_t r = r0 + ri, c = c0 + ci;
      t[ri][ci] = (r < rows && c < cols) ? (float)X[r * ldx + c] : 0.f;
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 8; ++i) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int ci = threadIdx.y + 8 * i, ri = threadIdx.x + 32 * h;
      const int64_t c = c0 + ci, r = r0 + ri;
      if (r < rows && c < cols) Y[c * ldy + r] = (TO)t[ri][ci];
    }
  }
}

template <typename TI, typename TO>
__global__ void cast_kernel(const TI* __restrict__ X, int64_t rows, int64_t cols, int64_t ldx, TO* __restrict__ Y,
                            int64_t ldy) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= rows * cols) return;
  const int64_t r = e / cols, c = e % cols;
  Y[r * ldy + c] = (TO)(float)X[r * ldx + c];
}

template <typename TI, typename TO>
static cudaError_t transpose_cast(const TI* X, int64_t rows, int64_t cols, int64_t ldx, TO* Y, int64_t ldy,
                                  cudaStream_t st) {
  AMM_TRACE_W("transpose", st, 0.0, (double)rows * cols * (sizeof(TI) + sizeof(TO)), nullptr);
  dim3 grid((unsigned)((cols + 63) / 64), (unsigned)((rows + 63) / 64));
  transpose_cast_kernel<TI, TO><<<grid, dim3(32, 8), 0, st>>>(X, rows, cols, ldx, Y, ldy);
  return cudaGetLastError();
}

cudaError_t sumsq_f32(const float* X, int64_t rows, int64_t cols, int64_t ld, double* out, cudaStream_t st) {
  return sumsq<float>(X, rows, cols, ld, out, st);
}

cudaError_t transpose_f32(const float* X, int64_t rows, int64_t cols, int64_t ldx, float* Y, int64_t ldy,
                          cudaStream_t st) {
  return transpose_cast<float, float>(X, rows, cols, ldx, Y, ldy, st);
}

template <typename TI, typename TO>
static cudaError_t cast(const TI* X, int64_t rows, int64_t cols, int64_t ldx, TO* Y, int64_t ldy, cudaStream_t st) {
  AMM_TRACE_W("cast", st, 0.0, (double)rows * cols * (sizeof(TI) + sizeof(TO)), nullptr);
  const int64_t tot = rows * cols;
  cast_kernel<TI, TO><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(X, rows, cols, ldx, Y, ldy);
  return cudaGetLastError();
}

cudaError_t widen_bf16(const void* X, int64_t rows, int64_t cols, int64_t ldx, float* Y, int64_t ldy,
                       cudaStream_t st) {
  return cast<__nv_bfloat16, float>((const __nv_bfloat16*)X, rows, cols, ldx, Y, ldy, st);
}

// Y = [X1 | X2 | 0] (rows x kpad, E): two thin matrices side by side, zero-padded to kpad columns,
// so that one K-major GEMM evaluates X1 Z1^T + X2 Z2^T with a single pass over its output.
template <typename T1, typename T2, typename E>
__global__ void concat_cols_kernel(const T1* __restrict__ X1, int64_t ld1, int c1, const T2* __restrict__ X2,
                                   int64_t ld2, int c2, int64_t rows, E* __restrict__ Y, int kpad) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= rows * kpad) return;
  const int64_t r = e / kpad;
  const int c = (int)(e % kpad);
  float v = 0.f;
  if (c < c1) v = (float)X1[r * ld1 + c];
  else if (c < c1 + c2) v = (float)X2[r * ld2 + (c - c1)];
  Y[e] = (E)v;
}

template <typename T1, typename T2, typename E>
static cudaError_t concat_cols(const T1* X1, int64_t ld1, int c1, const T2* X2, int64_t ld2, int c2, int64_t rows,
                               E* Y, int kpad, cudaStream_t st) {
  AMM_TRACE_W("concat", st, 0.0, (double)rows * (c1 * sizeof(T1) + c2 * sizeof(T2) + kpad * sizeof(E)), nullptr);
  const int64_t tot = rows * kpad;
  concat_cols_kernel<T1, T2, E><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(X1, ld1, c1, X2, ld2, c2, rows, Y, kpad);
  return cudaGetLastError();
}

static int pad8(int k) { return (k + 7) / 8 * 8; }

// C = alpha A B^T + beta C with A (M x K, lda) and B (N x K, ldb) K-major in the compute type E.
// tcgen05 when every row starts 16-byte aligned, the SIMT kernel otherwise.  (Routing the small
// projections, about 8 MFLOP at n = 4096, to the SIMT kernel was measured no faster: about 18 us
// per product there against 15 - 24 us on the tensor cores.)
template <typename E>
static cudaError_t gemm_tn(int M, int N, int K, float alpha, const E* A, int64_t lda, const E* B, int64_t ldb,
                           float beta, float* C, int64_t ldc, int* err, cudaStream_t st) {
  cudaError_t se = cudaSuccess;
  if (skinny_gemm<E>(true, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, st, &se)) return se;
  const bool aligned = ((uintptr_t)A % 16 == 0) && ((uintptr_t)B % 16 == 0) && (lda * sizeof(E)) % 16 == 0 &&
                       (ldb * sizeof(E)) % 16 == 0;
  if (aligned && K > 0)
    return umma_gemm_tn(std::is_same<E, float>::value, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, err, st);
  return sgemm<E>(false, true, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, st);
}

// FP32 -> E copy of a small matrix (no copy when E is float)
template <typename E>
static cudaError_t to_e(Handle* h, const float* X, int64_t rows, int64_t cols, const E** out, cudaStream_t st) {
  if constexpr (std::is_same<E, float>::value) {
    *out = X;
    return cudaSuccess;
  } else {
    E* y = nullptr;
    cudaError_t e = h ? h->alloc((void**)&y, sizeof(E) * rows * cols) : dev_alloc((void**)&y, sizeof(E) * rows * cols, st);
    if (e != cudaSuccess) return e;
    *out = y;
    return cast<float, E>(X, rows, cols, cols, y, cols, st);
  }
}

template <typename E>
static cudaError_t svd_build_tc(Handle* h) {
  auto& s = h->svd;
  cudaStream_t st = h->stream;
  const int64_t m = h->rows, n = h->cols;
  const int k = (int)h->k;
  cudaError_t e;
  // operand copies: X in E (K-major), X^T in E, phi^T in E
  const bool in_bf16 = h->dtype == AMM_BF16;
  const bool direct = (std::is_same<E, float>::value != in_bf16) && ((uintptr_t)h->A % 16 == 0) &&
                      (h->lda * (int64_t)sizeof(E)) % 16 == 0;
  if (direct) {
    s.Xe = h->A;
    s.ldxe = h->lda;
  } else {
    E* xe = nullptr;
    if ((e = h->alloc((void**)&xe, sizeof(E) * m * n)) != cudaSuccess) return e;
    e = in_bf16 ? cast<__nv_bfloat16, E>((const __nv_bfloat16*)h->A, m, n, h->lda, xe, n, st)
                : cast<float, E>((const float*)h->A, m, n, h->lda, xe, n, st);
    if (e != cudaSuccess) return e;
    s.Xe = xe;
    s.ldxe = n;
  }
  E* xte = nullptr;
  E* phit = nullptr;
  if ((e = h->alloc((void**)&xte, sizeof(E) * m * n)) != cudaSuccess) return e;
  if ((e = h->alloc((void**)&phit, sizeof(E) * n * k)) != cudaSuccess) return e;
  s.XTe = xte;
  e = in_bf16 ? transpose_cast<__nv_bfloat16, E>((const __nv_bfloat16*)h->A, m, n, h->lda, xte, m, st)
              : transpose_cast<float, E>((const float*)h->A, m, n, h->lda, xte, m, st);
  if (e == cudaSuccess) e = transpose_cast<float, E>(s.phi, n, k, k, phit, n, st);
  if (e != cudaSuccess) return e;
  const E* Xe = (const E*)s.Xe;
  // Y = X phi  -> rows x k
  float* Y = nullptr;
  if ((e = dev_alloc((void**)&Y, sizeof(float) * m * k, st)) != cudaSuccess) return e;
  e = gemm_tn<E>((int)m, k, (int)n, 1.f, Xe, s.ldxe, phit, n, 0.f, Y, k, s.err, st);
  if (e == cudaSuccess) e = orthonormalize(m, k, Y, s.Q, st);
  dev_free(Y, st);
  if (e != cudaSuccess) return e;
  const E* qe = nullptr;
  if ((e = to_e<E>(h, s.Q, m, k, &qe, st)) != cudaSuccess) return e;
  s.Qe = (void*)qe;
  E* qte = nullptr;
  if ((e = h->alloc((void**)&qte, sizeof(E) * m * k)) != cudaSuccess) return e;
  if ((e = transpose_cast<float, E>(s.Q, m, k, k, qte, m, st)) != cudaSuccess) return e;
  s.QTe = qte;
  // Z = Q^T X (k x n) and Z^T (n x k), FP32 and E
  float* ZT = nullptr;
  if ((e = h->alloc((void**)&ZT, sizeof(float) * n * k)) != cudaSuccess) return e;
  if (h->role == AMM_LEFT) {
    e = gemm_tn<E>(k, (int)n, (int)m, 1.f, qte, m, xte, m, 0.f, s.X, n, s.err, st);
    if (e == cudaSuccess) e = transpose_cast<float, float>(s.X, k, n, n, ZT, k, st);
  } else {
    e = gemm_tn<E>((int)n, k, (int)m, 1.f, xte, m, qte, m, 0.f, ZT, k, s.err, st);
    if (e == cudaSuccess) e = transpose_cast<float, float>(ZT, n, k, k, s.X, n, st);
  }
  if (e != cudaSuccess) return e;
  const E *ze = nullptr, *zte = nullptr;
  if ((e = to_e<E>(h, s.X, k, n, &ze, st)) != cudaSuccess) return e;
  if ((e = to_e<E>(h, ZT, n, k, &zte, st)) != cudaSuccess) return e;
  s.Ze = (void*)ze;
  s.ZTe = (void*)zte;
  return e;  // the norms of amm_handle_info are computed when asked (svd_info)
}

template <typename E>
static cudaError_t svd_matmul_tc(Handle* a, Handle* b, float* C, int64_t ldc, cudaStream_t st) {
  const int m = (int)a->rows, n = (int)a->cols, p = (int)b->cols;
  const int ka = (int)a->k, kb = (int)b->k, kk = pad8(ka + kb);
  auto &sa = a->svd, &sb = b->svd;
  int* err = sa.err;
  float *T1T = nullptr, *W = nullptr, *ZZ = nullptr;
  E *L = nullptr, *R = nullptr;
  const E* zze = nullptr;
  cudaError_t e = dev_alloc((void**)&T1T, sizeof(float) * (size_t)p * ka, st);
  if (e == cudaSuccess) e = dev_alloc((void**)&W, sizeof(float) * (size_t)m * kb, st);
  if (e == cudaSuccess) e = dev_alloc((void**)&ZZ, sizeof(float) * (size_t)kb * ka, st);
  if (e == cudaSuccess) e = dev_alloc((void**)&L, sizeof(E) * (size_t)m * kk, st);
  if (e == cudaSuccess) e = dev_alloc((void**)&R, sizeof(E) * (size_t)p * kk, st);
  // T1^T = B^T Z_A^T ; W = A Q_B ; (Z_A Q_B)^T = Q_B^T Z_A^T ; W -= Q_A (Z_A Q_B)
  if (e == cudaSuccess) e = gemm_tn<E>(p, ka, n, 1.f, (const E*)sb.XTe, n, (const E*)sa.Ze, n, 0.f, T1T, ka, err, st);
  if (e == cudaSuccess) e = gemm_tn<E>(m, kb, n, 1.f, (const E*)sa.Xe, sa.ldxe, (const E*)sb.QTe, n, 0.f, W, kb, err, st);
  if (e == cudaSuccess) e = gemm_tn<E>(kb, ka, n, 1.f, (const E*)sb.QTe, n, (const E*)sa.Ze, n, 0.f, ZZ, ka, err, st);
  if (e == cudaSuccess) e = to_e<E>(nullptr, ZZ, kb, ka, &zze, st);
  if (e == cudaSuccess) e = gemm_tn<E>(m, kb, ka, -1.f, (const E*)sa.Qe, ka, zze, ka, 1.f, W, kb, err, st);
  // C = Q_A T1 + W Z_B = [Q_A | W] [T1^T | Z_B^T]^T: one pass over C
  if (e == cudaSuccess) e = concat_cols<E, float, E>((const E*)sa.Qe, ka, ka, W, kb, kb, m, L, kk, st);
  if (e == cudaSuccess) e = concat_cols<float, E, E>(T1T, ka, ka, (const E*)sb.ZTe, kb, kb, p, R, kk, st);
  if (e == cudaSuccess) e = gemm_tn<E>(m, p, kk, 1.f, L, kk, R, kk, 0.f, C, ldc, err, st);
  if constexpr (!std::is_same<E, float>::value) dev_free((void*)zze, st);
  for (float* q : {T1T, W, ZZ}) dev_free(q, st);
  dev_free(L, st);
  dev_free(R, st);
  return e;
}

template <typename E>
static cudaError_t svd_backward_tc(Handle* a, Handle* b, const float* G, int64_t ldg, float* dA, int64_t ldda,
                                   float* dB, int64_t lddb, cudaStream_t st) {
  const int m = (int)a->rows, n = (int)a->cols, p = (int)b->cols;
  const int ka = (int)a->k, kb = (int)b->k;
  auto &sa = a->svd, &sb = b->svd;
  int* err = sa.err;
  std::vector<void*> tmp;
  cudaError_t e = cudaSuccess;
  auto al = [&](size_t bytes) -> void* {
    void* q = nullptr;
    if (e == cudaSuccess) e = dev_alloc(&q, bytes, st);
    if (q) tmp.push_back(q);
    return q;
  };
  auto as_e = [&](const float* X, int64_t r, int64_t c) -> const E* {
    const E* y = nullptr;
    if (e == cudaSuccess) e = to_e<E>(nullptr, X, r, c, &y, st);
    if constexpr (!std::is_same<E, float>::value) tmp.push_back((void*)y);
    return y;
  };
  // G and G^T in E
  const E* Ge = nullptr;
  int64_t ldge = ldg;
  if constexpr (std::is_same<E, float>::value) {
    Ge = G;
  } else {
    E* g = (E*)al(sizeof(E) * (size_t)m * p);
    if (e == cudaSuccess) e = cast<float, E>(G, m, p, ldg, g, p, st);
    Ge = g;
    ldge = p;
  }
  E* GTe = (E*)al(sizeof(E) * (size_t)m * p);
  if (e == cudaSuccess) e = transpose_cast<float, E>(G, m, p, ldg, GTe, m, st);
  // H2^T = G^T Q_A (p x ka), H2 = (H2^T)^T
  float* H2T = (float*)al(sizeof(float) * (size_t)p * ka);
  float* H2 = (float*)al(sizeof(float) * (size_t)p * ka);
  if (e == cudaSuccess) e = gemm_tn<E>(p, ka, m, 1.f, GTe, m, (const E*)sa.QTe, m, 0.f, H2T, ka, err, st);
  if (e == cudaSuccess) e = transpose_cast<float, float>(H2T, p, ka, ka, H2, p, st);
  const E* H2e = as_e(H2, ka, p);
  if (dA) {
    // dA = (G Z_B^T) Q_B^T + Q_A [ H2 B^T - (H2 Z_B^T) Q_B^T ]
    float* H1 = (float*)al(sizeof(float) * (size_t)m * kb);
    if (e == cudaSuccess) e = gemm_tn<E>(m, kb, p, 1.f, Ge, ldge, (const E*)sb.Ze, p, 0.f, H1, kb, err, st);
    float* H3T = (float*)al(sizeof(float) * (size_t)n * ka);
    float* H4 = (float*)al(sizeof(float) * (size_t)ka * kb);
    if (e == cudaSuccess)
      e = gemm_tn<E>(n, ka, p, 1.f, (const E*)sb.Xe, sb.ldxe, H2e, p, 0.f, H3T, ka, err, st);  // B H2^T
    if (e == cudaSuccess) e = gemm_tn<E>(ka, kb, p, 1.f, H2e, p, (const E*)sb.Ze, p, 0.f, H4, kb, err, st);
    const E* H4e = as_e(H4, ka, kb);
    if (e == cudaSuccess) e = gemm_tn<E>(n, ka, kb, -1.f, (const E*)sb.Qe, kb, H4e, kb, 1.f, H3T, ka, err, st);
    // dA = [H1 | Q_A] [Q_B | H3^T]^T: one pass over dA
    const int kk = pad8(ka + kb);
    E* Lc = (E*)al(sizeof(E) * (size_t)m * kk);
    E* Rc = (E*)al(sizeof(E) * (size_t)n * kk);
    if (e == cudaSuccess) e = concat_cols<float, E, E>(H1, kb, kb, (const E*)sa.Qe, ka, ka, m, Lc, kk, st);
    if (e == cudaSuccess) e = concat_cols<E, float, E>((const E*)sb.Qe, kb, kb, H3T, ka, ka, n, Rc, kk, st);
    if (e == cudaSuccess) e = gemm_tn<E>(m, n, kk, 1.f, Lc, kk, Rc, kk, 0.f, dA, ldda, err, st);
  }
  if (dB) {
    // W^T = Q_B^T A^T - (Z_A Q_B)^T Q_A^T ; dB = Z_A^T H2 + Q_B (W^T G)
    float* WT = (float*)al(sizeof(float) * (size_t)kb * m);
    float* ZZ = (float*)al(sizeof(float) * (size_t)kb * ka);
    if (e == cudaSuccess) e = gemm_tn<E>(kb, m, n, 1.f, (const E*)sb.QTe, n, (const E*)sa.Xe, sa.ldxe, 0.f, WT, m, err, st);
    if (e == cudaSuccess) e = gemm_tn<E>(kb, ka, n, 1.f, (const E*)sb.QTe, n, (const E*)sa.Ze, n, 0.f, ZZ, ka, err, st);
    const E* ZZe = as_e(ZZ, kb, ka);
    if (e == cudaSuccess) e = gemm_tn<E>(kb, m, ka, -1.f, ZZe, ka, (const E*)sa.Qe, ka, 1.f, WT, m, err, st);
    const E* WTe = as_e(WT, kb, m);
    float* H5T = (float*)al(sizeof(float) * (size_t)p * kb);
    if (e == cudaSuccess) e = gemm_tn<E>(p, kb, m, 1.f, GTe, m, WTe, m, 0.f, H5T, kb, err, st);
    // dB = Z_A^T H2 + Q_B H5 = [Z_A^T | Q_B] [H2^T | H5^T]^T: one pass over dB
    const int kk = pad8(ka + kb);
    E* Lc = (E*)al(sizeof(E) * (size_t)n * kk);
    E* Rc = (E*)al(sizeof(E) * (size_t)p * kk);
    if (e == cudaSuccess) e = concat_cols<E, E, E>((const E*)sa.ZTe, ka, ka, (const E*)sb.Qe, kb, kb, n, Lc, kk, st);
    if (e == cudaSuccess) e = concat_cols<float, float, E>(H2T, ka, ka, H5T, kb, kb, p, Rc, kk, st);
    if (e == cudaSuccess) e = gemm_tn<E>(n, p, kk, 1.f, Lc, kk, Rc, kk, 0.f, dB, lddb, err, st);
  }
  for (void* q : tmp) dev_free(q, st);
  return e;
}

// ============================================================================ mixed-method pieces
// Applies of one SVD truncation to a dense FP32 matrix, for products whose other operand uses a
// different method.  A~ = Q_A Z_A with Z_A = Q_A^T A (k x n); B~ = Q_B Z_B.
template <typename E>
static cudaError_t as_kmajor(const float* X, int64_t rows, int64_t cols, int64_t ldx, const E** out, E** owned,
                             cudaStream_t st) {
  *owned = nullptr;
  if (std::is_same<E, float>::value && ((uintptr_t)X % 16) == 0 && (ldx * 4) % 16 == 0) {
    *out = (const E*)X;
    return cudaSuccess;
  }
  E* y = nullptr;
  cudaError_t e = dev_alloc((void**)&y, sizeof(E) * rows * cols, st);
  if (e != cudaSuccess) return e;
  *owned = y;
  *out = y;
  return cast<float, E>(X, rows, cols, ldx, y, cols, st);
}

// C = Q_A (Z_A X) + beta C for X (n x p)
template <typename E>
static cudaError_t svd_left_apply_t(Handle* a, const float* X, int64_t ldx, int64_t p, float* C, int64_t ldc, float beta,
                                    cudaStream_t st) {
  const int m = (int)a->rows, n = (int)a->cols, k = (int)a->k;
  E* xt = nullptr;
  float* TT = nullptr;
  const E* tte = nullptr;
  cudaError_t e = dev_alloc((void**)&xt, sizeof(E) * (size_t)p * n, st);
  if (e == cudaSuccess) e = dev_alloc((void**)&TT, sizeof(float) * (size_t)p * k, st);
  if (e == cudaSuccess) e = transpose_cast<float, E>(X, n, p, ldx, xt, n, st);  // X^T, K-major over n
  if (e == cudaSuccess) e = gemm_tn<E>((int)p, k, n, 1.f, xt, n, (const E*)a->svd.Ze, n, 0.f, TT, k, a->svd.err, st);
  if (e == cudaSuccess) e = to_e<E>(nullptr, TT, p, k, &tte, st);
  if (e == cudaSuccess)
    e = gemm_tn<E>(m, (int)p, k, 1.f, (const E*)a->svd.Qe, k, tte, k, beta, C, ldc, a->svd.err, st);
  if constexpr (!std::is_same<E, float>::value) dev_free((void*)tte, st);
  dev_free(xt, st);
  dev_free(TT, st);
  return e;
}

// C = (Y Q_B) Z_B + beta C for Y (m x n)
template <typename E>
static cudaError_t svd_right_apply_t(Handle* b, const float* Y, int64_t ldy, int64_t m, float* C, int64_t ldc,
                                     float beta, cudaStream_t st) {
  const int n = (int)b->rows, p = (int)b->cols, k = (int)b->k;
  const E* ye = nullptr;
  E* yown = nullptr;
  float* W = nullptr;
  const E* we = nullptr;
  cudaError_t e = as_kmajor<E>(Y, m, n, ldy, &ye, &yown, st);
  const int64_t ldye = yown ? n : ldy;
  if (e == cudaSuccess) e = dev_alloc((void**)&W, sizeof(float) * (size_t)m * k, st);
  if (e == cudaSuccess) e = gemm_tn<E>((int)m, k, n, 1.f, ye, ldye, (const E*)b->svd.QTe, n, 0.f, W, k, b->svd.err, st);
  if (e == cudaSuccess) e = to_e<E>(nullptr, W, m, k, &we, st);
  if (e == cudaSuccess)
    e = gemm_tn<E>((int)m, p, k, 1.f, we, k, (const E*)b->svd.ZTe, k, beta, C, ldc, b->svd.err, st);
  if constexpr (!std::is_same<E, float>::value) dev_free((void*)we, st);
  dev_free(yown, st);
  dev_free(W, st);
  return e;
}

// D = A - Q_A Z_A (m x n, FP32)
template <typename E>
static cudaError_t svd_residual_t(Handle* a, float* D, int64_t ldd, cudaStream_t st) {
  const int m = (int)a->rows, n = (int)a->cols, k = (int)a->k;
  cudaError_t e = a->dtype == AMM_BF16
                      ? cast<__nv_bfloat16, float>((const __nv_bfloat16*)a->A, m, n, a->lda, D, ldd, st)
                      : cast<float, float>((const float*)a->A, m, n, a->lda, D, ldd, st);
  if (e == cudaSuccess)
    e = gemm_tn<E>(m, n, k, -1.f, (const E*)a->svd.Qe, k, (const E*)a->svd.ZTe, k, 1.f, D, ldd, a->svd.err, st);
  return e;
}

// Pieces of the backward of a mixed-method product (thin GEMMs on the handle's Q and Z).
// Scratch helpers: a float buffer and a K-major copy in E of a float matrix.
template <typename E>
struct SvdScratch {
  cudaStream_t st;
  std::vector<void*> bufs;
  cudaError_t e = cudaSuccess;
  explicit SvdScratch(cudaStream_t s) : st(s) {}
  float* f(size_t cnt) {
    void* q = nullptr;
    if (e == cudaSuccess) e = dev_alloc(&q, sizeof(float) * cnt, st);
    if (q) bufs.push_back(q);
    return (float*)q;
  }
  // Y = X^T in E (cols x rows)
  const E* tr(const float* X, int64_t rows, int64_t cols, int64_t ldx) {
    void* q = nullptr;
    if (e == cudaSuccess) e = dev_alloc(&q, sizeof(E) * rows * cols, st);
    if (q) bufs.push_back(q);
    if (e == cudaSuccess) e = transpose_cast<float, E>(X, rows, cols, ldx, (E*)q, rows, st);
    return (const E*)q;
  }
  // X in E, K-major as it is (rows x cols, leading dimension cols when copied)
  const E* km(const float* X, int64_t rows, int64_t cols, int64_t ldx, int64_t* ld) {
    const E* out = nullptr;
    E* own = nullptr;
    if (e == cudaSuccess) e = as_kmajor<E>(X, rows, cols, ldx, &out, &own, st);
    if (own) bufs.push_back(own);
    *ld = own ? cols : ldx;
    return out;
  }
  const E* ke(const float* X, int64_t rows, int64_t cols) {  // contiguous float -> E
    const E* out = nullptr;
    if (e == cudaSuccess) e = to_e<E>(nullptr, X, rows, cols, &out, st);
    if (!std::is_same<E, float>::value && out) bufs.push_back((void*)out);
    return out;
  }
  ~SvdScratch() {
    for (void* q : bufs) dev_free(q, st);
  }
};

// out = G B~^T = (G Z_B^T) Q_B^T, G (m x p), out (m x n)
template <typename E>
static cudaError_t svd_rt_apply_t(Handle* b, const float* G, int64_t ldg, int64_t m, float* out, int64_t ldo,
                                  cudaStream_t st) {
  const int n = (int)b->rows, p = (int)b->cols, k = (int)b->k;
  SvdScratch<E> sc(st);
  int64_t ldge = 0;
  const E* ge = sc.km(G, m, p, ldg, &ldge);
  float* T = sc.f((size_t)m * k);
  if (sc.e == cudaSuccess) sc.e = gemm_tn<E>((int)m, k, p, 1.f, ge, ldge, (const E*)b->svd.Ze, p, 0.f, T, k, b->svd.err, st);
  const E* te = sc.ke(T, m, k);
  if (sc.e == cudaSuccess) sc.e = gemm_tn<E>((int)m, n, k, 1.f, te, k, (const E*)b->svd.Qe, k, 0.f, out, ldo, b->svd.err, st);
  return sc.e;
}

// out = A~^T G = Z_A^T (Q_A^T G), G (m x p), out (n x p)
template <typename E>
static cudaError_t svd_lt_apply_t(Handle* a, const float* G, int64_t ldg, int64_t p, float* out, int64_t ldo,
                                  cudaStream_t st) {
  const int m = (int)a->rows, n = (int)a->cols, k = (int)a->k;
  SvdScratch<E> sc(st);
  const E* gt = sc.tr(G, m, p, ldg);  // p x m
  float* T = sc.f((size_t)k * p);
  if (sc.e == cudaSuccess) sc.e = gemm_tn<E>(k, (int)p, m, 1.f, (const E*)a->svd.QTe, m, gt, m, 0.f, T, p, a->svd.err, st);
  const E* tt = sc.tr(T, k, p, p);    // p x k
  if (sc.e == cudaSuccess) sc.e = gemm_tn<E>(n, (int)p, k, 1.f, (const E*)a->svd.ZTe, k, tt, k, 0.f, out, ldo, a->svd.err, st);
  return sc.e;
}

// out += Q_A Q_A^T (G D^T), G (m x p), D (n x p), out (m x n)
template <typename E>
static cudaError_t svd_proj_left_t(Handle* a, const float* G, int64_t ldg, const float* D, int64_t ldd, int64_t p,
                                   float* out, int64_t ldo, cudaStream_t st) {
  const int m = (int)a->rows, n = (int)a->cols, k = (int)a->k;
  SvdScratch<E> sc(st);
  const E* gt = sc.tr(G, m, p, ldg);
  float* T = sc.f((size_t)k * p);
  if (sc.e == cudaSuccess) sc.e = gemm_tn<E>(k, (int)p, m, 1.f, (const E*)a->svd.QTe, m, gt, m, 0.f, T, p, a->svd.err, st);
  const E* te = sc.ke(T, k, p);
  int64_t ldde = 0;
  const E* de = sc.km(D, n, p, ldd, &ldde);
  float* U = sc.f((size_t)k * n);
  if (sc.e == cudaSuccess) sc.e = gemm_tn<E>(k, n, (int)p, 1.f, te, p, de, ldde, 0.f, U, n, a->svd.err, st);
  const E* ut = sc.tr(U, k, n, n);    // n x k
  if (sc.e == cudaSuccess) sc.e = gemm_tn<E>(m, n, k, 1.f, (const E*)a->svd.Qe, k, ut, k, 1.f, out, ldo, a->svd.err, st);
  return sc.e;
}

// out += Q_B Q_B^T (D^T G), D (m x n), G (m x p), out (n x p)
template <typename E>
static cudaError_t svd_proj_right_t(Handle* b, const float* D, int64_t ldd, const float* G, int64_t ldg, int64_t m,
                                    float* out, int64_t ldo, cudaStream_t st) {
  const int n = (int)b->rows, p = (int)b->cols, k = (int)b->k;
  SvdScratch<E> sc(st);
  int64_t ldde = 0;
  const E* de = sc.km(D, m, n, ldd, &ldde);
  float* V = sc.f((size_t)m * k);
  if (sc.e == cudaSuccess) sc.e = gemm_tn<E>((int)m, k, n, 1.f, de, ldde, (const E*)b->svd.QTe, n, 0.f, V, k, b->svd.err, st);
  const E* vt = sc.tr(V, m, k, k);    // k x m
  const E* gt = sc.tr(G, m, p, ldg);  // p x m
  float* U = sc.f((size_t)k * p);
  if (sc.e == cudaSuccess) sc.e = gemm_tn<E>(k, p, (int)m, 1.f, vt, m, gt, m, 0.f, U, p, b->svd.err, st);
  const E* ut = sc.tr(U, k, p, p);    // p x k
  if (sc.e == cudaSuccess) sc.e = gemm_tn<E>(n, p, k, 1.f, (const E*)b->svd.Qe, k, ut, k, 1.f, out, ldo, b->svd.err, st);
  return sc.e;
}

cudaError_t svd_rt_apply(Handle* b, const float* G, int64_t ldg, int64_t m, float* out, int64_t ldo, cudaStream_t st) {
  return b->svd.bf16 ? svd_rt_apply_t<__nv_bfloat16>(b, G, ldg, m, out, ldo, st)
                     : svd_rt_apply_t<float>(b, G, ldg, m, out, ldo, st);
}
cudaError_t svd_lt_apply(Handle* a, const float* G, int64_t ldg, int64_t p, float* out, int64_t ldo, cudaStream_t st) {
  return a->svd.bf16 ? svd_lt_apply_t<__nv_bfloat16>(a, G, ldg, p, out, ldo, st)
                     : svd_lt_apply_t<float>(a, G, ldg, p, out, ldo, st);
}
cudaError_t svd_proj_left(Handle* a, const float* G, int64_t ldg, const float* D, int64_t ldd, int64_t p, float* out,
                          int64_t ldo, cudaStream_t st) {
  return a->svd.bf16 ? svd_proj_left_t<__nv_bfloat16>(a, G, ldg, D, ldd, p, out, ldo, st)
                     : svd_proj_left_t<float>(a, G, ldg, D, ldd, p, out, ldo, st);
}
cudaError_t svd_proj_right(Handle* b, const float* D, int64_t ldd, const float* G, int64_t ldg, int64_t m, float* out,
                           int64_t ldo, cudaStream_t st) {
  return b->svd.bf16 ? svd_proj_right_t<__nv_bfloat16>(b, D, ldd, G, ldg, m, out, ldo, st)
                     : svd_proj_right_t<float>(b, D, ldd, G, ldg, m, out, ldo, st);
}

cudaError_t svd_left_apply(Handle* a, const float* X, int64_t ldx, int64_t p, float* C, int64_t ldc, float beta,
                           cudaStream_t st) {
  return a->svd.bf16 ? svd_left_apply_t<__nv_bfloat16>(a, X, ldx, p, C, ldc, beta, st)
                     : svd_left_apply_t<float>(a, X, ldx, p, C, ldc, beta, st);
}
cudaError_t svd_right_apply(Handle* b, const float* Y, int64_t ldy, int64_t m, float* C, int64_t ldc, float beta,
                            cudaStream_t st) {
  return b->svd.bf16 ? svd_right_apply_t<__nv_bfloat16>(b, Y, ldy, m, C, ldc, beta, st)
                     : svd_right_apply_t<float>(b, Y, ldy, m, C, ldc, beta, st);
}
cudaError_t svd_residual(Handle* a, float* D, int64_t ldd, cudaStream_t st) {
  return a->svd.bf16 ? svd_residual_t<__nv_bfloat16>(a, D, ldd, st) : svd_residual_t<float>(a, D, ldd, st);
}

// ============================================================================ ABI glue
amm_status_t decompose_svd(Handle* h, const amm_opts_t* o) {
  if (h->k > 1024) return fail(AMM_ERR_UNSUPPORTED_SIZE, "svd: k=%lld > 1024", (long long)h->k);
  const int compute = o ? o->compute : AMM_F32;
  if (compute != AMM_F32 && compute != AMM_BF16) return fail(AMM_ERR_INVALID_ARG, "svd: bad compute mode %d", compute);
  auto& s = h->svd;
  const int64_t m = h->rows, n = h->cols, k = h->k;
  cudaError_t e;
  if ((e = h->alloc((void**)&s.phi, sizeof(float) * (size_t)n * k)) != cudaSuccess ||
      (e = h->alloc((void**)&s.Q, sizeof(float) * (size_t)m * k)) != cudaSuccess ||
      (e = h->alloc((void**)&s.X, sizeof(float) * (size_t)k * n)) != cudaSuccess ||
      (e = h->alloc((void**)&s.norms, sizeof(double) * 2)) != cudaSuccess)
    return cuda_fail(e, "svd: device allocation");
  if (o && o->sketch) {
    e = cudaMemcpyAsync(s.phi, o->sketch, sizeof(float) * (size_t)n * k, cudaMemcpyDeviceToDevice, h->stream);
  } else {
    const int64_t cnt = n * k;
    AMM_TRACE("philox", h->stream);
    philox_normal_kernel<<<(unsigned)((cnt / 4 + 256) / 256), 256, 0, h->stream>>>(s.phi, cnt, o ? o->seed : 0);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return cuda_fail(e, "svd: sketch");
  if ((e = h->alloc((void**)&s.err, sizeof(int))) != cudaSuccess) return cuda_fail(e, "svd: device allocation");
  if ((e = cudaMemsetAsync(s.err, 0, sizeof(int), h->stream)) != cudaSuccess) return cuda_fail(e, "svd: memset");
  s.bf16 = compute == AMM_BF16;
  e = s.bf16 ? svd_build_tc<__nv_bfloat16>(h) : svd_build_tc<float>(h);
  if (e != cudaSuccess) return cuda_fail(e, "svd: decomposition");
  return AMM_OK;
}

amm_status_t svd_matmul(Handle* a, Handle* b, float* C, int64_t ldc, cudaStream_t st) {
  if (a->svd.bf16 != b->svd.bf16) return fail(AMM_ERR_STATE, "svd: both operands need the same compute mode");
  cudaError_t e = a->svd.bf16 ? svd_matmul_tc<__nv_bfloat16>(a, b, C, ldc, st) : svd_matmul_tc<float>(a, b, C, ldc, st);
  if (e != cudaSuccess) return cuda_fail(e, "svd product");
  return AMM_OK;
}

amm_status_t svd_backward(Handle* a, Handle* b, const float* G, int64_t ldg, float* dA, int64_t ldda, float* dB,
                          int64_t lddb, cudaStream_t st) {
  if (a->svd.bf16 != b->svd.bf16) return fail(AMM_ERR_STATE, "svd: both operands need the same compute mode");
  cudaError_t e = a->svd.bf16 ? svd_backward_tc<__nv_bfloat16>(a, b, G, ldg, dA, ldda, dB, lddb, st)
                              : svd_backward_tc<float>(a, b, G, ldg, dA, ldda, dB, lddb, st);
  if (e != cudaSuccess) return cuda_fail(e, "svd backward");
  return AMM_OK;
}

amm_status_t svd_info(Handle* h, amm_info_t* info) {
  // ||A||_F^2 and ||Q^T A||_F^2, on the handle's stream (A is borrowed and still alive)
  const int64_t m = h->rows, n = h->cols;
  cudaError_t e = h->dtype == AMM_BF16
                      ? sumsq<__nv_bfloat16>((const __nv_bfloat16*)h->A, m, n, h->lda, h->svd.norms + 0, h->stream)
                      : sumsq<float>((const float*)h->A, m, n, h->lda, h->svd.norms + 0, h->stream);
  if (e == cudaSuccess) e = sumsq<float>(h->svd.X, h->k, n, n, h->svd.norms + 1, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  double nr[2];
  if (e == cudaSuccess) e = cudaMemcpy(nr, h->svd.norms, sizeof(nr), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "svd_info");
  if (h->svd.err) {
    int flag = 0;
    if ((e = cudaMemcpy(&flag, h->svd.err, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
      return cuda_fail(e, "svd_info");
    if (flag) return fail(AMM_ERR_TIMEOUT, "a tensor-core kernel of this handle gave up waiting (bounded wait)");
  }
  info->fro2 = nr[0];
  info->resid_fro2 = nr[0] - nr[1];  // ||A - Q Q^T A||^2 = ||A||^2 - ||Q^T A||^2
  info->boundary_gap = -1.0;
  return AMM_OK;
}

amm_status_t svd_get_sketch(Handle* h, float* host_phi, int64_t cap) {
  const int64_t cnt = h->cols * h->k;
  if (cap < cnt) return fail(AMM_ERR_INVALID_ARG, "sketch capacity %lld < %lld", (long long)cap, (long long)cnt);
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e == cudaSuccess) e = cudaMemcpy(host_phi, h->svd.phi, sizeof(float) * cnt, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "svd_get_sketch");
  return AMM_OK;
}

}  // namespace amm
