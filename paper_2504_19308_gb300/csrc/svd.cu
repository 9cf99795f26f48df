// Randomized truncated SVD path (Alg. 1 and Section 2.2 of arXiv 2504.19308) for sm_103a.
//
// Decomposition of one operand X (rows x cols), test matrix phi (cols x k):
//   Y = X phi                      FP32 GEMM
//   Q = orth(Y)                    CholeskyQR2 in FP64 (k x k Gram, Cholesky, triangular apply)
//   Z = Q^T X                      FP32 GEMM            ->  X~ = Q Z = Q Q^T X
// The small SVD of Z (Alg. 1 steps 8-10) rotates Q and Z by the same k x k factors and does
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
  for (int z = 0; z < splits; ++z) s += (double)ws[(int64_t)z * M * N + e];
  float* c = C + (int64_t)row * ldc + col;
  *c = (beta == 0.f) ? (float)(alpha * s) : (float)fma((double)alpha, s, (double)beta * *c);
}

static int g_num_sms = 0;
static int num_sms() {
  if (g_num_sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_num_sms <= 0) g_num_sms = 148;
  }
  return g_num_sms;
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

// ============================================================================ FP64 small GEMM
// C[M x N] = sum_l opA(i, l) opB(l, j), FP64 accumulation, 32 x 32 tiles, K split over grid.z
// (partials to ws, reduced in fixed order).  Used for Gram matrices and triangular applies.
template <bool TA, bool TB, typename TA_t, typename TB_t>
__global__ void __launch_bounds__(256) dgemm_small_kernel(int M, int N, int K, const TA_t* __restrict__ A,
                                                          int64_t lda, const TB_t* __restrict__ B, int64_t ldb,
                                                          int kchunk, double* __restrict__ ws) {
  __shared__ double As[32][33];
  __shared__ double Bs[32][33];
  const int tid = threadIdx.x;
  const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
  const int kbeg = blockIdx.z * kchunk, kend = min(K, kbeg + kchunk);
  double acc[4] = {0, 0, 0, 0};
  const int ci = tid >> 3, cj = (tid & 7) * 4;  // thread computes (ci, cj..cj+3)
  for (int k0 = kbeg; k0 < kend; k0 += 32) {
    for (int e = tid; e < 32 * 32; e += 256) {
      int r = e >> 5, c = e & 31;
      // As[i][l]
      int gi = i0 + r, gl = k0 + c;
      double va = 0.0;
      if (gi < M && gl < kend) va = (double)(TA ? A[(int64_t)gl * lda + gi] : A[(int64_t)gi * lda + gl]);
      As[r][c] = va;
      // Bs[l][j]
      int bl = k0 + r, bj = j0 + c;
      double vb = 0.0;
      if (bj < N && bl < kend) vb = (double)(TB ? B[(int64_t)bj * ldb + bl] : B[(int64_t)bl * ldb + bj]);
      Bs[r][c] = vb;
    }
    __syncthreads();
#pragma unroll 8
    for (int l = 0; l < 32; ++l) {
      double a = As[ci][l];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] = fma(a, Bs[l][cj + q], acc[q]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    int i = i0 + ci, j = j0 + cj + q;
    if (i < M && j < N) ws[((int64_t)blockIdx.z * M + i) * N + j] = acc[q];
  }
}

template <typename TOut>
__global__ void dreduce_kernel(int M, int N, int splits, const double* __restrict__ ws, TOut* __restrict__ C,
                               int64_t ldc) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)M * N) return;
  double s = 0.0;
  for (int z = 0; z < splits; ++z) s += ws[(int64_t)z * M * N + e];
  C[(e / N) * ldc + (e % N)] = (TOut)s;
}

template <bool TA, bool TB, typename TA_t, typename TB_t, typename TOut>
static cudaError_t dgemm_small(int M, int N, int K, const TA_t* A, int64_t lda, const TB_t* B, int64_t ldb, TOut* C,
                               int64_t ldc, cudaStream_t st) {
  const int tiles = ((M + 31) / 32) * ((N + 31) / 32);
  int splits = std::max(1, std::min(K / 256, (2 * num_sms() + tiles - 1) / tiles));
  int kchunk = (K + splits - 1) / splits;
  kchunk = ((kchunk + 31) / 32) * 32;
  splits = std::max(1, (K + kchunk - 1) / kchunk);
  double* ws = nullptr;
  cudaError_t e = dev_alloc((void**)&ws, sizeof(double) * (size_t)splits * M * N, st);
  if (e != cudaSuccess) return e;
  dim3 grid((N + 31) / 32, (M + 31) / 32, splits);
  {
    AMM_TRACE_W("dgemm_small", st, 2.0 * M * N * (double)K, 0.0, nullptr);
    dgemm_small_kernel<TA, TB, TA_t, TB_t><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, kchunk, ws);
  }
  e = cudaGetLastError();
  if (e == cudaSuccess) {
    const int64_t tot = (int64_t)M * N;
    AMM_TRACE("dreduce", st);
    dreduce_kernel<TOut><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(M, N, splits, ws, C, ldc);
    e = cudaGetLastError();
  }
  dev_free(ws, st);
  return e;
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
// formed from the double sum so that the small entries of G - I keep their accuracy.
__global__ void gram_reduce_kernel(int k, int splits, const double* __restrict__ ws, float* __restrict__ G, int ns) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= k * k) return;
  double s = 0.0;
  for (int z = 0; z < splits; ++z) s += ws[(int64_t)z * k * k + e];
  if (ns) s = -0.5 * (s - ((e / k) == (e % k) ? 1.0 : 0.0));
  G[e] = (float)s;
}

static cudaError_t gram_dot2(int64_t m, int k, const float* X, float* G, cudaStream_t st, int ns = 0) {
  const int tiles = ((k + 31) / 32) * ((k + 31) / 32);
  int splits = std::max(1, std::min((int)(m / 256), (2 * num_sms() + tiles - 1) / tiles));
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
    gram_reduce_kernel<<<(k * k + 255) / 256, 256, 0, st>>>(k, splits, ws, G, ns);
    e = cudaGetLastError();
  }
  dev_free(ws, st);
  return e;
}

// ============================================================================ Cholesky + inverse (FP32, one CTA)
// G (k x k, symmetric positive semi-definite) -> Linv = L^{-1} with G + s I = L L^T,
// s = shift_rel * trace(G).  Shared memory holds W (k x k; L ends in its lower triangle), Linv
// (k x k, row-major) and the current column of L, so every inner loop reads consecutive or
// broadcast words (no bank conflicts).  One warp per row in the trailing update; the inverse is
// built row by row (thread c forms Linv[i][c] from Linv[c..i-1][c]).  For k > CHOL_SMEM_K the
// same arrays live in a global work area (2 k^2 + k floats).
constexpr int CHOL_SMEM_K = 160;
constexpr int CHOL_T = 1024;

__global__ void __launch_bounds__(CHOL_T) chol_inv_kernel(int k, const float* __restrict__ G, float shift_rel,
                                                          float* __restrict__ Linv_out, float* __restrict__ gwork) {
  extern __shared__ float sh_dyn[];
  float* sh = (k <= CHOL_SMEM_K) ? sh_dyn : gwork;  // larger k: same layout in global memory
  float* W = sh;              // k * k
  float* Li = sh + k * k;     // k * k
  float* col = Li + k * k;    // k
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
  for (int e = tid; e < k * k; e += CHOL_T) {
    const int i = e / k, j = e - i * k;
    W[e] = G[e] + (i == j ? shift : 0.f);
    Li[e] = 0.f;
  }
  __syncthreads();
  // right-looking Cholesky
  for (int j = 0; j < k; ++j) {
    const float djj = sqrtf(fmaxf(W[j * k + j], shift));
    const float rdj = 1.f / djj;
    for (int i = j + tid; i < k; i += CHOL_T) {
      const float v = (i == j) ? djj : W[i * k + j] * rdj;
      col[i] = v;
      W[i * k + j] = v;
    }
    __syncthreads();
    for (int i = j + 1 + warp; i < k; i += CHOL_T / 32) {
      const float ci = col[i];
      for (int l = j + 1 + lane; l <= i; l += 32) W[i * k + l] = fmaf(-ci, col[l], W[i * k + l]);
    }
    __syncthreads();
  }
  // Linv: diagonal, then rows i = 1..k-1
  for (int i = tid; i < k; i += CHOL_T) Li[i * k + i] = 1.f / W[i * k + i];
  __syncthreads();
  for (int i = 1; i < k; ++i) {
    const float di = Li[i * k + i];
    for (int c = tid; c < i; c += CHOL_T) {
      float s0 = 0.f, s1 = 0.f;
      int l = c;
      for (; l + 1 < i; l += 2) {
        s0 = fmaf(W[i * k + l], Li[l * k + c], s0);
        s1 = fmaf(W[i * k + l + 1], Li[(l + 1) * k + c], s1);
      }
      if (l < i) s0 = fmaf(W[i * k + l], Li[l * k + c], s0);
      Li[i * k + c] = -(s0 + s1) * di;
    }
    __syncthreads();
  }
  for (int e = tid; e < k * k; e += CHOL_T) Linv_out[e] = Li[e];
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

// W: global work area of at least 2 k^2 + k floats (used when k > CHOL_SMEM_K)
static cudaError_t chol_inv(int k, const float* G, float shift_rel, float* W, float* Li, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute((const void*)chol_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (2 * CHOL_SMEM_K * CHOL_SMEM_K + CHOL_SMEM_K) * (int)sizeof(float));
    if (e != cudaSuccess) return e;
    attr = true;
  }
  AMM_TRACE_W("chol_inv", st, (double)k * k * k / 3.0 * 2.0 * 2.0, 0.0, nullptr);
  const size_t sm = k <= CHOL_SMEM_K ? sizeof(float) * (2 * (size_t)k * k + k) : 0;
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
  al(&W, 2 * (size_t)k * k + k);
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
      e = sgemm<float>(false, true, (int)m, k, k, 1.f, src, k, Li, k, 0.f, dsts[pass], k, st);  // src Linv^T
    src = dsts[pass];
  }
  if (e == cudaSuccess) e = gram_dot2(m, k, Q2, G, st, 1);  // G <- -(Q2^T Q2 - I) / 2
  if (e == cudaSuccess) e = cudaMemcpyAsync(Q, Q2, sizeof(float) * (size_t)m * k, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = sgemm<float>(false, false, (int)m, k, k, 1.f, Q2, k, G, k, 1.f, Q, k, st);
  for (float* p : {G, W, Li, Q1, Q2}) dev_free(p, st);
  return e;
}

// ============================================================================ tensor-core path
// Y[c][r] = X[r][c] (cols x rows), 32 x 32 tiles through shared memory, with a type cast.
template <typename TI, typename TO>
__global__ void transpose_cast_kernel(const TI* __restrict__ X, int64_t rows, int64_t cols, int64_t ldx,
                                      TO* __restrict__ Y, int64_t ldy) {
  __shared__ float t[32][33];
  const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int64_t r = r0 + i, c = c0 + threadIdx.x;
    float v = 0.f;
    if (r < rows && c < cols) v = (float)X[r * ldx + c];
    t[i][threadIdx.x] = v;
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int64_t c = c0 + i, r = r0 + threadIdx.x;
    if (r < rows && c < cols) Y[c * ldy + r] = (TO)t[threadIdx.x][i];
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
  dim3 grid((unsigned)((cols + 31) / 32), (unsigned)((rows + 31) / 32));
  transpose_cast_kernel<TI, TO><<<grid, dim3(32, 8), 0, st>>>(X, rows, cols, ldx, Y, ldy);
  return cudaGetLastError();
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

// C = alpha A B^T + beta C with A (M x K, lda) and B (N x K, ldb) K-major in the compute type E.
// tcgen05 when every row starts 16-byte aligned, the SIMT kernel otherwise.
template <typename E>
static cudaError_t gemm_tn(int M, int N, int K, float alpha, const E* A, int64_t lda, const E* B, int64_t ldb,
                           float beta, float* C, int64_t ldc, int* err, cudaStream_t st) {
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
  if (in_bf16) e = sumsq<__nv_bfloat16>((const __nv_bfloat16*)h->A, m, n, h->lda, s.norms + 0, st);
  else e = sumsq<float>((const float*)h->A, m, n, h->lda, s.norms + 0, st);
  if (e == cudaSuccess) e = sumsq<float>(s.X, k, n, n, s.norms + 1, st);
  return e;
}

template <typename E>
static cudaError_t svd_matmul_tc(Handle* a, Handle* b, float* C, int64_t ldc, cudaStream_t st) {
  const int m = (int)a->rows, n = (int)a->cols, p = (int)b->cols;
  const int ka = (int)a->k, kb = (int)b->k;
  auto &sa = a->svd, &sb = b->svd;
  int* err = sa.err;
  float *T1T = nullptr, *W = nullptr, *ZZ = nullptr;
  const E *t1te = nullptr, *we = nullptr, *zze = nullptr;
  cudaError_t e = dev_alloc((void**)&T1T, sizeof(float) * (size_t)p * ka, st);
  if (e == cudaSuccess) e = dev_alloc((void**)&W, sizeof(float) * (size_t)m * kb, st);
  if (e == cudaSuccess) e = dev_alloc((void**)&ZZ, sizeof(float) * (size_t)kb * ka, st);
  // T1^T = B^T Z_A^T ; W = A Q_B ; (Z_A Q_B)^T = Q_B^T Z_A^T ; W -= Q_A (Z_A Q_B) ; C = Q_A T1 + W Z_B
  if (e == cudaSuccess) e = gemm_tn<E>(p, ka, n, 1.f, (const E*)sb.XTe, n, (const E*)sa.Ze, n, 0.f, T1T, ka, err, st);
  if (e == cudaSuccess) e = gemm_tn<E>(m, kb, n, 1.f, (const E*)sa.Xe, sa.ldxe, (const E*)sb.QTe, n, 0.f, W, kb, err, st);
  if (e == cudaSuccess) e = gemm_tn<E>(kb, ka, n, 1.f, (const E*)sb.QTe, n, (const E*)sa.Ze, n, 0.f, ZZ, ka, err, st);
  if (e == cudaSuccess) e = to_e<E>(nullptr, ZZ, kb, ka, &zze, st);
  if (e == cudaSuccess) e = gemm_tn<E>(m, kb, ka, -1.f, (const E*)sa.Qe, ka, zze, ka, 1.f, W, kb, err, st);
  if (e == cudaSuccess) e = to_e<E>(nullptr, T1T, p, ka, &t1te, st);
  if (e == cudaSuccess) e = to_e<E>(nullptr, W, m, kb, &we, st);
  if (e == cudaSuccess) e = gemm_tn<E>(m, p, ka, 1.f, (const E*)sa.Qe, ka, t1te, ka, 0.f, C, ldc, err, st);
  if (e == cudaSuccess) e = gemm_tn<E>(m, p, kb, 1.f, we, kb, (const E*)sb.ZTe, kb, 1.f, C, ldc, err, st);
  if constexpr (!std::is_same<E, float>::value) {
    for (const E* q : {t1te, we, zze}) dev_free((void*)q, st);
  }
  for (float* q : {T1T, W, ZZ}) dev_free(q, st);
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
  const E* H2Te = as_e(H2T, p, ka);
  if (dA) {
    // dA = (G Z_B^T) Q_B^T + Q_A [ H2 B^T - (H2 Z_B^T) Q_B^T ]
    float* H1 = (float*)al(sizeof(float) * (size_t)m * kb);
    if (e == cudaSuccess) e = gemm_tn<E>(m, kb, p, 1.f, Ge, ldge, (const E*)sb.Ze, p, 0.f, H1, kb, err, st);
    const E* H1e = as_e(H1, m, kb);
    if (e == cudaSuccess) e = gemm_tn<E>(m, n, kb, 1.f, H1e, kb, (const E*)sb.Qe, kb, 0.f, dA, ldda, err, st);
    float* H3T = (float*)al(sizeof(float) * (size_t)n * ka);
    float* H4 = (float*)al(sizeof(float) * (size_t)ka * kb);
    if (e == cudaSuccess)
      e = gemm_tn<E>(n, ka, p, 1.f, (const E*)sb.Xe, sb.ldxe, H2e, p, 0.f, H3T, ka, err, st);  // B H2^T
    if (e == cudaSuccess) e = gemm_tn<E>(ka, kb, p, 1.f, H2e, p, (const E*)sb.Ze, p, 0.f, H4, kb, err, st);
    const E* H4e = as_e(H4, ka, kb);
    if (e == cudaSuccess) e = gemm_tn<E>(n, ka, kb, -1.f, (const E*)sb.Qe, kb, H4e, kb, 1.f, H3T, ka, err, st);
    const E* H3Te = as_e(H3T, n, ka);
    if (e == cudaSuccess) e = gemm_tn<E>(m, n, ka, 1.f, (const E*)sa.Qe, ka, H3Te, ka, 1.f, dA, ldda, err, st);
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
    const E* H5Te = as_e(H5T, p, kb);
    if (e == cudaSuccess) e = gemm_tn<E>(n, p, ka, 1.f, (const E*)sa.ZTe, ka, H2Te, ka, 0.f, dB, lddb, err, st);
    if (e == cudaSuccess) e = gemm_tn<E>(n, p, kb, 1.f, (const E*)sb.Qe, kb, H5Te, kb, 1.f, dB, lddb, err, st);
  }
  for (void* q : tmp) dev_free(q, st);
  return e;
}

// ============================================================================ ABI glue
static cudaError_t svd_build(Handle* h, const float* A) {
  auto& s = h->svd;
  const int64_t m = h->rows, n = h->cols;
  const int k = (int)h->k;
  float* Y = nullptr;
  cudaError_t e = dev_alloc((void**)&Y, sizeof(float) * (size_t)m * k, h->stream);
  if (e != cudaSuccess) return e;
  e = sgemm<float>(false, false, (int)m, k, (int)n, 1.f, A, h->lda, s.phi, k, 0.f, Y, k, h->stream);  // Y = A phi
  if (e == cudaSuccess) e = orthonormalize(m, k, Y, s.Q, h->stream);                                          // Q = orth(Y)
  if (e == cudaSuccess)
    e = sgemm<float>(true, false, k, (int)n, (int)m, 1.f, s.Q, k, A, h->lda, 0.f, s.X, n, h->stream);  // X = Q^T A
  if (e == cudaSuccess) e = sumsq<float>(A, m, n, h->lda, s.norms + 0, h->stream);
  if (e == cudaSuccess) e = sumsq<float>(s.X, k, n, n, s.norms + 1, h->stream);
  dev_free(Y, h->stream);
  return e;
}

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
  s.tc = true;
  s.bf16 = compute == AMM_BF16;
  e = s.bf16 ? svd_build_tc<__nv_bfloat16>(h) : svd_build_tc<float>(h);
  if (e != cudaSuccess) return cuda_fail(e, "svd: decomposition");
  return AMM_OK;
}

amm_status_t svd_matmul(Handle* a, Handle* b, float* C, int64_t ldc, cudaStream_t st) {
  if (a->svd.tc && b->svd.tc) {
    if (a->svd.bf16 != b->svd.bf16) return fail(AMM_ERR_STATE, "svd: both operands need the same compute mode");
    cudaError_t e = a->svd.bf16 ? svd_matmul_tc<__nv_bfloat16>(a, b, C, ldc, st) : svd_matmul_tc<float>(a, b, C, ldc, st);
    if (e != cudaSuccess) return cuda_fail(e, "svd product");
    return AMM_OK;
  }
  const int m = (int)a->rows, n = (int)a->cols, p = (int)b->cols;
  const int ka = (int)a->k, kb = (int)b->k;
  const float* A = (const float*)a->A;
  const float* B = (const float*)b->A;
  float *T1 = nullptr, *W = nullptr, *Z = nullptr;
  cudaError_t e = dev_alloc((void**)&T1, sizeof(float) * (size_t)ka * p, st);
  if (e == cudaSuccess) e = dev_alloc((void**)&W, sizeof(float) * (size_t)m * kb, st);
  if (e == cudaSuccess) e = dev_alloc((void**)&Z, sizeof(float) * (size_t)ka * kb, st);
  // T1 = Z_A B ; W = A Q_B - Q_A (Z_A Q_B) ; C = Q_A T1 + W Z_B
  if (e == cudaSuccess) e = sgemm<float>(false, false, ka, p, n, 1.f, a->svd.X, n, B, b->lda, 0.f, T1, p, st);
  if (e == cudaSuccess) e = sgemm<float>(false, false, m, kb, n, 1.f, A, a->lda, b->svd.Q, kb, 0.f, W, kb, st);
  if (e == cudaSuccess) e = sgemm<float>(false, false, ka, kb, n, 1.f, a->svd.X, n, b->svd.Q, kb, 0.f, Z, kb, st);
  if (e == cudaSuccess) e = sgemm<float>(false, false, m, kb, ka, -1.f, a->svd.Q, ka, Z, kb, 1.f, W, kb, st);
  if (e == cudaSuccess) e = sgemm<float>(false, false, m, p, ka, 1.f, a->svd.Q, ka, T1, p, 0.f, C, ldc, st);
  if (e == cudaSuccess) e = sgemm<float>(false, false, m, p, kb, 1.f, W, kb, b->svd.X, p, 1.f, C, ldc, st);
  dev_free(T1, st);
  dev_free(W, st);
  dev_free(Z, st);
  if (e != cudaSuccess) return cuda_fail(e, "svd product");
  return AMM_OK;
}

amm_status_t svd_backward(Handle* a, Handle* b, const float* G, int64_t ldg, float* dA, int64_t ldda, float* dB,
                          int64_t lddb, cudaStream_t st) {
  if (a->svd.tc && b->svd.tc) {
    if (a->svd.bf16 != b->svd.bf16) return fail(AMM_ERR_STATE, "svd: both operands need the same compute mode");
    cudaError_t e = a->svd.bf16 ? svd_backward_tc<__nv_bfloat16>(a, b, G, ldg, dA, ldda, dB, lddb, st)
                                : svd_backward_tc<float>(a, b, G, ldg, dA, ldda, dB, lddb, st);
    if (e != cudaSuccess) return cuda_fail(e, "svd backward");
    return AMM_OK;
  }
  const int m = (int)a->rows, n = (int)a->cols, p = (int)b->cols;
  const int ka = (int)a->k, kb = (int)b->k;
  const float* A = (const float*)a->A;
  const float* B = (const float*)b->A;
  const float *QA = a->svd.Q, *ZA = a->svd.X, *QB = b->svd.Q, *ZB = b->svd.X;
  float *H1 = nullptr, *H2 = nullptr, *H3 = nullptr, *H4 = nullptr, *W = nullptr, *Z = nullptr, *H5 = nullptr;
  cudaError_t e = cudaSuccess;
  auto al = [&](float** ptr, size_t cnt) {
    if (e == cudaSuccess) e = dev_alloc((void**)ptr, sizeof(float) * cnt, st);
  };
  al(&H2, (size_t)ka * p);  // Q_A^T G
  if (e == cudaSuccess) e = sgemm<float>(true, false, ka, p, m, 1.f, QA, ka, G, ldg, 0.f, H2, p, st);
  if (dA) {
    al(&H1, (size_t)m * kb);
    al(&H3, (size_t)ka * n);
    al(&H4, (size_t)ka * kb);
    // dA = (G Z_B^T) Q_B^T + Q_A [ H2 B^T - (H2 Z_B^T) Q_B^T ]
    if (e == cudaSuccess) e = sgemm<float>(false, true, m, kb, p, 1.f, G, ldg, ZB, p, 0.f, H1, kb, st);
    if (e == cudaSuccess) e = sgemm<float>(false, true, m, n, kb, 1.f, H1, kb, QB, kb, 0.f, dA, ldda, st);
    if (e == cudaSuccess) e = sgemm<float>(false, true, ka, n, p, 1.f, H2, p, B, b->lda, 0.f, H3, n, st);
    if (e == cudaSuccess) e = sgemm<float>(false, true, ka, kb, p, 1.f, H2, p, ZB, p, 0.f, H4, kb, st);
    if (e == cudaSuccess) e = sgemm<float>(false, true, ka, n, kb, -1.f, H4, kb, QB, kb, 1.f, H3, n, st);
    if (e == cudaSuccess) e = sgemm<float>(false, false, m, n, ka, 1.f, QA, ka, H3, n, 1.f, dA, ldda, st);
  }
  if (dB) {
    al(&W, (size_t)m * kb);
    al(&Z, (size_t)ka * kb);
    al(&H5, (size_t)kb * p);
    // W = A Q_B - Q_A (Z_A Q_B) ; dB = Z_A^T H2 + Q_B (W^T G)
    if (e == cudaSuccess) e = sgemm<float>(false, false, m, kb, n, 1.f, A, a->lda, QB, kb, 0.f, W, kb, st);
    if (e == cudaSuccess) e = sgemm<float>(false, false, ka, kb, n, 1.f, ZA, n, QB, kb, 0.f, Z, kb, st);
    if (e == cudaSuccess) e = sgemm<float>(false, false, m, kb, ka, -1.f, QA, ka, Z, kb, 1.f, W, kb, st);
    if (e == cudaSuccess) e = sgemm<float>(true, false, kb, p, m, 1.f, W, kb, G, ldg, 0.f, H5, p, st);
    if (e == cudaSuccess) e = sgemm<float>(true, false, n, p, ka, 1.f, ZA, n, H2, p, 0.f, dB, lddb, st);
    if (e == cudaSuccess) e = sgemm<float>(false, false, n, p, kb, 1.f, QB, kb, H5, p, 1.f, dB, lddb, st);
  }
  for (float* ptr : {H1, H2, H3, H4, W, Z, H5}) dev_free(ptr, st);
  if (e != cudaSuccess) return cuda_fail(e, "svd backward");
  return AMM_OK;
}

amm_status_t svd_info(Handle* h, amm_info_t* info) {
  double nr[2];
  cudaError_t e = cudaMemcpy(nr, h->svd.norms, sizeof(nr), cudaMemcpyDeviceToHost);
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
