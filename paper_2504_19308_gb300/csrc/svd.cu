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

__global__ void splitk_reduce_kernel(int M, int N, int splits, const float* __restrict__ ws, float alpha, float beta,
                                     float* __restrict__ C, int64_t ldc) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)M * N) return;
  const int row = (int)(e / N), col = (int)(e % N);
  float s = 0.f;
  for (int z = 0; z < splits; ++z) s += ws[(int64_t)z * M * N + e];
  float* c = C + (int64_t)row * ldc + col;
  *c = (beta == 0.f) ? alpha * s : fmaf(alpha, s, beta * *c);
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

// ============================================================================ Cholesky + inverse (FP64, one CTA)
// G (k x k, symmetric positive semi-definite) -> Linv = L^{-1} with G + s I = L L^T,
// s = 1e-15 trace(G) / k (keeps rank-deficient sketches factorisable; the second CholQR pass
// restores orthonormality).  For k <= CHOL_SMEM_K the work matrix lives in shared memory:
// L in the lower triangle, L^{-1} transposed in the strict upper triangle, 1/L_ii aside.
// Larger k use the global scratch W the same way.
constexpr int CHOL_SMEM_K = 128;
constexpr int CHOL_T = 1024;

__global__ void __launch_bounds__(CHOL_T) chol_inv_kernel(int k, const double* __restrict__ G,
                                                          double* __restrict__ Wg, double* __restrict__ Linv) {
  extern __shared__ double sW[];
  __shared__ double dinv_s[CHOL_SMEM_K];
  __shared__ double red[32];
  __shared__ double shift_s;
  const bool in_smem = k <= CHOL_SMEM_K;
  double* W = in_smem ? sW : Wg;
  double* dinv = in_smem ? dinv_s : Linv;  // global case: diagonal stashed in Linv's first row
  const int tid = threadIdx.x;
  double tr = 0.0;
  for (int i = tid; i < k; i += CHOL_T) tr += G[(int64_t)i * k + i];
  for (int o = 16; o > 0; o >>= 1) tr += __shfl_xor_sync(0xffffffffu, tr, o);
  if ((tid & 31) == 0) red[tid >> 5] = tr;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int w = 0; w < CHOL_T / 32; ++w) t += red[w];
    shift_s = 1e-15 * t / k + 1e-300;
  }
  __syncthreads();
  const double shift = shift_s;
  for (int e = tid; e < k * k; e += CHOL_T) {
    const int i = e / k, j = e % k;
    W[e] = G[e] + (i == j ? shift : 0.0);
  }
  __syncthreads();
  // right-looking Cholesky, L overwrites the lower triangle
  for (int j = 0; j < k; ++j) {
    const double djj = sqrt(fmax(W[(int64_t)j * k + j], shift));
    __syncthreads();
    for (int i = j + 1 + tid; i < k; i += CHOL_T) W[(int64_t)i * k + j] /= djj;
    if (tid == 0) W[(int64_t)j * k + j] = djj;
    __syncthreads();
    const int rem = k - j - 1;
    for (int e = tid; e < rem * rem; e += CHOL_T) {
      const int i = j + 1 + e / rem, l = j + 1 + e % rem;
      if (l <= i) W[(int64_t)i * k + l] -= W[(int64_t)i * k + j] * W[(int64_t)l * k + j];
    }
    __syncthreads();
  }
  // L^{-1} row by row: Linv[i][c] = -(sum_{l=c}^{i-1} L[i][l] Linv[l][c]) / L[i][i]; stored at W[c][i]
  double* dv = in_smem ? dinv_s : nullptr;
  for (int i = tid; i < k; i += CHOL_T) {
    const double d = 1.0 / W[(int64_t)i * k + i];
    if (in_smem) dv[i] = d;
    else Linv[(int64_t)i * k + i] = d;
  }
  __syncthreads();
  for (int i = 1; i < k; ++i) {
    const double di = in_smem ? dv[i] : Linv[(int64_t)i * k + i];
    for (int c = tid; c < i; c += CHOL_T) {
      double s = W[(int64_t)i * k + c] * (in_smem ? dv[c] : Linv[(int64_t)c * k + c]);
      for (int l = c + 1; l < i; ++l) s += W[(int64_t)i * k + l] * W[(int64_t)c * k + l];
      W[(int64_t)c * k + i] = -s * di;
    }
    __syncthreads();
  }
  for (int e = tid; e < k * k; e += CHOL_T) {
    const int i = e / k, c = e % k;
    double v = 0.0;
    if (c < i) v = W[(int64_t)c * k + i];
    else if (c == i) v = in_smem ? dv[i] : Linv[(int64_t)i * k + i];
    if (in_smem || c != i) Linv[e] = v;
  }
  (void)dinv;
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

__global__ void sum_partials_kernel(const double* __restrict__ p, int n, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += p[i];
    *out = s;
  }
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

static cudaError_t chol_inv(int k, const double* G, double* W, double* Li, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute((const void*)chol_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         CHOL_SMEM_K * CHOL_SMEM_K * (int)sizeof(double));
    if (e != cudaSuccess) return e;
    attr = true;
  }
  AMM_TRACE_W("chol_inv", st, (double)k * k * k / 3.0 * 2.0, 0.0, nullptr);
  const size_t sm = k <= CHOL_SMEM_K ? sizeof(double) * k * k : 0;
  chol_inv_kernel<<<1, CHOL_T, sm, st>>>(k, G, W, Li);
  return cudaGetLastError();
}

// ============================================================================ orth(Y) by CholeskyQR2
// Y (m x k, FP32) -> Q (m x k, FP32 with orthonormal columns, same span).
// Each pass: G = Y^T Y accumulated in FP64, G + sI = L L^T and L^{-1} in FP64 (one CTA),
// then Y <- Y L^{-T} with the FP32 GEMM.  Any invertible triangular factor keeps span(Y);
// the FP32 rounding of the apply only costs orthogonality, which the second pass restores.
__global__ void d2f_kernel(const double* __restrict__ x, float* __restrict__ y, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = (float)x[i];
}

static cudaError_t cholqr2(int64_t m, int k, const float* Y, float* Q, cudaStream_t st) {
  double *G = nullptr, *W = nullptr, *Li = nullptr;
  float *Lf = nullptr, *Q1 = nullptr;
  cudaError_t e = cudaSuccess;
  auto al = [&](void** p, size_t bytes) {
    if (e == cudaSuccess) e = dev_alloc(p, bytes, st);
  };
  al((void**)&G, sizeof(double) * k * k);
  al((void**)&W, sizeof(double) * k * k);
  al((void**)&Li, sizeof(double) * k * k);
  al((void**)&Lf, sizeof(float) * k * k);
  al((void**)&Q1, sizeof(float) * m * k);
  const float* src = Y;
  for (int pass = 0; pass < 2 && e == cudaSuccess; ++pass) {
    float* dst = pass == 0 ? Q1 : Q;
    e = dgemm_small<true, false>((int)k, k, (int)m, src, k, src, k, G, k, st);  // src^T src
    if (e == cudaSuccess) e = chol_inv(k, G, W, Li, st);
    if (e == cudaSuccess) {
      AMM_TRACE("d2f", st);
      d2f_kernel<<<(k * k + 255) / 256, 256, 0, st>>>(Li, Lf, k * k);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess)
      e = sgemm<float>(false, true, (int)m, k, k, 1.f, src, k, Lf, k, 0.f, dst, k, st);  // src Linv^T
    src = dst;
  }
  dev_free(G, st);
  dev_free(W, st);
  dev_free(Li, st);
  dev_free(Lf, st);
  dev_free(Q1, st);
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
  if (e == cudaSuccess) e = cholqr2(m, k, Y, s.Q, h->stream);                                          // Q = orth(Y)
  if (e == cudaSuccess)
    e = sgemm<float>(true, false, k, (int)n, (int)m, 1.f, s.Q, k, A, h->lda, 0.f, s.X, n, h->stream);  // X = Q^T A
  if (e == cudaSuccess) e = sumsq<float>(A, m, n, h->lda, s.norms + 0, h->stream);
  if (e == cudaSuccess) e = sumsq<float>(s.X, k, n, n, s.norms + 1, h->stream);
  dev_free(Y, h->stream);
  return e;
}

amm_status_t decompose_svd(Handle* h, const amm_opts_t* o) {
  if (h->dtype != AMM_F32) return fail(AMM_ERR_NOT_IMPLEMENTED, "svd: BF16 inputs are not built yet");
  if (h->k > 1024) return fail(AMM_ERR_UNSUPPORTED_SIZE, "svd: k=%lld > 1024", (long long)h->k);
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
  e = svd_build(h, (const float*)h->A);
  if (e != cudaSuccess) return cuda_fail(e, "svd: decomposition");
  return AMM_OK;
}

amm_status_t svd_matmul(Handle* a, Handle* b, float* C, int64_t ldc, cudaStream_t st) {
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
