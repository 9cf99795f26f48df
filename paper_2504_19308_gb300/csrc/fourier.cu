// Fourier-domain sparsification (Section 2.4, Alg. 4 and Alg. 5 of arXiv 2504.19308), sm_103a.
//
//   A~ = A W^*  (row transforms),  B~ = W B  (column transforms),  W(p,q) = n^{-1/2} e^{-2 pi i pq/n}
//   A~_a keeps the k largest |A~(i, q)| of each row, B~_a the k largest |B~(q, c)| of each column
//   M = A~_a B~ + (A~ - A~_a) B~_a,   C = Re(M)
// Real inputs make each transformed row/column Hermitian, so only q = 0..n/2 is stored and the
// magnitudes of q and n-q are the same number (exact tie, lower index first).
//
// HBM layout (kh = n/2 + 1):  At [m][kh] c64, AtT [kh][m] c64, magA [m][kh] f32,
//   Bt [kh][p] c64, magBT [p][kh] f32, sel [rows][k] i32 (ascending q), maskT [n][ceil(rows/32)] u32.
#include <cuda_runtime.h>

#include "api_internal.h"
#include "common.cuh"
#include "fft.cuh"
#include "kernels.h"
#include "trace.h"

namespace amm {

// ============================================================================ transforms
// ROW: rows r0..r0+2S of A (m x n); COL: columns c0..c0+2S of B (n x p).  Packed pairs.
template <int N, int S, int NT, bool ROW>
__global__ void __launch_bounds__(NT) ft_transform_kernel(const float* __restrict__ X, int64_t ldx, int nvec,
                                                          const float2* __restrict__ tw, float2* __restrict__ T,
                                                          float2* __restrict__ TT, float* __restrict__ mag) {
  extern __shared__ float2 smem[];
  constexpr int LD = fft_padded_len(N);
  constexpr int KH = N / 2 + 1;
  const int base = blockIdx.x * 2 * S;
#pragma unroll 8
  for (int it = 0; it < N * S / NT; ++it) {
    const int e = threadIdx.x + it * NT;
    int s, l;
    if (ROW) { s = e / N; l = e % N; } else { l = e / S; s = e % S; }
    const int v0 = base + 2 * s, v1 = v0 + 1;
    float x0 = 0.f, x1 = 0.f;
    if (ROW) {
      if (v0 < nvec) x0 = __ldg(X + (int64_t)v0 * ldx + l);
      if (v1 < nvec) x1 = __ldg(X + (int64_t)v1 * ldx + l);
    } else {
      if (v0 < nvec) x0 = __ldg(X + (int64_t)l * ldx + v0);
      if (v1 < nvec) x1 = __ldg(X + (int64_t)l * ldx + v1);
    }
    smem[s * LD + fpad(l)] = make_float2(x0, x1);
  }
  __syncthreads();
  fft_smem<N, S, NT, false>(smem, tw);
  const float sc = rsqrtf((float)N);
  for (int e = threadIdx.x; e < KH * 2 * S; e += NT) {
    int q, m;
    if (ROW) { m = e / KH; q = e % KH; } else { q = e / (2 * S); m = e % (2 * S); }
    const int v = base + m;
    if (v >= nvec) continue;
    const float2* z = smem + (m >> 1) * LD;
    const float2 a = z[fpad(q)];
    const float2 b = cconj(z[fpad(wrapN<N>(N - q))]);
    float2 x;
    if ((m & 1) == 0) x = cscale(cadd(a, b), 0.5f * sc);
    else { float2 d = csub(a, b); x = make_float2(0.5f * sc * d.y, -0.5f * sc * d.x); }
    if (ROW) x = cconj(x);  // A W^* = conj(F A^T)^T / sqrt(n) for real rows
    const float mg = x.x * x.x + x.y * x.y;
    if (ROW) {
      T[(int64_t)v * KH + q] = x;
      TT[(int64_t)q * nvec + v] = x;
      mag[(int64_t)v * KH + q] = mg;
    } else {
      T[(int64_t)q * nvec + v] = x;
      mag[(int64_t)v * KH + q] = mg;
    }
  }
}

// ============================================================================ exact top-k per row
// Keys are the float bit patterns of |z|^2 (non-negative, so unsigned order = numeric order) of
// the virtual row q = 0..n-1 with key(q) = mag[min(q, n-q)].  Four 8-bit MSB radix passes find
// the k-th largest key tau exactly; the selection is {key > tau} plus the lowest-index entries
// with key == tau, written in ascending q.  One warp per row (ft_select_warp_kernel below).

// ============================================================================ T1 = Re(A~_a B~)
// CTA: RB rows x 256 columns; thread per column, RB accumulators.
constexpr int T1_RB = 8;
__global__ void __launch_bounds__(256) ft_t1_kernel(const float2* __restrict__ At, const int32_t* __restrict__ selA,
                                                    int k, const float2* __restrict__ Bt, int n, int m, int p,
                                                    float* __restrict__ C, int64_t ldc) {
  extern __shared__ unsigned char sm[];
  int32_t* qs = reinterpret_cast<int32_t*>(sm);                   // RB x k
  float2* as = reinterpret_cast<float2*>(qs + T1_RB * k + (T1_RB * k & 1));  // RB x k
  const int kh = n / 2 + 1;
  const int i0 = blockIdx.y * T1_RB;
  const int c = blockIdx.x * 256 + threadIdx.x;
  for (int e = threadIdx.x; e < T1_RB * k; e += 256) {
    const int rr = e / k, i = i0 + rr;
    int q = 0;
    float2 a = make_float2(0.f, 0.f);
    if (i < m) {
      q = selA[(int64_t)i * k + (e % k)];
      const bool mir = q > n / 2;
      a = At[(int64_t)i * kh + (mir ? n - q : q)];
      if (mir) a = cconj(a);
    }
    qs[e] = q;
    as[e] = a;
  }
  __syncthreads();
  if (c >= p) return;
  float acc[T1_RB];
#pragma unroll
  for (int rr = 0; rr < T1_RB; ++rr) acc[rr] = 0.f;
#pragma unroll
  for (int rr = 0; rr < T1_RB; ++rr) {
#pragma unroll 8
    for (int u = 0; u < k; ++u) {
      const int q = qs[rr * k + u];
      const float2 a = as[rr * k + u];
      const bool mir = q > n / 2;
      float2 b = __ldg(Bt + (int64_t)(mir ? n - q : q) * p + c);
      if (mir) b.y = -b.y;
      acc[rr] = fmaf(a.x, b.x, fmaf(-a.y, b.y, acc[rr]));
    }
  }
#pragma unroll
  for (int rr = 0; rr < T1_RB; ++rr)
    if (i0 + rr < m) C[(int64_t)(i0 + rr) * ldc + c] = acc[rr];
}

// ============================================================================ T2 = Re((A~ - A~_a) B~_a)
// CTA: CB columns x 512 rows; a thread takes rows i, i + 1 (one 16-byte load of A~^T(q, i..i+1)
// per kept entry when m is even) with CB accumulators each; A~(i, q) read from At^T.  Entries kept
// in A~_a are zeroed after the load (no branch between the mask and the operand load, so the
// loads of consecutive kept entries stay in flight together).  maskT NULL: nothing of A~ is
// excluded (the dense left operand of a mixed product).  IMAG: the imaginary part instead of the
// real part.
constexpr int T2_CB = 8;
template <bool IMAG, bool VEC>
__global__ void __launch_bounds__(256) ft_t2_kernel(const float2* __restrict__ AtT, const uint32_t* __restrict__ maskT,
                                                    int mask_words, const int32_t* __restrict__ selB, int k,
                                                    const float2* __restrict__ Bt, int n, int m, int p,
                                                    float* __restrict__ C, int64_t ldc) {
  extern __shared__ unsigned char sm[];
  int32_t* qs = reinterpret_cast<int32_t*>(sm);                   // CB x k
  float2* bs = reinterpret_cast<float2*>(qs + T2_CB * k + (T2_CB * k & 1));
  const int c0 = blockIdx.x * T2_CB;
  const int i = 2 * (blockIdx.y * 256 + threadIdx.x);
  for (int e = threadIdx.x; e < T2_CB * k; e += 256) {
    const int cc = e / k, c = c0 + cc;
    int q = 0;
    float2 b = make_float2(0.f, 0.f);
    if (c < p) {
      q = selB[(int64_t)c * k + (e % k)];
      const bool mir = q > n / 2;
      b = Bt[(int64_t)(mir ? n - q : q) * p + c];
      if (mir) b = cconj(b);
    }
    qs[e] = q;
    bs[e] = b;
  }
  __syncthreads();
  if (i >= m) return;
  const bool two = i + 1 < m;
  float acc0[T2_CB], acc1[T2_CB];
#pragma unroll
  for (int cc = 0; cc < T2_CB; ++cc) acc0[cc] = acc1[cc] = 0.f;
  // entry u of all T2_CB columns together: each column's kept entries are in ascending q, and
  // columns with similar spectra keep mostly the same frequencies, so the loads of one step hit
  // the same A~^T rows (merged in L1); every accumulator still adds its column's entries in order
#pragma unroll 2
  for (int u = 0; u < k; ++u) {
#pragma unroll
    for (int cc = 0; cc < T2_CB; ++cc) {
      const int q = qs[cc * k + u];
      const bool mir = q > n / 2;
      const float2* row = AtT + (int64_t)(mir ? n - q : q) * m + i;
      float2 a0, a1;
      if (VEC) {
        const float4 a = __ldg(reinterpret_cast<const float4*>(row));
        a0 = make_float2(a.x, a.y);
        a1 = make_float2(a.z, a.w);
      } else {
        a0 = __ldg(row);
        a1 = two ? __ldg(row + 1) : make_float2(0.f, 0.f);
      }
      if (mir) { a0.y = -a0.y; a1.y = -a1.y; }
      if (maskT != nullptr) {  // (i, q) kept in A~_a: not part of the residue
        const uint32_t w = __ldg(maskT + (int64_t)q * mask_words + (i >> 5));
        if ((w >> (i & 31)) & 1u) a0 = make_float2(0.f, 0.f);
        if ((w >> ((i + 1) & 31)) & 1u) a1 = make_float2(0.f, 0.f);
      }
      const float2 b = bs[cc * k + u];
      if (IMAG) {
        acc0[cc] = fmaf(a0.x, b.y, fmaf(a0.y, b.x, acc0[cc]));
        acc1[cc] = fmaf(a1.x, b.y, fmaf(a1.y, b.x, acc1[cc]));
      } else {
        acc0[cc] = fmaf(a0.x, b.x, fmaf(-a0.y, b.y, acc0[cc]));
        acc1[cc] = fmaf(a1.x, b.x, fmaf(-a1.y, b.y, acc1[cc]));
      }
    }
  }
#pragma unroll
  for (int cc = 0; cc < T2_CB; ++cc) {
    if (c0 + cc < p) {
      C[(int64_t)i * ldc + c0 + cc] += acc0[cc];
      if (two) C[(int64_t)(i + 1) * ldc + c0 + cc] += acc1[cc];
    }
  }
}

// T2 launch: rows in pairs (512 per CTA), the 16-byte form when every A~^T row starts 16-byte aligned
template <bool IMAG>
static void ft_t2_launch(const float2* AtT, const uint32_t* maskT, int mask_words, const int32_t* selB, int k,
                         const float2* Bt, int n, int m, int p, float* C, int64_t ldc, cudaStream_t st) {
  dim3 grid((p + T2_CB - 1) / T2_CB, (m + 511) / 512);
  const size_t sm = (size_t)T2_CB * k * (4 + 8) + 8;
  if ((m % 2) == 0 && (reinterpret_cast<uintptr_t>(AtT) & 15) == 0)
    ft_t2_kernel<IMAG, true><<<grid, 256, sm, st>>>(AtT, maskT, mask_words, selB, k, Bt, n, m, p, C, ldc);
  else
    ft_t2_kernel<IMAG, false><<<grid, 256, sm, st>>>(AtT, maskT, mask_words, selB, k, Bt, n, m, p, C, ldc);
}

// ============================================================================ launchers
template <int N> struct FtCfg {
  static constexpr int S = (N >= 6144) ? 2 : 4;
  static constexpr int NT = fft_threads(N);
  static constexpr size_t SMEM = sizeof(float2) * S * fft_padded_len(N);
};

template <int N> struct FtOps {
  using C = FtCfg<N>;
  static cudaError_t transform(bool row, const float* X, int64_t ldx, int nvec, const float2* tw, float2* T,
                               float2* TT, float* mag, cudaStream_t st) {
    static DeviceOnce once;
    const cudaError_t attr = once([] {
      cudaError_t e = cudaFuncSetAttribute((const void*)ft_transform_kernel<N, C::S, C::NT, true>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute((const void*)ft_transform_kernel<N, C::S, C::NT, false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
      return e;
    });
    if (attr != cudaSuccess) return attr;
    dim3 grid((nvec + 2 * C::S - 1) / (2 * C::S));
    if (row)
      ft_transform_kernel<N, C::S, C::NT, true><<<grid, C::NT, C::SMEM, st>>>(X, ldx, nvec, tw, T, TT, mag);
    else
      ft_transform_kernel<N, C::S, C::NT, false><<<grid, C::NT, C::SMEM, st>>>(X, ldx, nvec, tw, T, TT, mag);
    return cudaGetLastError();
  }
};

#define AMM_FT_DISPATCH(n, EXPR)                  \
  switch (n) {                                    \
    case 16: { constexpr int NN = 16; EXPR; }     \
    case 32: { constexpr int NN = 32; EXPR; }     \
    case 64: { constexpr int NN = 64; EXPR; }     \
    case 128: { constexpr int NN = 128; EXPR; }   \
    case 256: { constexpr int NN = 256; EXPR; }   \
    case 512: { constexpr int NN = 512; EXPR; }   \
    case 1024: { constexpr int NN = 1024; EXPR; } \
    case 2048: { constexpr int NN = 2048; EXPR; } \
    case 4096: { constexpr int NN = 4096; EXPR; } \
    case 8192: { constexpr int NN = 8192; EXPR; } \
    case 48: { constexpr int NN = 48; EXPR; }     \
    case 96: { constexpr int NN = 96; EXPR; } \
    case 192: { constexpr int NN = 192; EXPR; } \
    case 384: { constexpr int NN = 384; EXPR; } \
    case 768: { constexpr int NN = 768; EXPR; } \
    case 1536: { constexpr int NN = 1536; EXPR; } \
    case 3072: { constexpr int NN = 3072; EXPR; } \
    case 6144: { constexpr int NN = 6144; EXPR; } \
    default: return cudaErrorInvalidValue;        \
  }

cudaError_t ft_transform(int n, bool row, const float* X, int64_t ldx, int nvec, const float2* tw, float2* T,
                         float2* TT, float* mag, cudaStream_t st) {
  AMM_TRACE_W(row ? "ft_row_transform" : "ft_col_transform", st, 0.0,
              (double)n * nvec * 4 + (n / 2 + 1.0) * nvec * (row ? 20 : 12), nullptr);
  AMM_FT_DISPATCH(n, return FtOps<NN>::transform(row, X, ldx, nvec, tw, T, TT, mag, st));
}

// The selection with one warp per row (SELW_ROWS rows per CTA): the radix passes of a row
// synchronise its warp only and the rows of a CTA proceed independently (a CTA per row waiting at
// block barriers between the short steps measured 10% slower).  Keys in shared memory per warp,
// the 256-bin histogram per warp; the entries are then taken in rounds of 32 consecutive q
// (ballots give the order): tau, the lowest-q rule for ties, ascending q.
constexpr int SELW_ROWS = 4;
__global__ void __launch_bounds__(32 * SELW_ROWS) ft_select_warp_kernel(const float* __restrict__ mag, int n,
                                                                       int k, int rows, int32_t* __restrict__ sel,
                                                                       uint32_t* __restrict__ maskT,
                                                                       int mask_words) {
  extern __shared__ uint32_t selw_sm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int kh = n / 2 + 1;
  const int kpad = (kh + 3) & ~3;
  uint32_t* keys = selw_sm + warp * (kpad + 256);
  uint32_t* hist = keys + kpad;
  const int row = blockIdx.x * SELW_ROWS + warp;
  if (row >= rows) return;  // whole warps: nothing below synchronises across warps
  for (int q = lane; q < kh; q += 32) keys[q] = __float_as_uint(__ldg(mag + (int64_t)row * kh + q));
  uint32_t prefix = 0, need = (uint32_t)k, mask = 0;
  for (int shift = 24; shift >= 0; shift -= 8) {
    for (int b = lane; b < 256; b += 32) hist[b] = 0;
    __syncwarp();
    // each stored key stands for q and n - q (counted twice), q = 0 and q = n/2 corrected below
    for (int q0 = 0; q0 < kh; q0 += 32) {
      const int q = q0 + lane;
      const uint32_t key = q < kh ? keys[q] : 0u;
      const bool part = q < kh && (key & mask) == prefix;
      const unsigned pm = __ballot_sync(0xffffffffu, part);
      if (part) {
        const uint32_t bkt = (key >> shift) & 255u;
        const unsigned peers = __match_any_sync(pm, bkt);
        if (lane == __ffs(peers) - 1) atomicAdd(&hist[bkt], 2u * __popc(peers));
      }
    }
    __syncwarp();
    if (lane == 0) {
      if ((keys[0] & mask) == prefix) hist[(keys[0] >> shift) & 255u] -= 1u;
      if ((n & 1) == 0 && (keys[n / 2] & mask) == prefix) hist[(keys[n / 2] >> shift) & 255u] -= 1u;
    }
    __syncwarp();
    unsigned above;
    const int b = radix_bucket_warp(hist, need, &above);
    need -= above;
    prefix |= (uint32_t)b << shift;
    mask |= 255u << shift;
    __syncwarp();
  }
  const uint32_t tau = prefix;
  const uint32_t need_eq = need;  // how many entries equal to tau are taken (lowest q first)
  uint32_t eq_seen = 0, pos = 0;
  const unsigned lt = (1u << lane) - 1u;
  for (int q0 = 0; q0 < n && pos < (uint32_t)k; q0 += 32) {
    const int q = q0 + lane;
    const uint32_t key = q < n ? keys[q <= n / 2 ? q : n - q] : 0u;
    const bool gt = q < n && key > tau, eq = q < n && key == tau;
    const unsigned eqm = __ballot_sync(0xffffffffu, eq);
    const bool take = gt || (eq && eq_seen + (uint32_t)__popc(eqm & lt) < need_eq);
    const unsigned tm = __ballot_sync(0xffffffffu, take);
    if (take) {
      const uint32_t at = pos + (uint32_t)__popc(tm & lt);
      if (at < (uint32_t)k) sel[(int64_t)row * k + at] = q;
      if (maskT) atomicOr(maskT + (int64_t)q * mask_words + (row >> 5), 1u << (row & 31));
    }
    eq_seen += (uint32_t)__popc(eqm);
    pos += (uint32_t)__popc(tm);
  }
}

cudaError_t ft_select(int n, int k, int rows, const float* mag, int32_t* sel, uint32_t* maskT, int mask_words,
                      cudaStream_t st) {
  AMM_TRACE_W("ft_select", st, 0.0, (double)rows * (n / 2 + 1) * 4, nullptr);
  if (maskT) {
    cudaError_t e = cudaMemsetAsync(maskT, 0, sizeof(uint32_t) * (size_t)n * mask_words, st);
    if (e != cudaSuccess) return e;
  }
  const int kpad = (n / 2 + 1 + 3) & ~3;
  const size_t smw = sizeof(uint32_t) * (size_t)SELW_ROWS * (kpad + 256);
  static DeviceOnce once;
  const cudaError_t attr = once([] {
    return cudaFuncSetAttribute((const void*)ft_select_warp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(sizeof(uint32_t) * SELW_ROWS * ((8192 / 2 + 1 + 3) / 4 * 4 + 256)));
  });
  if (attr != cudaSuccess) return attr;
  ft_select_warp_kernel<<<(rows + SELW_ROWS - 1) / SELW_ROWS, 32 * SELW_ROWS, smw, st>>>(mag, n, k, rows, sel, maskT,
                                                                                        mask_words);
  return cudaGetLastError();
}

cudaError_t ft_product(int n, int m, int p, int k_a, int k_b, const float2* At, const float2* AtT,
                       const int32_t* selA, const uint32_t* maskT, int mask_words, const float2* Bt,
                       const int32_t* selB, float* C, int64_t ldc, cudaStream_t st) {
  {
    // work: the real part of each kept product (2 FMAs); bytes: the minimal HBM traffic (kept entries
    // of A~, the half spectrum B~, C written)
    AMM_TRACE_W("ft_t1", st, 4.0 * m * (double)p * k_a, 12.0 * m * (double)k_a + 8.0 * (n / 2 + 1.0) * p + 4.0 * m * p,
                nullptr);
    dim3 grid((p + 255) / 256, (m + T1_RB - 1) / T1_RB);
    size_t sm = (size_t)T1_RB * k_a * (4 + 8) + 8;
    ft_t1_kernel<<<grid, 256, sm, st>>>(At, selA, k_a, Bt, n, m, p, C, ldc);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  {
    // bytes: A~^T and its mask, the kept entries of B~, C read and written
    AMM_TRACE_W("ft_t2", st, 4.0 * m * (double)p * k_b,
                8.0 * (n / 2 + 1.0) * m + n * (double)m / 8 + 12.0 * p * (double)k_b + 8.0 * m * p, nullptr);
    ft_t2_launch<false>(AtT, maskT, mask_words, selB, k_b, Bt, n, m, p, C, ldc, st);
  }
  return cudaGetLastError();
}

// ============================================================================ truncation norms
// Per row of magnitudes |A~(i, q)|^2 (q = 0..n/2): the row's squared norm (Parseval: q and n - q
// both count except q = 0 and q = n/2) and the squared norm of its kept entries.  Rows are
// summed afterwards in a fixed order (deterministic).
__global__ void __launch_bounds__(256) ft_norm_rows_kernel(const float* __restrict__ mag, const int32_t* __restrict__ sel,
                                                           int n, int k, double* __restrict__ part) {
  __shared__ double red[2][8];
  const int row = blockIdx.x, kh = n / 2 + 1;
  const float* m = mag + (int64_t)row * kh;
  double tot = 0.0, kept = 0.0;
  for (int q = threadIdx.x; q < kh; q += 256) tot += (q == 0 || q == n / 2 ? 1.0 : 2.0) * (double)__ldg(m + q);
  for (int u = threadIdx.x; u < k; u += 256) {
    const int q = __ldg(sel + (int64_t)row * k + u);
    kept += (double)__ldg(m + (q > n / 2 ? n - q : q));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    tot += __shfl_xor_sync(0xffffffffu, tot, o);
    kept += __shfl_xor_sync(0xffffffffu, kept, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = tot;
    red[1][threadIdx.x >> 5] = kept;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < 8; ++w) {
      a += red[0][w];
      b += red[1][w];
    }
    part[2 * row] = a;
    part[2 * row + 1] = b;
  }
}

__global__ void ft_norm_sum_kernel(const double* __restrict__ part, int rows, double* __restrict__ out) {
  if (threadIdx.x < 2) {
    double s = 0.0;
    for (int r = 0; r < rows; ++r) s += part[2 * r + threadIdx.x];
    out[threadIdx.x] = s;
  }
}

cudaError_t ft_norms(int n, int k, int nvec, const float* mag, const int32_t* sel, double* out, cudaStream_t st) {
  double* part = nullptr;
  cudaError_t e = dev_alloc((void**)&part, sizeof(double) * 2 * (size_t)nvec, st);
  if (e != cudaSuccess) return e;
  {
    AMM_TRACE("ft_norms", st);
    ft_norm_rows_kernel<<<nvec, 256, 0, st>>>(mag, sel, n, k, part);
  }
  ft_norm_sum_kernel<<<1, 32, 0, st>>>(part, nvec, out);
  e = cudaGetLastError();
  dev_free(part, st);
  return e;
}

// ============================================================================ mixed-method pieces
// Dense real or imaginary part of A_s = A~_a W (the sparse rows back in the space domain):
// part 0: y = Re(A~_a W) through the Hermitian part H(q) = (X(q) + conj X(-q))/2 of each row;
// part 1: y = Im(A~_a W) through K(q) = -i (X(q) - conj X(-q))/2.  Two rows share one complex
// FFT (Z = P_{v0} + i P_{v1}).  D = A - y when A is given, else D = y.
template <int N, int S, int NT>
__global__ void __launch_bounds__(NT) ft_dense_kernel(const float2* __restrict__ At, const int32_t* __restrict__ sel,
                                                      int k, int m, const float2* __restrict__ tw, int part,
                                                      const float* __restrict__ A, int64_t lda, float* __restrict__ D,
                                                      int64_t ldd) {
  extern __shared__ float2 smem[];
  constexpr int LD = fft_padded_len(N);
  constexpr int KH = N / 2 + 1;
  const int base = blockIdx.x * 2 * S;
  for (int e = threadIdx.x; e < S * LD; e += NT) smem[e] = make_float2(0.f, 0.f);
  __syncthreads();
  if (threadIdx.x < S) {  // one thread per packed pair: its two rows' entries, in order
    const int s = threadIdx.x;
    for (int h = 0; h < 2; ++h) {
      const int r = base + 2 * s + h;
      if (r >= m) break;
      for (int u = 0; u < k; ++u) {
        const int q = __ldg(sel + (int64_t)r * k + u);
        const bool mir = q > N / 2;
        float2 x = __ldg(At + (int64_t)r * KH + (mir ? N - q : q));
        if (mir) x.y = -x.y;
        float2 cq, cn;  // contributions at q and at -q
        if (part == 0) { cq = cscale(x, 0.5f); cn = cscale(cconj(x), 0.5f); }
        else { cq = make_float2(0.5f * x.y, -0.5f * x.x); cn = make_float2(0.5f * x.y, 0.5f * x.x); }
        if (h == 1) {  // times i
          cq = make_float2(-cq.y, cq.x);
          cn = make_float2(-cn.y, cn.x);
        }
        float2* zq = smem + s * LD + fpad(q);
        float2* zn = smem + s * LD + fpad(wrapN<N>(N - q));
        *zq = cadd(*zq, cq);
        *zn = cadd(*zn, cn);
      }
    }
  }
  __syncthreads();
  fft_smem<N, S, NT, false>(smem, tw);
  const float sc = rsqrtf((float)N);
  for (int e = threadIdx.x; e < N * 2 * S; e += NT) {
    const int mm = e / N, l = e % N;
    const int v = base + mm;
    if (v >= m) continue;
    const float2 z = smem[(mm >> 1) * LD + fpad(l)];
    const float y = sc * ((mm & 1) ? z.y : z.x);
    D[(int64_t)v * ldd + l] = A ? __ldg(A + (int64_t)v * lda + l) - y : y;
  }
}

template <int N> struct FtMixOps {
  using C = FtCfg<N>;
  static cudaError_t dense(const float2* At, const int32_t* sel, int k, int m, const float2* tw, int part,
                           const float* A, int64_t lda, float* D, int64_t ldd, cudaStream_t st) {
    static DeviceOnce once;
    const cudaError_t attr = once([] {
      return cudaFuncSetAttribute((const void*)ft_dense_kernel<N, C::S, C::NT>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    });
    if (attr != cudaSuccess) return attr;
    ft_dense_kernel<N, C::S, C::NT><<<(m + 2 * C::S - 1) / (2 * C::S), C::NT, C::SMEM, st>>>(At, sel, k, m, tw, part,
                                                                                             A, lda, D, ldd);
    return cudaGetLastError();
  }
};

cudaError_t ft_dense(int n, const float2* At, const int32_t* sel, int k, int m, const float2* tw, int part,
                     const float* A, int64_t lda, float* D, int64_t ldd, cudaStream_t st) {
  AMM_TRACE_W(part ? "ft_dense_imag" : "ft_dense_real", st, 0.0, (double)m * n * (A ? 8 : 4), nullptr);
  AMM_FT_DISPATCH(n, return FtMixOps<NN>::dense(At, sel, k, m, tw, part, A, lda, D, ldd, st));
}

// C = Re(A~_a (W X)) for X (n x p): column transforms of X, then T1
cudaError_t ft_left_apply(int n, int m, const float2* At, const int32_t* selA, int ka, const float2* tw,
                          const float* X, int64_t ldx, int p, float* C, int64_t ldc, cudaStream_t st) {
  const size_t kh = (size_t)n / 2 + 1;
  float2* Xt = nullptr;
  float* mag = nullptr;
  cudaError_t e = dev_alloc((void**)&Xt, sizeof(float2) * kh * p, st);
  if (e == cudaSuccess) e = dev_alloc((void**)&mag, sizeof(float) * kh * p, st);
  if (e == cudaSuccess) e = ft_transform(n, false, X, ldx, p, tw, Xt, nullptr, mag, st);
  if (e == cudaSuccess) {
    AMM_TRACE_W("ft_t1", st, 4.0 * m * (double)p * ka, 12.0 * m * (double)ka + 8.0 * (n / 2 + 1.0) * p + 4.0 * m * p,
                nullptr);
    dim3 grid((p + 255) / 256, (m + T1_RB - 1) / T1_RB);
    ft_t1_kernel<<<grid, 256, (size_t)T1_RB * ka * (4 + 8) + 8, st>>>(At, selA, ka, Xt, n, m, p, C, ldc);
    e = cudaGetLastError();
  }
  dev_free(Xt, st);
  dev_free(mag, st);
  return e;
}

// C += Re (or Im) of (Y W^*) B~_a for Y (m x n): row transforms of Y, then T2 without a mask
cudaError_t ft_right_apply(int n, int p, const float2* Bt, const int32_t* selB, int kb, const float2* tw,
                           const float* Y, int64_t ldy, int m, bool imag, float* C, int64_t ldc, cudaStream_t st) {
  const size_t kh = (size_t)n / 2 + 1;
  float2 *Yt = nullptr, *YtT = nullptr;
  float* mag = nullptr;
  cudaError_t e = dev_alloc((void**)&Yt, sizeof(float2) * kh * m, st);
  if (e == cudaSuccess) e = dev_alloc((void**)&YtT, sizeof(float2) * kh * m, st);
  if (e == cudaSuccess) e = dev_alloc((void**)&mag, sizeof(float) * kh * m, st);
  if (e == cudaSuccess) e = ft_transform(n, true, Y, ldy, m, tw, Yt, YtT, mag, st);
  if (e == cudaSuccess) {
    AMM_TRACE_W(imag ? "ft_t2_imag" : "ft_t2", st, 4.0 * m * (double)p * kb,
                8.0 * (n / 2 + 1.0) * m + 12.0 * p * (double)kb + 8.0 * m * p, nullptr);
    if (imag) ft_t2_launch<true>(YtT, nullptr, 0, selB, kb, Bt, n, m, p, C, ldc, st);
    else ft_t2_launch<false>(YtT, nullptr, 0, selB, kb, Bt, n, m, p, C, ldc, st);
    e = cudaGetLastError();
  }
  dev_free(Yt, st);
  dev_free(YtT, st);
  dev_free(mag, st);
  return e;
}

}  // namespace amm
