// Backward of the Fourier-domain sparsified product (Section 2.4, Alg. 5) with the element masks
// frozen, sm_103a.
//
// M = A~_a B~ + (A~ - A~_a) B~_a with A~ = A W^*, B~ = W B, W(p,q) = n^{-1/2} e^{-2 pi i pq/n};
// P_A, P_B keep the selected entries.  For the upstream gradient G of C = Re(M):
//   dA = Re[ (G B~_a^T + P_A(G dB~^T)) conj(W) ],   dB = Re[ W (A~_a^T G + P_B(dA~^T G)) ]
// with dB~ = B~ - B~_a, dA~ = A~ - A~_a.  Each bracket is a sparse-times-dense product (the kept
// entries of one operand) plus a sampled product on the kept entries of the other; neither forms
// a dense n x n x p contraction.  The brackets live on the full frequency range q = 0..n-1 (the
// masks need not be mirror-symmetric: ties between q and n-q keep the lower index), so the last
// step takes the real part of a complex transform: Re F(X) = F(H) with the Hermitian part
// H(q) = (X(q) + conj X(n-q)) / 2, two real outputs per complex FFT.
//
// Workspace (freed on the stream at the end):  GT [p][m] f32 (G transposed),
//   XAT [n][m] c64 (dA bracket, frequency-major), XB [n][p] c64 (dB bracket).
#include <cuda_runtime.h>

#include "api_internal.h"
#include "common.cuh"
#include "fft.cuh"
#include "kernels.h"
#include "trace.h"

namespace amm {

// B~(q, c) of a real B from the half spectrum Bt [n/2+1][p]
__device__ __forceinline__ float2 half_spec(const float2* __restrict__ T, int n, int q, int64_t ld, int64_t col) {
  const bool mir = q > n / 2;
  float2 v = __ldg(T + (int64_t)(mir ? n - q : q) * ld + col);
  if (mir) v.y = -v.y;
  return v;
}

// ============================================================================ sparse x dense
// out[q][v] = sum over the set bits x of mask[q]:  T~(q, x) D[x][v]   (T~ from a half spectrum).
//   G B~_a^T :  D = G^T [p][m], T = B~ [n/2+1][p], mask = B~_a bits  -> XAT[q][i]
//   A~_a^T G :  D = G [m][p],   T = A~^T [n/2+1][m], mask = A~_a bits -> XB[q][c]
// The set bits of each mask row are cut into units of at most SP_UNIT entries, one CTA per (unit,
// 1024 outputs): a row kept by every vector (the DC term of data with a non-zero mean is kept
// everywhere, 4096 entries against about k elsewhere) spreads over several CTAs instead of running
// on one.  A row of one unit is stored; the units of a longer row add their partial sums atomically
// to the row, which the counting kernel zeroes first.  Per unit the entries are compacted in shared
// memory (index and coefficient), then every thread streams the selected rows of D for its 4
// outputs, four entries at a time (16 loads in flight per thread).
constexpr int SP_UNIT = 256;  // entries per unit
constexpr int SP_RPT = 4;     // outputs per thread

// cnt[q] = set bits of mask row q.  With out given, a row without set bits (no unit writes it) or of
// more than one unit (its units add to it) is zeroed in out.  Warp per row.
__global__ void __launch_bounds__(256) ft_bw_count_kernel(const uint32_t* __restrict__ mask, int mw, int n, int nout,
                                                          int unit, int32_t* __restrict__ cnt,
                                                          float2* __restrict__ out) {
  const int q = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (q >= n) return;
  int c = 0;
  for (int w = lane; w < mw; w += 32) c += __popc(__ldg(mask + (int64_t)q * mw + w));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if (lane == 0) cnt[q] = c;
  if (out != nullptr && (c == 0 || c > unit)) {
    float2* row = out + (int64_t)q * nout;
    for (int v = lane; v < nout; v += 32) row[v] = make_float2(0.f, 0.f);
  }
}

// Exclusive scan of x over the CTA (blockDim.x a multiple of 32, at most 1024); *total receives
// the sum.  s_warp: 32 ints of shared memory.  Every thread of the CTA must call it.
__device__ __forceinline__ int block_excl_scan(int x, int* s_warp, int* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int y = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, y, o);
    if (lane >= o) y += t;
  }
  if (lane == 31) s_warp[warp] = y;
  __syncthreads();
  if (warp == 0) {
    int w = lane < nw ? s_warp[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += t;
    }
    if (lane < nw) s_warp[lane] = w;
  }
  __syncthreads();
  const int excl = y - x + (warp > 0 ? s_warp[warp - 1] : 0);
  *total = s_warp[nw - 1];
  __syncthreads();  // s_warp may be reused by the next call
  return excl;
}

// uoff[q] = units of rows 0..q-1 (exclusive scan of ceil(cnt / unit)), uoff[n] = the total.
// One CTA of 1024 threads.
__global__ void __launch_bounds__(1024) ft_bw_plan_kernel(const int32_t* __restrict__ cnt, int n, int unit,
                                                          int32_t* __restrict__ uoff) {
  __shared__ int s_warp[32];
  int carry = 0;
  for (int base = 0; base < n; base += 1024) {
    const int q = base + threadIdx.x;
    const int u = q < n ? (cnt[q] + unit - 1) / unit : 0;
    int tot = 0;
    const int ex = block_excl_scan(u, s_warp, &tot);
    if (q < n) uoff[q] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) uoff[n] = carry;
}

// The row q of unit u and the unit's entry range [row[1], row[2]) among the row's set bits: q is the
// largest row with uoff[q] <= u (a row without units shares its offset with the next row, so the
// largest such q is the row that owns u).
__device__ __forceinline__ void unit_row(int u, int n, int unit, const int32_t* __restrict__ cnt,
                                         const int32_t* __restrict__ uoff, int* row) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(uoff + mid) <= u) lo = mid;
    else hi = mid - 1;
  }
  const int j = u - __ldg(uoff + lo);
  row[0] = lo;
  row[1] = j * unit;
  row[2] = min(__ldg(cnt + lo), (j + 1) * unit);
}

// The set bits of mask row mrow (mw words) with ranks in [elo, ehi), in increasing order, to
// s_idx[rank - elo] (and, with T given, T~(q, x) to s_val).  Walks 256 words at a time; every thread
// of the CTA (256) must call it.
__device__ __forceinline__ void compact_bits(const uint32_t* __restrict__ mrow, int mw, int elo, int ehi,
                                             const float2* __restrict__ T, int n, int q, int64_t ldt, int* s_warp,
                                             int32_t* s_idx, float2* s_val) {
  int base = 0;  // set bits before the current 256-word chunk
  for (int w0 = 0; w0 < mw && base < ehi; w0 += 256) {
    const int w = w0 + threadIdx.x;
    const uint32_t bits = w < mw ? __ldg(mrow + w) : 0u;
    int tot = 0;
    int rank = base + block_excl_scan(__popc(bits), s_warp, &tot);
    if (rank < ehi && rank + __popc(bits) > elo) {
      uint32_t b = bits;
      while (b) {
        const int x = w * 32 + __ffs(b) - 1;
        b &= b - 1;
        if (rank >= elo && rank < ehi) {
          s_idx[rank - elo] = x;
          if (T != nullptr) s_val[rank - elo] = half_spec(T, n, q, ldt, x);
        }
        ++rank;
      }
    }
    base += tot;
  }
}

// One unit (blockIdx.x) x 1024 outputs (blockIdx.y).
__global__ void __launch_bounds__(256) ft_bw_spmm_kernel(const float* __restrict__ D, int64_t ldd, int nout,
                                                         const float2* __restrict__ T, int64_t ldt,
                                                         const uint32_t* __restrict__ mask, int mw, int n,
                                                         const int32_t* __restrict__ cnt,
                                                         const int32_t* __restrict__ uoff, float2* __restrict__ out) {
  __shared__ int32_t s_idx[SP_UNIT];
  __shared__ float2 s_val[SP_UNIT];
  __shared__ int s_warp[32];
  __shared__ int s_row[3];
  const int u = blockIdx.x;
  if (u >= __ldg(uoff + n)) return;  // the grid is an upper bound on the units
  if (threadIdx.x == 0) unit_row(u, n, SP_UNIT, cnt, uoff, s_row);
  __syncthreads();
  const int q = s_row[0], elo = s_row[1], ehi = s_row[2];
  compact_bits(mask + (int64_t)q * mw, mw, elo, ehi, T, n, q, ldt, s_warp, s_idx, s_val);
  __syncthreads();
  const int ne = ehi - elo;
  const int v0 = blockIdx.y * (256 * SP_RPT) + threadIdx.x;
  float2 acc[SP_RPT];
#pragma unroll
  for (int r = 0; r < SP_RPT; ++r) acc[r] = make_float2(0.f, 0.f);
  int e = 0;
  for (; e + 4 <= ne; e += 4) {
    float d[4][SP_RPT];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const float* drow = D + (int64_t)s_idx[e + s] * ldd;
#pragma unroll
      for (int r = 0; r < SP_RPT; ++r) {
        const int v = v0 + r * 256;
        d[s][r] = v < nout ? __ldg(drow + v) : 0.f;
      }
    }
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const float2 c = s_val[e + s];
#pragma unroll
      for (int r = 0; r < SP_RPT; ++r) {
        acc[r].x = fmaf(d[s][r], c.x, acc[r].x);
        acc[r].y = fmaf(d[s][r], c.y, acc[r].y);
      }
    }
  }
  for (; e < ne; ++e) {
    const float* drow = D + (int64_t)s_idx[e] * ldd;
    const float2 c = s_val[e];
#pragma unroll
    for (int r = 0; r < SP_RPT; ++r) {
      const int v = v0 + r * 256;
      if (v < nout) {
        const float dv = __ldg(drow + v);
        acc[r].x = fmaf(dv, c.x, acc[r].x);
        acc[r].y = fmaf(dv, c.y, acc[r].y);
      }
    }
  }
  const bool split = __ldg(cnt + q) > SP_UNIT;
#pragma unroll
  for (int r = 0; r < SP_RPT; ++r) {
    const int v = v0 + r * 256;
    if (v >= nout) continue;
    float2* o = out + (int64_t)q * nout + v;
    if (split) {
      atomicAdd(&o->x, acc[r].x);
      atomicAdd(&o->y, acc[r].y);
    } else {
      *o = acc[r];
    }
  }
}

// out [n][nout] = the product above for a mask whose rows hold nbits set bits in total (the units
// number at most n + nbits / SP_UNIT)
static cudaError_t ft_bw_spmm(const float* D, int64_t ldd, int nout, const float2* T, int64_t ldt,
                              const uint32_t* mask, int mw, int n, int64_t nbits, float2* out, cudaStream_t st) {
  int32_t* cnt = nullptr;
  cudaError_t e = dev_alloc((void**)&cnt, sizeof(int32_t) * (2 * (size_t)n + 1), st);
  if (e != cudaSuccess) return e;
  int32_t* uoff = cnt + n;
  ft_bw_count_kernel<<<(n + 7) / 8, 256, 0, st>>>(mask, mw, n, nout, SP_UNIT, cnt, out);
  e = cudaGetLastError();
  if (e == cudaSuccess) {
    ft_bw_plan_kernel<<<1, 1024, 0, st>>>(cnt, n, SP_UNIT, uoff);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    const int64_t units = (int64_t)n + (nbits + SP_UNIT - 1) / SP_UNIT;
    ft_bw_spmm_kernel<<<dim3((unsigned)units, (nout + 256 * SP_RPT - 1) / (256 * SP_RPT)), 256, 0, st>>>(
        D, ldd, nout, T, ldt, mask, mw, n, cnt, uoff, out);
    e = cudaGetLastError();
  }
  dev_free(cnt, st);
  return e;
}

// ============================================================================ sampled products
// For each set bit v of sel row q (a kept entry of one operand):
//   X[q][v] += f * sum_x Dm[v][x] T~(q, x) [x not set in excl row q]
// with f = 1, +i or -i (IMAG = 0, 1, -1; MASKED = false: no excluded entries).
//   P_A(G dB~^T):  Dm = G [m][p],   T = B~ [n/2+1][p],   excl = B~_a bits, sel = A~_a bits -> XAT[q][i]
//   P_B(dA~^T G):  Dm = G^T [p][m], T = A~^T [n/2+1][m], excl = A~_a bits, sel = B~_a bits -> XB[q][c]
// The kept entries of each row q are cut into units of at most SS_UNIT (counted and planned as for
// the sparse x dense product; every entry belongs to one unit, so the update is a plain
// read-modify-write).  Per unit the CTA stages row q of T~ in shared memory with the excluded
// entries zeroed, and every warp takes two kept entries at a time and streams their rows of Dm
// against the staged row (one shared-memory read serves both rows).  Grouped by q this way, each
// kept entry moves its real row of Dm from L2 once, where grouping by v would move a complex row
// of T~ per entry, twice the bytes.
constexpr int SS_UNIT = 64;
constexpr int SS_MAX_LEN = 8192;  // staged row length (64 KB of shared memory)

template <bool MASKED, int IMAG, bool VEC4>
__global__ void __launch_bounds__(256) ft_bw_sampled_kernel(const float* __restrict__ Dm, int64_t ldd, int len,
                                                            const float2* __restrict__ T, int64_t ldt,
                                                            const uint32_t* __restrict__ excl, int mwx,
                                                            const uint32_t* __restrict__ sel, int mws, int n,
                                                            int nout, const int32_t* __restrict__ cnt,
                                                            const int32_t* __restrict__ uoff,
                                                            float2* __restrict__ X) {
  extern __shared__ float2 s_t[];  // len entries: row q of T~, excluded entries zeroed
  __shared__ int32_t s_idx[SS_UNIT];
  __shared__ int s_warp[32];
  __shared__ int s_row[3];
  const int u = blockIdx.x;
  if (u >= __ldg(uoff + n)) return;  // the grid is an upper bound on the units
  if (threadIdx.x == 0) unit_row(u, n, SS_UNIT, cnt, uoff, s_row);
  __syncthreads();
  const int q = s_row[0], elo = s_row[1], ehi = s_row[2];
  const bool mir = q > n / 2;
  const float2* trow = T + (int64_t)(mir ? n - q : q) * ldt;
  const uint32_t* xrow = MASKED ? excl + (int64_t)q * mwx : nullptr;
  for (int x = threadIdx.x; x < len; x += 256) {
    float2 v = __ldg(trow + x);
    if (mir) v.y = -v.y;
    if (MASKED && ((__ldg(xrow + (x >> 5)) >> (x & 31)) & 1u)) v = make_float2(0.f, 0.f);
    s_t[x] = v;
  }
  compact_bits(sel + (int64_t)q * mws, mws, elo, ehi, nullptr, n, q, 0, s_warp, s_idx, nullptr);
  __syncthreads();
  const int ne = ehi - elo;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int e0 = 2 * warp; e0 < ne; e0 += 16) {
    const bool two = e0 + 1 < ne;
    const int v1 = s_idx[e0], v2 = two ? s_idx[e0 + 1] : v1;
    const float* r1 = Dm + (int64_t)v1 * ldd;
    const float* r2 = Dm + (int64_t)v2 * ldd;
    float a1x = 0.f, a1y = 0.f, a2x = 0.f, a2y = 0.f;
    if (VEC4) {  // len % 4 == 0, rows 16-byte aligned
#pragma unroll 2
      for (int x = lane * 4; x < len; x += 128) {
        const float4 g1 = __ldg(reinterpret_cast<const float4*>(r1 + x));
        const float4 g2 = __ldg(reinterpret_cast<const float4*>(r2 + x));
        const float4 t01 = *reinterpret_cast<const float4*>(s_t + x);
        const float4 t23 = *reinterpret_cast<const float4*>(s_t + x + 2);
        a1x = fmaf(g1.x, t01.x, a1x); a1y = fmaf(g1.x, t01.y, a1y);
        a1x = fmaf(g1.y, t01.z, a1x); a1y = fmaf(g1.y, t01.w, a1y);
        a1x = fmaf(g1.z, t23.x, a1x); a1y = fmaf(g1.z, t23.y, a1y);
        a1x = fmaf(g1.w, t23.z, a1x); a1y = fmaf(g1.w, t23.w, a1y);
        a2x = fmaf(g2.x, t01.x, a2x); a2y = fmaf(g2.x, t01.y, a2y);
        a2x = fmaf(g2.y, t01.z, a2x); a2y = fmaf(g2.y, t01.w, a2y);
        a2x = fmaf(g2.z, t23.x, a2x); a2y = fmaf(g2.z, t23.y, a2y);
        a2x = fmaf(g2.w, t23.z, a2x); a2y = fmaf(g2.w, t23.w, a2y);
      }
    } else {
#pragma unroll 4
      for (int x = lane; x < len; x += 32) {
        const float g1 = __ldg(r1 + x), g2 = __ldg(r2 + x);
        const float2 t = s_t[x];
        a1x = fmaf(g1, t.x, a1x); a1y = fmaf(g1, t.y, a1y);
        a2x = fmaf(g2, t.x, a2x); a2y = fmaf(g2, t.y, a2y);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a1x += __shfl_xor_sync(0xffffffffu, a1x, o);
      a1y += __shfl_xor_sync(0xffffffffu, a1y, o);
      a2x += __shfl_xor_sync(0xffffffffu, a2x, o);
      a2y += __shfl_xor_sync(0xffffffffu, a2y, o);
    }
    if (lane == 0) {
      float2* x1 = X + (int64_t)q * nout + v1;
      const float2 o1 = *x1;
      *x1 = IMAG > 0 ? make_float2(o1.x - a1y, o1.y + a1x)
                     : IMAG < 0 ? make_float2(o1.x + a1y, o1.y - a1x) : make_float2(o1.x + a1x, o1.y + a1y);
      if (two) {
        float2* x2 = X + (int64_t)q * nout + v2;
        const float2 o2 = *x2;
        *x2 = IMAG > 0 ? make_float2(o2.x - a2y, o2.y + a2x)
                       : IMAG < 0 ? make_float2(o2.x + a2y, o2.y - a2x) : make_float2(o2.x + a2x, o2.y + a2y);
      }
    }
  }
}

template <bool MASKED, int IMAG, bool VEC4>
static cudaError_t sampled_launch(dim3 grid, size_t smem, cudaStream_t st, const float* Dm, int64_t ldd, int len,
                                  const float2* T, int64_t ldt, const uint32_t* excl, int mwx, const uint32_t* sel,
                                  int mws, int n, int nout, const int32_t* cnt, const int32_t* uoff, float2* X) {
  static DeviceOnce once;
  const cudaError_t attr = once([] {
    return cudaFuncSetAttribute((const void*)ft_bw_sampled_kernel<MASKED, IMAG, VEC4>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(sizeof(float2) * SS_MAX_LEN));
  });
  if (attr != cudaSuccess) return attr;
  ft_bw_sampled_kernel<MASKED, IMAG, VEC4><<<grid, 256, smem, st>>>(Dm, ldd, len, T, ldt, excl, mwx, sel, mws, n,
                                                                     nout, cnt, uoff, X);
  return cudaGetLastError();
}

// X [n][nout] += the sampled product above; sel holds nbits set bits in total (the units number at
// most n + nbits / SS_UNIT); excl NULL: no excluded entries; imag in {0, 1, -1}.  len <= SS_MAX_LEN.
static cudaError_t ft_bw_sampled(const float* Dm, int64_t ldd, int len, const float2* T, int64_t ldt,
                                 const uint32_t* excl, int mwx, const uint32_t* sel, int mws, int n, int nout,
                                 int64_t nbits, int imag, float2* X, cudaStream_t st) {
  if (len > SS_MAX_LEN || (excl != nullptr && imag != 0)) return cudaErrorInvalidValue;
  int32_t* cnt = nullptr;
  cudaError_t e = dev_alloc((void**)&cnt, sizeof(int32_t) * (2 * (size_t)n + 1), st);
  if (e != cudaSuccess) return e;
  int32_t* uoff = cnt + n;
  ft_bw_count_kernel<<<(n + 7) / 8, 256, 0, st>>>(sel, mws, n, nout, SS_UNIT, cnt, nullptr);
  e = cudaGetLastError();
  if (e == cudaSuccess) {
    ft_bw_plan_kernel<<<1, 1024, 0, st>>>(cnt, n, SS_UNIT, uoff);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    const dim3 grid((unsigned)((int64_t)n + (nbits + SS_UNIT - 1) / SS_UNIT));
    const size_t smem = sizeof(float2) * (size_t)len;
    const bool vec = ((uintptr_t)Dm % 16) == 0 && ldd % 4 == 0 && len % 4 == 0;
#define AMM_SS(MK, IM, V) \
  e = sampled_launch<MK, IM, V>(grid, smem, st, Dm, ldd, len, T, ldt, excl, mwx, sel, mws, n, nout, cnt, uoff, X)
    if (excl != nullptr) {
      if (vec) AMM_SS(true, 0, true);
      else AMM_SS(true, 0, false);
    } else if (imag == 0) {
      if (vec) AMM_SS(false, 0, true);
      else AMM_SS(false, 0, false);
    } else if (imag > 0) {
      if (vec) AMM_SS(false, 1, true);
      else AMM_SS(false, 1, false);
    } else {
      if (vec) AMM_SS(false, -1, true);
      else AMM_SS(false, -1, false);
    }
#undef AMM_SS
  }
  dev_free(cnt, st);
  return e;
}

// ============================================================================ P_A(G dB~^T)
// For each kept (i, q) of A~_a:  XAT[q][i] += sum_c G(i, c) B~(q, c) [(q, c) not kept in B~_a].
// CTA per row i (G row shared through L1), warp per kept entry, lanes over c.  MASKED = false: no
// entry excluded (B~ the transform of a dense residual, for mixed-method gradients); IMAG = +1 / -1:
// the sum is multiplied by +i / -i before it is added.  Both are template flags so that the
// masked loop of the plain backward carries no extra test.
template <bool MASKED, int IMAG>
__global__ void __launch_bounds__(256) ft_bw_pa_kernel(const float* __restrict__ G, int64_t ldg,
                                                       const float2* __restrict__ Bt, const uint32_t* __restrict__ maskB,
                                                       int mwB, const int32_t* __restrict__ selA, int ka, int n, int m,
                                                       int p, float2* __restrict__ XAT) {
  const int i = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float* grow = G + (int64_t)i * ldg;
  for (int u = warp; u < ka; u += 8) {
    const int q = __ldg(selA + (int64_t)i * ka + u);
    const bool mir = q > n / 2;
    const float2* brow = Bt + (int64_t)(mir ? n - q : q) * p;
    const uint32_t* mrow = MASKED ? maskB + (int64_t)q * mwB : nullptr;
    float ax = 0.f, ay = 0.f;
    for (int c = lane; c < p; c += 32) {
      if (MASKED && ((__ldg(mrow + (c >> 5)) >> (c & 31)) & 1u)) continue;  // kept in B~_a: not in dB~
      const float g = __ldg(grow + c);
      const float2 b = __ldg(brow + c);
      ax = fmaf(g, b.x, ax);
      ay = fmaf(g, b.y, ay);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      ax += __shfl_xor_sync(0xffffffffu, ax, o);
      ay += __shfl_xor_sync(0xffffffffu, ay, o);
    }
    if (lane == 0) {
      float2* x = XAT + (int64_t)q * m + i;
      const float2 v = *x;
      const float2 d = make_float2(ax, mir ? -ay : ay);
      *x = IMAG > 0 ? make_float2(v.x - d.y, v.y + d.x)
                    : IMAG < 0 ? make_float2(v.x + d.y, v.y - d.x) : make_float2(v.x + d.x, v.y + d.y);
    }
  }
}

// ============================================================================ P_B(dA~^T G)
// For each kept (q, c) of B~_a:  XB[q][c] += sum_i A~(i, q) [(i, q) not kept in A~_a] G(i, c).
// CTA per column c (GT row shared through L1), warp per kept entry, lanes over i.  MASKED and IMAG
// as for ft_bw_pa_kernel.
template <bool MASKED, int IMAG>
__global__ void __launch_bounds__(256) ft_bw_pb_kernel(const float* __restrict__ GT, const float2* __restrict__ AtT,
                                                       const uint32_t* __restrict__ maskA, int mwA,
                                                       const int32_t* __restrict__ selB, int kb, int n, int m, int p,
                                                       float2* __restrict__ XB) {
  const int c = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float* grow = GT + (int64_t)c * m;
  for (int u = warp; u < kb; u += 8) {
    const int q = __ldg(selB + (int64_t)c * kb + u);
    const bool mir = q > n / 2;
    const float2* arow = AtT + (int64_t)(mir ? n - q : q) * m;
    const uint32_t* mrow = MASKED ? maskA + (int64_t)q * mwA : nullptr;
    float ax = 0.f, ay = 0.f;
    for (int i = lane; i < m; i += 32) {
      if (MASKED && ((__ldg(mrow + (i >> 5)) >> (i & 31)) & 1u)) continue;  // kept in A~_a: not in dA~
      const float g = __ldg(grow + i);
      const float2 a = __ldg(arow + i);
      ax = fmaf(g, a.x, ax);
      ay = fmaf(g, a.y, ay);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      ax += __shfl_xor_sync(0xffffffffu, ax, o);
      ay += __shfl_xor_sync(0xffffffffu, ay, o);
    }
    if (lane == 0) {
      float2* x = XB + (int64_t)q * p + c;
      const float2 v = *x;
      const float2 d = make_float2(ax, mir ? -ay : ay);
      *x = IMAG > 0 ? make_float2(v.x - d.y, v.y + d.x)
                    : IMAG < 0 ? make_float2(v.x + d.y, v.y - d.x) : make_float2(v.x + d.x, v.y + d.y);
    }
  }
}

// ============================================================================ real part of a transform
// X [n][nvec] complex, frequency-major.  For each vector v: y_v(l) = n^{-1/2} Re sum_q X(q, v)
// e^{-+2 pi i q l/n} (INV selects +).  Vectors v0, v0+1 share one complex FFT of
// Z = H_{v0} + i H_{v1}.  OUT_ROW writes y_v to out[v][l], otherwise to out[l][v].
template <int N, int S, int NT, bool INV, bool OUT_ROW>
__global__ void __launch_bounds__(NT) ft_bw_real_kernel(const float2* __restrict__ X, int nvec,
                                                        const float2* __restrict__ tw, float* __restrict__ out,
                                                        int64_t ldo) {
  extern __shared__ float2 smem[];
  constexpr int LD = fft_padded_len(N);
  const int base = blockIdx.x * 2 * S;
  for (int e = threadIdx.x; e < (N / 2 + 1) * S; e += NT) {
    const int q = e / S, s = e % S;
    const int r = wrapN<N>(N - q);
    const int v0 = base + 2 * s, v1 = v0 + 1;
    float2 x0q = make_float2(0.f, 0.f), x0r = x0q, x1q = x0q, x1r = x0q;
    if (v0 < nvec) { x0q = X[(int64_t)q * nvec + v0]; x0r = X[(int64_t)r * nvec + v0]; }
    if (v1 < nvec) { x1q = X[(int64_t)q * nvec + v1]; x1r = X[(int64_t)r * nvec + v1]; }
    // H(q) = (x(q) + conj x(r)) / 2, H(r) = conj H(q)
    const float2 h0 = make_float2(0.5f * (x0q.x + x0r.x), 0.5f * (x0q.y - x0r.y));
    const float2 h1 = make_float2(0.5f * (x1q.x + x1r.x), 0.5f * (x1q.y - x1r.y));
    smem[s * LD + fpad(q)] = make_float2(h0.x - h1.y, h0.y + h1.x);  // h0 + i h1
    smem[s * LD + fpad(r)] = make_float2(h0.x + h1.y, h1.x - h0.y);  // conj h0 + i conj h1
  }
  __syncthreads();
  fft_smem<N, S, NT, INV>(smem, tw);
  const float sc = rsqrtf((float)N);
  for (int e = threadIdx.x; e < N * 2 * S; e += NT) {
    int l, mm;
    if (OUT_ROW) { mm = e / N; l = e % N; } else { l = e / (2 * S); mm = e % (2 * S); }
    const int v = base + mm;
    if (v >= nvec) continue;
    const float2 z = smem[(mm >> 1) * LD + fpad(l)];
    const float y = sc * ((mm & 1) ? z.y : z.x);
    if (OUT_ROW) out[(int64_t)v * ldo + l] = y;
    else out[(int64_t)l * ldo + v] = y;
  }
}

template <int N> struct FtBwCfg {
  static constexpr int S = (N >= 6144) ? 2 : 4;
  static constexpr int NT = fft_threads(N);
  static constexpr size_t SMEM = sizeof(float2) * S * fft_padded_len(N);
};

template <int N> struct FtBwOps {
  using C = FtBwCfg<N>;
  template <bool INV, bool OUT_ROW>
  static cudaError_t real(const float2* X, int nvec, const float2* tw, float* out, int64_t ldo, cudaStream_t st) {
    static DeviceOnce once;
    const cudaError_t attr = once([] {
      return cudaFuncSetAttribute((const void*)ft_bw_real_kernel<N, C::S, C::NT, INV, OUT_ROW>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    });
    if (attr != cudaSuccess) return attr;
    dim3 grid((nvec + 2 * C::S - 1) / (2 * C::S));
    ft_bw_real_kernel<N, C::S, C::NT, INV, OUT_ROW><<<grid, C::NT, C::SMEM, st>>>(X, nvec, tw, out, ldo);
    return cudaGetLastError();
  }
  static cudaError_t inv_rows(const float2* X, int nvec, const float2* tw, float* out, int64_t ldo, cudaStream_t st) {
    return real<true, true>(X, nvec, tw, out, ldo, st);
  }
  static cudaError_t fwd_cols(const float2* X, int nvec, const float2* tw, float* out, int64_t ldo, cudaStream_t st) {
    return real<false, false>(X, nvec, tw, out, ldo, st);
  }
  static cudaError_t inv_cols(const float2* X, int nvec, const float2* tw, float* out, int64_t ldo, cudaStream_t st) {
    return real<true, false>(X, nvec, tw, out, ldo, st);
  }
};

#define AMM_FTB_DISPATCH(n, EXPR)                 \
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

static cudaError_t ft_bw_real(int n, bool inv, const float2* X, int nvec, const float2* tw, float* out, int64_t ldo,
                              cudaStream_t st) {
  AMM_TRACE_W(inv ? "ft_bw_idft_rows" : "ft_bw_dft_cols", st, 0.0, (double)n * nvec * 12, nullptr);
  if (inv) { AMM_FTB_DISPATCH(n, return FtBwOps<NN>::inv_rows(X, nvec, tw, out, ldo, st)); }
  AMM_FTB_DISPATCH(n, return FtBwOps<NN>::fwd_cols(X, nvec, tw, out, ldo, st));
}

// out[l][v] = n^{-1/2} Re sum_q X(q, v) e^{+2 pi i q l/n}: the inverse transform of each column of
// X [n][nvec], written as a column (the dense form of a right Fourier truncation)
static cudaError_t ft_bw_real_inv_cols(int n, const float2* X, int nvec, const float2* tw, float* out, int64_t ldo,
                                       cudaStream_t st) {
  AMM_TRACE_W("ft_idft_cols", st, 0.0, (double)n * nvec * 12, nullptr);
  AMM_FTB_DISPATCH(n, return FtBwOps<NN>::inv_cols(X, nvec, tw, out, ldo, st));
}

// ============================================================================ mixed-method pieces
// out[r][c] += t[r][c]
__global__ void ft_add_kernel(float* __restrict__ out, int64_t ldo, const float* __restrict__ t, int64_t ldt,
                              int64_t rows, int64_t cols) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= rows * cols) return;
  const int64_t r = e / cols, c = e - r * cols;
  out[r * ldo + c] += t[r * ldt + c];
}

// d[r][c] -= t[r][c]
__global__ void ft_sub_kernel(float* __restrict__ d, int64_t ldd, const float* __restrict__ t, int64_t ldt,
                              int64_t rows, int64_t cols) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= rows * cols) return;
  const int64_t r = e / cols, c = e - r * cols;
  d[r * ldd + c] -= t[r * ldt + c];
}

static cudaError_t add_into(float* out, int64_t ldo, const float* t, int64_t ldt, int64_t rows, int64_t cols,
                            cudaStream_t st) {
  const int64_t cnt = rows * cols;
  ft_add_kernel<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(out, ldo, t, ldt, rows, cols);
  return cudaGetLastError();
}

// X[q][c] = f * B~(q, c) on the kept entries of each column (selB [p][kb]), 0 elsewhere, q = 0..n-1;
// f = 1 (part 0) or -i (part 1).  One thread per kept entry; X must be zero on entry.
__global__ void ft_scatter_cols_kernel(const float2* __restrict__ Bt, const int32_t* __restrict__ selB, int kb, int n,
                                       int p, int part, float2* __restrict__ X) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)p * kb) return;
  const int c = (int)(e / kb);
  const int q = __ldg(selB + e);
  const float2 v = half_spec(Bt, n, q, p, c);
  X[(int64_t)q * p + c] = part ? make_float2(v.y, -v.x) : v;
}

// Dense parts of a right Fourier truncation B_s = W^* B~_a (n x p): part 0 writes D = B - Re B_s,
// part 1 D = Im B_s.
cudaError_t ft_right_dense(int n, int p, const float2* Bt, const int32_t* selB, int kb, const float2* tw, int part,
                           const float* B, int64_t ldb, float* D, int64_t ldd, cudaStream_t st) {
  float2* X = nullptr;
  float* Y = nullptr;
  cudaError_t e = dev_alloc((void**)&X, sizeof(float2) * (size_t)n * p, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(X, 0, sizeof(float2) * (size_t)n * p, st);
  if (e == cudaSuccess) {
    ft_scatter_cols_kernel<<<(unsigned)(((int64_t)p * kb + 255) / 256), 256, 0, st>>>(Bt, selB, kb, n, p, part, X);
    e = cudaGetLastError();
  }
  if (part == 0) {
    if (e == cudaSuccess) e = dev_alloc((void**)&Y, sizeof(float) * (size_t)n * p, st);
    if (e == cudaSuccess) e = ft_bw_real_inv_cols(n, X, p, tw, Y, p, st);  // Re(W^* X)
    if (e == cudaSuccess) e = cudaMemcpy2DAsync(D, sizeof(float) * ldd, B, sizeof(float) * ldb, sizeof(float) * p, n,
                                                cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) {  // D -= Y
      const int64_t cnt = (int64_t)n * p;
      ft_sub_kernel<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(D, ldd, Y, p, n, p);
      e = cudaGetLastError();
    }
  } else if (e == cudaSuccess) {
    e = ft_bw_real_inv_cols(n, X, p, tw, D, ldd, st);  // Re(W^* (-i X)) = Im(W^* X)
  }
  dev_free(X, st);
  if (Y) dev_free(Y, st);
  return e;
}

// out = Re(G B~^T) for a right Fourier truncation (G m x p, out m x n): the sparse x dense product
// over the kept entries of B~_a, then the inverse row transforms (the first term of dA above)
cudaError_t ft_rt_apply_bw(int n, int m, int p, const float2* Bt, const uint32_t* maskB, int kb, const float2* tw,
                           const float* G, int64_t ldg, float* out, int64_t ldo, cudaStream_t st) {
  const int mwB = (p + 31) / 32;
  float *GT = nullptr;
  float2* XAT = nullptr;
  cudaError_t e = dev_alloc((void**)&GT, sizeof(float) * (size_t)p * m, st);
  if (e == cudaSuccess) e = dev_alloc((void**)&XAT, sizeof(float2) * (size_t)n * m, st);
  if (e == cudaSuccess) e = transpose_f32(G, m, p, ldg, GT, m, st);
  if (e == cudaSuccess) {
    AMM_TRACE_W("ft_bw_gba", st, 4.0 * p * (double)kb * m, 4.0 * m * (double)p + 8.0 * p * (double)kb + 8.0 * n * m,
                nullptr);
    e = ft_bw_spmm(GT, m, m, Bt, p, maskB, mwB, n, (int64_t)kb * p, XAT, st);
  }
  if (e == cudaSuccess) e = ft_bw_real(n, true, XAT, m, tw, out, ldo, st);
  dev_free(GT, st);
  dev_free(XAT, st);
  return e;
}

// out = Re(A~^T G) for a left Fourier truncation (G m x p, out n x p): the sparse x dense product
// over the kept entries of A~_a, then the forward column transforms (the first term of dB above)
cudaError_t ft_lt_apply_bw(int n, int m, int p, const float2* AtT, const uint32_t* maskA, int ka, const float2* tw,
                           const float* G, int64_t ldg, float* out, int64_t ldo, cudaStream_t st) {
  const int mwA = (m + 31) / 32;
  float2* XB = nullptr;
  cudaError_t e = dev_alloc((void**)&XB, sizeof(float2) * (size_t)n * p, st);
  if (e == cudaSuccess) {
    AMM_TRACE_W("ft_bw_aag", st, 4.0 * m * (double)ka * p, 4.0 * m * (double)p + 8.0 * m * (double)ka + 8.0 * n * p,
                nullptr);
    e = ft_bw_spmm(G, ldg, p, AtT, m, maskA, mwA, n, (int64_t)ka * m, XB, st);
  }
  if (e == cudaSuccess) e = ft_bw_real(n, false, XB, p, tw, out, ldo, st);
  dev_free(XB, st);
  return e;
}

// out (m x n) += Re P_A'(G D^T) for a left Fourier truncation with kept entries selA (m x ka), where
// D = Dre + s i Dim (n x p, Dim may be NULL; s = sign_im = +1 / -1) and P_A'(Y) = (M o (Y W)) conj(W):
// (Y W)(i, q) = sum_c G(i, c) (W D)(q, c) is sampled at the kept (i, q) from the column transforms
// of D, and the last step is the inverse row transform.
cudaError_t ft_proj_left(int n, int m, int p, const int32_t* selA, const uint32_t* maskA, int ka, const float2* tw,
                         const float* G, int64_t ldg, const float* Dre, const float* Dim, int sign_im, int64_t ldd,
                         float* out, int64_t ldo, cudaStream_t st) {
  const size_t kh = (size_t)n / 2 + 1;
  float2 *T = nullptr, *XAT = nullptr;
  float *mag = nullptr, *Y = nullptr;
  cudaError_t e = dev_alloc((void**)&T, sizeof(float2) * kh * p, st);
  if (e == cudaSuccess) e = dev_alloc((void**)&mag, sizeof(float) * kh * p, st);
  if (e == cudaSuccess) e = dev_alloc((void**)&XAT, sizeof(float2) * (size_t)n * m, st);
  if (e == cudaSuccess) e = dev_alloc((void**)&Y, sizeof(float) * (size_t)m * n, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(XAT, 0, sizeof(float2) * (size_t)n * m, st);
  for (int part = 0; part < 2 && e == cudaSuccess; ++part) {
    const float* D = part ? Dim : Dre;
    if (!D) continue;
    e = ft_transform(n, false, D, ldd, p, tw, T, nullptr, mag, st);  // W D, half spectrum [kh][p]
    if (e == cudaSuccess) {
      AMM_TRACE_W("ft_bw_pa", st, 4.0 * m * (double)ka * p, 4.0 * m * (double)p + 8.0 * kh * p, nullptr);
      const int imag = part == 0 ? 0 : sign_im > 0 ? 1 : -1;
      if (p <= SS_MAX_LEN) {
        e = ft_bw_sampled(G, ldg, p, T, p, nullptr, 0, maskA, (m + 31) / 32, n, m, (int64_t)ka * m, imag, XAT, st);
      } else {
        if (imag == 0) ft_bw_pa_kernel<false, 0><<<m, 256, 0, st>>>(G, ldg, T, nullptr, 0, selA, ka, n, m, p, XAT);
        else if (imag > 0) ft_bw_pa_kernel<false, 1><<<m, 256, 0, st>>>(G, ldg, T, nullptr, 0, selA, ka, n, m, p, XAT);
        else ft_bw_pa_kernel<false, -1><<<m, 256, 0, st>>>(G, ldg, T, nullptr, 0, selA, ka, n, m, p, XAT);
        e = cudaGetLastError();
      }
    }
  }
  if (e == cudaSuccess) e = ft_bw_real(n, true, XAT, m, tw, Y, n, st);
  if (e == cudaSuccess) e = add_into(out, ldo, Y, n, m, n, st);
  for (void* q : {(void*)T, (void*)mag, (void*)XAT, (void*)Y})
    if (q) dev_free(q, st);
  return e;
}

// out (n x p) += Re P_B'(D^T G) for a right Fourier truncation with kept entries selB (p x kb), where
// D = Dre + s i Dim (m x n) and P_B'(Y) = W (M o (conj(W) Y)): (conj(W) Y)(q, c) = sum_i (D W^*)(i, q)
// G(i, c) is sampled at the kept (q, c) from the row transforms of D, and the last step is the
// forward column transform.
cudaError_t ft_proj_right(int n, int m, int p, const int32_t* selB, const uint32_t* maskB, int kb,
                          const float2* tw, const float* Dre, const float* Dim, int sign_im, int64_t ldd,
                          const float* G, int64_t ldg, float* out, int64_t ldo, cudaStream_t st) {
  const size_t kh = (size_t)n / 2 + 1;
  float2 *T = nullptr, *TT = nullptr, *XB = nullptr;
  float *mag = nullptr, *GT = nullptr, *Y = nullptr;
  cudaError_t e = dev_alloc((void**)&T, sizeof(float2) * kh * m, st);
  if (e == cudaSuccess) e = dev_alloc((void**)&TT, sizeof(float2) * kh * m, st);
  if (e == cudaSuccess) e = dev_alloc((void**)&mag, sizeof(float) * kh * m, st);
  if (e == cudaSuccess) e = dev_alloc((void**)&GT, sizeof(float) * (size_t)p * m, st);
  if (e == cudaSuccess) e = dev_alloc((void**)&XB, sizeof(float2) * (size_t)n * p, st);
  if (e == cudaSuccess) e = dev_alloc((void**)&Y, sizeof(float) * (size_t)n * p, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(XB, 0, sizeof(float2) * (size_t)n * p, st);
  if (e == cudaSuccess) e = transpose_f32(G, m, p, ldg, GT, m, st);
  for (int part = 0; part < 2 && e == cudaSuccess; ++part) {
    const float* D = part ? Dim : Dre;
    if (!D) continue;
    e = ft_transform(n, true, D, ldd, m, tw, T, TT, mag, st);  // D W^*, transposed half spectrum [kh][m]
    if (e == cudaSuccess) {
      AMM_TRACE_W("ft_bw_pb", st, 4.0 * p * (double)kb * m, 4.0 * m * (double)p + 8.0 * kh * m, nullptr);
      const int imag = part == 0 ? 0 : sign_im > 0 ? 1 : -1;
      if (m <= SS_MAX_LEN) {
        e = ft_bw_sampled(GT, m, m, TT, m, nullptr, 0, maskB, (p + 31) / 32, n, p, (int64_t)kb * p, imag, XB, st);
      } else {
        if (imag == 0) ft_bw_pb_kernel<false, 0><<<p, 256, 0, st>>>(GT, TT, nullptr, 0, selB, kb, n, m, p, XB);
        else if (imag > 0) ft_bw_pb_kernel<false, 1><<<p, 256, 0, st>>>(GT, TT, nullptr, 0, selB, kb, n, m, p, XB);
        else ft_bw_pb_kernel<false, -1><<<p, 256, 0, st>>>(GT, TT, nullptr, 0, selB, kb, n, m, p, XB);
        e = cudaGetLastError();
      }
    }
  }
  if (e == cudaSuccess) e = ft_bw_real(n, false, XB, p, tw, Y, p, st);
  if (e == cudaSuccess) e = add_into(out, ldo, Y, p, n, p, st);
  for (void* q : {(void*)T, (void*)TT, (void*)mag, (void*)GT, (void*)XB, (void*)Y})
    if (q) dev_free(q, st);
  return e;
}

// Trace work of the kernels below: FLOPs of the real or complex products actually formed, bytes the
// minimal HBM traffic (each operand read once, each output written once); the kernels themselves
// are bound by L2 gathers, which neither figure counts.
cudaError_t ft_backward(const FtBwArgs& a, cudaStream_t st) {
  const int n = a.n, m = a.m, p = a.p;
  const int mwA = (m + 31) / 32, mwB = (p + 31) / 32;
  float* GT = nullptr;
  float2* XAT = nullptr;
  float2* XB = nullptr;
  cudaError_t e = dev_alloc((void**)&GT, sizeof(float) * (size_t)p * m, st);
  if (e == cudaSuccess && a.dA) e = dev_alloc((void**)&XAT, sizeof(float2) * (size_t)n * m, st);
  if (e == cudaSuccess && a.dB) e = dev_alloc((void**)&XB, sizeof(float2) * (size_t)n * p, st);
  if (e == cudaSuccess) e = transpose_f32(a.G, m, p, a.ldg, GT, m, st);
  if (e == cudaSuccess && a.dA) {
    {
      AMM_TRACE_W("ft_bw_gba", st, 4.0 * p * (double)a.kb * m, 4.0 * m * (double)p + 8.0 * p * (double)a.kb + 8.0 * n * m,
                  nullptr);
      e = ft_bw_spmm(GT, m, m, a.Bt, p, a.maskB, mwB, n, (int64_t)a.kb * p, XAT, st);
    }
    if (e == cudaSuccess) {
      AMM_TRACE_W("ft_bw_pa", st, 4.0 * m * (double)a.ka * p,
                  4.0 * m * (double)p + 8.0 * (n / 2 + 1.0) * p + 16.0 * m * (double)a.ka, nullptr);
      if (p <= SS_MAX_LEN) {
        e = ft_bw_sampled(a.G, a.ldg, p, a.Bt, p, a.maskB, mwB, a.maskA, mwA, n, m, (int64_t)a.ka * m, 0, XAT, st);
      } else {
        ft_bw_pa_kernel<true, 0><<<m, 256, 0, st>>>(a.G, a.ldg, a.Bt, a.maskB, mwB, a.selA, a.ka, n, m, p, XAT);
        e = cudaGetLastError();
      }
    }
    if (e == cudaSuccess) e = ft_bw_real(n, true, XAT, m, a.tw, a.dA, a.ldda, st);
  }
  if (e == cudaSuccess && a.dB) {
    {
      AMM_TRACE_W("ft_bw_aag", st, 4.0 * m * (double)a.ka * p, 4.0 * m * (double)p + 8.0 * m * (double)a.ka + 8.0 * n * p,
                  nullptr);
      e = ft_bw_spmm(a.G, a.ldg, p, a.AtT, m, a.maskA, mwA, n, (int64_t)a.ka * m, XB, st);
    }
    if (e == cudaSuccess) {
      AMM_TRACE_W("ft_bw_pb", st, 4.0 * p * (double)a.kb * m,
                  4.0 * m * (double)p + 8.0 * (n / 2 + 1.0) * m + 16.0 * p * (double)a.kb, nullptr);
      if (m <= SS_MAX_LEN) {
        e = ft_bw_sampled(GT, m, m, a.AtT, m, a.maskA, mwA, a.maskB, mwB, n, p, (int64_t)a.kb * p, 0, XB, st);
      } else {
        ft_bw_pb_kernel<true, 0><<<p, 256, 0, st>>>(GT, a.AtT, a.maskA, mwA, a.selB, a.kb, n, m, p, XB);
        e = cudaGetLastError();
      }
    }
    if (e == cudaSuccess) e = ft_bw_real(n, false, XB, p, a.tw, a.dB, a.lddb, st);
  }
  dev_free(GT, st);
  dev_free(XAT, st);
  dev_free(XB, st);
  return e;
}

}  // namespace amm
