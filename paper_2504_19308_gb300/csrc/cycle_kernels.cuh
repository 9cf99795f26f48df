// Tile bodies of the cycle-sparsifier forward kernels (Section 1.2.2; Eq. (2.4)-(2.5) of
// arXiv 2504.19308), shared by the kernels of cycle.cu (one tile per CTA) and by the batch's
// persistent executor (tiles taken from a work queue): the same arithmetic in the same order, so
// both give bit-identical results.  Every body takes its tile index explicitly and is called by
// all CYC_NT threads of a CTA (256 for the key and gather tiles).
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

namespace amm {

constexpr int CYC_CW = 4;    // columns per CTA (A_s B)
constexpr int CYC_RW = 4;    // rows per CTA (dA B_s)
constexpr int CYC_NT = 256;
constexpr int CYC_RG = 8;    // rows (or columns) per thread per pass of the component loop

// Loads of the selections, selected cycles and kept-cycle flags.  PC (produced in this launch):
// the persistent executor writes them in an earlier stage of the same kernel, so they are read
// with ordinary cached loads (ld.global.ca), which the executor's acquire of the stage counter
// orders after the writes; the read-only path (ld.global.nc), which assumes data that no thread
// writes during the launch, serves the one-tile-per-CTA kernels.
template <bool PC, typename T> AMM_DEV T ldp(const T* p) {
  if constexpr (PC) return __ldca(p);
  else return __ldg(p);
}

// part[rb][j] = sum over rows r of block rb of A(r, (r - j) mod n)^2 for the 256 cycles of block
// jb (thread per cycle j: a warp reads 32 consecutive columns of one row).
AMM_DEV void cyc_keys_tile(const float* __restrict__ A, int64_t lda, int n, int rows_per, float* __restrict__ part,
                           int jb, int rb) {
  const int j = jb * 256 + threadIdx.x;
  if (j >= n) return;
  const int r0 = rb * rows_per;
  float s = 0.f;
  for (int r = r0; r < min(n, r0 + rows_per); ++r) {
    const float v = __ldg(A + (int64_t)r * lda + cwrap<false>(r - j, n));
    s = fmaf(v, v, s);
  }
  part[(int64_t)rb * n + j] = s;
}

// cyc[u][l] = A((l + t_u) mod n, l) for selected cycle u, l = x0, x0 + xs, ... (x0 = the thread's
// first column, xs the stride); the tile with x0 == threadIdx.x of thread 0 sets insel[t_u] = 1.
template <bool PC>
AMM_DEV void cyc_gather_tile(const float* __restrict__ A, int64_t lda, int n, const int32_t* __restrict__ sel,
                             float* __restrict__ cyc, unsigned char* __restrict__ insel, int u, int x0, int xs,
                             bool mark) {
  const int t = ldp<PC>(sel + u);
  for (int l = x0; l < n; l += xs) cyc[(int64_t)u * n + l] = __ldg(A + (int64_t)cwrap<false>(l + t, n) * lda + l);
  if (mark && threadIdx.x == 0) insel[t] = 1;
}

// out(:, c0..c0+3) = sum_u cyc[u][r - t_u] B(r - t_u, c), c0 = cb * CYC_CW.  bp: shared memory of
// n float4 plus k ints.
template <bool P2, bool PC>
AMM_DEV void cyc_apply_col_tile(const float* __restrict__ B, int64_t ldb, int n, const int32_t* __restrict__ sel,
                                int k, const float* __restrict__ cyc, float* __restrict__ out, int64_t ldo, int ncols,
                                int cb, float4* bp) {
  int* s_sel = reinterpret_cast<int*>(bp + n);
  const int c0 = cb * CYC_CW;
  for (int r = threadIdx.x; r < n; r += CYC_NT) {
    const float* src = B + (int64_t)r * ldb + c0;
    float4 v;
    v.x = c0 + 0 < ncols ? __ldg(src + 0) : 0.f;
    v.y = c0 + 1 < ncols ? __ldg(src + 1) : 0.f;
    v.z = c0 + 2 < ncols ? __ldg(src + 2) : 0.f;
    v.w = c0 + 3 < ncols ? __ldg(src + 3) : 0.f;
    bp[r] = v;
  }
  for (int u = threadIdx.x; u < k; u += CYC_NT) s_sel[u] = ldp<PC>(sel + u);
  __syncthreads();
  // CYC_RG rows per thread at a time, components in the outer loop: CYC_RG independent gathers
  // of cyc in flight per component
  for (int r0 = threadIdx.x; r0 < n; r0 += CYC_NT * CYC_RG) {
    float4 acc[CYC_RG];
#pragma unroll
    for (int i = 0; i < CYC_RG; ++i) acc[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    // unrolled over components: the gathers of several components are issued before the FMAs
    // that wait on them (the loads are L2 hits whose latency, not bandwidth, set the time)
#pragma unroll 2
    for (int u = 0; u < k; ++u) {
      const int t = s_sel[u];
      const float* crow = cyc + (int64_t)u * n;
#pragma unroll
      for (int i = 0; i < CYC_RG; ++i) {
        const int r = r0 + i * CYC_NT;
        if (r < n) {
          const int l = cwrap<P2>(r - t, n);
          const float a = ldp<PC>(crow + l);
          const float4 b = bp[l];
          acc[i].x = fmaf(a, b.x, acc[i].x);
          acc[i].y = fmaf(a, b.y, acc[i].y);
          acc[i].z = fmaf(a, b.z, acc[i].z);
          acc[i].w = fmaf(a, b.w, acc[i].w);
        }
      }
    }
#pragma unroll
    for (int i = 0; i < CYC_RG; ++i) {
      const int r = r0 + i * CYC_NT;
      if (r >= n) continue;
      float* o = out + (int64_t)r * ldo + c0;
      if (c0 + 0 < ncols) o[0] = acc[i].x;
      if (c0 + 1 < ncols) o[1] = acc[i].y;
      if (c0 + 2 < ncols) o[2] = acc[i].z;
      if (c0 + 3 < ncols) o[3] = acc[i].w;
    }
  }
}

// out(r0..r0+3, :) += sum_u dA(r, c + s_u) cycB[u][c], r0 = rb * CYC_RW; dA = A with the kept
// cycles of A masked (inselA), or A itself when inselA is NULL.  ar: shared memory of CYC_RW x n
// floats.
template <bool P2, bool PC>
AMM_DEV void cyc_apply_row_tile(const float* __restrict__ A, int64_t lda, int n,
                                const unsigned char* __restrict__ inselA, const int32_t* __restrict__ selB, int kb,
                                const float* __restrict__ cycB, float* __restrict__ out, int64_t ldo, int nrows,
                                int rb, float* ar) {
  const int r0 = rb * CYC_RW;
  for (int e = threadIdx.x; e < CYC_RW * n; e += CYC_NT) {
    const int rr = e / n, q = e % n, r = r0 + rr;
    float v = 0.f;
    if (r < nrows && (inselA == nullptr || !ldp<PC>(inselA + cwrap<P2>(r - q, n)))) v = __ldg(A + (int64_t)r * lda + q);
    ar[e] = v;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < n; c += CYC_NT) {
    float acc[CYC_RW] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 8
    for (int u = 0; u < kb; ++u) {
      const int q = cwrap<P2>(c + ldp<PC>(selB + u), n);
      const float b = ldp<PC>(cycB + (int64_t)u * n + c);
#pragma unroll
      for (int rr = 0; rr < CYC_RW; ++rr) acc[rr] = fmaf(ar[rr * n + q], b, acc[rr]);
    }
#pragma unroll
    for (int rr = 0; rr < CYC_RW; ++rr) {
      if (r0 + rr >= nrows) continue;
      float* o = out + (int64_t)(r0 + rr) * ldo + c;  // written by the column tiles (PC: this launch)
      *o = (PC ? __ldcg(o) : *o) + acc[rr];
    }
  }
}

}  // namespace amm
