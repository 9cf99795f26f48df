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
// CTA per (q, 1024 outputs): the mask row is compacted in shared memory chunk by chunk (index and
// coefficient per set bit), then every thread streams the selected rows of D for its 4 outputs.
constexpr int MW_CHUNK = 64;  // mask words per chunk (2048 bits)
constexpr int MW_RPT = 4;     // outputs per thread
__global__ void __launch_bounds__(256) ft_bw_maskwalk_kernel(const float* __restrict__ D, int64_t ldd, int nout,
                                                             const float2* __restrict__ T, int64_t ldt,
                                                             const uint32_t* __restrict__ mask, int mw, int n,
                                                             float2* __restrict__ out) {
  __shared__ int32_t s_idx[MW_CHUNK * 32];
  __shared__ float2 s_val[MW_CHUNK * 32];
  __shared__ int32_t s_off[MW_CHUNK + 1];
  const int q = blockIdx.y;
  const int v0 = blockIdx.x * (256 * MW_RPT) + threadIdx.x;
  const uint32_t* mrow = mask + (int64_t)q * mw;
  float2 acc[MW_RPT];
#pragma unroll
  for (int r = 0; r < MW_RPT; ++r) acc[r] = make_float2(0.f, 0.f);
  for (int w0 = 0; w0 < mw; w0 += MW_CHUNK) {
    uint32_t bits = 0;
    if (threadIdx.x < MW_CHUNK && w0 + threadIdx.x < mw) bits = __ldg(mrow + w0 + threadIdx.x);
    if (threadIdx.x < 32) {  // exclusive scan of the popcounts of 64 words (two per lane)
      const uint32_t b0 = __ldg(mrow + min(w0 + 2 * (int)threadIdx.x, mw - 1));
      const uint32_t b1 = __ldg(mrow + min(w0 + 2 * (int)threadIdx.x + 1, mw - 1));
      const int c0 = (w0 + 2 * (int)threadIdx.x < mw) ? __popc(b0) : 0;
      const int c1 = (w0 + 2 * (int)threadIdx.x + 1 < mw) ? __popc(b1) : 0;
      int x = c0 + c1;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if ((int)threadIdx.x >= o) x += y;
      }
      s_off[2 * threadIdx.x] = x - c0 - c1;
      s_off[2 * threadIdx.x + 1] = x - c1;
      if (threadIdx.x == 31) s_off[MW_CHUNK] = x;
    }
    __syncthreads();
    if (threadIdx.x < MW_CHUNK) {
      int o = s_off[threadIdx.x];
      while (bits) {
        const int x = (w0 + threadIdx.x) * 32 + __ffs(bits) - 1;
        bits &= bits - 1;
        s_idx[o] = x;
        s_val[o] = half_spec(T, n, q, ldt, x);
        ++o;
      }
    }
    __syncthreads();
    const int cnt = s_off[MW_CHUNK];
    for (int e = 0; e < cnt; ++e) {
      const int x = s_idx[e];
      const float2 c = s_val[e];
      const float* drow = D + (int64_t)x * ldd;
#pragma unroll
      for (int r = 0; r < MW_RPT; ++r) {
        const int v = v0 + r * 256;
        if (v < nout) {
          const float d = __ldg(drow + v);
          acc[r].x = fmaf(d, c.x, acc[r].x);
          acc[r].y = fmaf(d, c.y, acc[r].y);
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < MW_RPT; ++r) {
    const int v = v0 + r * 256;
    if (v < nout) out[(int64_t)q * nout + v] = acc[r];
  }
}

// ============================================================================ P_A(G dB~^T)
// For each kept (i, q) of A~_a:  XAT[q][i] += sum_c G(i, c) B~(q, c) [(q, c) not kept in B~_a].
// CTA per row i (G row shared through L1), warp per kept entry, lanes over c.  maskB NULL: no
// entry excluded (B~ the transform of a dense residual, for mixed-method gradients); imag = +1 / -1:
// the sum is multiplied by +i / -i before it is added.
__global__ void __launch_bounds__(256) ft_bw_pa_kernel(const float* __restrict__ G, int64_t ldg,
                                                       const float2* __restrict__ Bt, const uint32_t* __restrict__ maskB,
                                                       int mwB, const int32_t* __restrict__ selA, int ka, int n, int m,
                                                       int p, float2* __restrict__ XAT, int imag) {
  const int i = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float* grow = G + (int64_t)i * ldg;
  for (int u = warp; u < ka; u += 8) {
    const int q = __ldg(selA + (int64_t)i * ka + u);
    const bool mir = q > n / 2;
    const float2* brow = Bt + (int64_t)(mir ? n - q : q) * p;
    const uint32_t* mrow = maskB ? maskB + (int64_t)q * mwB : nullptr;
    float ax = 0.f, ay = 0.f;
    for (int c = lane; c < p; c += 32) {
      if (maskB != nullptr && ((__ldg(mrow + (c >> 5)) >> (c & 31)) & 1u)) continue;  // kept in B~_a: not in dB~
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
      *x = imag > 0 ? make_float2(v.x - d.y, v.y + d.x)
                    : imag < 0 ? make_float2(v.x + d.y, v.y - d.x) : make_float2(v.x + d.x, v.y + d.y);
    }
  }
}

// ============================================================================ P_B(dA~^T G)
// For each kept (q, c) of B~_a:  XB[q][c] += sum_i A~(i, q) [(i, q) not kept in A~_a] G(i, c).
// CTA per column c (GT row shared through L1), warp per kept entry, lanes over i.  maskA NULL: no
// entry excluded; imag = +1 / -1: the sum is multiplied by +i / -i before it is added.
__global__ void __launch_bounds__(256) ft_bw_pb_kernel(const float* __restrict__ GT, const float2* __restrict__ AtT,
                                                       const uint32_t* __restrict__ maskA, int mwA,
                                                       const int32_t* __restrict__ selB, int kb, int n, int m, int p,
                                                       float2* __restrict__ XB, int imag) {
  const int c = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float* grow = GT + (int64_t)c * m;
  for (int u = warp; u < kb; u += 8) {
    const int q = __ldg(selB + (int64_t)c * kb + u);
    const bool mir = q > n / 2;
    const float2* arow = AtT + (int64_t)(mir ? n - q : q) * m;
    const uint32_t* mrow = maskA ? maskA + (int64_t)q * mwA : nullptr;
    float ax = 0.f, ay = 0.f;
    for (int i = lane; i < m; i += 32) {
      if (maskA != nullptr && ((__ldg(mrow + (i >> 5)) >> (i & 31)) & 1u)) continue;  // kept in A~_a: not in dA~
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
      *x = imag > 0 ? make_float2(v.x - d.y, v.y + d.x)
                    : imag < 0 ? make_float2(v.x + d.y, v.y - d.x) : make_float2(v.x + d.x, v.y + d.y);
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
    ft_bw_maskwalk_kernel<<<dim3((m + 256 * MW_RPT - 1) / (256 * MW_RPT), n), 256, 0, st>>>(GT, m, m, Bt, p, maskB,
                                                                                           mwB, n, XAT);
    e = cudaGetLastError();
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
    ft_bw_maskwalk_kernel<<<dim3((p + 256 * MW_RPT - 1) / (256 * MW_RPT), n), 256, 0, st>>>(G, ldg, p, AtT, m, maskA,
                                                                                           mwA, n, XB);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = ft_bw_real(n, false, XB, p, tw, out, ldo, st);
  dev_free(XB, st);
  return e;
}

// out (m x n) += Re P_A'(G D^T) for a left Fourier truncation with kept entries selA (m x ka), where
// D = Dre + s i Dim (n x p, Dim may be NULL; s = sign_im = +1 / -1) and P_A'(Y) = (M o (Y W)) conj(W):
// (Y W)(i, q) = sum_c G(i, c) (W D)(q, c) is sampled at the kept (i, q) from the column transforms
// of D, and the last step is the inverse row transform.
cudaError_t ft_proj_left(int n, int m, int p, const int32_t* selA, int ka, const float2* tw, const float* G,
                         int64_t ldg, const float* Dre, const float* Dim, int sign_im, int64_t ldd, float* out,
                         int64_t ldo, cudaStream_t st) {
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
      ft_bw_pa_kernel<<<m, 256, 0, st>>>(G, ldg, T, nullptr, 0, selA, ka, n, m, p, XAT, part ? sign_im : 0);
      e = cudaGetLastError();
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
cudaError_t ft_proj_right(int n, int m, int p, const int32_t* selB, int kb, const float2* tw, const float* Dre,
                          const float* Dim, int sign_im, int64_t ldd, const float* G, int64_t ldg, float* out,
                          int64_t ldo, cudaStream_t st) {
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
      ft_bw_pb_kernel<<<p, 256, 0, st>>>(GT, TT, nullptr, 0, selB, kb, n, m, p, XB, part ? sign_im : 0);
      e = cudaGetLastError();
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
      ft_bw_maskwalk_kernel<<<dim3((m + 256 * MW_RPT - 1) / (256 * MW_RPT), n), 256, 0, st>>>(
          GT, m, m, a.Bt, p, a.maskB, mwB, n, XAT);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
      AMM_TRACE_W("ft_bw_pa", st, 4.0 * m * (double)a.ka * p,
                  4.0 * m * (double)p + 8.0 * (n / 2 + 1.0) * p + 16.0 * m * (double)a.ka, nullptr);
      ft_bw_pa_kernel<<<m, 256, 0, st>>>(a.G, a.ldg, a.Bt, a.maskB, mwB, a.selA, a.ka, n, m, p, XAT, 0);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = ft_bw_real(n, true, XAT, m, a.tw, a.dA, a.ldda, st);
  }
  if (e == cudaSuccess && a.dB) {
    {
      AMM_TRACE_W("ft_bw_aag", st, 4.0 * m * (double)a.ka * p, 4.0 * m * (double)p + 8.0 * m * (double)a.ka + 8.0 * n * p,
                  nullptr);
      ft_bw_maskwalk_kernel<<<dim3((p + 256 * MW_RPT - 1) / (256 * MW_RPT), n), 256, 0, st>>>(
          a.G, a.ldg, p, a.AtT, m, a.maskA, mwA, n, XB);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
      AMM_TRACE_W("ft_bw_pb", st, 4.0 * p * (double)a.kb * m,
                  4.0 * m * (double)p + 8.0 * (n / 2 + 1.0) * m + 16.0 * p * (double)a.kb, nullptr);
      ft_bw_pb_kernel<<<p, 256, 0, st>>>(GT, a.AtT, a.maskA, mwA, a.selB, a.kb, n, m, p, XB, 0);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = ft_bw_real(n, false, XB, p, a.tw, a.dB, a.lddb, st);
  }
  dev_free(GT, st);
  dev_free(XAT, st);
  dev_free(XB, st);
  return e;
}

}  // namespace amm
