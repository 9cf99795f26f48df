// The circulant decomposition, product and backward at any length n in [16, 4096] that is neither
// 2^a nor 3 * 2^a (the lengths the fused kernels are compiled for).  Thm 2.1 and Alg. 2 / 3 hold for
// every n; only the FFT of length n changes.  Here a length-n DFT is computed by the chirp-z
// (Bluestein) identity
//
//     j k = (j^2 + k^2 - (k - j)^2) / 2   =>   X_k = w_k sum_j (x_j w_j) h_{k-j},
//     w_j = e^{-i pi j^2 / n},  h_m = e^{+i pi m^2 / n}   (the inverse DFT conjugates w and h),
//
// a circular convolution evaluated with power-of-two FFTs of length L >= 2n - 1 (L. I. Bluestein,
// "A linear filtering approach to the computation of the discrete Fourier transform", 1970).  The
// steps around the transforms -- the cycle gather of Alg. 7, the spectrum split and key partials,
// the spectral MAC of Alg. 3's applies, the inverse cycle transform, the backward SDDMM and the
// component spectra -- are separate small kernels that pass their operands through global
// scratch, one pass per step, where the fixed-length paths fuse them into one kernel: this is the
// general-length path, not the fast one.
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <map>
#include <mutex>
#include <vector>

#include "api_internal.h"
#include "common.cuh"
#include "fft.cuh"
#include "kernels.h"
#include "trace.h"

namespace amm {

bool cd_any_length_ok(int64_t n) { return n >= 16 && n <= CD_ANY_MAX_N; }

namespace {

// FFT length of the chirp convolution: the smallest power of two >= 2n - 1 (at least 256)
int chirp_len(int n) {
  int L = 256;
  while (L < 2 * n - 1) L <<= 1;
  return L;
}

// Bluestein tables of one length n (per device, kept for the process): w[j] = e^{-i pi j^2/n}
// (j < n); hf = FFT_L(h) / L and hi = FFT_L(conj h) / L with h[m] = e^{+i pi m^2/n} placed
// circularly (h at m and L - m for 0 <= m < n, zero between); twL the length-L twiddles.
struct Chirp {
  int n = 0, L = 0;
  float2* w = nullptr;
  float2* hf = nullptr;
  float2* hi = nullptr;
  const float2* twL = nullptr;
};

// e^{-+ i pi (j^2 mod 2n) / n} in double, rounded to float (the exponent reduced exactly first)
__global__ void chirp_w_kernel(float2* __restrict__ w, int n) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const long long jj = ((long long)j * j) % (2LL * n);
  double s, c;
  sincospi((double)jj / (double)n, &s, &c);
  w[j] = make_float2((float)c, (float)-s);
}

template <int L>
__global__ void __launch_bounds__(fft_threads(L)) chirp_hat_kernel(int n, const float2* __restrict__ twL,
                                                                   float2* __restrict__ hf, float2* __restrict__ hi) {
  extern __shared__ float2 sm[];
  constexpr int NT = fft_threads(L);
  const bool inv = blockIdx.x == 1;  // CTA 0: the forward filter h, CTA 1: conj h
  for (int m = threadIdx.x; m < L; m += NT) {
    const int d = m < n ? m : (L - m < n ? L - m : -1);  // |m| on the circle, if within (-n, n)
    float2 v = make_float2(0.f, 0.f);
    if (d >= 0) {
      const long long dd = ((long long)d * d) % (2LL * n);
      double s, c;
      sincospi((double)dd / (double)n, &s, &c);
      v = make_float2((float)c, (float)(inv ? -s : s));
    }
    sm[fpad(m)] = v;
  }
  __syncthreads();
  fft_smem<L, 1, NT, false>(sm, twL);
  const float sc = 1.f / (float)L;
  float2* out = inv ? hi : hf;
  for (int m = threadIdx.x; m < L; m += NT) out[m] = cscale(sm[fpad(m)], sc);
}

#define AMM_ANY_DISPATCH_L(L_, EXPR)                  \
  switch (L_) {                                       \
    case 256: { constexpr int LL = 256; EXPR; }       \
    case 512: { constexpr int LL = 512; EXPR; }       \
    case 1024: { constexpr int LL = 1024; EXPR; }     \
    case 2048: { constexpr int LL = 2048; EXPR; }     \
    case 4096: { constexpr int LL = 4096; EXPR; }     \
    case 8192: { constexpr int LL = 8192; EXPR; }     \
    default: return cudaErrorInvalidValue;            \
  }

std::mutex g_chirp_mu;
std::map<std::pair<int, int>, Chirp> g_chirp;

template <int L>
cudaError_t chirp_hat(int n, const float2* twL, float2* hf, float2* hi, cudaStream_t st) {
  constexpr size_t SM = sizeof(float2) * fft_padded_len(L);
  static DeviceOnce once;
  const cudaError_t a = once([] {
    return cudaFuncSetAttribute((const void*)chirp_hat_kernel<L>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)SM);
  });
  if (a != cudaSuccess) return a;
  chirp_hat_kernel<L><<<2, fft_threads(L), SM, st>>>(n, twL, hf, hi);
  return cudaGetLastError();
}

cudaError_t chirp_tables(int n, cudaStream_t st, Chirp* out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(g_chirp_mu);
  auto it = g_chirp.find({dev, n});
  if (it != g_chirp.end()) {
    *out = it->second;
    return cudaSuccess;
  }
  Chirp c;
  c.n = n;
  c.L = chirp_len(n);
  e = twiddles(c.L, st, &c.twL);
  float2* buf = nullptr;
  if (e == cudaSuccess) e = cudaMalloc(&buf, sizeof(float2) * ((size_t)n + 2 * (size_t)c.L));
  if (e != cudaSuccess) return e;
  c.w = buf;
  c.hf = buf + n;
  c.hi = c.hf + c.L;
  chirp_w_kernel<<<(n + 255) / 256, 256, 0, st>>>(c.w, n);
  e = cudaGetLastError();
  if (e == cudaSuccess) {
    AMM_ANY_DISPATCH_L(c.L, e = chirp_hat<LL>(n, c.twL, c.hf, c.hi, st); break);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaFree(buf);
    return e;
  }
  g_chirp[{dev, n}] = c;
  *out = c;
  return cudaSuccess;
}

// ============================================================================ DFT of rows
// out[row][k] = sum_j x_row[j] e^{-+2 pi i j k/n} (INV selects +, no scaling), k < n, one CTA per
// row.  REALPAIR: x_row[j] = re[2 row * rs + j * es] + i re[(2 row + 1) * rs + j * es] (two real
// vectors packed as one complex signal; the second is zero past nreal); otherwise x_row[j] =
// in[row * ldi + j].  With a gate given, a gated-off launch writes nothing.
template <int L, bool INV, bool REALPAIR>
__global__ void __launch_bounds__(fft_threads(L)) any_dft_kernel(const float2* __restrict__ in, int64_t ldi,
                                                                 const float* __restrict__ re, int64_t rs,
                                                                 int64_t es, int nreal, int n,
                                                                 const float2* __restrict__ w,
                                                                 const float2* __restrict__ hhat,
                                                                 const float2* __restrict__ twL,
                                                                 float2* __restrict__ out, int64_t ldo,
                                                                 const int32_t* __restrict__ gate0,
                                                                 const int32_t* __restrict__ gate1) {
  extern __shared__ float2 sm[];
  constexpr int NT = fft_threads(L);
  if (gate0 != nullptr && (*gate0 == 0 || *gate1 == 0)) return;
  const int row = blockIdx.x;
  for (int j = threadIdx.x; j < L; j += NT) {
    float2 a = make_float2(0.f, 0.f);
    if (j < n) {
      float2 x;
      if (REALPAIR) {
        const int v0 = 2 * row, v1 = 2 * row + 1;
        x.x = __ldg(re + (int64_t)v0 * rs + (int64_t)j * es);
        x.y = v1 < nreal ? __ldg(re + (int64_t)v1 * rs + (int64_t)j * es) : 0.f;
      } else {
        x = __ldg(in + (int64_t)row * ldi + j);
      }
      float2 c = __ldg(w + j);
      if (INV) c.y = -c.y;
      a = cmul(x, c);
    }
    sm[fpad(j)] = a;
  }
  __syncthreads();
  fft_smem<L, 1, NT, false>(sm, twL);
  for (int m = threadIdx.x; m < L; m += NT) sm[fpad(m)] = cmul(sm[fpad(m)], __ldg(hhat + m));
  __syncthreads();
  fft_smem<L, 1, NT, true>(sm, twL);
  for (int k = threadIdx.x; k < n; k += NT) {
    float2 c = __ldg(w + k);
    if (INV) c.y = -c.y;
    out[(int64_t)row * ldo + k] = cmul(sm[fpad(k)], c);
  }
}

template <int L, bool INV, bool REALPAIR>
cudaError_t any_dft_launch(int rows, const float2* in, int64_t ldi, const float* re, int64_t rs, int64_t es,
                           int nreal, const Chirp& c, float2* out, int64_t ldo, const int32_t* g0, const int32_t* g1,
                           cudaStream_t st) {
  constexpr size_t SM = sizeof(float2) * fft_padded_len(L);
  static DeviceOnce once;
  const cudaError_t a = once([] {
    return cudaFuncSetAttribute((const void*)any_dft_kernel<L, INV, REALPAIR>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM);
  });
  if (a != cudaSuccess) return a;
  if (rows <= 0) return cudaSuccess;
  any_dft_kernel<L, INV, REALPAIR><<<rows, fft_threads(L), SM, st>>>(in, ldi, re, rs, es, nreal, c.n, c.w,
                                                                     INV ? c.hi : c.hf, c.twL, out, ldo, g0, g1);
  return cudaGetLastError();
}

template <bool INV, bool REALPAIR>
cudaError_t any_dft_len(int rows, const float2* in, int64_t ldi, const float* re, int64_t rs, int64_t es, int nreal,
                        const Chirp& c, float2* out, int64_t ldo, const int32_t* g0, const int32_t* g1,
                        cudaStream_t st) {
  switch (c.L) {
    case 256: return any_dft_launch<256, INV, REALPAIR>(rows, in, ldi, re, rs, es, nreal, c, out, ldo, g0, g1, st);
    case 512: return any_dft_launch<512, INV, REALPAIR>(rows, in, ldi, re, rs, es, nreal, c, out, ldo, g0, g1, st);
    case 1024: return any_dft_launch<1024, INV, REALPAIR>(rows, in, ldi, re, rs, es, nreal, c, out, ldo, g0, g1, st);
    case 2048: return any_dft_launch<2048, INV, REALPAIR>(rows, in, ldi, re, rs, es, nreal, c, out, ldo, g0, g1, st);
    case 4096: return any_dft_launch<4096, INV, REALPAIR>(rows, in, ldi, re, rs, es, nreal, c, out, ldo, g0, g1, st);
    case 8192: return any_dft_launch<8192, INV, REALPAIR>(rows, in, ldi, re, rs, es, nreal, c, out, ldo, g0, g1, st);
    default: return cudaErrorInvalidValue;
  }
}

// rows DFTs of length n (complex rows of in, or pairs of real vectors of re: see any_dft_kernel)
cudaError_t any_dft(bool inv, bool realpair, int rows, const float2* in, int64_t ldi, const float* re, int64_t rs,
                    int64_t es, int nreal, const Chirp& c, float2* out, int64_t ldo, cudaStream_t st,
                    const int32_t* g0 = nullptr, const int32_t* g1 = nullptr) {
  AMM_TRACE_W("any_dft", st, 0.0, (double)rows * c.n * 16, nullptr);
  if (inv)
    return realpair ? any_dft_len<true, true>(rows, in, ldi, re, rs, es, nreal, c, out, ldo, g0, g1, st)
                    : any_dft_len<true, false>(rows, in, ldi, re, rs, es, nreal, c, out, ldo, g0, g1, st);
  return realpair ? any_dft_len<false, true>(rows, in, ldi, re, rs, es, nreal, c, out, ldo, g0, g1, st)
                  : any_dft_len<false, false>(rows, in, ldi, re, rs, es, nreal, c, out, ldo, g0, g1, st);
}

// ============================================================================ step kernels
template <typename T> __device__ __forceinline__ float any_ld(const T* p);
template <> __device__ __forceinline__ float any_ld<float>(const float* p) { return __ldg(p); }
template <> __device__ __forceinline__ float any_ld<__nv_bfloat16>(const __nv_bfloat16* p) {
  return __bfloat162float(*p);
}

// Cycle layout (Alg. 7), cycle-major: C[j][l] = A((l + j) mod n, l).  CTA: 32 cycles x 64 rows of A;
// row r of A holds cycles j at the contiguous (wrapping) columns (r - j) mod n, so the reads go
// along rows and the writes along cycles, through a shared tile.
template <typename T>
__global__ void __launch_bounds__(256) any_gather_cycles_kernel(const T* __restrict__ A, int64_t lda, int n,
                                                                float* __restrict__ C) {
  __shared__ float tile[64][33];
  const int j0 = blockIdx.x * 32, r0 = blockIdx.y * 64;
  for (int e = threadIdx.x; e < 64 * 32; e += 256) {
    const int rr = e >> 5, jj = e & 31, r = r0 + rr, j = j0 + jj;
    float v = 0.f;
    if (r < n && j < n) {
      const int c = r - j < 0 ? r - j + n : r - j;
      v = any_ld<T>(A + (int64_t)r * lda + c);
    }
    tile[rr][jj] = v;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 32 * 64; e += 256) {
    const int jj = e >> 6, rr = e & 63, r = r0 + rr, j = j0 + jj;
    if (r < n && j < n) {
      const int l = r - j < 0 ? r - j + n : r - j;
      C[(int64_t)j * n + l] = tile[rr][jj];
    }
  }
}

// Two real spectra from each packed one: Z[q] = F(x_2q + i x_2q+1) gives, for k <= n/2,
// out[k][2q] = sc (Z(k) + conj Z(-k)) / 2 and out[k][2q + 1] = sc (Z(k) - conj Z(-k)) / 2i
// (out row length ldo >= nvec).  kpart (optional): kpart[b][k] = sum of |out[k][v]|^2 over the
// vectors v of block b (8 vectors).  Thread per (k, block).
__global__ void __launch_bounds__(256) any_split_kernel(const float2* __restrict__ Z, int n, int nvec, float sc,
                                                        float2* __restrict__ out, int64_t ldo,
                                                        float* __restrict__ kpart, const int32_t* __restrict__ gate0,
                                                        const int32_t* __restrict__ gate1) {
  if (gate0 != nullptr && (*gate0 == 0 || *gate1 == 0)) return;
  const int kh = n / 2 + 1;
  const int k = blockIdx.x * 256 + threadIdx.x, b = blockIdx.y;
  if (k >= kh) return;
  const int kr = k == 0 ? 0 : n - k;
  const float h = 0.5f * sc;
  float p = 0.f;
  for (int v = 8 * b; v < min(nvec, 8 * b + 8); v += 2) {
    const float2* z = Z + (int64_t)(v >> 1) * n;
    const float2 a = __ldg(z + k), c = cconj(__ldg(z + kr));
    const float2 x0 = cscale(cadd(a, c), h);
    const float2 d = csub(a, c);
    const float2 x1 = make_float2(h * d.y, -h * d.x);
    out[(int64_t)k * ldo + v] = x0;
    p += x0.x * x0.x + x0.y * x0.y;
    if (v + 1 < nvec) {
      out[(int64_t)k * ldo + v + 1] = x1;
      p += x1.x * x1.x + x1.y * x1.y;
    }
  }
  if (kpart) kpart[(int64_t)b * kh + k] = p;
}

// Packed signals of the inverse cycle transform: Z[q][k] = g'_k (r_{2q,k} + i r_{2q+1,k}), k < n,
// from the half spectrum R (row k > n/2 is conj of row n - k) with g'_k by mode (0: 1 - g_k,
// 1: -i g_k, 2: g_k, 3: +i g_k).  Rows with a zero coefficient are not read.  CTA: 32 k x 32 q
// through a shared tile (reads along spectrum rows, writes along signals).
__global__ void __launch_bounds__(256) any_cycle_pairs_kernel(const float2* __restrict__ R,
                                                              const float* __restrict__ g, int mode, int n,
                                                              float2* __restrict__ Z) {
  __shared__ float2 tile[32][33];
  const int k0 = blockIdx.x * 32, q0 = blockIdx.y * 32, npair = (n + 1) / 2;
  for (int e = threadIdx.x; e < 32 * 32; e += 256) {
    const int kk = e >> 5, qq = e & 31, k = k0 + kk, q = q0 + qq;
    float2 z = make_float2(0.f, 0.f);
    if (k < n && q < npair) {
      const float gk = __ldg(g + k);
      const float c = mode == 0 ? 1.f - gk : gk;
      if (c != 0.f) {
        const bool mir = k > n / 2;
        const float2* row = R + (int64_t)(mir ? n - k : k) * n;
        float2 ra = __ldg(row + 2 * q);
        float2 rb = 2 * q + 1 < n ? __ldg(row + 2 * q + 1) : make_float2(0.f, 0.f);
        if (mir) {
          ra = cconj(ra);
          rb = cconj(rb);
        }
        z = make_float2(ra.x - rb.y, ra.y + rb.x);
        switch (mode) {
          case 0: case 2: z = cscale(z, c); break;
          case 1: z = make_float2(c * z.y, -c * z.x); break;
          default: z = make_float2(-c * z.y, c * z.x); break;
        }
      }
    }
    tile[kk][qq] = z;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 32 * 32; e += 256) {
    const int qq = e >> 5, kk = e & 31, k = k0 + kk, q = q0 + qq;
    if (k < n && q < npair) Z[(int64_t)q * n + k] = tile[kk][qq];
  }
}

// Inverse of the cycle layout for packed results: X((c + j) mod n, c) (+)= Lambda_j(c), where
// Lambda_2q + i Lambda_2q+1 = Z[q].  CTA: 32 cycles x 64 rows of X through a shared tile (reads
// along cycles, writes along rows of X).  Writes nothing when the residual's gates say so: odd
// modes with *dcount == 0 (no unpaired component), any mode with *dcount2 == 0.
__global__ void __launch_bounds__(256) any_cycle_scatter_kernel(const float2* __restrict__ Z, int n,
                                                                float* __restrict__ X, int64_t ldx, int accumulate,
                                                                int mode, const int32_t* __restrict__ dcount,
                                                                const int32_t* __restrict__ dcount2) {
  if ((mode & 1) && dcount != nullptr && *dcount == 0) return;
  if (dcount2 != nullptr && *dcount2 == 0) return;
  __shared__ float tile[64][33];
  const int j0 = blockIdx.x * 32, r0 = blockIdx.y * 64;
  for (int e = threadIdx.x; e < 32 * 64; e += 256) {
    const int jj = e >> 6, rr = e & 63, r = r0 + rr, j = j0 + jj;
    float v = 0.f;
    if (r < n && j < n) {
      const int l = r - j < 0 ? r - j + n : r - j;
      const float2 z = __ldg(Z + (int64_t)(j >> 1) * n + l);
      v = (j & 1) ? z.y : z.x;
    }
    tile[rr][jj] = v;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 64 * 32; e += 256) {
    const int rr = e >> 5, jj = e & 31, r = r0 + rr, j = j0 + jj;
    if (r < n && j < n) {
      const int c = r - j < 0 ? r - j + n : r - j;
      float* x = X + (int64_t)r * ldx + c;
      *x = accumulate ? *x + tile[rr][jj] : tile[rr][jj];
    }
  }
}

// G[u][j] = row t_u of the half spectrum R (conj of row n - t for t > n/2), u < count; zero rows
// beyond count
__global__ void __launch_bounds__(256) any_gather_rows_kernel(const float2* __restrict__ R, int n,
                                                              const int32_t* __restrict__ list,
                                                              const int32_t* __restrict__ count,
                                                              float2* __restrict__ G) {
  const int u = blockIdx.y;
  const int j = blockIdx.x * 256 + threadIdx.x;
  if (j >= n) return;
  float2 v = make_float2(0.f, 0.f);
  if (u < *count) {
    const int t = __ldg(list + u);
    const bool mir = t > n / 2;
    v = __ldg(R + (int64_t)(mir ? n - t : t) * n + j);
    if (mir) v = cconj(v);
  }
  G[(int64_t)u * n + j] = v;
}

// L[u][p] = c_u Y[u][p] (imag: -i c_u Y[u][p]) for u < count
__global__ void __launch_bounds__(256) any_scale_rows_kernel(const float2* __restrict__ Y, int n,
                                                             const float* __restrict__ coef,
                                                             const int32_t* __restrict__ count, int imag,
                                                             float2* __restrict__ L) {
  const int u = blockIdx.y;
  const int p = blockIdx.x * 256 + threadIdx.x;
  if (p >= n || u >= *count) return;
  const float c = __ldg(coef + u);
  const float2 y = __ldg(Y + (int64_t)u * n + p);
  L[(int64_t)u * n + p] = imag ? make_float2(c * y.y, -c * y.x) : cscale(y, c);
}

// Spectral MAC of the apply (Alg. 3): Y[s][p] = sum_u Lc[u][i_u(p)] Xh[s][(p - t_u) mod n]
// with i_u(p) = (t_u - p) mod n (rev) or p.  CTA per packed signal s, its spectrum staged in
// shared memory.
__global__ void __launch_bounds__(256) any_mac_kernel(const float2* __restrict__ Xh, int n,
                                                      const int32_t* __restrict__ list,
                                                      const float2* __restrict__ Lc,
                                                      const int32_t* __restrict__ count, int rev,
                                                      float2* __restrict__ Y) {
  extern __shared__ float2 sx[];
  const int s = blockIdx.x;
  for (int p = threadIdx.x; p < n; p += 256) sx[p] = __ldg(Xh + (int64_t)s * n + p);
  __syncthreads();
  const int nu = *count;
  for (int p = threadIdx.x; p < n; p += 256) {
    float2 acc = make_float2(0.f, 0.f);
    for (int u = 0; u < nu; ++u) {
      const int t = __ldg(list + u);
      int q = p - t;
      if (q < 0) q += n;
      int i = t - p;
      if (i < 0) i += n;
      cmac(acc, __ldg(Lc + (int64_t)u * n + (rev ? i : p)), sx[q]);
    }
    Y[(int64_t)s * n + p] = acc;
  }
}

// Unpacking of the applied signals, Z[s] = x_2s + i x_2s+1 (times n), into the output: rows
// (row = true: out[v][l]) or columns (out[l][v], through a shared tile of 32 signals x 32 l);
// scaled by 1/n, overwriting or adding; a gated-off launch writes nothing.
__global__ void __launch_bounds__(256) any_unpack_kernel(const float2* __restrict__ Z, int n, int nvec, int row,
                                                         float* __restrict__ out, int64_t ldo, int accumulate,
                                                         const int32_t* __restrict__ gate0,
                                                         const int32_t* __restrict__ gate1) {
  if (gate0 != nullptr && (*gate0 == 0 || *gate1 == 0)) return;
  __shared__ float2 tile[32][33];
  const int l0 = blockIdx.x * 32, s0 = blockIdx.y * 32, npair = (nvec + 1) / 2;
  const float sc = 1.f / (float)n;
  auto put = [&](float* o, float v) { *o = accumulate ? *o + v : v; };
  if (row) {
    for (int e = threadIdx.x; e < 32 * 32; e += 256) {
      const int ss = e >> 5, ll = e & 31, s = s0 + ss, l = l0 + ll;
      if (s < npair && l < n) {
        const float2 z = __ldg(Z + (int64_t)s * n + l);
        put(out + (int64_t)(2 * s) * ldo + l, sc * z.x);
        if (2 * s + 1 < nvec) put(out + (int64_t)(2 * s + 1) * ldo + l, sc * z.y);
      }
    }
    return;
  }
  for (int e = threadIdx.x; e < 32 * 32; e += 256) {
    const int ss = e >> 5, ll = e & 31, s = s0 + ss, l = l0 + ll;
    tile[ss][ll] = (s < npair && l < n) ? __ldg(Z + (int64_t)s * n + l) : make_float2(0.f, 0.f);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 32 * 32; e += 256) {
    const int ll = e >> 5, ss = e & 31, s = s0 + ss, l = l0 + ll;
    if (s < npair && l < n) {
      const float2 z = tile[ss][ll];
      put(out + (int64_t)l * ldo + 2 * s, sc * z.x);
      if (2 * s + 1 < nvec) put(out + (int64_t)l * ldo + 2 * s + 1, sc * z.y);
    }
  }
}

// SDDMM on half spectra at length n (the backward, reading R10): K[u][p] = sum_m Xh(p, m)
// Yh((t_u - p) mod n, m) for listed t_u <= n/2, p < n; warp per p, lanes over m.
__global__ void __launch_bounds__(256) any_sddmm_kernel(const float2* __restrict__ Xh, const float2* __restrict__ Yh,
                                                        int n, const int32_t* __restrict__ list,
                                                        const int32_t* __restrict__ count, float2* __restrict__ K,
                                                        const int32_t* __restrict__ gate0,
                                                        const int32_t* __restrict__ gate1) {
  if (gate0 != nullptr && (*gate0 == 0 || *gate1 == 0)) return;
  const int u = blockIdx.x;
  if (u >= *count) return;
  const int t = __ldg(list + u);
  if (t > n / 2) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int p = blockIdx.y * 8 + warp;
  if (p >= n) return;
  int q = t - p;
  if (q < 0) q += n;
  const bool xm = p > n / 2, ym = q > n / 2;
  const float2* xr = Xh + (int64_t)(xm ? n - p : p) * n;
  const float2* yr = Yh + (int64_t)(ym ? n - q : q) * n;
  float2 acc = make_float2(0.f, 0.f);
  for (int m = lane; m < n; m += 32) {
    float2 x = __ldg(xr + m), y = __ldg(yr + m);
    if (xm) x.y = -x.y;
    if (ym) y.y = -y.y;
    cmac(acc, x, y);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
  }
  if (lane == 0) K[(int64_t)u * n + p] = acc;
}

// Component spectra from the inverse DFTs of the K rows: RX[t_u][j] = Kt[u][j] / n^2 for listed
// t_u <= n/2
__global__ void __launch_bounds__(256) any_rho_out_kernel(const float2* __restrict__ Kt, int n,
                                                          const int32_t* __restrict__ list,
                                                          const int32_t* __restrict__ count,
                                                          float2* __restrict__ RX, const int32_t* __restrict__ gate0,
                                                          const int32_t* __restrict__ gate1) {
  if (gate0 != nullptr && (*gate0 == 0 || *gate1 == 0)) return;
  const int u = blockIdx.y;
  const int j = blockIdx.x * 256 + threadIdx.x;
  if (j >= n || u >= *count) return;
  const int t = __ldg(list + u);
  if (t > n / 2) return;
  const float sc = 1.f / ((float)n * (float)n);
  RX[(int64_t)t * n + j] = cscale(__ldg(Kt + (int64_t)u * n + j), sc);
}

// Scratch buffers of one call, released at the end (stream-ordered).
struct AnyScratch {
  cudaStream_t st;
  std::vector<void*> bufs;
  cudaError_t e = cudaSuccess;
  explicit AnyScratch(cudaStream_t s) : st(s) {}
  template <typename T>
  T* get(size_t count) {
    void* q = nullptr;
    if (e == cudaSuccess) e = dev_alloc(&q, sizeof(T) * count, st);
    if (q) bufs.push_back(q);
    return (T*)q;
  }
  ~AnyScratch() {
    for (void* q : bufs) dev_free(q, st);
  }
};

unsigned cdiv(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }

}  // namespace

// ============================================================================ the steps at any n
// Each mirrors the fixed-length step of the same name (circulant.cu, cd_backward.cu) and writes the
// same outputs in the same layouts.

cudaError_t cd_spectrum_any(int n, const void* A, int64_t lda, bool bf16, float2* R, float* kpart, cudaStream_t st) {
  Chirp c;
  cudaError_t e = chirp_tables(n, st, &c);
  if (e != cudaSuccess) return e;
  const int npair = (n + 1) / 2, kh = n / 2 + 1;
  AnyScratch s(st);
  float* C = s.get<float>((size_t)n * n);
  float2* Z = s.get<float2>((size_t)npair * n);
  if (s.e != cudaSuccess) return s.e;
  const dim3 gg(cdiv(n, 32), cdiv(n, 64));
  if (bf16) any_gather_cycles_kernel<__nv_bfloat16><<<gg, 256, 0, st>>>((const __nv_bfloat16*)A, lda, n, C);
  else any_gather_cycles_kernel<float><<<gg, 256, 0, st>>>((const float*)A, lda, n, C);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = any_dft(false, true, npair, nullptr, 0, C, n, 1, n, c, Z, n, st);
  if (e == cudaSuccess) {
    any_split_kernel<<<dim3(cdiv(kh, 256), cdiv(n, 8)), 256, 0, st>>>(Z, n, n, 1.f / (float)n, R, n, kpart, nullptr,
                                                                      nullptr);
    e = cudaGetLastError();
  }
  return e;
}

cudaError_t cd_eigen_any(int n, const float2* R, const int32_t* list, const float* coef, const int32_t* count,
                         int cap, int imag_coef, float2* L, cudaStream_t st) {
  if (cap <= 0) return cudaSuccess;
  Chirp c;
  cudaError_t e = chirp_tables(n, st, &c);
  if (e != cudaSuccess) return e;
  AnyScratch s(st);
  float2* G = s.get<float2>((size_t)cap * n);
  float2* Y = s.get<float2>((size_t)cap * n);
  if (s.e != cudaSuccess) return s.e;
  any_gather_rows_kernel<<<dim3(cdiv(n, 256), cap), 256, 0, st>>>(R, n, list, count, G);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = any_dft(false, false, cap, G, n, nullptr, 0, 0, 0, c, Y, n, st);
  if (e == cudaSuccess) {
    any_scale_rows_kernel<<<dim3(cdiv(n, 256), cap), 256, 0, st>>>(Y, n, coef, count, imag_coef, L);
    e = cudaGetLastError();
  }
  return e;
}

cudaError_t cd_residual_any(int n, const float2* R, const float* g, int mode, const int32_t* dcount,
                            const int32_t* dcount2, float* X, int64_t ldx, int accumulate, cudaStream_t st) {
  Chirp c;
  cudaError_t e = chirp_tables(n, st, &c);
  if (e != cudaSuccess) return e;
  const int npair = (n + 1) / 2;
  AnyScratch s(st);
  float2* Z1 = s.get<float2>((size_t)npair * n);
  float2* Z2 = s.get<float2>((size_t)npair * n);
  if (s.e != cudaSuccess) return s.e;
  any_cycle_pairs_kernel<<<dim3(cdiv(n, 32), cdiv(npair, 32)), 256, 0, st>>>(R, g, mode, n, Z1);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = any_dft(true, false, npair, Z1, n, nullptr, 0, 0, 0, c, Z2, n, st);
  if (e == cudaSuccess) {
    any_cycle_scatter_kernel<<<dim3(cdiv(n, 32), cdiv(n, 64)), 256, 0, st>>>(Z2, n, X, ldx, accumulate, mode, dcount,
                                                                          dcount2);
    e = cudaGetLastError();
  }
  return e;
}

cudaError_t cd_apply_any(int n, bool row, const void* X, int64_t ldx, bool bf16, int64_t nvec, const int32_t* list,
                         const float2* Lc, const int32_t* count, const int32_t* gate0, const int32_t* gate1,
                         float* out, int64_t ldo, int accumulate, int rev, cudaStream_t st) {
  if (nvec <= 0) return cudaSuccess;
  Chirp c;
  cudaError_t e = chirp_tables(n, st, &c);
  if (e != cudaSuccess) return e;
  const int npair = (int)((nvec + 1) / 2);
  AnyScratch s(st);
  const float* Xf = (const float*)X;
  int64_t ldf = ldx;
  if (bf16) {  // widened once; the transforms run in FP32 as on the fixed-length path
    const int64_t rows = row ? nvec : n, cols = row ? n : nvec;
    float* w = s.get<float>((size_t)(rows * cols));
    if (s.e != cudaSuccess) return s.e;
    if ((e = widen_bf16(X, rows, cols, ldx, w, cols, st)) != cudaSuccess) return e;
    Xf = w;
    ldf = cols;
  }
  float2* Xh = s.get<float2>((size_t)npair * n);
  float2* Y = s.get<float2>((size_t)npair * n);
  if (s.e != cudaSuccess) return s.e;
  e = any_dft(false, true, npair, nullptr, 0, Xf, row ? ldf : 1, row ? 1 : ldf, (int)nvec, c, Xh, n, st);
  if (e == cudaSuccess) {
    any_mac_kernel<<<npair, 256, sizeof(float2) * (size_t)n, st>>>(Xh, n, list, Lc, count, rev < 0 ? (int)row : rev,
                                                                  Y);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = any_dft(true, false, npair, Y, n, nullptr, 0, 0, 0, c, Xh, n, st);
  if (e == cudaSuccess) {
    any_unpack_kernel<<<dim3(cdiv(n, 32), cdiv(npair, 32)), 256, 0, st>>>(Xh, n, (int)nvec, row ? 1 : 0, out, ldo,
                                                                          accumulate, gate0, gate1);
    e = cudaGetLastError();
  }
  return e;
}

cudaError_t bw_spectrum_any(int n, bool row, const float* X, int64_t ldx, float2* Xh, const int32_t* gate0,
                            const int32_t* gate1, cudaStream_t st) {
  Chirp c;
  cudaError_t e = chirp_tables(n, st, &c);
  if (e != cudaSuccess) return e;
  const int npair = (n + 1) / 2, kh = n / 2 + 1;
  AnyScratch s(st);
  float2* Z = s.get<float2>((size_t)npair * n);
  if (s.e != cudaSuccess) return s.e;
  e = any_dft(false, true, npair, nullptr, 0, X, row ? ldx : 1, row ? 1 : ldx, n, c, Z, n, st, gate0, gate1);
  if (e == cudaSuccess) {
    any_split_kernel<<<dim3(cdiv(kh, 256), cdiv(n, 8)), 256, 0, st>>>(Z, n, n, 1.f, Xh, n, nullptr, gate0, gate1);
    e = cudaGetLastError();
  }
  return e;
}

cudaError_t cd_sddmm_any(int n, const float2* Xh, const float2* Yh, const int32_t* list, const int32_t* count,
                         int cap, float2* K, const int32_t* gate0, const int32_t* gate1, cudaStream_t st) {
  if (cap <= 0) return cudaSuccess;
  any_sddmm_kernel<<<dim3(cap, cdiv(n, 8)), 256, 0, st>>>(Xh, Yh, n, list, count, K, gate0, gate1);
  return cudaGetLastError();
}

cudaError_t cd_rho_any(int n, const float2* K, const int32_t* list, const int32_t* count, int cap, float2* RX,
                       const int32_t* gate0, const int32_t* gate1, cudaStream_t st) {
  if (cap <= 0) return cudaSuccess;
  Chirp c;
  cudaError_t e = chirp_tables(n, st, &c);
  if (e != cudaSuccess) return e;
  AnyScratch s(st);
  float2* Kt = s.get<float2>((size_t)cap * n);
  if (s.e != cudaSuccess) return s.e;
  e = any_dft(true, false, cap, K, n, nullptr, 0, 0, 0, c, Kt, n, st, gate0, gate1);
  if (e == cudaSuccess) {
    any_rho_out_kernel<<<dim3(cdiv(n, 256), cap), 256, 0, st>>>(Kt, n, list, count, RX, gate0, gate1);
    e = cudaGetLastError();
  }
  return e;
}

}  // namespace amm
