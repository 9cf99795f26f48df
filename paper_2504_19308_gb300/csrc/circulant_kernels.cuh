// N-templated kernels of the circulant decomposition and product (cycle spectrum, eigen-spectra,
// inverse cycle transform, spectral apply) and their launch configuration.  Included by
// circulant.cu (N = 2^a) and circulant_r3.cu (N = 3 * 2^a), which instantiate them for their
// lengths in separate translation units.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include "api_internal.h"
#include "common.cuh"
#include "fft.cuh"
#include "kernels.h"
#include "trace.h"
#include "tune.cuh"

namespace amm {

template <typename T> AMM_DEV float ld_as_float(const T* p);
template <> AMM_DEV float ld_as_float<float>(const float* p) { return __ldg(p); }
template <> AMM_DEV float ld_as_float<__nv_bfloat16>(const __nv_bfloat16* p) { return __bfloat162float(*p); }

// outputs per store batch of a thread: the largest divisor of its per-thread count up to 8
__host__ __device__ constexpr int store_batch(int it) { return it % 8 == 0 ? 8 : it % 6 == 0 ? 6 : it % 4 == 0 ? 4 : it % 3 == 0 ? 3 : it % 2 == 0 ? 2 : 1; }

// ============================================================================ K1: cycle spectrum
// CTA b handles cycles j0 = b*J .. j0+J-1 (J = 2S), packed in pairs as complex signals.
// Reads row r of A at columns (r - j) mod n for the J cycles (a contiguous, wrapping segment).
template <int N, int S, int NT, typename T>
__global__ void __launch_bounds__(NT) cd_spectrum_kernel(const T* __restrict__ A, int64_t lda,
                                                         const float2* __restrict__ tw,
                                                         float2* __restrict__ R, float* __restrict__ kpart) {
  extern __shared__ float2 smem[];
  constexpr int J = 2 * S;
  constexpr int LD = fft_padded_len(N);
  const int j0 = blockIdx.x * J;
  float* fs = reinterpret_cast<float*>(smem);
  // gather: element (r, q): column c = (r - j0 - (J-1) + q) mod n holds cycle m = J-1-q at l = c.
  // With J = 8 a warp covers four rows; they are taken as r, r + 1, r + 8, r + 9 (a permutation of
  // each 16 consecutive rows), whose shared-memory stores fall on disjoint banks.
  static_assert((N * J) % NT == 0, "whole iterations");
#pragma unroll 16
  for (int it = 0; it < N * J / NT; ++it) {  // unrolled: several loads in flight per thread
    const int e = threadIdx.x + it * NT;
    const int r0 = e / J, q = e % J;
    const int r = (J == 8 && N % 16 == 0) ? ((r0 & ~15) | (((r0 >> 2) & 3) << 1) | (r0 & 1) | (((r0 >> 1) & 1) << 3))
                                          : r0;
    const int c = wrapN<N>(r - j0 - (J - 1) + q);
    const int m = J - 1 - q;
    const float v = ld_as_float<T>(A + (int64_t)r * lda + c);
    fs[2 * ((m >> 1) * LD + fpad(c)) + (m & 1)] = v;
  }
  __syncthreads();
  fft_smem<N, S, NT, false>(smem, tw);
  // separate the two real spectra of each packed signal, scale by 1/n, store k = 0..n/2
  constexpr float inv_n = 1.0f / (float)N;
  constexpr int KH = N / 2 + 1;
  constexpr int ITER = (KH * J + NT - 1) / NT;  // whole warps iterate together (shuffles below)
  for (int it = 0; it < ITER; ++it) {
    const int e = threadIdx.x + it * NT;
    const bool valid = e < KH * J;
    const int k = e / J, m = e % J;
    float p = 0.f;
    if (valid) {
      const float2* z = smem + (m >> 1) * LD;
      const float2 a = z[fpad(k)];
      const float2 b = cconj(z[fpad(wrapN<N>(N - k))]);
      float2 x;
      if ((m & 1) == 0) x = cscale(cadd(a, b), 0.5f * inv_n);  // (Z + conj Z(-k)) / 2
      else { float2 d = csub(a, b); x = make_float2(0.5f * inv_n * d.y, -0.5f * inv_n * d.x); }  // (Z - conj Z(-k)) / 2i
      R[(int64_t)k * N + j0 + m] = x;
      p = x.x * x.x + x.y * x.y;
    }
    // J consecutive lanes share k (J divides 32): reduce to the first of them
    constexpr unsigned MASK = (NT >= 32) ? 0xffffffffu : ((1u << NT) - 1u);  // CTAs of 16 threads at n = 16
#pragma unroll
    for (int o = J / 2; o > 0; o >>= 1) p += __shfl_xor_sync(MASK, p, o, J);
    if (valid && m == 0) kpart[(int64_t)blockIdx.x * KH + k] = p;
  }
}

// ============================================================================ K3: eigen-spectra
// CTA u: L = F R_A[t_u] for t_u in the union (coefficient w) or in the unpaired set
// (coefficient -i v).  Writes coef * L_t.
template <int N, int NT>
__global__ void __launch_bounds__(NT) cd_eigen_kernel(const float2* __restrict__ R, const float2* __restrict__ tw,
                                                      const int32_t* __restrict__ list, const float* __restrict__ coef,
                                                      const int32_t* __restrict__ count, int imag_coef,
                                                      float2* __restrict__ L) {
  extern __shared__ float2 smem[];
  const int u = blockIdx.x;
  if (u >= *count) return;
  const int t = list[u];
  const bool mir = t > N / 2;
  const int tr = mir ? N - t : t;
  for (int j = threadIdx.x; j < N; j += NT) {
    float2 v = R[(int64_t)tr * N + j];
    smem[fpad(j)] = mir ? cconj(v) : v;
  }
  __syncthreads();
  fft_smem<N, 1, NT, false>(smem, tw);
  const float c = coef[u];
  for (int p = threadIdx.x; p < N; p += NT) {
    float2 l = smem[fpad(p)];
    L[(int64_t)u * N + p] = imag_coef ? make_float2(c * l.y, -c * l.x) /* -i c l */ : cscale(l, c);
  }
}

// ============================================================================ K6: dense residual
// For cycles j0..j0+J-1: Lambda_j(c) = sum_k g_k r_{j,k} omega^{k c}, with g_k = 1 - w_k (mode 0,
// gfull = w, giving dB_w) or g_k = -i v_k (mode 1, gfull = v, giving V = Im B~_S).
// Writes X((c+j) mod n, c).
// Modes: 0 coefficient 1 - g, 1 coefficient -i g, 2 coefficient g, 3 coefficient +i g (the last two
// serve the backward); accumulate adds into X (leading dimension ldx).  Modes 1 and 3 return early
// when *dcount is zero (no unpaired component).
template <int N, int S, int NT>
__global__ void __launch_bounds__(NT) cd_residual_kernel(const float2* __restrict__ R, const float2* __restrict__ tw,
                                                         const float* __restrict__ gfull, int mode,
                                                         const int32_t* __restrict__ dcount,
                                                         const int32_t* __restrict__ dcount2,
                                                         float* __restrict__ X, int64_t ldx, int accumulate) {
  extern __shared__ float2 smem[];
  if ((mode & 1) && dcount != nullptr && *dcount == 0) return;
  if (dcount2 != nullptr && *dcount2 == 0) return;
  constexpr int J = 2 * S;
  constexpr int LD = fft_padded_len(N);
  const int j0 = blockIdx.x * J;
  // the coefficients of all n rows, staged once: the row loads below then wait on shared memory
  // only, not on a global load of their coefficient
  float* coef = reinterpret_cast<float*>(smem + S * LD);
  for (int k = threadIdx.x; k < N; k += NT) {
    const float g = __ldg(gfull + k);
    coef[k] = mode == 0 ? 1.f - g : g;
  }
  __syncthreads();
  // packed signal s: Z(k) = g_k (r_{j0+2s,k} + i r_{j0+2s+1,k}), k in [0, n)
#pragma unroll 16
  for (int it = 0; it < N * S / NT; ++it) {
    const int e = threadIdx.x + it * NT;
    const int k = e / S, s = e % S;
    const float c = coef[k];
    float2 z = make_float2(0.f, 0.f);
    if (c != 0.f) {  // rows with a zero coefficient are neither read nor required to be set
      const bool mir = k > N / 2;
      const int kr = mir ? N - k : k;
      const float4 rr = *reinterpret_cast<const float4*>(R + (int64_t)kr * N + j0 + 2 * s);
      float2 r1 = make_float2(rr.x, rr.y), r2 = make_float2(rr.z, rr.w);
      if (mir) { r1 = cconj(r1); r2 = cconj(r2); }
      z = make_float2(r1.x - r2.y, r1.y + r2.x);
      switch (mode) {
        case 0: z = cscale(z, c); break;                         // (1 - w_k)
        case 1: z = make_float2(c * z.y, -c * z.x); break;       // -i v_k
        case 2: z = cscale(z, c); break;                         // w_k
        default: z = make_float2(-c * z.y, c * z.x); break;      // +i v_k
      }
    }
    smem[s * LD + fpad(k)] = z;
  }
  __syncthreads();
  fft_smem<N, S, NT, true>(smem, tw);
  const float* fs = reinterpret_cast<const float*>(smem);
  constexpr int IT = N * J / NT, B = store_batch(IT);  // B outputs per batch: loads all in flight
  static_assert(IT % B == 0, "whole batches");
  // element e of the output: row r = e / J, column c = (r - j0 - (J - 1) + q) mod n, q = e % J
  auto addr = [&](int e) { return (int64_t)(e / J) * ldx + wrapN<N>(e / J - j0 - (J - 1) + e % J); };
  auto value = [&](int e) {
    const int q = e % J, m = J - 1 - q;
    return fs[2 * ((m >> 1) * LD + fpad(wrapN<N>(e / J - j0 - (J - 1) + q))) + (m & 1)];
  };
  for (int i0 = 0; i0 < IT; i0 += B) {
    float v[B];
#pragma unroll
    for (int b = 0; b < B; ++b) v[b] = value(threadIdx.x + (i0 + b) * NT);
    if (accumulate) {
      float old[B];
#pragma unroll
      for (int b = 0; b < B; ++b) old[b] = X[addr(threadIdx.x + (i0 + b) * NT)];
#pragma unroll
      for (int b = 0; b < B; ++b) v[b] += old[b];
    }
#pragma unroll
    for (int b = 0; b < B; ++b) X[addr(threadIdx.x + (i0 + b) * NT)] = v[b];
  }
}

// ============================================================================ K5: spectral apply
// COL: out(:, c0..c0+2S) (+)= (sum_u Lc_u-weighted) applied to X's columns (Alg. 3, zeroth-order term).
// ROW: out(r0..r0+2S, :) (+)= rows of X times (sum_s c_s R_s D^s).
// Packed pairs of real columns/rows form complex signals; the output pair comes out of one
// inverse FFT as (real, imag).  Coefficients Lc[u][p] = c_u L_{t_u}(p) (c conjugate-symmetric).
// REV selects the coefficient index: L_u((t_u - p) mod n) (REV) or L_u(p).  The forward product
// uses REV = ROW; the backward's adjoint applies use the other pairing.
template <int N, int S, int NT, bool ROW, bool REV, typename T>
__global__ void __launch_bounds__(NT) cd_apply_kernel(const T* __restrict__ X, int64_t ldx,
                                                      const float2* __restrict__ tw,
                                                      const int32_t* __restrict__ list, const float2* __restrict__ Lc,
                                                      const int32_t* __restrict__ count,
                                                      const int32_t* __restrict__ gate0,
                                                      const int32_t* __restrict__ gate1, float* __restrict__ out,
                                                      int64_t ldo, int accumulate, int nvec) {
  extern __shared__ float2 smem[];
  if (gate0 != nullptr && (*gate0 == 0 || *gate1 == 0)) return;
  constexpr int LD = fft_padded_len(N);
  constexpr int PT = N / NT;  // output frequencies per thread
  static_assert(N % NT == 0, "NT must divide N");
  const int base = blockIdx.x * 2 * S;
  if (!ROW) {
#pragma unroll 8
    for (int it = 0; it < N * S / NT; ++it) {
      const int e = threadIdx.x + it * NT;
      const int l = e / S, s = e % S;
      const int v = base + 2 * s;
      const T* p = X + (int64_t)l * ldx + v;
      smem[s * LD + fpad(l)] = make_float2(v < nvec ? ld_as_float<T>(p) : 0.f, v + 1 < nvec ? ld_as_float<T>(p + 1) : 0.f);
    }
  } else {
#pragma unroll 8
    for (int it = 0; it < N * S / NT; ++it) {
      const int e = threadIdx.x + it * NT;
      const int s = e / N, l = e % N;
      const int v = base + 2 * s;
      const T* p = X + (int64_t)v * ldx + l;
      smem[s * LD + fpad(l)] = make_float2(v < nvec ? ld_as_float<T>(p) : 0.f, v + 1 < nvec ? ld_as_float<T>(p + ldx) : 0.f);
    }
  }
  __syncthreads();
  fft_smem<N, S, NT, false, true>(smem, tw);  // spectrum left unpadded: shifted reads below
  float2 acc[PT][S];
#pragma unroll
  for (int i = 0; i < PT; ++i)
#pragma unroll
    for (int s = 0; s < S; ++s) acc[i][s] = make_float2(0.f, 0.f);
  const int nu = *count;
  for (int u = 0; u < nu; ++u) {
    const int t = __ldg(list + u);
    const float2* lrow = Lc + (int64_t)u * N;
#pragma unroll
    for (int i = 0; i < PT; ++i) {
      const int p = threadIdx.x + i * NT;
      const float2 l = __ldg(lrow + (REV ? wrapN<N>(t - p) : p));
      const int q = wrapN<N>(p - t);
#pragma unroll
      for (int s = 0; s < S; ++s) cmac(acc[i][s], l, smem[s * LD + q]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < PT; ++i)
#pragma unroll
    for (int s = 0; s < S; ++s) smem[s * LD + fpad(threadIdx.x + i * NT)] = acc[i][s];
  __syncthreads();
  fft_smem<N, S, NT, true>(smem, tw);
  constexpr float inv_n = 1.0f / (float)N;
  if (!ROW) {
    const bool vec2 = ((ldo & 1) == 0) && ((reinterpret_cast<uintptr_t>(out) & 7) == 0);  // pairs as float2
    constexpr int IT = N * S / NT, B = store_batch(IT);  // B outputs per batch, loads in flight
    static_assert(IT % B == 0, "whole batches");
    for (int i0 = 0; i0 < IT; i0 += B) {
      float2 z[B];
      float* o[B];
      int v[B];
#pragma unroll
      for (int b = 0; b < B; ++b) {
        const int e = threadIdx.x + (i0 + b) * NT;
        const int l = e / S, s = e % S;
        v[b] = base + 2 * s;
        z[b] = cscale(smem[s * LD + fpad(l)], inv_n);
        o[b] = out + (int64_t)l * ldo + v[b];
      }
      if (accumulate) {
        float2 old[B];
#pragma unroll
        for (int b = 0; b < B; ++b) {
          if (v[b] + 1 < nvec && vec2) old[b] = *reinterpret_cast<const float2*>(o[b]);
          else old[b] = make_float2(v[b] < nvec ? o[b][0] : 0.f, v[b] + 1 < nvec ? o[b][1] : 0.f);
        }
#pragma unroll
        for (int b = 0; b < B; ++b) {
          z[b].x += old[b].x;
          z[b].y += old[b].y;
        }
      }
#pragma unroll
      for (int b = 0; b < B; ++b) {
        if (v[b] + 1 < nvec && vec2) {
          *reinterpret_cast<float2*>(o[b]) = z[b];
        } else {
          if (v[b] < nvec) o[b][0] = z[b].x;
          if (v[b] + 1 < nvec) o[b][1] = z[b].y;
        }
      }
    }
  } else {
    constexpr int IT = N * S / NT, B = store_batch(IT);  // B outputs per batch, loads in flight
    static_assert(IT % B == 0, "whole batches");
    for (int i0 = 0; i0 < IT; i0 += B) {
      float2 z[B];
      float* o0[B];
      int v[B];
#pragma unroll
      for (int b = 0; b < B; ++b) {
        const int e = threadIdx.x + (i0 + b) * NT;
        const int s = e / N, l = e % N;
        v[b] = base + 2 * s;
        z[b] = cscale(smem[s * LD + fpad(l)], inv_n);
        o0[b] = out + (int64_t)v[b] * ldo + l;
      }
      if (accumulate) {
        float a0[B], a1[B];
#pragma unroll
        for (int b = 0; b < B; ++b) {
          a0[b] = v[b] < nvec ? *o0[b] : 0.f;
          a1[b] = v[b] + 1 < nvec ? o0[b][ldo] : 0.f;
        }
#pragma unroll
        for (int b = 0; b < B; ++b) {
          z[b].x += a0[b];
          z[b].y += a1[b];
        }
      }
#pragma unroll
      for (int b = 0; b < B; ++b) {
        if (v[b] < nvec) *o0[b] = z[b].x;
        if (v[b] + 1 < nvec) o0[b][ldo] = z[b].y;
      }
    }
  }
}

// ============================================================================ host launchers

template <int N> struct CdCfg {
  static constexpr int S = (N >= 16384) ? 1 : (N >= 6144) ? 2 : 4;  // packed signals per CTA
  static constexpr int NT = fft_threads(N);          // threads per CTA
  static constexpr size_t SMEM = sizeof(float2) * S * fft_padded_len(N);
  // inverse cycle transform: the spectral configuration (variant 0) or half the packed signals at
  // the same threads (variant 1, measured faster at N = 4096: 96 vs 115 us); autotuned, variant 1
  // by default at N = 4096
  static constexpr int S_RES1 = S >= 2 ? S / 2 : S;
  static constexpr bool HAS_RES1 = S >= 2;
  static constexpr size_t SMEM_RES = sizeof(float2) * S * fft_padded_len(N) + sizeof(float) * N;  // + coefficients
  static constexpr size_t SMEM_RES1 = sizeof(float2) * S_RES1 * fft_padded_len(N) + sizeof(float) * N;
  // second spectral-apply variant for the autotuner: half the packed signals and threads per CTA
  // (more, smaller CTAs per SM; each coefficient load serves half as many signals)
  static constexpr bool HAS_V1 = S >= 2 && NT >= 64;
  static constexpr int S1 = HAS_V1 ? S / 2 : S, NT1A = HAS_V1 ? NT / 2 : NT;
  static constexpr size_t SMEM1 = sizeof(float2) * S1 * fft_padded_len(N);
  static constexpr int NT1 = (N >= 1024) ? 256 : (N >= 64 ? 64 : N);  // eigen-spectrum kernel
};

template <int N> static cudaError_t set_smem_attrs_now() {
  using C = CdCfg<N>;
  cudaError_t e = cudaSuccess;
  auto s = [&](const void* f, size_t b) {
    if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b);
  };
  s((const void*)cd_spectrum_kernel<N, C::S, C::NT, float>, C::SMEM);
  s((const void*)cd_spectrum_kernel<N, C::S, C::NT, __nv_bfloat16>, C::SMEM);
  s((const void*)cd_residual_kernel<N, C::S, C::NT>, C::SMEM_RES);
  s((const void*)cd_residual_kernel<N, C::S_RES1, C::NT>, C::SMEM_RES1);
  s((const void*)cd_apply_kernel<N, C::S, C::NT, false, false, float>, C::SMEM);
  s((const void*)cd_apply_kernel<N, C::S, C::NT, true, true, float>, C::SMEM);
  s((const void*)cd_apply_kernel<N, C::S, C::NT, true, true, __nv_bfloat16>, C::SMEM);
  s((const void*)cd_apply_kernel<N, C::S, C::NT, false, false, __nv_bfloat16>, C::SMEM);
  s((const void*)cd_apply_kernel<N, C::S, C::NT, false, true, float>, C::SMEM);
  s((const void*)cd_apply_kernel<N, C::S, C::NT, true, false, float>, C::SMEM);
  s((const void*)cd_apply_kernel<N, C::S1, C::NT1A, false, false, float>, C::SMEM1);
  s((const void*)cd_apply_kernel<N, C::S1, C::NT1A, true, true, float>, C::SMEM1);
  s((const void*)cd_apply_kernel<N, C::S1, C::NT1A, true, true, __nv_bfloat16>, C::SMEM1);
  s((const void*)cd_apply_kernel<N, C::S1, C::NT1A, false, false, __nv_bfloat16>, C::SMEM1);
  s((const void*)cd_apply_kernel<N, C::S1, C::NT1A, false, true, float>, C::SMEM1);
  s((const void*)cd_apply_kernel<N, C::S1, C::NT1A, true, false, float>, C::SMEM1);
  s((const void*)cd_eigen_kernel<N, CdCfg<N>::NT1>, sizeof(float2) * fft_padded_len(N));
  return e;
}

// the attributes above, set once per device
template <int N> static cudaError_t set_smem_attrs() {
  static DeviceOnce once;
  return once([] { return set_smem_attrs_now<N>(); });
}

template <int N> struct CdOps {
  using C = CdCfg<N>;
  static cudaError_t spectrum(const void* A, int64_t lda, bool bf16, const float2* tw, float2* R, float* kpart,
                              cudaStream_t st) {
    const cudaError_t attr = set_smem_attrs<N>();
    if (attr != cudaSuccess) return attr;
    dim3 grid(N / (2 * C::S));
    if (bf16)
      cd_spectrum_kernel<N, C::S, C::NT, __nv_bfloat16><<<grid, C::NT, C::SMEM, st>>>(
          (const __nv_bfloat16*)A, lda, tw, R, kpart);
    else
      cd_spectrum_kernel<N, C::S, C::NT, float><<<grid, C::NT, C::SMEM, st>>>((const float*)A, lda, tw, R, kpart);
    return cudaGetLastError();
  }
  static cudaError_t eigen(const float2* R, const float2* tw, const int32_t* list, const float* coef,
                           const int32_t* count, int cap, int imag_coef, float2* L, cudaStream_t st) {
    const cudaError_t attr = set_smem_attrs<N>();
    if (attr != cudaSuccess) return attr;
    constexpr int NT1 = C::NT1;
    size_t sm = sizeof(float2) * fft_padded_len(N);
    if (cap <= 0) return cudaSuccess;
    cd_eigen_kernel<N, NT1><<<cap, NT1, sm, st>>>(R, tw, list, coef, count, imag_coef, L);
    return cudaGetLastError();
  }
  template <int V>
  static cudaError_t residual_v(const float2* R, const float2* tw, const float* g, int mode, const int32_t* dcount,
                                const int32_t* dcount2, float* X, int64_t ldx, int accumulate, cudaStream_t st) {
    constexpr int S_ = V ? C::S_RES1 : C::S;
    constexpr size_t SM_ = V ? C::SMEM_RES1 : C::SMEM_RES;
    cd_residual_kernel<N, S_, C::NT><<<N / (2 * S_), C::NT, SM_, st>>>(R, tw, g, mode, dcount, dcount2, X, ldx,
                                                                       accumulate);
    return cudaGetLastError();
  }
  static cudaError_t residual(const float2* R, const float2* tw, const float* g, int mode, const int32_t* dcount,
                              const int32_t* dcount2, float* X, int64_t ldx, int accumulate, cudaStream_t st) {
    const cudaError_t attr = set_smem_attrs<N>();
    if (attr != cudaSuccess) return attr;
    int v = 0;
    if (C::HAS_RES1) {
      // one key for the overwriting and one for the accumulating form (flag 1: the read-modify-write
      // of 16-byte row segments favours the full variant); timed with mode 0 on a scratch output --
      // the variants differ in CTA shape only
      const int acc = accumulate ? 1 : 0;
      float* scratch = nullptr;
      v = tune_pick(tune_key(TUNE_RESIDUAL, N, acc), 2, (N == 4096 && !acc) ? 1 : 0, st, [&](int cand) -> cudaError_t {
        if (!scratch) {
          cudaError_t e = dev_alloc((void**)&scratch, sizeof(float) * (size_t)N * N, st);
          if (e == cudaSuccess) e = cudaMemsetAsync(scratch, 0, sizeof(float) * (size_t)N * N, st);
          if (e != cudaSuccess) return e;
        }
        return cand ? residual_v<1>(R, tw, g, 0, nullptr, nullptr, scratch, N, acc, st)
                    : residual_v<0>(R, tw, g, 0, nullptr, nullptr, scratch, N, acc, st);
      });
      if (scratch) dev_free(scratch, st);
    }
    return v ? residual_v<1>(R, tw, g, mode, dcount, dcount2, X, ldx, accumulate, st)
             : residual_v<0>(R, tw, g, mode, dcount, dcount2, X, ldx, accumulate, st);
  }
  template <int V>
  static cudaError_t apply_v(bool row, const void* X, int64_t ldx, bool bf16, int64_t nvec, const float2* tw,
                             const int32_t* list, const float2* Lc, const int32_t* count, const int32_t* gate0,
                             const int32_t* gate1, float* out, int64_t ldo, int accumulate, int rev, cudaStream_t st) {
    constexpr int S_ = V ? C::S1 : C::S, NT_ = V ? C::NT1A : C::NT;
    constexpr size_t SM_ = V ? C::SMEM1 : C::SMEM;
    dim3 grid((unsigned)((nvec + 2 * S_ - 1) / (2 * S_)));
    const bool r = rev < 0 ? row : rev != 0;
#define AMM_APPLY_LAUNCH(ROW_, REV_, T_)                                                                    \
  cd_apply_kernel<N, S_, NT_, ROW_, REV_, T_><<<grid, NT_, SM_, st>>>((const T_*)X, ldx, tw, list, Lc, count, gate0, \
                                                                      gate1, out, ldo, accumulate, (int)nvec)
    if (row && r) {
      if (bf16) AMM_APPLY_LAUNCH(true, true, __nv_bfloat16);
      else AMM_APPLY_LAUNCH(true, true, float);
    } else if (!row && !r) {
      if (bf16) AMM_APPLY_LAUNCH(false, false, __nv_bfloat16);
      else AMM_APPLY_LAUNCH(false, false, float);
    } else if (row) {
      if (bf16) return cudaErrorInvalidValue;
      AMM_APPLY_LAUNCH(true, false, float);
    } else {
      if (bf16) return cudaErrorInvalidValue;
      AMM_APPLY_LAUNCH(false, true, float);
    }
#undef AMM_APPLY_LAUNCH
    return cudaGetLastError();
  }
  // The variant for this (N, direction, coefficient pairing, element type): the tuned choice when
  // the autotuner has timed it, else the default.  With the autotuner on and the stream not being
  // captured, an untimed key is timed here once on the call's own operands, writing a scratch output.
  static int variant(bool row, const void* X, int64_t ldx, bool bf16, int64_t nvec, const float2* tw,
                     const int32_t* list, const float2* Lc, const int32_t* count, int rev, cudaStream_t st) {
    if (!C::HAS_V1) return 0;
    const int key = tune_key(TUNE_APPLY, N, (row ? 4 : 0) + ((rev < 0 ? row : rev != 0) ? 2 : 0) + (bf16 ? 1 : 0));
    const int64_t lds = row ? N : nvec;
    float* scratch = nullptr;
    const int v = tune_pick(key, 2, 0, st, [&](int cand) -> cudaError_t {
      if (!scratch) {
        cudaError_t e = dev_alloc((void**)&scratch, sizeof(float) * (size_t)N * nvec, st);
        if (e != cudaSuccess) return e;
      }
      return cand ? apply_v<1>(row, X, ldx, bf16, nvec, tw, list, Lc, count, nullptr, nullptr, scratch, lds, 0, rev, st)
                  : apply_v<0>(row, X, ldx, bf16, nvec, tw, list, Lc, count, nullptr, nullptr, scratch, lds, 0, rev, st);
    });
    if (scratch) dev_free(scratch, st);
    return v;
  }
  static cudaError_t apply(bool row, const void* X, int64_t ldx, bool bf16, int64_t nvec, const float2* tw,
                           const int32_t* list, const float2* Lc, const int32_t* count, const int32_t* gate0,
                           const int32_t* gate1, float* out, int64_t ldo, int accumulate, int rev, cudaStream_t st) {
    const cudaError_t attr = set_smem_attrs<N>();
    if (attr != cudaSuccess) return attr;
    const int v = gate0 ? 0 : variant(row, X, ldx, bf16, nvec, tw, list, Lc, count, rev, st);
    if (v) return apply_v<1>(row, X, ldx, bf16, nvec, tw, list, Lc, count, gate0, gate1, out, ldo, accumulate, rev, st);
    return apply_v<0>(row, X, ldx, bf16, nvec, tw, list, Lc, count, gate0, gate1, out, ldo, accumulate, rev, st);
  }
};

// lengths 3 * 2^a, 48 <= n <= 6144 (circulant_r3.cu); cudaErrorInvalidValue for other n
cudaError_t cd_spectrum_r3(int n, const void* A, int64_t lda, bool bf16, const float2* tw, float2* R, float* kpart,
                           cudaStream_t st);
cudaError_t cd_eigen_r3(int n, const float2* R, const float2* tw, const int32_t* list, const float* coef,
                        const int32_t* count, int cap, int imag_coef, float2* L, cudaStream_t st);
cudaError_t cd_residual_r3(int n, const float2* R, const float2* tw, const float* g, int mode, const int32_t* dcount,
                           const int32_t* dcount2, float* X, int64_t ldx, int accumulate, cudaStream_t st);
cudaError_t cd_apply_r3(int n, bool row, const void* X, int64_t ldx, bool bf16, int64_t nvec, const float2* tw,
                        const int32_t* list, const float2* Lc, const int32_t* count, const int32_t* gate0,
                        const int32_t* gate1, float* out, int64_t ldo, int accumulate, int rev, cudaStream_t st);

}  // namespace amm
