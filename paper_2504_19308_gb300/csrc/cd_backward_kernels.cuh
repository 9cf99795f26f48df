// Backward of the circulant first-order product with the selections frozen (sm_103a).
//
// With S the selection of A (weights w, unpaired coefficients v as in the forward) and G the
// upstream gradient, the gradients of <G, Re M> are (bilinear adjoint of P_S is P_{S-bar}):
//   dA = G B~_w^T + sum_{t in S u S-bar} w_t R_t(G dB_w^T) D^t + sum_{t unpaired} (i v_t) R_t(G V_B^T) D^t
//   dB = A~_w^T G + sum_{s} w_s R_s(dA_w^T G) D^s + sum_{s unpaired} (i v_s) R_s(Y_A^T G) D^s
// where dB_w = B - Re B~, V_B = Im B~, dA_w = A - Re A~, Y_A = Im A~.  The first terms are spectral
// applies with the adjoint coefficient pairing.  A component of a product matrix is an SDDMM on
// spectra: with column spectra Xh = F X, Yh = F Y (DFT along the row index),
//   r_{j,t}(X Y^T) = (1/n^2) sum_p e^{2 pi i p j/n} K_t(p),   K_t(p) = sum_m Xh(p, m) Yh(t - p, m),
// and for X^T Y the same with row spectra stored transposed ([frequency][row]).  Real products
// have Hermitian component spectra, so only t <= n/2 is formed; the dense result comes from the
// inverse cycle transform (cd_residual) with the coefficient w_t or i v_t.
//
// This header holds the N-templated kernels and their launch structs; cd_backward.cu instantiates
// them for N = 2^a and cd_backward_r3.cu for N = 3 * 2^a.
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"
#include "fft.cuh"
#include "kernels.h"
#include "trace.h"
#include "tune.cuh"

namespace amm {

// ============================================================================ half spectra
// COL: Xh[q][c] = sum_r e^{-2 pi i q r/n} X(r, c);  ROW: Xh[q][r] = sum_c e^{-2 pi i q c/n} X(r, c).
// Output layout [q][vector], q = 0..n/2.  Packed pairs of real vectors per complex FFT.
template <int N, int S, int NT, bool ROW>
__global__ void __launch_bounds__(NT) bw_spectrum_kernel(const float* __restrict__ X, int64_t ldx,
                                                         const float2* __restrict__ tw, float2* __restrict__ Xh,
                                                         const int32_t* __restrict__ gate0,
                                                         const int32_t* __restrict__ gate1) {
  extern __shared__ float2 smem[];
  if (gate0 != nullptr && (*gate0 == 0 || *gate1 == 0)) return;
  constexpr int LD = fft_padded_len(N);
  constexpr int KH = N / 2 + 1;
  const int base = blockIdx.x * 2 * S;
#pragma unroll 16
  for (int it = 0; it < N * S / NT; ++it) {
    const int e = threadIdx.x + it * NT;
    int s, l;
    if (ROW) { s = e / N; l = e % N; } else { l = e / S; s = e % S; }
    const int v0 = base + 2 * s;
    float x0, x1;
    if (ROW) { x0 = __ldg(X + (int64_t)v0 * ldx + l); x1 = __ldg(X + (int64_t)(v0 + 1) * ldx + l); }
    else { x0 = __ldg(X + (int64_t)l * ldx + v0); x1 = __ldg(X + (int64_t)l * ldx + v0 + 1); }
    smem[s * LD + fpad(l)] = make_float2(x0, x1);
  }
  __syncthreads();
  fft_smem<N, S, NT, false>(smem, tw);
  for (int e = threadIdx.x; e < KH * 2 * S; e += NT) {
    const int q = e / (2 * S), m = e % (2 * S);
    const float2* z = smem + (m >> 1) * LD;
    const float2 a = z[fpad(q)];
    const float2 b = cconj(z[fpad(wrapN<N>(N - q))]);
    float2 x;
    if ((m & 1) == 0) x = cscale(cadd(a, b), 0.5f);
    else { float2 d = csub(a, b); x = make_float2(0.5f * d.y, -0.5f * d.x); }
    Xh[(int64_t)q * N + base + m] = x;
  }
}

// ============================================================================ SDDMM on spectra
// K[u][p] = sum_m Xh(p, m) Yh((t_u - p) mod n, m) for t_u <= n/2, p = 0..n-1.  Half-spectrum rows
// q > n/2 are conj(row n - q).  One warp per (p, block of SD_UB listed components); lanes stride
// over m, so each Xh element is loaded once for SD_UB products (9 bytes per complex MAC instead
// of 16) and the SD_UB independent loads of Yh overlap.  The component blocks are the fast grid
// dimension: the CTAs in flight share a narrow window of p, so the Xh rows of the window and
// the Yh rows t - p (each used by every t whose window covers it) stay in L2 while the spectra
// themselves (2 x 64 MiB at n = 4096) do not fit.
constexpr int SD_UB = 8;
template <int N>
__global__ void __launch_bounds__(256) cd_sddmm_kernel(const float2* __restrict__ Xh, const float2* __restrict__ Yh,
                                                       const int32_t* __restrict__ list,
                                                       const int32_t* __restrict__ count, float2* __restrict__ K,
                                                       const int32_t* __restrict__ gate0,
                                                       const int32_t* __restrict__ gate1) {
  if (gate0 != nullptr && (*gate0 == 0 || *gate1 == 0)) return;
  const int cnt = *count;
  const int u0 = blockIdx.x * SD_UB;
  if (u0 >= cnt) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int p = blockIdx.y * 8 + warp;
  const bool xm = p > N / 2;
  const float2* xr = Xh + (int64_t)(xm ? N - p : p) * N;
  const float xs = xm ? -1.f : 1.f;
  const float2* yr[SD_UB];
  float ys[SD_UB];
  bool act[SD_UB];
#pragma unroll
  for (int j = 0; j < SD_UB; ++j) {
    const int u = u0 + j;
    const int t = u < cnt ? __ldg(list + u) : N;
    act[j] = t <= N / 2;
    // (t - p) mod N, written inline: through wrapN the compiler allocates ten more registers here
    const int q = ((N & (N - 1)) == 0) ? ((t - p) & (N - 1)) : ((t - p + N) % N);
    const bool ym = q > N / 2;
    yr[j] = Yh + (int64_t)(ym ? N - q : q) * N;
    ys[j] = ym ? -1.f : 1.f;
  }
  float2 acc[SD_UB];
#pragma unroll
  for (int j = 0; j < SD_UB; ++j) acc[j] = make_float2(0.f, 0.f);
  // SD_MU consecutive m of the lane's sequence m = lane, lane + 32, ... per step: their Xh loads,
  // then per component their Yh loads, are issued together (few listed components leave a warp
  // with little else to overlap); every accumulator still adds its products in increasing m
  constexpr int SD_MU = 4;
  for (int m0 = lane; m0 < N; m0 += 32 * SD_MU) {
    float2 x[SD_MU];
#pragma unroll
    for (int q = 0; q < SD_MU; ++q) {
      const int m = m0 + 32 * q;
      x[q] = m < N ? __ldg(xr + m) : make_float2(0.f, 0.f);
      x[q].y *= xs;
    }
#pragma unroll
    for (int j = 0; j < SD_UB; ++j) {
      if (!act[j]) continue;  // warp-uniform
      float2 y[SD_MU];
#pragma unroll
      for (int q = 0; q < SD_MU; ++q) {
        const int m = m0 + 32 * q;
        y[q] = m < N ? __ldg(yr[j] + m) : make_float2(0.f, 0.f);
        y[q].y *= ys[j];
      }
#pragma unroll
      for (int q = 0; q < SD_MU; ++q)
        if (m0 + 32 * q < N) cmac(acc[j], x[q], y[q]);
    }
  }
#pragma unroll
  for (int j = 0; j < SD_UB; ++j) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      acc[j].x += __shfl_xor_sync(0xffffffffu, acc[j].x, o);
      acc[j].y += __shfl_xor_sync(0xffffffffu, acc[j].y, o);
    }
  }
  if (lane == 0) {
#pragma unroll
    for (int j = 0; j < SD_UB; ++j)
      if (act[j]) K[(int64_t)(u0 + j) * N + p] = acc[j];
  }
}

// Tiled form for dense selections (many listed t per range of n/16).  A CTA takes a window of
// SDT_P frequencies p and a range of SDT_W component indices [T0, T0 + SDT_W): the Yh rows t - p
// of every listed t in the range and every p in the window are the SDT_P + SDT_W - 1 consecutive
// rows starting at T0 - p0 - SDT_P + 1.  Chunks of SDT_MC columns of those rows and of the SDT_P
// Xh rows are copied to shared memory with cp.async, double-buffered (the next chunk is in flight
// while the current one is used); rows are padded to SDT_MC + 1 complex (conflict-free column
// reads) and copied raw, with the conjugation of mirrored rows applied as a sign at use.  Each
// staged Yh element serves every listed t that reaches it, and each thread keeps its Xh row
// chunk in registers, so a complex MAC costs one shared load.  Warp w owns p = p0 + 32 (w & 1) +
// lane and the slots j = (w >> 1) + 4 i of the range's listed t's, in batches of 4 SDT_SLOTS.
constexpr int SDT_P = 64, SDT_W = 256, SDT_MC = 16, SDT_NT = 256, SDT_SLOTS = 16;
constexpr int SDT_LDM = SDT_MC + 1, SDT_YR = SDT_P + SDT_W - 1;
constexpr size_t SDT_STAGE = (size_t)(SDT_P + SDT_YR) * SDT_LDM;  // float2 per stage
constexpr size_t SDT_SMEM = sizeof(float2) * 2 * SDT_STAGE + sizeof(float) * (SDT_P + SDT_YR) +
                            sizeof(int) * 2 * SDT_W + 16;

__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gsrc) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(smem_dst)),
               "l"(gsrc)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int PENDING>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(PENDING) : "memory");
}

template <int N>
__global__ void __launch_bounds__(SDT_NT) cd_sddmm_tiled_kernel(const float2* __restrict__ Xh,
                                                               const float2* __restrict__ Yh,
                                                               const int32_t* __restrict__ list,
                                                               const int32_t* __restrict__ count,
                                                               float2* __restrict__ K,
                                                               const int32_t* __restrict__ gate0,
                                                               const int32_t* __restrict__ gate1) {
  extern __shared__ __align__(16) unsigned char sdt_raw[];
  float2* stage = reinterpret_cast<float2*>(sdt_raw);                       // 2 x [P + YR][LDM]
  float* sgn = reinterpret_cast<float*>(stage + 2 * SDT_STAGE);            // [P + YR] row signs
  int* s_u = reinterpret_cast<int*>(sgn + SDT_P + SDT_YR);                  // [W]
  int* s_t = s_u + SDT_W;                                                    // [W]
  __shared__ int s_cnt;
  if (gate0 != nullptr && (*gate0 == 0 || *gate1 == 0)) return;
  const int T0 = blockIdx.x * SDT_W, p0 = blockIdx.y * SDT_P;
  if (threadIdx.x == 0) s_cnt = 0;
  __syncthreads();
  const int nl = *count;
  for (int i = threadIdx.x; i < nl; i += SDT_NT) {
    const int t = __ldg(list + i);
    if (t >= T0 && t < T0 + SDT_W && t <= N / 2) {
      const int pos = atomicAdd(&s_cnt, 1);
      s_u[pos] = i;
      s_t[pos] = t;
    }
  }
  const int rlo = T0 - p0 - SDT_P + 1;  // first staged Yh row (mod N)
  for (int row = threadIdx.x; row < SDT_P + SDT_YR; row += SDT_NT) {
    const int q = row < SDT_P ? p0 + row : wrapN<N>(rlo + row - SDT_P);
    sgn[row] = q > N / 2 ? -1.f : 1.f;
  }
  __syncthreads();
  const int cnt = s_cnt;
  if (cnt == 0) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int pl = (warp & 1) * 32 + lane;  // p - p0
  const int sub = warp >> 1;
  const float xs = sgn[pl];
  auto load_chunk = [&](int m0, float2* buf) {
    for (int e = threadIdx.x; e < (SDT_P + SDT_YR) * SDT_MC; e += SDT_NT) {
      const int row = e / SDT_MC, m = e % SDT_MC;
      const int q = row < SDT_P ? p0 + row : wrapN<N>(rlo + row - SDT_P);
      const int qr = q > N / 2 ? N - q : q;
      cp_async8(buf + row * SDT_LDM + m, (row < SDT_P ? Xh : Yh) + (int64_t)qr * N + m0 + m);
    }
    cp_async_commit();
  };
  for (int tb0 = 0; tb0 < cnt; tb0 += 4 * SDT_SLOTS) {
    float2 acc[SDT_SLOTS];
#pragma unroll
    for (int i = 0; i < SDT_SLOTS; ++i) acc[i] = make_float2(0.f, 0.f);
    constexpr int NCH = N / SDT_MC;
    load_chunk(0, stage);
    for (int c = 0; c < NCH; ++c) {
      float2* cur = stage + (c & 1) * SDT_STAGE;
      if (c + 1 < NCH) {
        load_chunk((c + 1) * SDT_MC, stage + ((c + 1) & 1) * SDT_STAGE);
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
      __syncthreads();
      float2 x[SDT_MC];
#pragma unroll
      for (int m = 0; m < SDT_MC; ++m) {
        x[m] = cur[pl * SDT_LDM + m];
        x[m].y *= xs;
      }
      const float2* ybase = cur + SDT_P * SDT_LDM;
#pragma unroll
      for (int i = 0; i < SDT_SLOTS; ++i) {
        const int j = tb0 + sub + 4 * i;
        if (j >= cnt) break;  // warp-uniform
        const int yr = (s_t[j] - T0) + (SDT_P - 1) - pl;
        const float ys = sgn[SDT_P + yr];
        const float2* y = ybase + yr * SDT_LDM;
#pragma unroll
        for (int m = 0; m < SDT_MC; ++m) {
          float2 v = y[m];
          v.y *= ys;
          cmac(acc[i], x[m], v);
        }
      }
      __syncthreads();  // the buffer of chunk c is refilled next iteration
    }
#pragma unroll
    for (int i = 0; i < SDT_SLOTS; ++i) {
      const int j = tb0 + sub + 4 * i;
      if (j < cnt) K[(int64_t)s_u[j] * N + p0 + pl] = acc[i];
    }
  }
}

// ============================================================================ component spectra
// RX[t][j] = (1/n^2) sum_p e^{2 pi i p j/n} K[u][p] for t = list[u] <= n/2 (RX zeroed beforehand).
template <int N, int NT>
__global__ void __launch_bounds__(NT) cd_rho_kernel(const float2* __restrict__ K, const float2* __restrict__ tw,
                                                    const int32_t* __restrict__ list, const int32_t* __restrict__ count,
                                                    float2* __restrict__ RX, const int32_t* __restrict__ gate0,
                                                    const int32_t* __restrict__ gate1) {
  extern __shared__ float2 smem[];
  const int u = blockIdx.x;
  if (u >= *count) return;
  if (gate0 != nullptr && (*gate0 == 0 || *gate1 == 0)) return;
  const int t = list[u];
  if (t > N / 2) return;
  for (int p = threadIdx.x; p < N; p += NT) smem[fpad(p)] = K[(int64_t)u * N + p];
  __syncthreads();
  fft_smem<N, 1, NT, true>(smem, tw);
  const float sc = 1.0f / ((float)N * (float)N);
  for (int j = threadIdx.x; j < N; j += NT) RX[(int64_t)t * N + j] = cscale(smem[fpad(j)], sc);
}

// ============================================================================ launchers
template <int N> struct BwCfg {
  // variant 0: S signals per CTA of fft_threads(N); variant 1: half the signals and threads (two
  // CTAs per SM where one 512-thread CTA at 128 registers would fill the register file).  Both are
  // autotuned per direction; defaults measured at N = 4096: columns variant 0 (60 vs 70 us), rows
  // variant 1 for 1024 <= N < 6144 (47 vs 54 us)
  static constexpr int S = (N >= 16384) ? 1 : (N >= 6144) ? 2 : 4;
  static constexpr int NT = fft_threads(N);
  static constexpr bool HAS_V1 = S >= 2 && NT >= 64;
  static constexpr int S1 = HAS_V1 ? S / 2 : S, NT1S = HAS_V1 ? NT / 2 : NT;
  static constexpr size_t SMEM = sizeof(float2) * S * fft_padded_len(N);
  static constexpr size_t SMEM1 = sizeof(float2) * S1 * fft_padded_len(N);
  static constexpr int ROW_DEFAULT = (HAS_V1 && N >= 1024 && N < 6144) ? 1 : 0;
  static constexpr int NT1 = (N >= 1024) ? 256 : (N >= 64 ? 64 : N);
};

template <int N> struct BwOps {
  using C = BwCfg<N>;
  static cudaError_t attrs() {
    static DeviceOnce once;
    return once([] {
      cudaError_t r = cudaSuccess;
      for (const void* f : {(const void*)bw_spectrum_kernel<N, C::S, C::NT, true>,
                            (const void*)bw_spectrum_kernel<N, C::S, C::NT, false>})
        if (r == cudaSuccess) r = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
      for (const void* f : {(const void*)bw_spectrum_kernel<N, C::S1, C::NT1S, true>,
                            (const void*)bw_spectrum_kernel<N, C::S1, C::NT1S, false>})
        if (r == cudaSuccess) r = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM1);
      if (r == cudaSuccess)
        r = cudaFuncSetAttribute((const void*)cd_rho_kernel<N, C::NT1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(sizeof(float2) * fft_padded_len(N)));
      return r;
    });
  }
  template <int V>
  static cudaError_t spectrum_v(bool row, const float* X, int64_t ldx, const float2* tw, float2* Xh,
                                const int32_t* g0, const int32_t* g1, cudaStream_t st) {
    constexpr int S_ = V ? C::S1 : C::S, NT_ = V ? C::NT1S : C::NT;
    constexpr size_t SM_ = V ? C::SMEM1 : C::SMEM;
    if (row) bw_spectrum_kernel<N, S_, NT_, true><<<N / (2 * S_), NT_, SM_, st>>>(X, ldx, tw, Xh, g0, g1);
    else bw_spectrum_kernel<N, S_, NT_, false><<<N / (2 * S_), NT_, SM_, st>>>(X, ldx, tw, Xh, g0, g1);
    return cudaGetLastError();
  }
  static cudaError_t spectrum(bool row, const float* X, int64_t ldx, const float2* tw, float2* Xh,
                              const int32_t* g0, const int32_t* g1, cudaStream_t st) {
    cudaError_t e = attrs();
    if (e != cudaSuccess) return e;
    int v = 0;
    if (C::HAS_V1 && g0 == nullptr) {  // gated launches use the current choice (the gate may skip the work)
      float2* scratch = nullptr;
      v = tune_pick(tune_key(row ? TUNE_BW_ROW : TUNE_BW_COL, N, 0), 2, row ? C::ROW_DEFAULT : 0, st,
                    [&](int cand) -> cudaError_t {
                      if (!scratch) {
                        cudaError_t e2 = dev_alloc((void**)&scratch, sizeof(float2) * (N / 2 + 1) * (size_t)N, st);
                        if (e2 != cudaSuccess) return e2;
                      }
                      return cand ? spectrum_v<1>(row, X, ldx, tw, scratch, nullptr, nullptr, st)
                                  : spectrum_v<0>(row, X, ldx, tw, scratch, nullptr, nullptr, st);
                    });
      if (scratch) dev_free(scratch, st);
    } else if (C::HAS_V1) {
      const int t = cd_tune_get(tune_key(row ? TUNE_BW_ROW : TUNE_BW_COL, N, 0));
      v = t >= 0 ? t : (row ? C::ROW_DEFAULT : 0);
    }
    return v ? spectrum_v<1>(row, X, ldx, tw, Xh, g0, g1, st) : spectrum_v<0>(row, X, ldx, tw, Xh, g0, g1, st);
  }
  static cudaError_t sddmm(const float2* Xh, const float2* Yh, const int32_t* list, const int32_t* count, int cap,
                           float2* K, const int32_t* g0, const int32_t* g1, cudaStream_t st) {
    if (N >= 2 * SDT_W && (int64_t)cap * 12 >= N) {  // dense enough that a staged Yh row serves several t
      static DeviceOnce once;
      const cudaError_t attr = once([] {
        return cudaFuncSetAttribute((const void*)cd_sddmm_tiled_kernel<N>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SDT_SMEM);
      });
      if (attr != cudaSuccess) return attr;
      dim3 grid((N / 2 + SDT_W) / SDT_W, N / SDT_P);
      cd_sddmm_tiled_kernel<N><<<grid, SDT_NT, SDT_SMEM, st>>>(Xh, Yh, list, count, K, g0, g1);
      return cudaGetLastError();
    }
    dim3 grid((cap + SD_UB - 1) / SD_UB, N / 8);
    cd_sddmm_kernel<N><<<grid, 256, 0, st>>>(Xh, Yh, list, count, K, g0, g1);
    return cudaGetLastError();
  }
  static cudaError_t rho(const float2* K, const float2* tw, const int32_t* list, const int32_t* count, int cap,
                         float2* RX, const int32_t* g0, const int32_t* g1, cudaStream_t st) {
    cudaError_t e = attrs();
    if (e != cudaSuccess) return e;
    cd_rho_kernel<N, C::NT1><<<cap, C::NT1, sizeof(float2) * fft_padded_len(N), st>>>(K, tw, list, count, RX, g0,
                                                                                        g1);
    return cudaGetLastError();
  }
};

// lengths 3 * 2^a, 48 <= n <= 6144 (cd_backward_r3.cu); cudaErrorInvalidValue for other n
cudaError_t bw_spectrum_r3(int n, bool row, const float* X, int64_t ldx, const float2* tw, float2* Xh,
                           const int32_t* gate0, const int32_t* gate1, cudaStream_t st);
cudaError_t cd_sddmm_r3(int n, const float2* Xh, const float2* Yh, const int32_t* list, const int32_t* count, int cap,
                        float2* K, const int32_t* gate0, const int32_t* gate1, cudaStream_t st);
cudaError_t cd_rho_r3(int n, const float2* K, const float2* tw, const int32_t* list, const int32_t* count, int cap,
                      float2* RX, const int32_t* gate0, const int32_t* gate1, cudaStream_t st);

}  // namespace amm
