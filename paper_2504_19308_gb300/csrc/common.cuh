// Shared device helpers for libamm (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#define AMM_DEV __device__ __forceinline__

// ---------------------------------------------------------------- complex float2 arithmetic
AMM_DEV float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
AMM_DEV float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
AMM_DEV float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
AMM_DEV float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
AMM_DEV float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// acc += a * b
AMM_DEV void cmac(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x));
  acc.y = fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y));
}
// multiply by -i (s=-1) or +i (s=+1)
AMM_DEV float2 cmul_i(float2 a, int s) { return s > 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x); }

// Padded shared-memory index for FFT buffers: one float2 of padding every 16 elements.
// Makes the stride-R stores of the first radix-R Stockham pass bank-conflict free.
AMM_DEV int fpad(int e) { return e + (e >> 4); }
// Stride between the signals of a CTA: the padded length plus 4 float2, so that the same index of
// four consecutive signals falls on four different groups of 8 banks (2 * stride = 8 mod 32 for
// n >= 256) -- the reads of one frequency across the packed signals are then conflict free.
__host__ __device__ constexpr int fft_padded_len(int n) { return n + n / 16 + 4; }

constexpr int ilog2_c(int n) { return n <= 1 ? 0 : 1 + ilog2_c(n / 2); }

// Transform lengths of the shared-memory FFT: N = 3^c 2^a.
__host__ __device__ constexpr bool fft_len_ok(int n) {
  return n < 1 ? false : (n % 3 == 0) ? fft_len_ok(n / 3) : ((n & (n - 1)) == 0);
}
// x mod N for x in [-2N, ...): the indices of cyclic shifts (a mask when N is a power of two)
template <int N> AMM_DEV int wrapN(int x) {
  if constexpr ((N & (N - 1)) == 0) return x & (N - 1);
  else return (int)((unsigned)(x + 2 * N) % (unsigned)N);
}
// the conjugate partner n - t of component t (0 for t = 0), runtime n
AMM_DEV int mirror_idx(int t, int n) { return t == 0 ? 0 : n - t; }
// threads per CTA of the N-templated FFT kernels: the largest power of two dividing N, at most 512
__host__ __device__ constexpr int fft_threads(int n) { return (n & -n) >= 512 ? 512 : (n & -n); }
// x mod n for x in [-n, 2n), runtime n; P2: n is a power of two (a mask)
template <bool P2> AMM_DEV int cwrap(int x, int n) {
  if constexpr (P2) return x & (n - 1);
  else {
    x += (x < 0) ? n : 0;
    return x >= n ? x - n : x;
  }
}

// Host: runs a setup call (kernel attributes) once per device and returns its cached result on
// later calls with the same device current.  Kernel attributes belong to a device's context, so a
// process-wide "done" flag would skip them on a second device.  Thread-safe.
struct DeviceOnce {
  std::mutex mu;
  bool done[64] = {};
  cudaError_t res[64] = {};
  template <class F> cudaError_t operator()(F&& setup) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(mu);
    if (!done[dev]) {
      res[dev] = setup();
      done[dev] = true;
    }
    return res[dev];
  }
};

// Radix selection step over a 256-bin histogram: the bin b where the count from the top (bin 255
// down) first reaches need (need >= 1), and the count strictly above it in *above.  Called by one
// full warp (lane L scans bins 255 - 8L - q, q = 0..7, a shuffle scan finds the crossing lane);
// the result is valid on every lane.
AMM_DEV int radix_bucket_warp(const unsigned* hist, unsigned need, unsigned* above) {
  const int lane = threadIdx.x & 31;
  unsigned c[8], sum = 0;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    c[q] = hist[255 - 8 * lane - q];
    sum += c[q];
  }
  unsigned incl = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  const unsigned hit = __ballot_sync(0xffffffffu, incl - sum < need && need <= incl);
  const int src = hit ? __ffs(hit) - 1 : 31;
  unsigned acc = incl - sum;
  int b = 255 - 8 * lane;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    b = 255 - 8 * lane - q;
    if (acc + c[q] >= need || b == 0) break;
    acc += c[q];
  }
  *above = __shfl_sync(0xffffffffu, acc, src);
  return __shfl_sync(0xffffffffu, b, src);
}
