// Circulant-decomposition kernels (Thm 2.1, Alg. 2, Alg. 3 of arXiv 2504.19308) for sm_103a.
//
// Notation (paper): cycles A = sum_j C^j Lambda_j with Lambda_j(l) = A((l+j) mod n, l);
// spectrum r_{j,k} = (1/n) sum_l e^{-2 pi i k l/n} Lambda_j(l) stored as R[k][j] (row k = R_A[k]);
// eigen-spectra L_t = F R_A[t]; omega = e^{+2 pi i/n}.
//
// Data layout in HBM (n = FFT length, row-major everywhere):
//   R        (n/2+1) x n complex  -- half spectrum; R[n-k][j] = conj(R[k][j]) for real A
//   kpart    (n/J) x (n/2+1) f32  -- per-CTA partial sums of |r_{j,k}|^2 (deterministic keys)
//   Lw       cap x n complex      -- w_u L_{t_u} for the applied components t_u
//   resid    n x n f32            -- dB_w (right operand only)
//
// Product used (reading R5, real output):  with S the selection, S-bar = {n-t}, weights
// w_t = (1[t in S] + 1[n-t in S]) / 2 and v_t = (1[t in S] - 1[n-t in S]) / 2,
//   Re(A~_S B + dA_S B~_S) = A~_w dB_w + Y V + A B~_w,
//   A~_w = sum_t w_t R_t D^t (= Re A~_S),  Y = Im A~_S = sum_t (-i v_t) R_t D^t,  V = Im B~_S.
// The three terms are spectral applies (k complex MACs per output spectrum entry):
//   column apply  (Alg. 3, zeroth-order term): F(sum_t c_t R_t D^t X)(p,:) = sum_t c_t L_t(p) (F X)((p-t) mod n, :)
//   row apply     (X B~ by rows):  F_row(X sum_s c_s R_s D^s)(:,p) = sum_s c_s L_s((s-p) mod n) (F_row X)(:, (p-s) mod n)
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <fstream>
#include <mutex>
#include <sstream>
#include <string>
#include <unordered_map>
#include <vector>

#include "circulant_kernels.cuh"
#include "common.cuh"
#include "fft.cuh"
#include "kernels.h"
#include "trace.h"

namespace amm {

constexpr int SEL_SORT_MAX = 4096;  // selections up to this size are returned in key order

// ============================================================================ twiddles
__global__ void twiddle_kernel(float2* tw, int n) {
  int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m < n) {
    double s, c;
    sincospi(2.0 * (double)m / (double)n, &s, &c);
    tw[m] = make_float2((float)c, (float)-s);  // e^{-2 pi i m/n}
  }
}

// ============================================================================ K2: keys, top-k, weights
// One CTA of 1024 threads.  key2[t] = sum over the partial rows (fixed order, double).
// Top-k by (key desc, index asc): an exact MSB radix select over the 64-bit patterns of the
// non-negative double keys (8 passes of 8 bits) finds the k-th key tau; the selection is
// {key > tau} plus the lowest-index entries equal to tau.  The k winners are then ordered by
// a bitonic sort in shared memory.  Union / unpaired lists are compacted with block scans.
constexpr int SEL_T = 1024;

// exclusive block scan of one int per thread (SEL_T threads); returns the block total in *tot
__device__ int block_excl_scan(int v, int* wsum, int* tot) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[w] = x;
  __syncthreads();
  if (w == 0) {
    int y = lane < (SEL_T / 32) ? wsum[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int z = __shfl_up_sync(0xffffffffu, y, o);
      if (lane >= o) y += z;
    }
    wsum[lane] = y;  // inclusive warp-sum prefix
  }
  __syncthreads();
  const int before = (w > 0 ? wsum[w - 1] : 0) + x - v;
  *tot = wsum[SEL_T / 32 - 1];
  __syncthreads();
  return before;
}

__device__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < SEL_T / 32; ++w) s += red[w];
  __syncthreads();
  return s;  // valid in thread 0
}

// Circulant keys (mirror = 1): partial rows hold t = 0..n/2, T[n-t] = T[t], ||A||^2 = n sum T^2.
// Cycle keys (mirror = 0): partial rows hold all n cycles, ||A||^2 = sum T^2 (scale = 1).
// key2[t] = sum_c part[c][t] over the partial rows in a fixed order: 32 x 32 threads per CTA,
// thread (x, y) sums rows y, y+32, ..., then row 0 of the tile adds the 32 column sums in order.
// keys (optional): keys[t] = sqrt(key2[t]) in FP64, mirrored to keys[n - t] when mirror (the
// reported keys; taking the roots here spreads them over the CTAs instead of the selection's one).
__global__ void __launch_bounds__(1024) cd_keyreduce_kernel(const float* __restrict__ part, int nparts, int kh,
                                                            double* __restrict__ key2, double* __restrict__ keys,
                                                            int n, int mirror) {
  __shared__ double sm[32][33];
  const int t = blockIdx.x * 32 + threadIdx.x;
  double s = 0.0;
  if (t < kh)
    for (int c = threadIdx.y; c < nparts; c += 32) s += (double)part[(int64_t)c * kh + t];
  sm[threadIdx.y][threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.y == 0 && t < kh) {
    double v = 0.0;
    for (int y = 0; y < 32; ++y) v += sm[y][threadIdx.x];
    key2[t] = v;
    if (keys) {
      const double r = sqrt(v);
      keys[t] = r;
      if (mirror && t > 0 && t < n - t) keys[n - t] = r;
    }
  }
}

__global__ void __launch_bounds__(SEL_T) cd_select_kernel(const double* __restrict__ key2, int n,
                                                          int k, const int32_t* __restrict__ forced,
                                                          SelectOut out, int mirror, double scale,
                                                          int pair_closed) {
  extern __shared__ unsigned char sm[];
  double* key = reinterpret_cast<double*>(sm);                        // n (later: k sorted keys)
  unsigned char* in_s = reinterpret_cast<unsigned char*>(key + n);    // n
  __shared__ double red[32];
  __shared__ int wsum[32];
  __shared__ unsigned int hist[256];
  __shared__ unsigned long long s_prefix;
  __shared__ unsigned int s_need;
  __shared__ double s_kth;
  const int kh = mirror ? n / 2 + 1 : n;
  for (int t = threadIdx.x; t < kh; t += SEL_T) {
    const double s = key2[t];
    key[t] = s;
    if (mirror && t > 0 && t < n - t) key[n - t] = s;
  }
  for (int t = threadIdx.x; t < n; t += SEL_T) in_s[t] = 0;
  __syncthreads();
  double part = 0.0;  // (out.keys, the roots, were written by cd_keyreduce_kernel)
  for (int t = threadIdx.x; t < n; t += SEL_T) part += key[t];
  const double total = block_sum(part, red);
  if (threadIdx.x == 0) out.norms[0] = total * scale;
  // chunk ownership for compactions: thread owns [c0, c1)
  const int chunk = (n + SEL_T - 1) / SEL_T;
  const int c0 = min(n, threadIdx.x * chunk), c1 = min(n, c0 + chunk);
  if (forced == nullptr) {
    if (threadIdx.x == 0) { s_prefix = 0ull; s_need = (unsigned)k; }
    __syncthreads();
    unsigned long long mask = 0ull;
    for (int shift = 56; shift >= 0; shift -= 8) {
      for (int b = threadIdx.x; b < 256; b += SEL_T) hist[b] = 0;
      __syncthreads();
      const unsigned long long prefix = s_prefix;
      // lanes of a warp that fall into the same bucket add together: one atomic per bucket and warp
      // (the leading bytes of the keys crowd into few buckets)
      for (int t0 = 0; t0 < n; t0 += SEL_T) {
        const int t = t0 + threadIdx.x;
        const unsigned long long kb = t < n ? (unsigned long long)__double_as_longlong(key[t]) : 0ull;
        const bool part = t < n && (kb & mask) == prefix;
        const unsigned pm = __ballot_sync(0xffffffffu, part);
        if (part) {
          const unsigned bkt = (unsigned)((kb >> shift) & 255ull);
          const unsigned peers = __match_any_sync(pm, bkt);
          if ((threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&hist[bkt], (unsigned)__popc(peers));
        }
      }
      __syncthreads();
      if (threadIdx.x < 32) {
        unsigned above;
        const int b = radix_bucket_warp(hist, s_need, &above);
        if (threadIdx.x == 0) {
          s_need -= above;
          s_prefix = prefix | ((unsigned long long)b << shift);
        }
      }
      mask |= 255ull << shift;
      __syncthreads();
    }
    const unsigned long long tau = s_prefix;
    const unsigned need_eq = s_need;
    int eq = 0;
    for (int t = c0; t < c1; ++t) eq += (unsigned long long)__double_as_longlong(key[t]) == tau;
    int tot;
    int e = block_excl_scan(eq, wsum, &tot);
    for (int t = c0; t < c1; ++t) {
      const unsigned long long kb = (unsigned long long)__double_as_longlong(key[t]);
      if (kb > tau) in_s[t] = 1;
      else if (kb == tau) { if ((unsigned)e < need_eq) in_s[t] = 1; ++e; }
    }
    __syncthreads();
    // boundary gap: the k-th key is tau; the next key is the largest key not selected
    if (threadIdx.x == 0) s_kth = __longlong_as_double((long long)tau);
    __syncthreads();
    double nxt = -1.0;
    for (int t = threadIdx.x; t < n; t += SEL_T) if (!in_s[t]) nxt = fmax(nxt, key[t]);
    for (int o = 16; o > 0; o >>= 1) nxt = fmax(nxt, __shfl_xor_sync(0xffffffffu, nxt, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = nxt;
    __syncthreads();
    if (threadIdx.x == 0) {
      double m = -1.0;
      for (int w = 0; w < SEL_T / 32; ++w) m = fmax(m, red[w]);
      const double a = sqrt(s_kth);
      out.norms[2] = (m < 0.0) ? 1e300 : (a > 0 ? (a - sqrt(m)) / a : 0.0);
    }
    __syncthreads();
  } else {
    for (int t = threadIdx.x; t < k; t += SEL_T) in_s[forced[t]] = 1;
    if (threadIdx.x == 0) out.norms[2] = -1.0;
    __syncthreads();
  }
  // ||dA||^2 = ||A||^2 - scale * sum_{t in S} T[t]^2 (S u S-bar when the selection is pair-closed:
  // the partner's key equals the component's own)
  part = 0.0;
  for (int t = threadIdx.x; t < n; t += SEL_T) {
    if (in_s[t]) part += key[t];
    if (pair_closed && in_s[t] && !in_s[mirror_idx(t, n)]) part += key[t];
  }
  const double kept = block_sum(part, red);
  if (threadIdx.x == 0) out.norms[1] = total * scale - kept * scale;
  // compact the selection (ascending index), then order it by (key desc, index asc)
  int cnt = 0;
  for (int t = c0; t < c1; ++t) cnt += in_s[t];
  int tot;
  int pos = block_excl_scan(cnt, wsum, &tot);
  // stash (key, index) of the winners after the n keys are no longer needed: use idx area
  double* skey = reinterpret_cast<double*>(in_s + n + ((8 - (n & 7)) & 7));  // kp doubles
  int32_t* sidx = reinterpret_cast<int32_t*>(skey + SEL_SORT_MAX);           // kp ints
  int kp = 1;
  while (kp < k) kp <<= 1;
  const bool sortable = kp <= SEL_SORT_MAX;
  for (int t = c0; t < c1; ++t) {
    if (in_s[t]) {
      if (sortable) { skey[pos] = key[t]; sidx[pos] = t; }
      else out.sel[pos] = t;
      ++pos;
    }
  }
  __syncthreads();
  if (sortable && forced == nullptr) {
    for (int t = k + threadIdx.x; t < kp; t += SEL_T) { skey[t] = -1.0; sidx[t] = 0x7fffffff; }
    __syncthreads();
    for (int size = 2; size <= kp; size <<= 1) {
      for (int stride = size >> 1; stride > 0; stride >>= 1) {
        for (int i = threadIdx.x; i < kp; i += SEL_T) {
          const int p = i ^ stride;
          if (p > i) {
            const bool up = (i & size) == 0;
            const double ki = skey[i], kq = skey[p];
            const int ii = sidx[i], iq = sidx[p];
            const bool i_first = (ki > kq) || (ki == kq && ii < iq);
            if (up ? !i_first : i_first) { skey[i] = kq; skey[p] = ki; sidx[i] = iq; sidx[p] = ii; }
          }
        }
        __syncthreads();
      }
    }
    for (int t = threadIdx.x; t < k; t += SEL_T) out.sel[t] = sidx[t];
  } else if (forced != nullptr) {
    for (int t = threadIdx.x; t < k; t += SEL_T) out.sel[t] = forced[t];
  } else if (sortable) {
    for (int t = threadIdx.x; t < k; t += SEL_T) out.sel[t] = sidx[t];
  }
  if (pair_closed) {  // S <- S u S-bar: every kept component with its conjugate partner, M real
    unsigned char cl[(16384 + SEL_T - 1) / SEL_T];
    for (int t = c0; t < c1; ++t) cl[t - c0] = in_s[t] | in_s[mirror_idx(t, n)];
    __syncthreads();
    for (int t = c0; t < c1; ++t) in_s[t] = cl[t - c0];
    __syncthreads();
  }
  // union S u S-bar (weight w_t) and unpaired set (v_t), compacted in index order
  int nu = 0, nd = 0;
  for (int t = c0; t < c1; ++t) {
    const int a = in_s[t], b = in_s[mirror_idx(t, n)];
    out.wfull[t] = 0.5f * (float)(a + b);
    out.vfull[t] = 0.5f * (float)(a - b);
    nu += (a | b);
    nd += (a != b);
  }
  int totu, totd;
  int pu = block_excl_scan(nu, wsum, &totu);
  int pd = block_excl_scan(nd, wsum, &totd);
  for (int t = c0; t < c1; ++t) {
    const int a = in_s[t], b = in_s[mirror_idx(t, n)];
    if (a | b) { out.ulist[pu] = t; out.uw[pu] = 0.5f * (float)(a + b); ++pu; }
    if (a != b) { out.dlist[pd] = t; out.dv[pd] = 0.5f * (float)(a - b); ++pd; }
  }
  if (threadIdx.x == 0) {
    out.counts[0] = totu;
    out.counts[1] = totd;
  }
}

// ============================================================================ host launchers
#define AMM_DISPATCH_POW2(n, EXPR)                      \
  switch (n) {                                          \
    case 16: { constexpr int NN = 16; EXPR; }           \
    case 32: { constexpr int NN = 32; EXPR; }           \
    case 64: { constexpr int NN = 64; EXPR; }           \
    case 128: { constexpr int NN = 128; EXPR; }         \
    case 256: { constexpr int NN = 256; EXPR; }         \
    case 512: { constexpr int NN = 512; EXPR; }         \
    case 1024: { constexpr int NN = 1024; EXPR; }       \
    case 2048: { constexpr int NN = 2048; EXPR; }       \
    case 4096: { constexpr int NN = 4096; EXPR; }       \
    case 8192: { constexpr int NN = 8192; EXPR; }       \
    case 16384: { constexpr int NN = 16384; EXPR; }     \
    default: break;                                     \
  }

// ---------------------------------------------------------------------------- autotuner table
static bool cd_tune_parse(const char* text, bool (*length_ok)(int64_t));
// The table persists across processes through the text file named by the environment variable
// AMM_TUNE_CACHE: the first lookup loads it (a file that does not parse is ignored), and every
// newly timed choice rewrites it (written to a temporary name, then renamed).
namespace {
std::mutex g_tune_mu;
std::unordered_map<int, int> g_tune;
std::once_flag g_tune_loaded;

const char* tune_cache_path() {
  const char* p = std::getenv("AMM_TUNE_CACHE");
  return (p && *p) ? p : nullptr;
}

void tune_cache_load() {
  const char* path = tune_cache_path();
  if (!path) return;
  std::ifstream f(path);
  if (!f) return;
  std::string text((std::istreambuf_iterator<char>(f)), std::istreambuf_iterator<char>());
  cd_tune_parse(text.c_str(), cd_fft_length_ok);
}
}  // namespace

int cd_tune_get(int key) {
  std::call_once(g_tune_loaded, tune_cache_load);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune.find(key);
  return it == g_tune.end() ? -1 : it->second;
}

void cd_tune_set(int key, int variant) {
  std::call_once(g_tune_loaded, tune_cache_load);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = variant;
  }
  if (const char* path = tune_cache_path()) {
    const std::string tmp = std::string(path) + ".tmp";
    {
      std::ofstream f(tmp, std::ios::trunc);
      f << cd_tune_dump();
    }
    std::rename(tmp.c_str(), path);
  }
}

// The table as text: a header line, then "key variant" per line in ascending key order.
std::string cd_tune_dump() {
  std::call_once(g_tune_loaded, tune_cache_load);
  std::vector<std::pair<int, int>> v;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    v.assign(g_tune.begin(), g_tune.end());
  }
  std::sort(v.begin(), v.end());
  std::string out = "amm-autotune 1\n";
  for (const auto& kv : v) out += std::to_string(kv.first) + " " + std::to_string(kv.second) + "\n";
  return out;
}

// Parse text written by cd_tune_dump; every entry is checked before any is installed.  A key is
// kernel << 24 | N << 3 | flags (tune.cuh): kernel 0, the spectral apply, with flags (direction,
// reversed pairing, element type); kernel 1, the inverse cycle transform, with flag 1 for its
// accumulating form; kernels 2-3 (column and row backward spectra) with flags 0.  The variant is
// 0 or 1.
static bool cd_tune_parse(const char* text, bool (*length_ok)(int64_t));

bool cd_tune_load(const char* text, bool (*length_ok)(int64_t)) {
  std::call_once(g_tune_loaded, tune_cache_load);
  return cd_tune_parse(text, length_ok);
}

static bool cd_tune_parse(const char* text, bool (*length_ok)(int64_t)) {
  std::istringstream in(text);
  std::vector<std::string> tok;
  for (std::string t; in >> t;) tok.push_back(t);
  if (tok.size() < 2 || tok[0] != "amm-autotune" || tok[1] != "1" || tok.size() % 2 != 0) return false;
  // a whole token of decimal digits, at most 10 of them
  auto integer = [](const std::string& t, long long* out) {
    if (t.empty() || t.size() > 10) return false;
    long long x = 0;
    for (char c : t) {
      if (c < '0' || c > '9') return false;
      x = x * 10 + (c - '0');
    }
    *out = x;
    return true;
  };
  std::vector<std::pair<int, int>> v;
  for (size_t i = 2; i < tok.size(); i += 2) {
    long long key, var;
    if (!integer(tok[i], &key) || !integer(tok[i + 1], &var)) return false;
    const long long kid = key >> 24, n = (key >> 3) & 0x1FFFFF, flags = key & 7;
    const long long max_flags = kid == TUNE_APPLY ? 7 : kid == TUNE_RESIDUAL ? 1 : 0;
    if (kid > TUNE_BW_ROW || flags > max_flags || !length_ok(n) || (var != 0 && var != 1))
      return false;
    v.emplace_back((int)key, (int)var);
  }
  std::lock_guard<std::mutex> lk(g_tune_mu);
  for (const auto& kv : v) g_tune[kv.first] = kv.second;
  return true;
}

int cd_cols_per_cta(int n) { return n >= 16384 ? 2 : n >= 6144 ? 4 : 8; }

cudaError_t cd_twiddles(float2* tw, int n, cudaStream_t st) {
  AMM_TRACE("twiddle", st);
  twiddle_kernel<<<(n + 255) / 256, 256, 0, st>>>(tw, n);
  return cudaGetLastError();
}

cudaError_t cd_spectrum(int n, const void* A, int64_t lda, bool bf16, const float2* tw, float2* R, float* kpart,
                        cudaStream_t st) {
  const int J = cd_cols_per_cta(n);
  AMM_TRACE_W("cd_spectrum", st, 0.0,
              (double)n * n * (bf16 ? 2 : 4) + (n / 2 + 1.0) * n * 8 + (double)(n / J) * (n / 2 + 1) * 4, nullptr);
  AMM_DISPATCH_POW2(n, return CdOps<NN>::spectrum(A, lda, bf16, tw, R, kpart, st));
  if (cd_r3_length(n)) return cd_spectrum_r3(n, A, lda, bf16, tw, R, kpart, st);
  return cd_spectrum_any(n, A, lda, bf16, R, kpart, st);
}

cudaError_t cd_keys(int kh, const float* kpart, int nparts, double* key2, cudaStream_t st) {
  AMM_TRACE("cd_keyreduce", st);
  cd_keyreduce_kernel<<<(kh + 31) / 32, dim3(32, 32), 0, st>>>(kpart, nparts, kh, key2, nullptr, 0, 0);
  return cudaGetLastError();
}

cudaError_t cd_select(int n, int k, const float* kpart, int nparts, const int32_t* forced, const SelectOut& o,
                      cudaStream_t st, bool mirror, bool pair_closed) {
  auto bytes = [](int nn) {
    return (size_t)nn * (sizeof(double) + 1) + 8 + (size_t)SEL_SORT_MAX * (sizeof(double) + sizeof(int32_t));
  };
  static DeviceOnce once;
  const cudaError_t attr = once([&] {
    return cudaFuncSetAttribute((const void*)cd_select_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)bytes(16384));
  });
  if (attr != cudaSuccess) return attr;
  const int kh = mirror ? n / 2 + 1 : n;
  {
    AMM_TRACE("cd_keyreduce", st);
    cd_keyreduce_kernel<<<(kh + 31) / 32, dim3(32, 32), 0, st>>>(kpart, nparts, kh, o.key2, o.keys, n, mirror ? 1 : 0);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  AMM_TRACE("cd_select", st);
  cd_select_kernel<<<1, SEL_T, bytes(n), st>>>(o.key2, n, k, forced, o, mirror ? 1 : 0, mirror ? (double)n : 1.0,
                                                (mirror && pair_closed) ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t cd_eigen(int n, const float2* R, const float2* tw, const int32_t* list, const float* coef,
                     const int32_t* count, int cap, int imag_coef, float2* L, cudaStream_t st) {
  if (!R || !L) return cudaErrorInvalidValue;
  AMM_TRACE("cd_eigen", st);
  AMM_DISPATCH_POW2(n, return CdOps<NN>::eigen(R, tw, list, coef, count, cap, imag_coef, L, st));
  if (cd_r3_length(n)) return cd_eigen_r3(n, R, tw, list, coef, count, cap, imag_coef, L, st);
  return cd_eigen_any(n, R, list, coef, count, cap, imag_coef, L, st);
}

cudaError_t cd_residual(int n, const float2* R, const float2* tw, const float* g, int mode, const int32_t* dcount,
                        float* X, cudaStream_t st, int64_t ldx, int accumulate, const int32_t* dcount2) {
  if (!R || !X) return cudaErrorInvalidValue;  // e.g. a released spectrum (store_spectra = 0) not recomputed
  if (ldx <= 0) ldx = n;
  AMM_TRACE_W(mode == 0 ? "cd_residual" : (mode == 1 ? "cd_residual_imag" : "cd_project"), st, 0.0,
              (mode & 1) ? 0.0 : (n / 2 + 1.0) * n * 8 + (double)n * n * 4 * (accumulate ? 2 : 1), nullptr);
  AMM_DISPATCH_POW2(n, return CdOps<NN>::residual(R, tw, g, mode, dcount, dcount2, X, ldx, accumulate, st));
  if (cd_r3_length(n)) return cd_residual_r3(n, R, tw, g, mode, dcount, dcount2, X, ldx, accumulate, st);
  return cd_residual_any(n, R, g, mode, dcount, dcount2, X, ldx, accumulate, st);
}

// ============================================================================ direct inverse cycle transform
// The dense sum of a few listed components, without FFTs:
//   X(r, c) (+)= sum_{u < count} Re(g'_u r_{j, t_u} omega^{t_u c}),   j = (r - c) mod n,
// with r_{j, t} = R[t][j] (row n - t conjugated for t > n/2) and omega = e^{+2 pi i/n} (the inverse
// transform of Alg. 2's spectrum, term by term).  g'_u by mode as in cd_residual: 0 -> -w_u added
// to the operand A itself (A - sum w comp = the residual of (1 - w)), 1 -> -i v_u, 2 -> w_u,
// 3 -> +i v_u.  A CTA takes RD_ROWS rows x 256 columns: the cycles j = r - c it meets form one
// window of 256 + RD_ROWS - 1 consecutive j per listed component, staged in shared memory (each
// spectrum value then serves up to RD_ROWS outputs), and a thread takes one column, so each
// omega^{t c} serves all of its rows.  Gates as cd_residual: odd modes write nothing when *dcount
// is zero, every mode when *dcount2 is zero.
constexpr int RD_ROWS = 16;
constexpr int RD_MAX_U = 18;  // 2k at most: the direct form is taken for k <= 9
constexpr int RD_WIN = 256 + RD_ROWS - 1;

template <typename T>
__global__ void __launch_bounds__(256) cd_resid_direct_kernel(int n, const float2* __restrict__ R,
                                                              const float2* __restrict__ tw,
                                                              const int32_t* __restrict__ list,
                                                              const float* __restrict__ coef,
                                                              const int32_t* __restrict__ count, int mode,
                                                              const T* __restrict__ A, int64_t lda,
                                                              float* __restrict__ X, int64_t ldx, int accumulate,
                                                              const int32_t* __restrict__ dcount,
                                                              const int32_t* __restrict__ dcount2) {
  __shared__ float2 s_r[RD_MAX_U][RD_WIN];  // s_r[u][w] = r_{j0 + w, t_u} (conjugated for t_u > n/2)
  __shared__ int s_t[RD_MAX_U];
  __shared__ float s_g[RD_MAX_U];
  if ((mode & 1) && dcount != nullptr && *dcount == 0) return;
  if (dcount2 != nullptr && *dcount2 == 0) return;
  const int cnt = min(*count, RD_MAX_U);
  const int c0 = blockIdx.x * 256, r0 = blockIdx.y * RD_ROWS;
  const int c = c0 + threadIdx.x;
  // the column's base values first (A for the residual, X when accumulating), all loads in flight
  // together and overlapping the staging below; the listed terms are then added to them
  float acc[RD_ROWS];
#pragma unroll
  for (int i = 0; i < RD_ROWS; ++i) {
    const int r = r0 + i;
    float v = 0.f;
    if (c < n && r < n) {
      if (mode == 0) v = ld_as_float<T>(A + (int64_t)r * lda + c);
      else if (accumulate) v = X[(int64_t)r * ldx + c];
    }
    acc[i] = v;
  }
  const int j0 = (((r0 - c0 - 255) % n) + n) % n;  // the smallest r - c of the tile, mod n
  if (threadIdx.x < cnt) {
    s_t[threadIdx.x] = __ldg(list + threadIdx.x);
    s_g[threadIdx.x] = __ldg(coef + threadIdx.x);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < cnt * RD_WIN; e += 256) {
    const int u = e / RD_WIN, w = e - u * RD_WIN;
    const int t = s_t[u];
    const bool mir = t > n / 2;
    const int j = (j0 + w) % n;
    float2 v = __ldg(R + (int64_t)(mir ? n - t : t) * n + j);
    if (mir) v.y = -v.y;
    s_r[u][w] = v;
  }
  __syncthreads();
  if (c >= n) return;
  const bool p2 = (n & (n - 1)) == 0;
  for (int u = 0; u < cnt; ++u) {
    const int t = s_t[u];
    const float g = s_g[u];
    // e^{-2 pi i t c/n} (omega^{t c} is its conjugate); t c < n^2 <= 2^28: 32-bit index arithmetic
    const unsigned tc = (unsigned)t * (unsigned)c;
    const float2 w = __ldg(tw + (p2 ? (tc & (unsigned)(n - 1)) : tc % (unsigned)n));
    const float2* rw = s_r[u] + (255 - threadIdx.x);  // row r0 + i meets window entry 255 - tid + i
    // z = v conj(w): Re z = v.x w.x + v.y w.y, Im z = v.y w.x - v.x w.y; even modes add g' Re z,
    // odd modes Re(-+ i v z) = +- v Im z
    if (mode & 1) {
      const float gx = (mode == 1 ? g : -g) * w.x, gy = (mode == 1 ? g : -g) * w.y;
#pragma unroll
      for (int i = 0; i < RD_ROWS; ++i) acc[i] = fmaf(rw[i].y, gx, fmaf(-rw[i].x, gy, acc[i]));
    } else {
      const float gx = (mode == 0 ? -g : g) * w.x, gy = (mode == 0 ? -g : g) * w.y;
#pragma unroll
      for (int i = 0; i < RD_ROWS; ++i) acc[i] = fmaf(rw[i].x, gx, fmaf(rw[i].y, gy, acc[i]));
    }
  }
#pragma unroll
  for (int i = 0; i < RD_ROWS; ++i) {
    const int r = r0 + i;
    if (r >= n) break;
    X[(int64_t)r * ldx + c] = acc[i];
  }
}

bool cd_residual_direct_ok(int64_t k) { return 2 * k <= RD_MAX_U; }

cudaError_t cd_residual_direct(int n, const float2* R, const float2* tw, const int32_t* list, const float* coef,
                               const int32_t* count, int mode, const void* A, int64_t lda, bool bf16, float* X,
                               int64_t ldx, int accumulate, const int32_t* dcount, const int32_t* dcount2,
                               cudaStream_t st) {
  if (!R || !X || !tw || (mode == 0 && !A)) return cudaErrorInvalidValue;
  if (ldx <= 0) ldx = n;
  AMM_TRACE_W(mode == 0 ? "cd_residual_direct" : (mode == 1 ? "cd_residual_imag_direct" : "cd_project_direct"), st, 0.0,
              (mode & 1) ? 0.0 : (double)n * n * 4 * (accumulate || mode == 0 ? 2 : 1), nullptr);
  const dim3 grid((unsigned)((n + 255) / 256), (unsigned)((n + RD_ROWS - 1) / RD_ROWS));
  if (bf16)
    cd_resid_direct_kernel<__nv_bfloat16><<<grid, 256, 0, st>>>(n, R, tw, list, coef, count, mode,
                                                               (const __nv_bfloat16*)A, lda, X, ldx, accumulate,
                                                               dcount, dcount2);
  else
    cd_resid_direct_kernel<float><<<grid, 256, 0, st>>>(n, R, tw, list, coef, count, mode, (const float*)A, lda, X,
                                                        ldx, accumulate, dcount, dcount2);
  return cudaGetLastError();
}

cudaError_t cd_apply(int n, bool row, const void* X, int64_t ldx, bool bf16, int64_t nvec, const float2* tw,
                     const int32_t* list, const float2* Lc, const int32_t* count, const int32_t* gate0,
                     const int32_t* gate1, float* out, int64_t ldo, int accumulate, cudaStream_t st, int rev) {
  // work: 8 flops per complex MAC, n frequencies x nvec/2 packed signals per applied component
  AMM_TRACE_W(gate0 ? "cd_apply_unpaired" : (row ? "cd_apply_row" : "cd_apply_col"), st, 4.0 * n * (double)nvec,
              (double)n * nvec * (bf16 ? 2 : 4) + (double)n * nvec * 4 * (accumulate ? 2 : 1), count);
  AMM_DISPATCH_POW2(n, return CdOps<NN>::apply(row, X, ldx, bf16, nvec, tw, list, Lc, count, gate0, gate1, out,
                                               ldo, accumulate, rev, st));
  if (cd_r3_length(n))
    return cd_apply_r3(n, row, X, ldx, bf16, nvec, tw, list, Lc, count, gate0, gate1, out, ldo, accumulate, rev, st);
  return cd_apply_any(n, row, X, ldx, bf16, nvec, list, Lc, count, gate0, gate1, out, ldo, accumulate, rev, st);
}

}  // namespace amm
