// C ABI of libamm (include/amm.h): argument checking, handle ownership, launch order.
// Every step of the numerical path runs in the kernels of circulant.cu / svd.cu; this
// file only validates, allocates (stream-ordered) and launches.
#include <cuda_runtime.h>

#include <cmath>

#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <set>
#include <utility>
#include <vector>

#include "../../include/amm.h"
#include "api_internal.h"
#include "kernels.h"

using namespace amm;

// ----------------------------------------------------------------------------- errors
static thread_local char g_last_error[512] = "";

amm_status_t amm::fail(amm_status_t s, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
  va_end(ap);
  return s;
}

amm_status_t amm::cuda_fail(cudaError_t e, const char* what) {
  if (e == cudaErrorMemoryAllocation) return fail(AMM_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
  return fail(AMM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// ----------------------------------------------------------------------------- allocation
static std::atomic<int> g_fail_after{0};

cudaError_t amm::dev_alloc(void** p, size_t bytes, cudaStream_t st) {
  int f = g_fail_after.load();
  if (f > 0) {
    if (f == 1) {
      g_fail_after.store(0);
      *p = nullptr;
      return cudaErrorMemoryAllocation;
    }
    g_fail_after.store(f - 1);
  }
  if (bytes == 0) bytes = 16;
  return cudaMallocAsync(p, bytes, st);
}

void amm::dev_free(void* p, cudaStream_t st) {
  if (p) cudaFreeAsync(p, st);
}

// Per (device, n) twiddle table e^{-2 pi i m/n}, built once and kept for the process.
static std::mutex g_tw_mu;
static std::map<std::pair<int, int>, float2*> g_tw;

cudaError_t amm::twiddles(int n, cudaStream_t st, const float2** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(g_tw_mu);
  auto it = g_tw.find({dev, n});
  if (it != g_tw.end()) {
    *out = it->second;
    return cudaSuccess;
  }
  float2* tw = nullptr;
  e = cudaMalloc(&tw, sizeof(float2) * (size_t)n);
  if (e != cudaSuccess) return e;
  e = cd_twiddles(tw, n, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaFree(tw);
    return e;
  }
  g_tw[{dev, n}] = tw;
  *out = tw;
  return cudaSuccess;
}

// ----------------------------------------------------------------------------- small public calls
extern "C" const char* amm_status_string(amm_status_t s) {
  switch (s) {
    case AMM_OK: return "AMM_OK";
    case AMM_ERR_INVALID_ARG: return "AMM_ERR_INVALID_ARG";
    case AMM_ERR_UNSUPPORTED_SIZE: return "AMM_ERR_UNSUPPORTED_SIZE";
    case AMM_ERR_OOM: return "AMM_ERR_OOM";
    case AMM_ERR_CUDA: return "AMM_ERR_CUDA";
    case AMM_ERR_TIMEOUT: return "AMM_ERR_TIMEOUT";
    case AMM_ERR_STATE: return "AMM_ERR_STATE";
    case AMM_ERR_NOT_IMPLEMENTED: return "AMM_ERR_NOT_IMPLEMENTED";
  }
  return "AMM_ERR_UNKNOWN";
}

extern "C" const char* amm_last_error(void) { return g_last_error; }
extern "C" int32_t amm_version(void) { return AMM_VERSION; }

extern "C" amm_status_t amm_opts_init(amm_opts_t* o) {
  if (!o) return fail(AMM_ERR_INVALID_ARG, "amm_opts_init: opts is NULL");
  memset(o, 0, sizeof(*o));
  o->struct_size = sizeof(amm_opts_t);
  o->role = AMM_LEFT;
  o->compute = AMM_F32;
  o->store_spectra = 1;
  return AMM_OK;
}

namespace {
std::atomic<bool> g_autotune{false};
}
bool amm::amm_autotune_enabled() { return g_autotune.load(); }

extern "C" amm_status_t amm_autotune_export(char* host_buf, int64_t cap, int64_t* len) {
  if (!host_buf || !len) return fail(AMM_ERR_INVALID_ARG, "amm_autotune_export: NULL argument");
  const std::string t = cd_tune_dump();
  *len = (int64_t)t.size();
  if (cap < (int64_t)t.size() + 1)
    return fail(AMM_ERR_INVALID_ARG, "amm_autotune_export: cap=%lld < %lld", (long long)cap,
                (long long)t.size() + 1);
  memcpy(host_buf, t.c_str(), t.size() + 1);
  return AMM_OK;
}

extern "C" amm_status_t amm_autotune_import(const char* host_text) {
  if (!host_text) return fail(AMM_ERR_INVALID_ARG, "amm_autotune_import: NULL argument");
  if (!cd_tune_load(host_text, cd_fft_length_ok))
    return fail(AMM_ERR_INVALID_ARG, "amm_autotune_import: malformed table (nothing installed)");
  return AMM_OK;
}

extern "C" amm_status_t amm_set_autotune(int32_t on) {
  g_autotune.store(on != 0);
  return AMM_OK;
}

extern "C" amm_status_t amm_debug_fail_alloc_after(int32_t n) {
  if (n < 0) return fail(AMM_ERR_INVALID_ARG, "amm_debug_fail_alloc_after: n < 0");
  g_fail_after.store(n);
  return AMM_OK;
}

// ----------------------------------------------------------------------------- handles
static bool pow2(int64_t n) { return n > 0 && (n & (n - 1)) == 0; }
bool amm::cyc_length_ok(int64_t n) { return n >= 16 && n <= 8192 && n % 4 == 0; }
bool amm::cd_fft_length_ok(int64_t n) {
  return (pow2(n) && n >= 16 && n <= 16384) || (n % 3 == 0 && pow2(n / 3) && n >= 48 && n <= 6144);
}
bool amm::cd_length_ok(int64_t n) { return cd_fft_length_ok(n) || cd_any_length_ok(n); }

void amm::Handle::release() {
  for (amm_handle* b : blk.sub) {
    b->release();
    delete b;
  }
  blk.sub.clear();
  for (void* p : owned) dev_free(p, stream);
  owned.clear();
  owned_bytes.clear();
}

cudaError_t amm::Handle::alloc(void** p, size_t bytes) {
  cudaError_t e = dev_alloc(p, bytes, stream);
  if (e == cudaSuccess) {
    owned.push_back(*p);
    owned_bytes.push_back(bytes);
  }
  return e;
}

void amm::Handle::release_one(void* p) {
  for (size_t i = 0; i < owned.size(); ++i)
    if (owned[i] == p) {
      dev_free(p, stream);
      owned.erase(owned.begin() + i);
      owned_bytes.erase(owned_bytes.begin() + i);
      return;
    }
}

int64_t amm::Handle::device_bytes() const {
  int64_t s = 0;
  for (size_t b : owned_bytes) s += (int64_t)b;
  for (const amm_handle* b : blk.sub) s += b->device_bytes();
  return s;
}

cudaError_t amm::cd_spectrum_of(Handle* h, const float2** R, float2** temp, cudaStream_t st) {
  *temp = nullptr;
  if (h->cd.R) {
    *R = h->cd.R;
    return cudaSuccess;
  }
  const int n = (int)h->rows;
  const size_t kh = (size_t)n / 2 + 1;
  float* kpart = nullptr;
  cudaError_t e = dev_alloc((void**)temp, sizeof(float2) * kh * n, st);
  if (e == cudaSuccess) e = dev_alloc((void**)&kpart, sizeof(float) * kh * h->cd.nparts, st);
  if (e == cudaSuccess) e = cd_spectrum(n, h->A, h->lda, h->dtype == AMM_BF16, h->cd.tw, *temp, kpart, st);
  if (kpart) dev_free(kpart, st);
  if (e != cudaSuccess && *temp) {
    dev_free(*temp, st);
    *temp = nullptr;
  }
  *R = *temp;
  return e;
}

// The inverse cycle transform of a circulant handle's listed components (mode as cd_residual; odd
// modes the unpaired set with v, even modes S u S-bar with w): term by term when there are few of
// them (2k <= 18), by FFTs over the whole spectrum otherwise.  Mode 0 reads the operand A itself
// (A - sum w comp) on the direct path.
static cudaError_t resid_of(Handle* h, const float2* R, int mode, const void* A, int64_t lda, bool bf16, float* X,
                            int64_t ldx, int accumulate, const int32_t* dcount, const int32_t* dcount2,
                            cudaStream_t st) {
  auto& c = h->cd;
  const int n = (int)h->rows;
  const bool odd = (mode & 1) != 0;
  if (cd_residual_direct_ok(h->k) && (mode != 0 || A != nullptr))
    return cd_residual_direct(n, R, c.tw, odd ? c.so.dlist : c.so.ulist, odd ? c.so.dv : c.so.uw,
                              c.so.counts + (odd ? 1 : 0), mode, A, lda, bf16, X, ldx, accumulate, dcount, dcount2, st);
  return cd_residual(n, R, c.tw, odd ? c.so.vfull : c.so.wfull, mode, dcount, X, st, ldx, accumulate, dcount2);
}

amm_status_t amm::decompose_circulant(Handle* h, const amm_opts_t* o) {
  const int n = (int)h->rows;
  if (!cd_length_ok(n))
    return fail(AMM_ERR_UNSUPPORTED_SIZE, "circulant: n=%d must be in [16, 4096], or 2^a up to 16384", n);
  auto& c = h->cd;
  const int J = cd_cols_per_cta(n);
  c.nparts = (n + J - 1) / J;
  c.cap = (int)std::min<int64_t>(2 * h->k, n);
  cudaError_t e = twiddles(n, h->stream, &c.tw);
  if (e != cudaSuccess) return cuda_fail(e, "twiddle table");
  const size_t kh = (size_t)n / 2 + 1;
#define AL(ptr, bytes)                                                              \
  do {                                                                              \
    e = h->alloc((void**)&(ptr), (bytes));                                          \
    if (e != cudaSuccess) return cuda_fail(e, "amm_decompose: device allocation");  \
  } while (0)
  AL(c.R, sizeof(float2) * kh * n);
  AL(c.kpart, sizeof(float) * kh * c.nparts);
  AL(c.so.keys, sizeof(double) * n);
  AL(c.so.norms, sizeof(double) * 4);
  AL(c.so.sel, sizeof(int32_t) * h->k);
  AL(c.so.ulist, sizeof(int32_t) * c.cap);
  AL(c.so.uw, sizeof(float) * c.cap);
  AL(c.so.dlist, sizeof(int32_t) * c.cap);
  AL(c.so.dv, sizeof(float) * c.cap);
  AL(c.so.wfull, sizeof(float) * n);
  AL(c.so.vfull, sizeof(float) * n);
  AL(c.so.counts, sizeof(int32_t) * 2);
  AL(c.so.key2, sizeof(double) * n);
  AL(c.Lw, sizeof(float2) * (size_t)c.cap * n);
  AL(c.Ld, sizeof(float2) * (size_t)c.cap * n);
  if (h->role == AMM_RIGHT) {
    AL(c.resid, sizeof(float) * (size_t)n * n);
    AL(c.imag, sizeof(float) * (size_t)n * n);
  }
  int32_t* forced = nullptr;
  if (o && o->forced_selection) {
    std::set<int32_t> seen;
    for (int64_t i = 0; i < h->k; ++i) {
      int32_t t = o->forced_selection[i];
      if (t < 0 || t >= n || !seen.insert(t).second)
        return fail(AMM_ERR_INVALID_ARG, "forced_selection[%lld]=%d out of range or repeated", (long long)i, t);
    }
    AL(forced, sizeof(int32_t) * h->k);
    e = cudaMemcpyAsync(forced, o->forced_selection, sizeof(int32_t) * h->k, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);  // host array may be freed after return
    if (e != cudaSuccess) return cuda_fail(e, "forced selection upload");
  }
#undef AL
  const bool bf16 = h->dtype == AMM_BF16;
  if ((e = cd_spectrum(n, h->A, h->lda, bf16, c.tw, c.R, c.kpart, h->stream)) != cudaSuccess)
    return cuda_fail(e, "cd_spectrum launch");
  const bool closed = o && o->pair_closed;
  if ((e = cd_select(n, (int)h->k, c.kpart, c.nparts, forced, c.so, h->stream, true, closed)) != cudaSuccess)
    return cuda_fail(e, "cd_select launch");
  if ((e = cd_eigen(n, c.R, c.tw, c.so.ulist, c.so.uw, c.so.counts, c.cap, 0, c.Lw, h->stream)) != cudaSuccess)
    return cuda_fail(e, "cd_eigen launch");
  if ((e = cd_eigen(n, c.R, c.tw, c.so.dlist, c.so.dv, c.so.counts + 1, c.cap, 1, c.Ld, h->stream)) != cudaSuccess)
    return cuda_fail(e, "cd_eigen launch");
  if (h->role == AMM_RIGHT) {
    if ((e = resid_of(h, c.R, 0, h->A, h->lda, bf16, c.resid, n, 0, nullptr, nullptr, h->stream)) != cudaSuccess)
      return cuda_fail(e, "cd_residual launch");
    if ((e = resid_of(h, c.R, 1, nullptr, 0, false, c.imag, n, 0, c.so.counts + 1, nullptr, h->stream)) !=
        cudaSuccess)
      return cuda_fail(e, "cd_residual launch");
  }
  if (o && o->store_spectra == 0) {  // the products and the backward do not read R again
    h->release_one(c.R);
    h->release_one(c.kpart);
    c.R = nullptr;
    c.kpart = nullptr;
  }
  return AMM_OK;
}

// BF16 operands of the sparsifiers: the handle keeps an FP32 copy (read once from the caller's
// BF16 matrix) and every kernel of the method runs on it in FP32.
static cudaError_t widen_input(Handle* h) {
  if (h->dtype != AMM_BF16) return cudaSuccess;
  float* y = nullptr;
  cudaError_t e = h->alloc((void**)&y, sizeof(float) * (size_t)h->rows * h->cols);
  if (e == cudaSuccess) e = widen_bf16(h->A, h->rows, h->cols, h->lda, y, h->cols, h->stream);
  if (e != cudaSuccess) return e;
  h->A = y;
  h->lda = h->cols;
  h->dtype = AMM_F32;
  return cudaSuccess;
}

static amm_status_t decompose_cycle(Handle* h, const amm_opts_t* o) {
  const int n = (int)h->rows;
  if (!cyc_length_ok(n))
    return fail(AMM_ERR_UNSUPPORTED_SIZE, "cycle: n=%d must be a multiple of 4 in [16, 8192]", n);
  auto& c = h->cy;
  const int rp = cyc_rows_per_part(n);
  c.nparts = (n + rp - 1) / rp;
  const int cap = (int)std::min<int64_t>(2 * h->k, n);
  cudaError_t e = widen_input(h);
  if (e != cudaSuccess) return cuda_fail(e, "cycle: BF16 input");
#define AL(ptr, bytes)                                                              \
  do {                                                                              \
    e = h->alloc((void**)&(ptr), (bytes));                                          \
    if (e != cudaSuccess) return cuda_fail(e, "amm_decompose: device allocation");  \
  } while (0)
  AL(c.kpart, sizeof(float) * (size_t)c.nparts * n);
  AL(c.so.keys, sizeof(double) * n);
  AL(c.so.norms, sizeof(double) * 4);
  AL(c.so.sel, sizeof(int32_t) * h->k);
  AL(c.so.ulist, sizeof(int32_t) * cap);
  AL(c.so.uw, sizeof(float) * cap);
  AL(c.so.dlist, sizeof(int32_t) * cap);
  AL(c.so.dv, sizeof(float) * cap);
  AL(c.so.wfull, sizeof(float) * n);
  AL(c.so.vfull, sizeof(float) * n);
  AL(c.so.counts, sizeof(int32_t) * 2);
  AL(c.so.key2, sizeof(double) * n);
  AL(c.cyc, sizeof(float) * (size_t)h->k * n);
  AL(c.insel, (size_t)n);
  int32_t* forced = nullptr;
  if (o && o->forced_selection) {
    std::set<int32_t> seen;
    for (int64_t i = 0; i < h->k; ++i) {
      int32_t t = o->forced_selection[i];
      if (t < 0 || t >= n || !seen.insert(t).second)
        return fail(AMM_ERR_INVALID_ARG, "forced_selection[%lld]=%d out of range or repeated", (long long)i, t);
    }
    AL(forced, sizeof(int32_t) * h->k);
    e = cudaMemcpyAsync(forced, o->forced_selection, sizeof(int32_t) * h->k, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "forced selection upload");
  }
#undef AL
  const float* A = (const float*)h->A;
  if ((e = cyc_keys(n, A, h->lda, c.kpart, h->stream)) != cudaSuccess) return cuda_fail(e, "cyc_keys launch");
  if ((e = cd_select(n, (int)h->k, c.kpart, c.nparts, forced, c.so, h->stream, false)) != cudaSuccess)
    return cuda_fail(e, "cycle select launch");
  if ((e = cyc_gather(n, (int)h->k, A, h->lda, c.so.sel, c.cyc, c.insel, h->stream)) != cudaSuccess)
    return cuda_fail(e, "cyc_gather launch");
  return AMM_OK;
}

static amm_status_t decompose_fourier(Handle* h, const amm_opts_t* o) {
  auto& f = h->ft;
  const bool left = h->role == AMM_LEFT;
  f.n = (int)(left ? h->cols : h->rows);
  f.nvec = (int)(left ? h->rows : h->cols);
  if (!cd_fft_length_ok(f.n) || f.n > 8192)
    return fail(AMM_ERR_UNSUPPORTED_SIZE, "fourier: inner dimension %d must be 2^a in [16, 8192] or 3 * 2^a in [48, 6144]",
                f.n);
  if (widen_input(h) != cudaSuccess) return cuda_fail(cudaGetLastError(), "fourier: BF16 input");
  if (o && o->forced_selection) return fail(AMM_ERR_NOT_IMPLEMENTED, "fourier: forced selection is not built");
  if (h->k > f.n) return fail(AMM_ERR_INVALID_ARG, "fourier: k=%lld > n=%d", (long long)h->k, f.n);
  cudaError_t e = twiddles(f.n, h->stream, &f.tw);
  if (e != cudaSuccess) return cuda_fail(e, "twiddle table");
  const size_t kh = (size_t)f.n / 2 + 1;
  f.mask_words = (f.nvec + 31) / 32;
#define AL(ptr, bytes)                                                              \
  do {                                                                              \
    e = h->alloc((void**)&(ptr), (bytes));                                          \
    if (e != cudaSuccess) return cuda_fail(e, "amm_decompose: device allocation");  \
  } while (0)
  AL(f.T, sizeof(float2) * kh * f.nvec);
  AL(f.mag, sizeof(float) * kh * f.nvec);
  AL(f.sel, sizeof(int32_t) * (size_t)h->k * f.nvec);
  if (left) AL(f.TT, sizeof(float2) * kh * f.nvec);
  AL(f.maskT, sizeof(uint32_t) * (size_t)f.n * f.mask_words);
#undef AL
  if ((e = ft_transform(f.n, left, (const float*)h->A, h->lda, f.nvec, f.tw, f.T, f.TT, f.mag, h->stream)) !=
      cudaSuccess)
    return cuda_fail(e, "ft_transform launch");
  if ((e = ft_select(f.n, (int)h->k, f.nvec, f.mag, f.sel, f.maskT, f.mask_words, h->stream)) !=
      cudaSuccess)
    return cuda_fail(e, "ft_select launch");
  return AMM_OK;
}

extern "C" amm_status_t amm_decompose(const void* A, int64_t rows, int64_t cols, int64_t lda, amm_dtype_t dtype,
                                      amm_method_t method, int64_t k, const amm_opts_t* opts, void* stream,
                                      amm_handle_t* out) {
  if (!out) return fail(AMM_ERR_INVALID_ARG, "amm_decompose: out is NULL");
  if (!A) return fail(AMM_ERR_INVALID_ARG, "amm_decompose: A is NULL");
  if (rows <= 0 || cols <= 0) return fail(AMM_ERR_INVALID_ARG, "amm_decompose: empty matrix %lldx%lld",
                                          (long long)rows, (long long)cols);
  if (lda < cols) return fail(AMM_ERR_INVALID_ARG, "amm_decompose: lda=%lld < cols=%lld", (long long)lda,
                              (long long)cols);
  if (dtype != AMM_F32 && dtype != AMM_BF16) return fail(AMM_ERR_INVALID_ARG, "amm_decompose: bad dtype %d", dtype);
  if (opts && opts->struct_size != sizeof(amm_opts_t))
    return fail(AMM_ERR_INVALID_ARG, "amm_decompose: opts->struct_size=%u, expected %zu", opts->struct_size,
                sizeof(amm_opts_t));
  const int role = opts ? opts->role : AMM_LEFT;
  if (role != AMM_LEFT && role != AMM_RIGHT) return fail(AMM_ERR_INVALID_ARG, "amm_decompose: bad role %d", role);
  const int64_t block = opts ? opts->block : 0;
  if (block < 0) return fail(AMM_ERR_INVALID_ARG, "amm_decompose: block=%lld < 0", (long long)block);
  if (block > 0 && method != AMM_CIRCULANT)
    return fail(AMM_ERR_INVALID_ARG, "amm_decompose: block is an option of AMM_CIRCULANT");
  const bool blocked = block > 0 && !(rows == block && cols == block);
  const int64_t kmax = (method == AMM_SVD) ? std::min(rows, cols) : blocked ? block : cols;
  if (k < 1 || k > kmax)
    return fail(AMM_ERR_INVALID_ARG, "amm_decompose: k=%lld outside [1, %lld]", (long long)k, (long long)kmax);
  Handle* h = new (std::nothrow) Handle();
  if (!h) return fail(AMM_ERR_OOM, "amm_decompose: host allocation");
  h->A = A;
  h->rows = rows;
  h->cols = cols;
  h->lda = lda;
  h->dtype = dtype;
  h->method = method;
  h->role = role;
  h->k = k;
  h->stream = (cudaStream_t)stream;
  amm_status_t s;
  switch (method) {
    case AMM_CIRCULANT:
      if (blocked) {
        s = decompose_circulant_blocked(h, opts);
        break;
      }
      if (rows != cols) {
        s = fail(AMM_ERR_UNSUPPORTED_SIZE, "circulant: matrix must be square (got %lldx%lld; set opts.block)",
                 (long long)rows, (long long)cols);
        break;
      }
      s = decompose_circulant(h, opts);
      break;
    case AMM_SVD:
      s = decompose_svd(h, opts);
      break;
    case AMM_SPARSE_CYCLE:
      if (rows != cols) {
        s = fail(AMM_ERR_UNSUPPORTED_SIZE, "cycle: matrix must be square (got %lldx%lld)", (long long)rows,
                 (long long)cols);
        break;
      }
      s = decompose_cycle(h, opts);
      break;
    case AMM_SPARSE_FOURIER:
      s = decompose_fourier(h, opts);
      break;
    default:
      s = fail(AMM_ERR_INVALID_ARG, "amm_decompose: bad method %d", (int)method);
  }
  if (s != AMM_OK) {
    h->release();
    delete h;
    return s;
  }
  *out = h;
  return AMM_OK;
}

static amm_status_t check_pair(Handle* a, Handle* b) {
  if (!a || !b) return fail(AMM_ERR_INVALID_ARG, "NULL handle");
  if (a->role != AMM_LEFT || b->role != AMM_RIGHT)
    return fail(AMM_ERR_STATE, "hA must have role LEFT and hB role RIGHT (got %d, %d)", a->role, b->role);
  if (a->cols != b->rows)
    return fail(AMM_ERR_STATE, "inner dimensions differ: A is %lldx%lld, B is %lldx%lld", (long long)a->rows,
                (long long)a->cols, (long long)b->rows, (long long)b->cols);
  return AMM_OK;
}

// Re M = A~_w dB_w  +  Y V  +  A B~_w for one square pair (Alg. 3's two terms in the column /
// row spectral form); acc = 1 adds the product to C.
cudaError_t amm::cd_first_order(Handle* a, Handle* b, float* C, int64_t ldc, int acc, cudaStream_t st) {
  const int n = (int)a->rows;
  auto &ca = a->cd, &cb = b->cd;
  cudaError_t e = cd_apply(n, false, cb.resid, n, false, n, ca.tw, ca.so.ulist, ca.Lw, ca.so.counts, nullptr,
                           nullptr, C, ldc, acc, st);
  if (e == cudaSuccess)
    e = cd_apply(n, false, cb.imag, n, false, n, ca.tw, ca.so.dlist, ca.Ld, ca.so.counts + 1, ca.so.counts + 1,
                 cb.so.counts + 1, C, ldc, 1, st);
  if (e == cudaSuccess)
    e = cd_apply(n, true, a->A, a->lda, a->dtype == AMM_BF16, n, ca.tw, cb.so.ulist, cb.Lw, cb.so.counts, nullptr,
                 nullptr, C, ldc, 1, st);
  return e;
}

extern "C" amm_status_t amm_approx_matmul(amm_handle_t hA, amm_handle_t hB, float* C, int64_t ldc, void* stream) {
  Handle* a = hA;
  Handle* b = hB;
  amm_status_t s = check_pair(a, b);
  if (s != AMM_OK) return s;
  if (!C) return fail(AMM_ERR_INVALID_ARG, "amm_approx_matmul: C is NULL");
  if (ldc < b->cols) return fail(AMM_ERR_INVALID_ARG, "amm_approx_matmul: ldc=%lld < %lld", (long long)ldc,
                                 (long long)b->cols);
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e;
  if (a->method != b->method) return mixed_matmul(a, b, C, ldc, st);
  if (a->method == AMM_CIRCULANT) {
    if (a->blk.b || b->blk.b) return blocked_matmul(a, b, C, ldc, st);
    if ((e = cd_first_order(a, b, C, ldc, 0, st)) != cudaSuccess) return cuda_fail(e, "circulant product launch");
    return AMM_OK;
  }
  if (a->method == AMM_SVD) return svd_matmul(a, b, C, ldc, st);
  if (a->method == AMM_SPARSE_FOURIER) {
    e = ft_product(a->ft.n, (int)a->rows, (int)b->cols, (int)a->k, (int)b->k, a->ft.T, a->ft.TT, a->ft.sel,
                   a->ft.maskT, a->ft.mask_words, b->ft.T, b->ft.sel, C, ldc, st);
    if (e != cudaSuccess) return cuda_fail(e, "fourier product launch");
    return AMM_OK;
  }
  if (a->method == AMM_SPARSE_CYCLE) {
    const int n = (int)a->rows;
    e = cyc_apply(n, (const float*)a->A, a->lda, (const float*)b->A, b->lda, a->cy.so.sel, (int)a->k, a->cy.cyc,
                  a->cy.insel, b->cy.so.sel, (int)b->k, b->cy.cyc, C, ldc, st);
    if (e != cudaSuccess) return cuda_fail(e, "cycle product launch");
    return AMM_OK;
  }
  return fail(AMM_ERR_NOT_IMPLEMENTED, "method %d", a->method);
}

// Circulant backward (see cd_backward.cu for the formulas); every step is a kernel launch.
amm_status_t amm::cd_backward(Handle* a, Handle* b, const float* G, int64_t ldg, float* dA, int64_t ldda, int acc_a,
                              float* dB, int64_t lddb, int acc_b, cudaStream_t st) {
  const int n = (int)a->rows;
  auto &ca = a->cd, &cb = b->cd;
  const float2* tw = ca.tw;
  const size_t kh = (size_t)n / 2 + 1;
  std::vector<void*> tmp;
  cudaError_t e = cudaSuccess;
  auto al = [&](size_t bytes) -> void* {
    void* q = nullptr;
    if (e == cudaSuccess) e = dev_alloc(&q, bytes, st);
    if (q) tmp.push_back(q);
    return q;
  };
  float2* X1 = (float2*)al(sizeof(float2) * kh * n);
  float2* X2 = (float2*)al(sizeof(float2) * kh * n);
  float2* RX = (float2*)al(sizeof(float2) * kh * n);
  float2* K = (float2*)al(sizeof(float2) * (size_t)std::max(ca.cap, cb.cap) * n);
  float* T = dB ? (float*)al(sizeof(float) * (size_t)n * n) : nullptr;
#define STEP(x) \
  if (e == cudaSuccess) e = (x)
  if (dA) {
    // G B~_w^T (rows of G, coefficient L^B_s(p)), then the projection terms of G dB^T
    STEP(cd_apply(n, true, G, ldg, false, n, tw, cb.so.ulist, cb.Lw, cb.so.counts, nullptr, nullptr, dA, ldda, acc_a,
                  st, 0));
    STEP(bw_spectrum(n, false, G, ldg, tw, X1, st));
    STEP(bw_spectrum(n, false, cb.resid, n, tw, X2, st));
    STEP(cd_sddmm(n, X1, X2, ca.so.ulist, ca.so.counts, ca.cap, K, nullptr, nullptr, st));
    STEP(cd_rho(n, K, tw, ca.so.ulist, ca.so.counts, ca.cap, RX, nullptr, nullptr, st));
    STEP(resid_of(a, RX, 2, nullptr, 0, false, dA, ldda, 1, nullptr, nullptr, st));
    // unpaired: (i v_t) R_t(G V_B^T) D^t, only when both selections split a pair (device gates)
    STEP(bw_spectrum(n, false, cb.imag, n, tw, X2, st, ca.so.counts + 1, cb.so.counts + 1));
    STEP(cd_sddmm(n, X1, X2, ca.so.dlist, ca.so.counts + 1, ca.cap, K, ca.so.counts + 1, cb.so.counts + 1, st));
    STEP(cd_rho(n, K, tw, ca.so.dlist, ca.so.counts + 1, ca.cap, RX, ca.so.counts + 1, cb.so.counts + 1, st));
    STEP(resid_of(a, RX, 3, nullptr, 0, false, dA, ldda, 1, ca.so.counts + 1, cb.so.counts + 1, st));
  }
  // the dense dA_w and Im A~ below come from A's half spectrum: the stored one, or (store_spectra = 0)
  // computed again from A
  const float2* RA = nullptr;
  float2* RA_temp = nullptr;
  if (dB && e == cudaSuccess) e = cd_spectrum_of(a, &RA, &RA_temp, st);
  if (RA_temp) tmp.push_back(RA_temp);
  if (dB) {
    // A~_w^T G (columns of G, coefficient L^A_t(t - p)), then the projection terms of dA^T G
    STEP(cd_apply(n, false, G, ldg, false, n, tw, ca.so.ulist, ca.Lw, ca.so.counts, nullptr, nullptr, dB, lddb, acc_b,
                  st, 1));
    STEP(bw_spectrum(n, true, G, ldg, tw, X1, st));
    STEP(resid_of(a, RA, 0, a->A, a->lda, a->dtype == AMM_BF16, T, n, 0, nullptr, nullptr, st));  // dA_w
    STEP(bw_spectrum(n, true, T, n, tw, X2, st));
    STEP(cd_sddmm(n, X2, X1, cb.so.ulist, cb.so.counts, cb.cap, K, nullptr, nullptr, st));
    STEP(cd_rho(n, K, tw, cb.so.ulist, cb.so.counts, cb.cap, RX, nullptr, nullptr, st));
    STEP(resid_of(b, RX, 2, nullptr, 0, false, dB, lddb, 1, nullptr, nullptr, st));
    // unpaired: (i v_s) R_s(Y_A^T G) D^s with Y_A = Im A~
    STEP(resid_of(a, RA, 1, nullptr, 0, false, T, n, 0, ca.so.counts + 1, cb.so.counts + 1, st));
    STEP(bw_spectrum(n, true, T, n, tw, X2, st, ca.so.counts + 1, cb.so.counts + 1));
    STEP(cd_sddmm(n, X2, X1, cb.so.dlist, cb.so.counts + 1, cb.cap, K, ca.so.counts + 1, cb.so.counts + 1, st));
    STEP(cd_rho(n, K, tw, cb.so.dlist, cb.so.counts + 1, cb.cap, RX, ca.so.counts + 1, cb.so.counts + 1, st));
    STEP(resid_of(b, RX, 3, nullptr, 0, false, dB, lddb, 1, cb.so.counts + 1, ca.so.counts + 1, st));
  }
#undef STEP
  for (void* q : tmp) dev_free(q, st);
  if (e != cudaSuccess) return cuda_fail(e, "circulant backward");
  return AMM_OK;
}

extern "C" amm_status_t amm_approx_matmul_backward(amm_handle_t hA, amm_handle_t hB, const float* dC, int64_t lddc,
                                                   float* dA, int64_t ldda, float* dB, int64_t lddb, void* stream) {
  Handle* a = hA;
  Handle* b = hB;
  amm_status_t s = check_pair(a, b);
  if (s != AMM_OK) return s;
  if (!dC) return fail(AMM_ERR_INVALID_ARG, "backward: dC is NULL");
  if (lddc < b->cols || (dA && ldda < a->cols) || (dB && lddb < b->cols))
    return fail(AMM_ERR_INVALID_ARG, "backward: leading dimension too small");
  if (a->method != b->method) return mixed_backward(a, b, dC, lddc, dA, ldda, dB, lddb, (cudaStream_t)stream);
  if (a->method == AMM_SVD) return svd_backward(a, b, dC, lddc, dA, ldda, dB, lddb, (cudaStream_t)stream);
  if (a->method == AMM_CIRCULANT) {
    if (a->blk.b || b->blk.b) return blocked_backward(a, b, dC, lddc, dA, ldda, dB, lddb, (cudaStream_t)stream);
    return cd_backward(a, b, dC, lddc, dA, ldda, 0, dB, lddb, 0, (cudaStream_t)stream);
  }
  if (a->method == AMM_SPARSE_CYCLE) {
    cudaError_t e = cyc_backward((int)a->rows, (const float*)a->A, a->lda, (const float*)b->A, b->lda, a->cy.so.sel,
                                 (int)a->k, a->cy.cyc, a->cy.insel, b->cy.so.sel, (int)b->k, b->cy.cyc, b->cy.insel,
                                 dC, lddc, dA, ldda, dB, lddb, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "cycle backward");
    return AMM_OK;
  }
  if (a->method == AMM_SPARSE_FOURIER) {
    FtBwArgs f;
    f.n = a->ft.n;
    f.m = (int)a->rows;
    f.p = (int)b->cols;
    f.ka = (int)a->k;
    f.kb = (int)b->k;
    f.tw = a->ft.tw;
    f.AtT = a->ft.TT;
    f.selA = a->ft.sel;
    f.maskA = a->ft.maskT;
    f.Bt = b->ft.T;
    f.selB = b->ft.sel;
    f.maskB = b->ft.maskT;
    f.G = dC;
    f.ldg = lddc;
    f.dA = dA;
    f.ldda = ldda;
    f.dB = dB;
    f.lddb = lddb;
    cudaError_t e = ft_backward(f, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "fourier backward");
    return AMM_OK;
  }
  return fail(AMM_ERR_NOT_IMPLEMENTED, "backward for method %d is not built yet", a->method);
}

extern "C" amm_status_t amm_handle_info(amm_handle_t h, amm_info_t* info) {
  if (!h || !info) return fail(AMM_ERR_INVALID_ARG, "amm_handle_info: NULL argument");
  memset(info, 0, sizeof(*info));
  info->method = h->method;
  info->role = h->role;
  info->dtype = h->dtype;
  info->rows = h->rows;
  info->cols = h->cols;
  info->k = h->k;
  if (h->blk.b) return blocked_info(h, info);
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "amm_handle_info: stream");
  if (h->method == AMM_CIRCULANT || h->method == AMM_SPARSE_CYCLE) {
    const SelectOut& so = h->method == AMM_CIRCULANT ? h->cd.so : h->cy.so;
    double nr[3];
    int32_t cnt[2];
    if ((e = cudaMemcpy(nr, so.norms, sizeof(nr), cudaMemcpyDeviceToHost)) != cudaSuccess ||
        (e = cudaMemcpy(cnt, so.counts, sizeof(cnt), cudaMemcpyDeviceToHost)) != cudaSuccess)
      return cuda_fail(e, "amm_handle_info: copy");
    info->fro2 = nr[0];
    info->resid_fro2 = nr[1];
    info->boundary_gap = nr[2];
    if (h->method == AMM_CIRCULANT) {
      info->n_union = cnt[0];
      info->n_unpaired = (cnt[1] + 1) / 2;
    }
  } else if (h->method == AMM_SVD) {
    return svd_info(h, info);
  } else if (h->method == AMM_SPARSE_FOURIER) {
    double* d = nullptr;
    double nr[2];
    if ((e = dev_alloc((void**)&d, sizeof(nr), h->stream)) != cudaSuccess) return cuda_fail(e, "amm_handle_info");
    e = ft_norms(h->ft.n, (int)h->k, h->ft.nvec, h->ft.mag, h->ft.sel, d, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(nr, d, sizeof(nr), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    dev_free(d, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "amm_handle_info: fourier norms");
    info->fro2 = nr[0];
    info->resid_fro2 = nr[0] - nr[1];  // W is unitary: the dropped entries carry the rest
  }
  return AMM_OK;
}

extern "C" amm_status_t amm_choose_k(const void* A, int64_t rows, int64_t cols, int64_t lda, amm_dtype_t dtype,
                                     amm_method_t method, double tol, void* stream, int64_t* k_out) {
  if (!A || !k_out) return fail(AMM_ERR_INVALID_ARG, "amm_choose_k: NULL argument");
  if (rows != cols)
    return fail(AMM_ERR_UNSUPPORTED_SIZE, "amm_choose_k: A must be square (got %lldx%lld)", (long long)rows,
                (long long)cols);
  if (method == AMM_CIRCULANT ? !cd_length_ok(rows) : !cyc_length_ok(rows))
    return fail(AMM_ERR_UNSUPPORTED_SIZE, "amm_choose_k: n=%lld is not a supported length for this method",
                (long long)rows);
  if (lda < cols) return fail(AMM_ERR_INVALID_ARG, "amm_choose_k: lda < cols");
  if (!(tol >= 0.0)) return fail(AMM_ERR_INVALID_ARG, "amm_choose_k: tol must be >= 0");
  if (dtype != AMM_F32 && dtype != AMM_BF16) return fail(AMM_ERR_INVALID_ARG, "amm_choose_k: bad dtype");
  if (method != AMM_CIRCULANT && method != AMM_SPARSE_CYCLE)
    return fail(AMM_ERR_NOT_IMPLEMENTED, "amm_choose_k: built for AMM_CIRCULANT and AMM_SPARSE_CYCLE");
  const int n = (int)rows;
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<void*> tmp;
  cudaError_t e = cudaSuccess;
  auto al = [&](size_t bytes) -> void* {
    void* q = nullptr;
    if (e == cudaSuccess) e = dev_alloc(&q, bytes, st);
    if (q) tmp.push_back(q);
    return q;
  };
  const bool circ = method == AMM_CIRCULANT;
  const int kh = circ ? n / 2 + 1 : n;
  int nparts = 0;
  double* key2 = (double*)al(sizeof(double) * kh);
  if (circ) {
    const float2* tw = nullptr;
    if (e == cudaSuccess) e = twiddles(n, st, &tw);
    nparts = (n + cd_cols_per_cta(n) - 1) / cd_cols_per_cta(n);
    float2* R = (float2*)al(sizeof(float2) * (size_t)kh * n);
    float* kpart = (float*)al(sizeof(float) * (size_t)kh * nparts);
    if (e == cudaSuccess) e = cd_spectrum(n, A, lda, dtype == AMM_BF16, tw, R, kpart, st);
    if (e == cudaSuccess) e = cd_keys(kh, kpart, nparts, key2, st);
  } else {
    const float* Af = (const float*)A;
    int64_t ldf = lda;
    if (dtype == AMM_BF16) {
      float* y = (float*)al(sizeof(float) * (size_t)n * n);
      if (e == cudaSuccess) e = widen_bf16(A, n, n, lda, y, n, st);
      Af = y;
      ldf = n;
    }
    const int rp = cyc_rows_per_part(n);
    nparts = (n + rp - 1) / rp;
    float* kpart = (float*)al(sizeof(float) * (size_t)nparts * n);
    if (e == cudaSuccess) e = cyc_keys(n, Af, ldf, kpart, st);
    if (e == cudaSuccess) e = cd_keys(n, kpart, nparts, key2, st);
  }
  std::vector<double> h(kh);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), key2, sizeof(double) * kh, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  for (void* q : tmp) dev_free(q, st);
  if (e != cudaSuccess) return cuda_fail(e, "amm_choose_k");
  // squared key of every component (conjugate partners share theirs); ||A||^2 and the truncation
  // error of the top-k set follow from the orthogonality of the components (Section 2.3)
  std::vector<std::pair<double, int>> keys(n);
  double total = 0.0;
  for (int t = 0; t < n; ++t) {
    const double v = circ ? h[std::min(t, n - t) % (n / 2 + 1)] : h[t];
    keys[t] = {v, t};
    total += v;
  }
  std::sort(keys.begin(), keys.end(), [](const std::pair<double, int>& x, const std::pair<double, int>& y) {
    return x.first > y.first || (x.first == y.first && x.second < y.second);
  });
  double kept = 0.0;
  int64_t k = n;
  for (int i = 0; i < n; ++i) {
    if (total - kept <= tol * tol * total) {
      k = i;
      break;
    }
    kept += keys[i].first;
  }
  *k_out = std::max<int64_t>(k, 1);
  return AMM_OK;
}

// k from a truncation tolerance (Section 2.5: more components while the error is not
// satisfactory).  Circulant / cycle: the exact minimal k from the keys (amm_choose_k).  SVD /
// Fourier sparsifier: k doubles from k0 until the handle's truncation error meets the tolerance,
// then bisection inside the last bracket; every trial is a full decomposition whose error comes
// from amm_handle_info.
extern "C" amm_status_t amm_decompose_to_tolerance(const void* A, int64_t rows, int64_t cols, int64_t lda,
                                                   amm_dtype_t dtype, amm_method_t method, double tol, int64_t k_max,
                                                   const amm_opts_t* opts, void* stream, amm_handle_t* out,
                                                   int64_t* k_out) {
  if (!out || !k_out) return fail(AMM_ERR_INVALID_ARG, "amm_decompose_to_tolerance: NULL output");
  if (!(tol >= 0.0)) return fail(AMM_ERR_INVALID_ARG, "amm_decompose_to_tolerance: tol must be >= 0");
  if (opts && opts->forced_selection)
    return fail(AMM_ERR_INVALID_ARG, "amm_decompose_to_tolerance: a forced selection fixes k");
  amm_status_t s;
  if (method == AMM_CIRCULANT || method == AMM_SPARSE_CYCLE) {
    if (opts && opts->block) return fail(AMM_ERR_NOT_IMPLEMENTED, "amm_decompose_to_tolerance: circulant blocks");
    int64_t k = 0;
    if ((s = amm_choose_k(A, rows, cols, lda, dtype, method, tol, stream, &k)) != AMM_OK) return s;
    if (k_max > 0) k = std::min(k, k_max);
    if ((s = amm_decompose(A, rows, cols, lda, dtype, method, k, opts, stream, out)) != AMM_OK) return s;
    *k_out = k;
    return AMM_OK;
  }
  if (method != AMM_SVD && method != AMM_SPARSE_FOURIER)
    return fail(AMM_ERR_INVALID_ARG, "amm_decompose_to_tolerance: bad method %d", (int)method);
  if (opts && opts->sketch)
    return fail(AMM_ERR_INVALID_ARG, "amm_decompose_to_tolerance: a caller sketch fixes k (use the seed)");
  const int64_t kcap0 = method == AMM_SVD ? std::min<int64_t>(std::min(rows, cols), 1024)
                                          : (opts && opts->role == AMM_RIGHT ? rows : cols);
  const int64_t kcap = k_max > 0 ? std::min(k_max, kcap0) : kcap0;
  // error of one trial; the handle is kept when it meets the tolerance
  auto trial = [&](int64_t k, amm_handle_t* h, bool* ok) -> amm_status_t {
    amm_status_t st = amm_decompose(A, rows, cols, lda, dtype, method, k, opts, stream, h);
    if (st != AMM_OK) return st;
    amm_info_t info;
    if ((st = amm_handle_info(*h, &info)) != AMM_OK) {
      amm_handle_destroy(*h);
      return st;
    }
    *ok = std::max(info.resid_fro2, 0.0) <= tol * tol * info.fro2;
    return AMM_OK;
  };
  int64_t lo = 0, hi = std::min<int64_t>(8, kcap);
  amm_handle_t best = nullptr;
  bool ok = false;
  for (;;) {
    amm_handle_t h = nullptr;
    if ((s = trial(hi, &h, &ok)) != AMM_OK) return s;
    if (ok || hi == kcap) {
      best = h;
      break;
    }
    amm_handle_destroy(h);
    lo = hi;
    hi = std::min(2 * hi, kcap);
  }
  // bisection in (lo, hi]: the smallest k of the bracket whose trial meets the tolerance
  while (ok && hi - lo > 1) {
    const int64_t mid = lo + (hi - lo) / 2;
    amm_handle_t h = nullptr;
    bool okm = false;
    if ((s = trial(mid, &h, &okm)) != AMM_OK) {
      amm_handle_destroy(best);
      return s;
    }
    if (okm) {
      amm_handle_destroy(best);
      best = h;
      hi = mid;
    } else {
      amm_handle_destroy(h);
      lo = mid;
    }
  }
  *out = best;
  *k_out = hi;
  return AMM_OK;
}

extern "C" amm_status_t amm_error_estimate(amm_handle_t hA, amm_handle_t hB, const float* C, int64_t ldc,
                                           void* stream, double* estimate) {
  if (!estimate) return fail(AMM_ERR_INVALID_ARG, "amm_error_estimate: estimate is NULL");
  if (!C) return fail(AMM_ERR_INVALID_ARG, "amm_error_estimate: C is NULL");
  amm_status_t s = check_pair(hA, hB);
  if (s != AMM_OK) return s;
  if (ldc < hB->cols) return fail(AMM_ERR_INVALID_ARG, "amm_error_estimate: ldc too small");
  amm_info_t ia, ib;
  if ((s = amm_handle_info(hA, &ia)) != AMM_OK) return s;
  if ((s = amm_handle_info(hB, &ib)) != AMM_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  double* d = nullptr;
  double c2 = 0.0;
  cudaError_t e = dev_alloc((void**)&d, sizeof(double), st);
  if (e == cudaSuccess) e = sumsq_f32(C, hA->rows, hB->cols, ldc, d, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&c2, d, sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  dev_free(d, st);
  if (e != cudaSuccess) return cuda_fail(e, "amm_error_estimate");
  if (c2 <= 0.0) return fail(AMM_ERR_STATE, "amm_error_estimate: ||C||_F = 0");
  const double ra = std::max(ia.resid_fro2, 0.0), rb = std::max(ib.resid_fro2, 0.0);
  *estimate = std::sqrt(ra * rb) / (std::sqrt((double)hA->cols) * std::sqrt(c2));
  return AMM_OK;
}

// A priori estimate of the relative error (Section 2.5, before the product is formed):
// E||dA dB||_F ~ c_resid ||dA||_F ||dB||_F and E||A B||_F ~ c_ab ||A||_F ||B||_F, the constants
// those of Section 3 for independent entries (1/sqrt(n) for zero mean; the appendix tabulates
// others, e.g. 3/4 for U(0,1)).  Only the handles' norms enter: no device work.
extern "C" amm_status_t amm_apriori_estimate(amm_handle_t hA, amm_handle_t hB, double c_ab, double c_resid,
                                             double* estimate) {
  if (!estimate) return fail(AMM_ERR_INVALID_ARG, "amm_apriori_estimate: estimate is NULL");
  if (!(c_ab > 0.0) || !(c_resid > 0.0))
    return fail(AMM_ERR_INVALID_ARG, "amm_apriori_estimate: the constants must be > 0");
  amm_status_t s = check_pair(hA, hB);
  if (s != AMM_OK) return s;
  amm_info_t ia, ib;
  if ((s = amm_handle_info(hA, &ia)) != AMM_OK) return s;
  if ((s = amm_handle_info(hB, &ib)) != AMM_OK) return s;
  if (!(ia.fro2 > 0.0) || !(ib.fro2 > 0.0)) return fail(AMM_ERR_STATE, "amm_apriori_estimate: ||A||_F ||B||_F = 0");
  const double ra = std::max(ia.resid_fro2, 0.0), rb = std::max(ib.resid_fro2, 0.0);
  *estimate = (c_resid * std::sqrt(ra * rb)) / (c_ab * std::sqrt(ia.fro2 * ib.fro2));
  return AMM_OK;
}

// The most suitable of several decompositions of one operand at a given k (Section 2.5: the
// relative truncation error ||dA||_F / ||A||_F of each candidate decides; the paper lets A and B
// use different ones).  Candidates that do not take this shape or k are skipped.
extern "C" amm_status_t amm_decompose_best_method(const void* A, int64_t rows, int64_t cols, int64_t lda,
                                                  amm_dtype_t dtype, const int32_t* host_methods,
                                                  int32_t n_methods, int64_t k, const amm_opts_t* opts,
                                                  void* stream, amm_handle_t* out, int32_t* method_out) {
  if (!out || !method_out) return fail(AMM_ERR_INVALID_ARG, "amm_decompose_best_method: NULL output");
  if (!A) return fail(AMM_ERR_INVALID_ARG, "amm_decompose_best_method: A is NULL");
  if (!host_methods || n_methods < 1)
    return fail(AMM_ERR_INVALID_ARG, "amm_decompose_best_method: no candidate methods");
  if (rows <= 0 || cols <= 0 || lda < cols)
    return fail(AMM_ERR_INVALID_ARG, "amm_decompose_best_method: bad shape %lldx%lld, lda=%lld", (long long)rows,
                (long long)cols, (long long)lda);
  if (dtype != AMM_F32 && dtype != AMM_BF16) return fail(AMM_ERR_INVALID_ARG, "amm_decompose_best_method: bad dtype");
  if (k < 1) return fail(AMM_ERR_INVALID_ARG, "amm_decompose_best_method: k=%lld < 1", (long long)k);
  for (int32_t i = 0; i < n_methods; ++i) {
    const int32_t m = host_methods[i];
    if (m != AMM_SVD && m != AMM_CIRCULANT && m != AMM_SPARSE_FOURIER && m != AMM_SPARSE_CYCLE)
      return fail(AMM_ERR_INVALID_ARG, "amm_decompose_best_method: bad method %d", (int)m);
  }
  if (opts && opts->struct_size != sizeof(amm_opts_t))
    return fail(AMM_ERR_INVALID_ARG, "amm_decompose_best_method: opts->struct_size=%u, expected %zu",
                opts->struct_size, sizeof(amm_opts_t));
  if (opts && (opts->forced_selection || opts->sketch))
    return fail(AMM_ERR_INVALID_ARG, "amm_decompose_best_method: forced selections and sketches are per method");
  amm_opts_t base;
  amm_opts_init(&base);
  if (opts) base = *opts;
  amm_handle_t best = nullptr;
  int32_t best_method = -1;
  double best_rel = 0.0;
  amm_status_t last = AMM_ERR_INVALID_ARG;
  for (int32_t i = 0; i < n_methods; ++i) {
    const amm_method_t m = (amm_method_t)host_methods[i];
    amm_opts_t o = base;
    if (m != AMM_CIRCULANT) o.block = 0;  // square blocks are an option of the circulant method only
    amm_handle_t h = nullptr;
    amm_status_t s = amm_decompose(A, rows, cols, lda, dtype, m, k, &o, stream, &h);
    if (s == AMM_ERR_UNSUPPORTED_SIZE || s == AMM_ERR_INVALID_ARG) {  // this shape / k is not one of m's
      last = s;
      continue;
    }
    if (s != AMM_OK) {
      if (best) amm_handle_destroy(best);
      return s;
    }
    amm_info_t info;
    if ((s = amm_handle_info(h, &info)) != AMM_OK) {
      amm_handle_destroy(h);
      if (best) amm_handle_destroy(best);
      return s;
    }
    const double rel = info.fro2 > 0.0 ? std::max(info.resid_fro2, 0.0) / info.fro2 : 0.0;
    if (!best || rel < best_rel) {  // ties keep the earlier candidate
      if (best) amm_handle_destroy(best);
      best = h;
      best_method = (int32_t)m;
      best_rel = rel;
    } else {
      amm_handle_destroy(h);
    }
  }
  if (!best) return last;  // amm_last_error() holds the last candidate's reason
  *out = best;
  *method_out = best_method;
  return AMM_OK;
}

extern "C" amm_status_t amm_handle_residual(amm_handle_t h, float* D, int64_t ldd, void* stream) {
  if (!h || !D) return fail(AMM_ERR_INVALID_ARG, "amm_handle_residual: NULL argument");
  if (ldd < h->cols)
    return fail(AMM_ERR_INVALID_ARG, "amm_handle_residual: ldd=%lld < cols=%lld", (long long)ldd, (long long)h->cols);
  return handle_residual(h, D, ldd, (cudaStream_t)stream);
}

extern "C" amm_status_t amm_refine_product(amm_handle_t hA, amm_handle_t hB, amm_handle_t hA2, amm_handle_t hB2,
                                           float* C, int64_t ldc, void* stream) {
  if (!C) return fail(AMM_ERR_INVALID_ARG, "amm_refine_product: C is NULL");
  amm_status_t s = check_pair(hA, hB);
  if (s != AMM_OK) return s;
  if ((s = check_pair(hA2, hB2)) != AMM_OK) return s;
  if (ldc < hB->cols) return fail(AMM_ERR_INVALID_ARG, "amm_refine_product: ldc too small");
  if (hA2->rows != hA->rows || hA2->cols != hA->cols || hB2->rows != hB->rows || hB2->cols != hB->cols)
    return fail(AMM_ERR_STATE, "amm_refine_product: the residues' handles must have the shapes of A and B");
  return refine_product(hA, hB, hA2, hB2, C, ldc, (cudaStream_t)stream);
}

extern "C" amm_status_t amm_handle_get_selection(amm_handle_t h, int32_t* host_idx, int64_t cap, int64_t* count) {
  if (!h || !host_idx || !count) return fail(AMM_ERR_INVALID_ARG, "amm_handle_get_selection: NULL argument");
  if (h->method == AMM_SPARSE_FOURIER) {
    const int64_t cnt = h->k * h->ft.nvec;
    if (cap < cnt) return fail(AMM_ERR_INVALID_ARG, "cap=%lld < rows*k=%lld", (long long)cap, (long long)cnt);
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e == cudaSuccess) e = cudaMemcpy(host_idx, h->ft.sel, sizeof(int32_t) * cnt, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "amm_handle_get_selection");
    *count = cnt;
    return AMM_OK;
  }
  if (h->method != AMM_CIRCULANT && h->method != AMM_SPARSE_CYCLE)
    return fail(AMM_ERR_STATE, "handle has no component selection");
  if (h->blk.b) return blocked_selection(h, host_idx, cap, count);
  if (cap < h->k) return fail(AMM_ERR_INVALID_ARG, "cap=%lld < k=%lld", (long long)cap, (long long)h->k);
  const int32_t* sel = h->method == AMM_CIRCULANT ? h->cd.so.sel : h->cy.so.sel;
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e == cudaSuccess) e = cudaMemcpy(host_idx, sel, sizeof(int32_t) * h->k, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "amm_handle_get_selection");
  *count = h->k;
  return AMM_OK;
}

extern "C" amm_status_t amm_handle_device_bytes(amm_handle_t h, int64_t* bytes) {
  if (!h || !bytes) return fail(AMM_ERR_INVALID_ARG, "amm_handle_device_bytes: NULL argument");
  *bytes = h->device_bytes();
  return AMM_OK;
}

extern "C" amm_status_t amm_handle_get_keys(amm_handle_t h, double* host_keys, int64_t cap, int64_t* count) {
  if (!h || !host_keys || !count) return fail(AMM_ERR_INVALID_ARG, "amm_handle_get_keys: NULL argument");
  if (h->method != AMM_CIRCULANT && h->method != AMM_SPARSE_CYCLE)
    return fail(AMM_ERR_STATE, "amm_handle_get_keys: handle has no component keys");
  if (h->blk.b) return fail(AMM_ERR_NOT_IMPLEMENTED, "amm_handle_get_keys: blocked circulant handle");
  const int64_t n = h->rows;
  if (cap < n) return fail(AMM_ERR_INVALID_ARG, "amm_handle_get_keys: cap=%lld < n=%lld", (long long)cap, (long long)n);
  const double* keys = h->method == AMM_CIRCULANT ? h->cd.so.keys : h->cy.so.keys;
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e == cudaSuccess) e = cudaMemcpy(host_keys, keys, sizeof(double) * n, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "amm_handle_get_keys");
  *count = n;
  return AMM_OK;
}

extern "C" amm_status_t amm_handle_get_sketch(amm_handle_t h, float* host_phi, int64_t cap) {
  if (!h || !host_phi) return fail(AMM_ERR_INVALID_ARG, "amm_handle_get_sketch: NULL argument");
  if (h->method != AMM_SVD) return fail(AMM_ERR_STATE, "handle has no sketch");
  return svd_get_sketch(h, host_phi, cap);
}

extern "C" amm_status_t amm_handle_destroy(amm_handle_t h) {
  if (!h) return fail(AMM_ERR_INVALID_ARG, "amm_handle_destroy: NULL handle");
  h->release();
  delete h;
  return AMM_OK;
}
