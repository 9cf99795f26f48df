// Rectangular circulant operands in square blocks.  The cycle decomposition (Thm 2.1) is defined
// for square matrices; Section 2.3 takes a rectangular or very large operand in square blocks.
// Both dimensions are cut into b x b blocks, a ragged edge is padded with zeros, and every block
// is an ordinary square circulant handle with its own top-k selection.  With A in blocks A_IJ
// and B in blocks B_JL (same b), Eq. (2.3) on the padded operands is blockwise
//
//   M_IL = sum_J ( A~_IJ B_JL + dA_IJ B~_JL ),
//
// the sum over inner blocks of the square first-order products, so every term runs through the
// square kernels (spectral applies on column / row spectra) with the first inner block writing
// its output block and the others adding to it.  The backward is blockwise too (the projector of
// a blocked truncation acts block by block):
//
//   dA_IJ = sum_L bwA(A_IJ, B_JL, G_IL),   dB_JL = sum_I bwB(A_IJ, B_JL, G_IL).
//
// Padded rows / columns of C, dA and dB are computed in a scratch buffer and dropped; G is read
// through a zero-padded copy when the output is ragged.
#include <cuda_runtime.h>

#include <algorithm>

#include "api_internal.h"
#include "kernels.h"

namespace amm {

namespace {

int64_t ceil_div(int64_t x, int64_t b) { return (x + b - 1) / b; }

// Block grid of a circulant handle; an unblocked square handle is a 1 x 1 grid of itself.
struct Grid {
  Handle* self;
  int64_t b, nbr, nbc;
  Handle* at(int64_t i, int64_t j) const {
    return self->blk.b ? self->blk.sub[(size_t)(i * nbc + j)] : self;
  }
};

Grid grid(Handle* h) {
  if (h->blk.b) return {h, h->blk.b, h->blk.nbr, h->blk.nbc};
  return {h, h->rows, 1, 1};
}

// Scratch buffers of one call, released at the end (stream-ordered).
struct Scratch {
  cudaStream_t st;
  std::vector<void*> bufs;
  cudaError_t e = cudaSuccess;
  explicit Scratch(cudaStream_t s) : st(s) {}
  float* get(size_t elems, bool zero) {
    void* q = nullptr;
    if (e == cudaSuccess) e = dev_alloc(&q, sizeof(float) * elems, st);
    if (q) bufs.push_back(q);
    if (e == cudaSuccess && zero) e = cudaMemsetAsync(q, 0, sizeof(float) * elems, st);
    return (float*)q;
  }
  ~Scratch() {
    for (void* q : bufs) dev_free(q, st);
  }
};

cudaError_t copy2d(float* dst, int64_t ldd, const float* src, int64_t lds, int64_t rows, int64_t cols,
                   cudaStream_t st) {
  return cudaMemcpy2DAsync(dst, sizeof(float) * ldd, src, sizeof(float) * lds, sizeof(float) * cols, rows,
                           cudaMemcpyDeviceToDevice, st);
}

}  // namespace

amm_status_t decompose_circulant_blocked(Handle* h, const amm_opts_t* o) {
  const int64_t b = o->block;
  if (!cd_length_ok(b))
    return fail(AMM_ERR_UNSUPPORTED_SIZE, "circulant: block=%lld must be in [16, 4096], or 2^a up to 16384",
                (long long)b);
  auto& g = h->blk;
  g.b = b;
  g.nbr = ceil_div(h->rows, b);
  g.nbc = ceil_div(h->cols, b);
  const size_t es = h->dtype == AMM_BF16 ? 2 : 4;
  g.base = h->A;
  g.ld = h->lda;
  cudaError_t e = cudaSuccess;
  if (h->rows % b || h->cols % b) {
    // ragged edge: a zero-padded copy of the whole operand (element type kept)
    const int64_t pr = g.nbr * b, pc = g.nbc * b;
    void* pad = nullptr;
    e = h->alloc(&pad, es * (size_t)pr * pc);
    if (e == cudaSuccess) e = cudaMemsetAsync(pad, 0, es * (size_t)pr * pc, h->stream);
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(pad, es * pc, h->A, es * h->lda, es * h->cols, h->rows, cudaMemcpyDeviceToDevice,
                            h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "circulant blocks: padded copy");
    g.base = pad;
    g.ld = pc;
  }
  amm_opts_t so = *o;
  so.block = 0;
  for (int64_t i = 0; i < g.nbr; ++i)
    for (int64_t j = 0; j < g.nbc; ++j) {
      Handle* s = new (std::nothrow) Handle();
      if (!s) return fail(AMM_ERR_OOM, "circulant blocks: host allocation");
      g.sub.push_back(s);  // released with h, also on a failure below
      s->A = (const char*)g.base + es * (size_t)(i * b * g.ld + j * b);
      s->rows = s->cols = b;
      s->lda = g.ld;
      s->dtype = h->dtype;
      s->method = AMM_CIRCULANT;
      s->role = h->role;
      s->k = h->k;
      s->stream = h->stream;
      so.forced_selection = o->forced_selection ? o->forced_selection + (size_t)(i * g.nbc + j) * h->k : nullptr;
      amm_status_t st = decompose_circulant(s, &so);
      if (st != AMM_OK) return st;
    }
  return AMM_OK;
}

amm_status_t blocked_matmul(Handle* a, Handle* b, float* C, int64_t ldc, cudaStream_t st) {
  const Grid ga = grid(a), gb = grid(b);
  if (ga.b != gb.b)
    return fail(AMM_ERR_UNSUPPORTED_SIZE, "circulant blocks differ: A in %lld, B in %lld", (long long)ga.b,
                (long long)gb.b);
  const int64_t bs = ga.b, m = a->rows, p = b->cols, mp = ga.nbr * bs, pp = gb.nbc * bs;
  Scratch sc(st);
  const bool crop = mp != m || pp != p;
  float* Cp = crop ? sc.get((size_t)mp * pp, false) : C;
  const int64_t ldp = crop ? pp : ldc;
  for (int64_t i = 0; i < ga.nbr && sc.e == cudaSuccess; ++i)
    for (int64_t l = 0; l < gb.nbc && sc.e == cudaSuccess; ++l)
      for (int64_t j = 0; j < ga.nbc && sc.e == cudaSuccess; ++j)
        sc.e = cd_first_order(ga.at(i, j), gb.at(j, l), Cp + i * bs * ldp + l * bs, ldp, j > 0, st);
  if (sc.e == cudaSuccess && crop) sc.e = copy2d(C, ldc, Cp, ldp, m, p, st);
  if (sc.e != cudaSuccess) return cuda_fail(sc.e, "blocked circulant product");
  return AMM_OK;
}

amm_status_t blocked_backward(Handle* a, Handle* b, const float* G, int64_t ldg, float* dA, int64_t ldda, float* dB,
                              int64_t lddb, cudaStream_t st) {
  const Grid ga = grid(a), gb = grid(b);
  if (ga.b != gb.b)
    return fail(AMM_ERR_UNSUPPORTED_SIZE, "circulant blocks differ: A in %lld, B in %lld", (long long)ga.b,
                (long long)gb.b);
  const int64_t bs = ga.b, m = a->rows, n = a->cols, p = b->cols;
  const int64_t mp = ga.nbr * bs, np = ga.nbc * bs, pp = gb.nbc * bs;
  Scratch sc(st);
  const float* Gp = G;
  int64_t ldgp = ldg;
  if (mp != m || pp != p) {
    float* t = sc.get((size_t)mp * pp, true);
    if (sc.e == cudaSuccess) sc.e = copy2d(t, pp, G, ldg, m, p, st);
    Gp = t;
    ldgp = pp;
  }
  const bool cropA = dA && (mp != m || np != n), cropB = dB && (np != n || pp != p);
  float* dAp = cropA ? sc.get((size_t)mp * np, false) : dA;
  float* dBp = cropB ? sc.get((size_t)np * pp, false) : dB;
  const int64_t lda_ = cropA ? np : ldda, ldb_ = cropB ? pp : lddb;
  amm_status_t s = AMM_OK;
  for (int64_t i = 0; i < ga.nbr && sc.e == cudaSuccess && s == AMM_OK; ++i)
    for (int64_t j = 0; j < ga.nbc && sc.e == cudaSuccess && s == AMM_OK; ++j)
      for (int64_t l = 0; l < gb.nbc && sc.e == cudaSuccess && s == AMM_OK; ++l)
        s = cd_backward(ga.at(i, j), gb.at(j, l), Gp + i * bs * ldgp + l * bs, ldgp,
                        dAp ? dAp + i * bs * lda_ + j * bs : nullptr, lda_, l > 0,
                        dBp ? dBp + j * bs * ldb_ + l * bs : nullptr, ldb_, i > 0, st);
  if (s != AMM_OK) return s;
  if (sc.e == cudaSuccess && cropA) sc.e = copy2d(dA, ldda, dAp, lda_, m, n, st);
  if (sc.e == cudaSuccess && cropB) sc.e = copy2d(dB, lddb, dBp, ldb_, n, p, st);
  if (sc.e != cudaSuccess) return cuda_fail(sc.e, "blocked circulant backward");
  return AMM_OK;
}

// Norms add over blocks (the blocks are disjoint, and so are their truncations); the boundary gap
// reported is the smallest of the blocks'.
amm_status_t blocked_info(Handle* h, amm_info_t* info) {
  double fro2 = 0.0, resid = 0.0, gap = 1e300;
  int64_t nu = 0, nunp = 0;
  for (Handle* s : h->blk.sub) {
    amm_info_t bi;
    amm_status_t st = amm_handle_info(s, &bi);
    if (st != AMM_OK) return st;
    fro2 += bi.fro2;
    resid += bi.resid_fro2;
    gap = std::min(gap, bi.boundary_gap);
    nu += bi.n_union;
    nunp += bi.n_unpaired;
  }
  info->fro2 = fro2;
  info->resid_fro2 = resid;
  info->boundary_gap = gap;
  info->n_union = nu;
  info->n_unpaired = nunp;
  return AMM_OK;
}

amm_status_t blocked_selection(Handle* h, int32_t* host_idx, int64_t cap, int64_t* count) {
  const int64_t total = (int64_t)h->blk.sub.size() * h->k;
  if (cap < total)
    return fail(AMM_ERR_INVALID_ARG, "cap=%lld < blocks*k=%lld", (long long)cap, (long long)total);
  int64_t off = 0;
  for (Handle* s : h->blk.sub) {
    int64_t c = 0;
    amm_status_t st = amm_handle_get_selection(s, host_idx + off, cap - off, &c);
    if (st != AMM_OK) return st;
    off += c;
  }
  *count = off;
  return AMM_OK;
}

// C_I = sum_J Re(A~_IJ) X_J for X with nbc*b rows; C has nbr*b rows.
cudaError_t blocked_left_apply(Handle* a, const float* X, int64_t ldx, int64_t p, float* C, int64_t ldc,
                               cudaStream_t st) {
  const Grid g = grid(a);
  const int bs = (int)g.b;
  cudaError_t e = cudaSuccess;
  for (int64_t i = 0; i < g.nbr && e == cudaSuccess; ++i)
    for (int64_t j = 0; j < g.nbc && e == cudaSuccess; ++j) {
      Handle* s = g.at(i, j);
      e = cd_apply(bs, false, X + j * bs * ldx, ldx, false, p, s->cd.tw, s->cd.so.ulist, s->cd.Lw, s->cd.so.counts,
                   nullptr, nullptr, C + i * bs * ldc, ldc, j > 0, st);
    }
  return e;
}

// C_L += sum_J Y_J Re(B~_JL) (imag: Y_J Im(B~_JL)) for Y with nbr*b columns; C has nbc*b columns.
cudaError_t blocked_right_apply(Handle* b, const float* Y, int64_t ldy, int64_t m, bool imag, float* C,
                                int64_t ldc, cudaStream_t st) {
  const Grid g = grid(b);
  const int bs = (int)g.b;
  cudaError_t e = cudaSuccess;
  for (int64_t l = 0; l < g.nbc && e == cudaSuccess; ++l)
    for (int64_t j = 0; j < g.nbr && e == cudaSuccess; ++j) {
      Handle* s = g.at(j, l);
      const auto& c = s->cd;
      if (imag)
        e = cd_apply(bs, true, Y + j * bs, ldy, false, m, c.tw, c.so.dlist, c.Ld, c.so.counts + 1, c.so.counts + 1,
                     c.so.counts + 1, C + l * bs, ldc, 1, st);
      else
        e = cd_apply(bs, true, Y + j * bs, ldy, false, m, c.tw, c.so.ulist, c.Lw, c.so.counts, nullptr, nullptr,
                     C + l * bs, ldc, 1, st);
    }
  return e;
}

// D = A - Re A~ (imag: D = Im A~) block by block, nbr*b x nbc*b.
cudaError_t blocked_residual(Handle* a, bool imag, float* D, int64_t ldd, cudaStream_t st) {
  const Grid g = grid(a);
  const int bs = (int)g.b;
  cudaError_t e = cudaSuccess;
  if (imag) e = cudaMemset2DAsync(D, sizeof(float) * ldd, 0, sizeof(float) * g.nbc * bs, g.nbr * bs, st);
  for (int64_t i = 0; i < g.nbr && e == cudaSuccess; ++i)
    for (int64_t j = 0; j < g.nbc && e == cudaSuccess; ++j) {
      Handle* s = g.at(i, j);
      const auto& c = s->cd;
      float* Dij = D + i * bs * ldd + j * bs;
      const float2* R = nullptr;
      float2* temp = nullptr;
      e = cd_spectrum_of(s, &R, &temp, st);
      if (e == cudaSuccess)
        e = imag ? cd_residual(bs, R, c.tw, c.so.vfull, 1, c.so.counts + 1, Dij, st, ldd, 0)
                 : cd_residual(bs, R, c.tw, c.so.wfull, 0, nullptr, Dij, st, ldd, 0);
      if (temp) dev_free(temp, st);
    }
  return e;
}

}  // namespace amm
