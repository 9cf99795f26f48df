// Export and import of a decomposition's device state (an offline weight decomposition reused by
// another process, Section 4: the weight is decomposed once, ahead of the products).
//
// The blob is a host byte string.  Each handle (and each block of a blocked circulant handle, in
// row-major block order) is written as a node:
//   scalar state   method, role, dtype, compute, sizes, per-method counts, block grid
//   buffers        every device buffer that one of the handle's pointer fields refers to, in the
//                  order of the handle's allocations: its size, then (after the field table) its
//                  bytes
//   field table    for each pointer field: null, an owned buffer (index, byte offset), a buffer of
//                  the enclosing handle (the zero-padded copy the blocks of a ragged operand read),
//                  the borrowed operand (byte offset from A) or the process's twiddle table of a
//                  length
// On import the buffers are allocated again (stream-ordered, owned by the new handle), the bytes
// copied in, and every field re-pointed: owned fields into the new buffers, borrowed fields into
// the caller's operand, twiddle fields to this process's tables.  Nothing is recomputed, so every
// later product and backward of the imported handle is bit-identical to the original's.
#include <cuda_runtime.h>

#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/amm.h"
#include "api_internal.h"

namespace amm {
namespace {

constexpr uint32_t kMagic = 0x484d4d41u;  // "AMMH"
constexpr int32_t kFormat = 1;

enum FieldKind : int32_t { F_NULL = 0, F_OWNED = 1, F_BORROWED = 2, F_TWIDDLE = 3, F_OUTER = 4 };

// The exported buffers of the enclosing handle, as seen by its blocks.
struct Outer {
  std::vector<const char*> base;
  std::vector<int64_t> bytes;
};

// Every device pointer field of a handle, in a fixed order (the blob's field table order).
std::vector<void**> pointer_fields(Handle* h) {
  auto& c = h->cd;
  auto& y = h->cy;
  auto& f = h->ft;
  auto& s = h->svd;
  std::vector<void**> v = {(void**)&h->A, (void**)&c.tw, (void**)&c.R, (void**)&c.kpart, (void**)&c.Lw,
                           (void**)&c.Ld, (void**)&c.resid, (void**)&c.imag, (void**)&y.kpart, (void**)&y.cyc,
                           (void**)&y.insel, (void**)&f.tw, (void**)&f.T, (void**)&f.TT, (void**)&f.mag,
                           (void**)&f.sel, (void**)&f.maskT, (void**)&s.phi, (void**)&s.Q, (void**)&s.X,
                           (void**)&s.norms, (void**)&s.Xe, (void**)&s.XTe, (void**)&s.Qe, (void**)&s.QTe,
                           (void**)&s.Ze, (void**)&s.ZTe, (void**)&s.err, (void**)&h->blk.base};
  for (SelectOut* so : {&c.so, &y.so}) {
    for (void** p : {(void**)&so->keys, (void**)&so->norms, (void**)&so->sel, (void**)&so->ulist, (void**)&so->uw,
                     (void**)&so->dlist, (void**)&so->dv, (void**)&so->wfull, (void**)&so->vfull,
                     (void**)&so->counts, (void**)&so->key2})
      v.push_back(p);
  }
  return v;
}

struct Writer {
  std::string out;
  template <class T> void put(T x) { out.append(reinterpret_cast<const char*>(&x), sizeof(T)); }
};

struct Reader {
  const unsigned char* p;
  size_t left;
  bool ok = true;
  template <class T> T get() {
    T x{};
    if (left < sizeof(T)) {
      ok = false;
      return x;
    }
    memcpy(&x, p, sizeof(T));
    p += sizeof(T);
    left -= sizeof(T);
    return x;
  }
};

// Bytes of the borrowed operand region [A, A + rows * lda elements).
int64_t borrowed_extent(const Handle* h) {
  const int64_t es = h->dtype == AMM_BF16 ? 2 : 4;
  return (h->rows > 0 ? (h->rows - 1) * h->lda + h->cols : 0) * es;
}

// A0 / ext: the caller's operand and its extent in bytes (the blocks of a blocked handle point into it)
cudaError_t write_node(Handle* h, const char* A0, int64_t ext, const Outer& outer, Writer& w) {
  w.put<int32_t>(h->method);
  w.put<int32_t>(h->role);
  w.put<int32_t>(h->dtype);
  w.put<int32_t>(h->compute);
  w.put<int64_t>(h->rows);
  w.put<int64_t>(h->cols);
  w.put<int64_t>(h->lda);
  w.put<int64_t>(h->k);
  w.put<int32_t>(h->cd.nparts);
  w.put<int32_t>(h->cd.cap);
  w.put<int32_t>(h->cy.nparts);
  w.put<int32_t>(h->ft.n);
  w.put<int32_t>(h->ft.nvec);
  w.put<int32_t>(h->ft.mask_words);
  w.put<int32_t>(h->svd.bf16 ? 1 : 0);
  w.put<int64_t>(h->svd.ldxe);
  w.put<int64_t>(h->blk.b);
  w.put<int64_t>(h->blk.nbr);
  w.put<int64_t>(h->blk.nbc);
  w.put<int64_t>(h->blk.ld);
  // the owned buffers some field refers to, in allocation order
  auto fields = pointer_fields(h);
  std::vector<int> used(h->owned.size(), 0);
  struct Ref {
    int32_t kind, index;
    int64_t offset;
  };
  std::vector<Ref> refs;
  for (void** fp : fields) {
    const char* v = (const char*)*fp;
    Ref r{F_NULL, -1, 0};
    if (v) {
      for (size_t i = 0; i < h->owned.size() && r.kind == F_NULL; ++i) {
        const char* b = (const char*)h->owned[i];
        if (v >= b && v < b + h->owned_bytes[i]) r = {F_OWNED, (int32_t)i, (int64_t)(v - b)};
      }
      for (size_t i = 0; i < outer.base.size() && r.kind == F_NULL; ++i)
        if (v >= outer.base[i] && v < outer.base[i] + outer.bytes[i]) r = {F_OUTER, (int32_t)i, (int64_t)(v - outer.base[i])};
      if (r.kind == F_NULL && A0 && v >= A0 && v < A0 + ext) r = {F_BORROWED, -1, (int64_t)(v - A0)};
      if (r.kind == F_NULL && (fp == (void**)&h->cd.tw || fp == (void**)&h->ft.tw))
        r = {F_TWIDDLE, fp == (void**)&h->cd.tw ? (int32_t)h->rows : h->ft.n, 0};
      if (r.kind == F_NULL) return cudaErrorInvalidValue;  // a pointer the format cannot place
      if (r.kind == F_OWNED) used[r.index] = 1;
    }
    refs.push_back(r);
  }
  // compact the buffer indices to the used ones
  std::vector<int32_t> remap(h->owned.size(), -1);
  int32_t nb = 0;
  for (size_t i = 0; i < used.size(); ++i)
    if (used[i]) remap[i] = nb++;
  w.put<int32_t>(nb);
  for (size_t i = 0; i < used.size(); ++i)
    if (used[i]) w.put<int64_t>((int64_t)h->owned_bytes[i]);
  w.put<int32_t>((int32_t)refs.size());
  for (const Ref& r : refs) {
    w.put<int32_t>(r.kind);
    w.put<int32_t>(r.kind == F_OWNED ? remap[r.index] : r.index);
    w.put<int64_t>(r.offset);
  }
  for (size_t i = 0; i < used.size(); ++i) {
    if (!used[i]) continue;
    const size_t at = w.out.size();
    w.out.resize(at + h->owned_bytes[i]);
    cudaError_t e = cudaMemcpy(&w.out[at], h->owned[i], h->owned_bytes[i], cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return e;
  }
  Outer mine;
  for (size_t i = 0; i < used.size(); ++i)
    if (used[i]) {
      mine.base.push_back((const char*)h->owned[i]);
      mine.bytes.push_back((int64_t)h->owned_bytes[i]);
    }
  w.put<int32_t>((int32_t)h->blk.sub.size());
  for (Handle* s : h->blk.sub) {
    cudaError_t e = write_node(s, A0, ext, mine, w);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Builds *h (allocated by the caller) from a node; A is the caller's operand, outer the buffers of
// the enclosing handle; *borrows is set when a field refers to A.
amm_status_t read_node(Reader& r, Handle* h, const char* A, const Outer& outer, bool* borrows, cudaStream_t st) {
  h->stream = st;
  h->method = r.get<int32_t>();
  h->role = r.get<int32_t>();
  h->dtype = r.get<int32_t>();
  h->compute = r.get<int32_t>();
  h->rows = r.get<int64_t>();
  h->cols = r.get<int64_t>();
  h->lda = r.get<int64_t>();
  h->k = r.get<int64_t>();
  h->cd.nparts = r.get<int32_t>();
  h->cd.cap = r.get<int32_t>();
  h->cy.nparts = r.get<int32_t>();
  h->ft.n = r.get<int32_t>();
  h->ft.nvec = r.get<int32_t>();
  h->ft.mask_words = r.get<int32_t>();
  h->svd.bf16 = r.get<int32_t>() != 0;
  h->svd.ldxe = r.get<int64_t>();
  h->blk.b = r.get<int64_t>();
  h->blk.nbr = r.get<int64_t>();
  h->blk.nbc = r.get<int64_t>();
  h->blk.ld = r.get<int64_t>();
  const int32_t nb = r.get<int32_t>();
  if (!r.ok || nb < 0 || nb > 4096 || h->rows <= 0 || h->cols <= 0 || h->k <= 0)
    return fail(AMM_ERR_INVALID_ARG, "amm_handle_import: malformed handle record");
  std::vector<int64_t> sizes(nb);
  for (int32_t i = 0; i < nb; ++i) {
    sizes[i] = r.get<int64_t>();
    if (!r.ok || sizes[i] <= 0) return fail(AMM_ERR_INVALID_ARG, "amm_handle_import: malformed buffer size");
  }
  auto fields = pointer_fields(h);
  const int32_t nf = r.get<int32_t>();
  if (!r.ok || nf != (int32_t)fields.size())
    return fail(AMM_ERR_INVALID_ARG, "amm_handle_import: field table of another format");
  struct Ref {
    int32_t kind, index;
    int64_t offset;
  };
  std::vector<Ref> refs(nf);
  for (int32_t i = 0; i < nf; ++i) {
    refs[i].kind = r.get<int32_t>();
    refs[i].index = r.get<int32_t>();
    refs[i].offset = r.get<int64_t>();
  }
  if (!r.ok) return fail(AMM_ERR_INVALID_ARG, "amm_handle_import: truncated field table");
  std::vector<void*> bufs(nb, nullptr);
  for (int32_t i = 0; i < nb; ++i) {
    if (r.left < (size_t)sizes[i]) return fail(AMM_ERR_INVALID_ARG, "amm_handle_import: truncated buffer");
    cudaError_t e = h->alloc(&bufs[i], (size_t)sizes[i]);
    if (e != cudaSuccess) return cuda_fail(e, "amm_handle_import: device allocation");
    e = cudaMemcpyAsync(bufs[i], r.p, (size_t)sizes[i], cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "amm_handle_import: upload");
    r.p += sizes[i];
    r.left -= (size_t)sizes[i];
  }
  for (int32_t i = 0; i < nf; ++i) {
    const Ref& f = refs[i];
    void* v = nullptr;
    switch (f.kind) {
      case F_NULL: break;
      case F_OWNED:
        if (f.index < 0 || f.index >= nb || f.offset < 0 || f.offset >= sizes[f.index])
          return fail(AMM_ERR_INVALID_ARG, "amm_handle_import: field outside its buffer");
        v = (char*)bufs[f.index] + f.offset;
        break;
      case F_BORROWED:
        if (f.offset < 0) return fail(AMM_ERR_INVALID_ARG, "amm_handle_import: bad operand offset");
        v = (void*)(A + f.offset);
        *borrows = true;
        break;
      case F_OUTER:
        if (f.index < 0 || f.index >= (int32_t)outer.base.size() || f.offset < 0 || f.offset >= outer.bytes[f.index])
          return fail(AMM_ERR_INVALID_ARG, "amm_handle_import: field outside the enclosing buffers");
        v = (void*)(outer.base[f.index] + f.offset);
        break;
      case F_TWIDDLE: {
        const float2* tw = nullptr;
        cudaError_t e = twiddles(f.index, st, &tw);
        if (e != cudaSuccess) return cuda_fail(e, "amm_handle_import: twiddle table");
        v = (void*)tw;
        break;
      }
      default: return fail(AMM_ERR_INVALID_ARG, "amm_handle_import: unknown field kind %d", f.kind);
    }
    *fields[i] = v;
  }
  const int32_t nsub = r.get<int32_t>();
  if (!r.ok || nsub < 0 || nsub != (int32_t)(h->blk.b ? h->blk.nbr * h->blk.nbc : 0))
    return fail(AMM_ERR_INVALID_ARG, "amm_handle_import: block count does not match the block grid");
  Outer mine;
  for (int32_t i = 0; i < nb; ++i) {
    mine.base.push_back((const char*)bufs[i]);
    mine.bytes.push_back(sizes[i]);
  }
  for (int32_t i = 0; i < nsub; ++i) {
    Handle* s = new (std::nothrow) Handle();
    if (!s) return fail(AMM_ERR_OOM, "amm_handle_import: host allocation");
    h->blk.sub.push_back(s);  // released with h on a failure below
    amm_status_t stt = read_node(r, s, A, mine, borrows, st);
    if (stt != AMM_OK) return stt;
  }
  return AMM_OK;
}

}  // namespace
}  // namespace amm

using namespace amm;

extern "C" amm_status_t amm_handle_export(amm_handle_t h, void* host_buf, int64_t cap, int64_t* len) {
  if (!h || !len) return fail(AMM_ERR_INVALID_ARG, "amm_handle_export: NULL argument");
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "amm_handle_export: synchronise");
  Writer w;
  w.put<uint32_t>(kMagic);
  w.put<int32_t>(kFormat);
  w.put<int32_t>(AMM_VERSION);
  e = write_node(h, (const char*)h->A, borrowed_extent(h), Outer{}, w);
  if (e == cudaErrorInvalidValue) return fail(AMM_ERR_STATE, "amm_handle_export: a field points outside the handle");
  if (e != cudaSuccess) return cuda_fail(e, "amm_handle_export: download");
  *len = (int64_t)w.out.size();
  if (!host_buf || cap < *len)
    return fail(AMM_ERR_INVALID_ARG, "amm_handle_export: cap=%lld < %lld bytes", (long long)cap, (long long)*len);
  memcpy(host_buf, w.out.data(), w.out.size());
  return AMM_OK;
}

extern "C" amm_status_t amm_handle_import(const void* host_buf, int64_t len, const void* A, int64_t rows,
                                          int64_t cols, int64_t lda, amm_dtype_t dtype, void* stream,
                                          amm_handle_t* out) {
  if (!host_buf || len <= 0 || !A || !out) return fail(AMM_ERR_INVALID_ARG, "amm_handle_import: NULL argument");
  Reader r{(const unsigned char*)host_buf, (size_t)len};
  if (r.get<uint32_t>() != kMagic || r.get<int32_t>() != kFormat)
    return fail(AMM_ERR_INVALID_ARG, "amm_handle_import: not a handle exported by this format");
  if (r.get<int32_t>() != AMM_VERSION)
    return fail(AMM_ERR_INVALID_ARG, "amm_handle_import: exported by another library version");
  Handle* h = new (std::nothrow) Handle();
  if (!h) return fail(AMM_ERR_OOM, "amm_handle_import: host allocation");
  bool borrows = false;
  amm_status_t st = read_node(r, h, (const char*)A, Outer{}, &borrows, (cudaStream_t)stream);
  if (st == AMM_OK && r.left != 0) st = fail(AMM_ERR_INVALID_ARG, "amm_handle_import: trailing bytes");
  // the operand is re-read only through borrowed fields (a sparsifier handle of a BF16 operand
  // keeps its own FP32 copy and borrows nothing)
  if (st == AMM_OK && (h->rows != rows || h->cols != cols || (borrows && (h->lda != lda || h->dtype != dtype))))
    st = fail(AMM_ERR_STATE, "amm_handle_import: operand is %lld x %lld (lda %lld, dtype %d), export was %lld x %lld "
              "(lda %lld, dtype %d)", (long long)rows, (long long)cols, (long long)lda, (int)dtype,
              (long long)h->rows, (long long)h->cols, (long long)h->lda, h->dtype);
  if (st != AMM_OK) {
    h->release();
    delete h;
    return st;
  }
  *out = h;
  return AMM_OK;
}
