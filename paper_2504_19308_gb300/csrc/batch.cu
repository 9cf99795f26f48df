// Batches of independent first-order products of uneven sizes (for example the layers of an
// LLM-shaped stack).  amm_batch_run executes every item (decompose A, decompose B, product, the
// backward for items added with amm_batch_add_grad, release) on a pool of 16 streams forked from
// the caller's stream, the largest items first, each on the least loaded stream.  The forward
// cycle-sparsifier products (FP32, square, n <= 4096) run instead in one persistent launch that
// takes (product, stage, tile) tasks from a device queue (batch_persistent.cu); that launch is
// placed on the pool like one item whose work is theirs.  With use_graph the first
// run executes eagerly once (building twiddle tables and setting kernel attributes, which must
// not happen inside a capture), then captures the same work into one CUDA graph; every later
// run is a single graph launch.  Device memory of the handles is stream-ordered, so inside the
// graph it becomes graph allocation nodes.
#include <cuda_runtime.h>

#include <algorithm>
#include <new>
#include <numeric>
#include <vector>

#include "../../include/amm.h"
#include "api_internal.h"
#include "persistent.h"

struct amm_batch {
  struct Item {
    const void* A;
    const void* B;
    float* C;
    int64_t m, n, p, lda, ldb, ldc, k;
    int dtype, method;
    amm_opts_t oa, ob;
    // optional backward of the item (amm_batch_add_grad): dC in, dA / dB out (either may be NULL)
    const float* dC = nullptr;
    float* dA = nullptr;
    float* dB = nullptr;
    int64_t lddc = 0, ldda = 0, lddb = 0;
  };
  std::vector<Item> items;
  int nstreams = 16;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> events;  // one per stream (join) + fork
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  bool captured = false;
  // persistent executor of the cycle-sparsifier items
  bool persistent = true;
  uint64_t wait_limit_ns = 2000000000ull;
  amm::PqPlan* pq = nullptr;
  size_t pq_built_for = 0;         // item count the plan was built for
  std::vector<size_t> pq_items;    // batch indices of the plan's products
  cudaStream_t last_parent = nullptr;
};

using namespace amm;

extern "C" amm_status_t amm_batch_create(amm_batch_t* out) {
  if (!out) return fail(AMM_ERR_INVALID_ARG, "amm_batch_create: out is NULL");
  amm_batch* b = new (std::nothrow) amm_batch();
  if (!b) return fail(AMM_ERR_OOM, "amm_batch_create: host allocation");
  *out = b;
  return AMM_OK;
}

extern "C" amm_status_t amm_batch_add(amm_batch_t b, const void* A, const void* B, float* C, int64_t m, int64_t n,
                                      int64_t p, int64_t lda, int64_t ldb, int64_t ldc, amm_dtype_t dtype,
                                      amm_method_t method, int64_t k, const amm_opts_t* opts_a,
                                      const amm_opts_t* opts_b) {
  if (!b || !A || !B || !C) return fail(AMM_ERR_INVALID_ARG, "amm_batch_add: NULL argument");
  if (b->captured) return fail(AMM_ERR_STATE, "amm_batch_add: batch already captured into a graph");
  if (m <= 0 || n <= 0 || p <= 0 || k <= 0 || lda < n || ldb < p || ldc < p)
    return fail(AMM_ERR_INVALID_ARG, "amm_batch_add: bad sizes");
  // checked here rather than when the batch runs, after earlier items have launched
  if (dtype != AMM_F32 && dtype != AMM_BF16) return fail(AMM_ERR_INVALID_ARG, "amm_batch_add: bad dtype %d", dtype);
  if (method != AMM_SVD && method != AMM_CIRCULANT && method != AMM_SPARSE_FOURIER && method != AMM_SPARSE_CYCLE)
    return fail(AMM_ERR_INVALID_ARG, "amm_batch_add: bad method %d", (int)method);
  if ((opts_a && opts_a->struct_size != sizeof(amm_opts_t)) || (opts_b && opts_b->struct_size != sizeof(amm_opts_t)))
    return fail(AMM_ERR_INVALID_ARG, "amm_batch_add: opts struct_size differs from sizeof(amm_opts_t)");
  amm_batch::Item it;
  it.A = A;
  it.B = B;
  it.C = C;
  it.m = m;
  it.n = n;
  it.p = p;
  it.lda = lda;
  it.ldb = ldb;
  it.ldc = ldc;
  it.k = k;
  it.dtype = dtype;
  it.method = method;
  amm_opts_init(&it.oa);
  amm_opts_init(&it.ob);
  if (opts_a) it.oa = *opts_a;
  if (opts_b) it.ob = *opts_b;
  it.oa.role = AMM_LEFT;
  it.ob.role = AMM_RIGHT;
  if (it.oa.forced_selection || it.ob.forced_selection)
    return fail(AMM_ERR_INVALID_ARG, "amm_batch_add: forced selections are not supported in batches");
  b->items.push_back(it);
  return AMM_OK;
}

extern "C" amm_status_t amm_batch_add_grad(amm_batch_t b, const void* A, const void* B, float* C, int64_t m,
                                           int64_t n, int64_t p, int64_t lda, int64_t ldb, int64_t ldc,
                                           amm_dtype_t dtype, amm_method_t method, int64_t k,
                                           const amm_opts_t* opts_a, const amm_opts_t* opts_b, const float* dC,
                                           int64_t lddc, float* dA, int64_t ldda, float* dB, int64_t lddb) {
  if (!b || !dC || (!dA && !dB)) return fail(AMM_ERR_INVALID_ARG, "amm_batch_add_grad: NULL dC, or both dA and dB NULL");
  if (lddc < p || (dA && ldda < n) || (dB && lddb < p))
    return fail(AMM_ERR_INVALID_ARG, "amm_batch_add_grad: bad leading dimension");
  const size_t before = b->captured ? 0 : b->items.size();
  amm_status_t st = amm_batch_add(b, A, B, C, m, n, p, lda, ldb, ldc, dtype, method, k, opts_a, opts_b);
  if (st != AMM_OK) return st;
  if (b->items.size() != before + 1) return fail(AMM_ERR_STATE, "amm_batch_add_grad: item not recorded");
  auto& it = b->items.back();
  it.dC = dC;
  it.lddc = lddc;
  it.dA = dA;
  it.ldda = ldda;
  it.dB = dB;
  it.lddb = lddb;
  return AMM_OK;
}

// (Re)build the persistent plan for the batch's eligible items when the item list changed.  Not
// called inside a capture (the first graph run executes eagerly first).
static amm_status_t plan_persistent(amm_batch* b) {
  if (!b->persistent || b->pq_built_for == b->items.size()) return AMM_OK;
  amm::pq_destroy(b->pq);  // cudaFree waits for earlier runs
  b->pq = nullptr;
  b->pq_items.clear();
  std::vector<amm::PqDesc> descs;
  for (size_t i = 0; i < b->items.size(); ++i) {
    const auto& it = b->items[i];
    if (!amm::pq_eligible(it.method, it.dtype, it.m, it.n, it.p, it.dC != nullptr) || it.k > it.n) continue;
    descs.push_back(amm::PqDesc{(const float*)it.A, (const float*)it.B, it.C, it.lda, it.ldb, it.ldc, it.n, it.k});
    b->pq_items.push_back(i);
  }
  cudaError_t e = amm::pq_build(descs, &b->pq);
  if (e != cudaSuccess) {
    b->pq_items.clear();
    return cuda_fail(e, "batch: persistent executor set-up");
  }
  b->pq_built_for = b->items.size();
  return AMM_OK;
}

static amm_status_t run_items(amm_batch* b, cudaStream_t parent) {
  cudaError_t e;
  if (b->streams.empty()) {
    for (int i = 0; i < b->nstreams; ++i) {
      cudaStream_t s;
      if ((e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != cudaSuccess) return cuda_fail(e, "batch stream");
      b->streams.push_back(s);
    }
    for (int i = 0; i <= b->nstreams; ++i) {
      cudaEvent_t ev;
      if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) return cuda_fail(e, "batch event");
      b->events.push_back(ev);
    }
  }
  // fork: every worker stream waits for the parent
  cudaEvent_t fork = b->events[b->nstreams];
  if ((e = cudaEventRecord(fork, parent)) != cudaSuccess) return cuda_fail(e, "batch fork");
  for (cudaStream_t s : b->streams)
    if ((e = cudaStreamWaitEvent(s, fork, 0)) != cudaSuccess) return cuda_fail(e, "batch fork wait");
  // Longest first: items in descending order of their exact-product work m n p, each on the worker
  // stream with the least work assigned so far (greedy longest-processing-time list scheduling), so
  // the large products start first and the small ones fill the other streams around them.  Every
  // item runs the same kernels whatever its stream, so the results do not depend on the order.
  std::vector<size_t> order(b->items.size());
  std::iota(order.begin(), order.end(), (size_t)0);
  auto work = [&](size_t i) {
    const auto& it = b->items[i];
    return (double)it.m * (double)it.n * (double)it.p * (it.dC ? 3.0 : 1.0);
  };
  std::vector<double> wk(b->items.size());
  for (size_t i = 0; i < b->items.size(); ++i) wk[i] = work(i);
  amm_status_t st = plan_persistent(b);
  if (st != AMM_OK) return st;
  // the persistent launch stands in the order for its products: their summed work, once
  std::vector<char> in_pq(b->items.size(), 0);
  double pq_w = 0.0;
  for (size_t i : b->pq_items) {
    in_pq[i] = 1;
    pq_w += wk[i];
  }
  const size_t PQ = (size_t)-1;
  order.erase(std::remove_if(order.begin(), order.end(), [&](size_t i) { return in_pq[i] != 0; }), order.end());
  if (b->pq) order.push_back(PQ);
  auto wof = [&](size_t i) { return i == PQ ? pq_w : wk[i]; };
  std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) { return wof(x) > wof(y); });
  std::vector<double> load(b->streams.size(), 0.0);
  for (size_t oi = 0; oi < order.size() && st == AMM_OK; ++oi) {
    const size_t si = (size_t)(std::min_element(load.begin(), load.end()) - load.begin());
    load[si] += wof(order[oi]);
    cudaStream_t s = b->streams[si];
    if (order[oi] == PQ) {
      if ((e = amm::pq_launch(b->pq, s, b->wait_limit_ns)) != cudaSuccess) st = cuda_fail(e, "batch: persistent launch");
      continue;
    }
    auto& it = b->items[order[oi]];
    amm_handle_t ha = nullptr, hb = nullptr;
    st = amm_decompose(it.A, it.m, it.n, it.lda, (amm_dtype_t)it.dtype, (amm_method_t)it.method, it.k, &it.oa, s, &ha);
    if (st == AMM_OK)
      st = amm_decompose(it.B, it.n, it.p, it.ldb, (amm_dtype_t)it.dtype, (amm_method_t)it.method, it.k, &it.ob, s, &hb);
    if (st == AMM_OK) st = amm_approx_matmul(ha, hb, it.C, it.ldc, s);
    if (st == AMM_OK && it.dC)
      st = amm_approx_matmul_backward(ha, hb, it.dC, it.lddc, it.dA, it.ldda, it.dB, it.lddb, s);
    if (ha) amm_handle_destroy(ha);
    if (hb) amm_handle_destroy(hb);
  }
  // join: the parent waits for every worker stream
  for (int i = 0; i < b->nstreams; ++i) {
    if ((e = cudaEventRecord(b->events[i], b->streams[i])) != cudaSuccess) return cuda_fail(e, "batch join");
    if ((e = cudaStreamWaitEvent(parent, b->events[i], 0)) != cudaSuccess) return cuda_fail(e, "batch join wait");
  }
  return st;
}

extern "C" amm_status_t amm_batch_set_persistent(amm_batch_t b, int32_t on, int64_t wait_limit_ns) {
  if (!b) return fail(AMM_ERR_INVALID_ARG, "amm_batch_set_persistent: NULL batch");
  if (b->captured) return fail(AMM_ERR_STATE, "amm_batch_set_persistent: batch already captured into a graph");
  if (wait_limit_ns <= 0) return fail(AMM_ERR_INVALID_ARG, "amm_batch_set_persistent: wait_limit_ns must be > 0");
  if ((on != 0) != b->persistent) {
    amm::pq_destroy(b->pq);
    b->pq = nullptr;
    b->pq_items.clear();
    b->pq_built_for = 0;
  }
  b->persistent = on != 0;
  b->wait_limit_ns = (uint64_t)wait_limit_ns;
  return AMM_OK;
}

extern "C" amm_status_t amm_batch_status(amm_batch_t b, int32_t* status, int64_t* item, int32_t* stage,
                                         int32_t* persistent_products) {
  if (!b || !status || !item || !stage || !persistent_products)
    return fail(AMM_ERR_INVALID_ARG, "amm_batch_status: NULL argument");
  *persistent_products = (int32_t)b->pq_items.size();
  cudaError_t e = b->last_parent ? cudaStreamSynchronize(b->last_parent) : cudaSuccess;
  int32_t it = -1;
  if (e == cudaSuccess) e = amm::pq_status(b->pq, status, &it, stage);
  if (e != cudaSuccess) return cuda_fail(e, "amm_batch_status");
  *item = (it >= 0 && (size_t)it < b->pq_items.size()) ? (int64_t)b->pq_items[(size_t)it] : -1;
  return AMM_OK;
}

extern "C" amm_status_t amm_batch_run(amm_batch_t b, void* stream, int32_t use_graph) {
  if (!b) return fail(AMM_ERR_INVALID_ARG, "amm_batch_run: NULL batch");
  cudaStream_t parent = (cudaStream_t)stream;
  b->last_parent = parent;
  if (!use_graph) return run_items(b, parent);
  cudaError_t e;
  if (!b->captured) {
    amm_status_t st = run_items(b, parent);  // eager pass: tables, attributes, allocator pool warm
    if (st != AMM_OK) return st;
    if ((e = cudaStreamSynchronize(parent)) != cudaSuccess) return cuda_fail(e, "batch warm-up");
    cudaStream_t cap = nullptr;
    if ((e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking)) != cudaSuccess) return cuda_fail(e, "capture stream");
    if ((e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) {
      cudaStreamDestroy(cap);
      return cuda_fail(e, "batch capture");
    }
    st = run_items(b, cap);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(cap, &g);
    cudaStreamDestroy(cap);
    if (st != AMM_OK) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    if (e != cudaSuccess) return cuda_fail(e, "batch end capture");
    if ((e = cudaGraphInstantiate(&b->exec, g, 0)) != cudaSuccess) {
      cudaGraphDestroy(g);
      return cuda_fail(e, "batch instantiate");
    }
    b->graph = g;
    b->captured = true;
  }
  if ((e = cudaGraphLaunch(b->exec, parent)) != cudaSuccess) return cuda_fail(e, "batch graph launch");
  return AMM_OK;
}

extern "C" amm_status_t amm_batch_destroy(amm_batch_t b) {
  if (!b) return fail(AMM_ERR_INVALID_ARG, "amm_batch_destroy: NULL batch");
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  amm::pq_destroy(b->pq);
  for (auto s : b->streams) cudaStreamDestroy(s);
  for (auto ev : b->events) cudaEventDestroy(ev);
  delete b;
  return AMM_OK;
}
