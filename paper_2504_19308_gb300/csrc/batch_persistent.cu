// Persistent work-queue executor of a batch's cycle-sparsifier products (the batch scheduler of
// arXiv 2504.19308's hot path, for Section 1.2.2's sparsifier): one launch whose CTAs take
// (product, stage, tile) tasks from a device queue until it is empty.
//
// Every product C = A_s B + dA B_s (n x n, FP32) runs six stages, each cut into tiles:
//   KEYS    partial sums of squares of the cycles of A and of B over row blocks;
//   REDUCE  the squared keys from the partials, in the order amm_decompose reduces them;
//   SELECT  the top-k cycles of A and of B ordered by (key desc, index asc), kept-cycle flags zeroed;
//   GATHER  the selected cycles of A and B (k x n each), the kept-cycle flags of A set;
//   COL     C(:, 4 columns) = A_s B (column panels);
//   ROW     C(4 rows, :) += dA B_s (row panels).
// The tiles are the bodies of the one-tile-per-CTA kernels of cycle.cu (cycle_kernels.cuh), the
// key reduction follows amm_decompose's order and the selection its ordering, so a product made
// here is bit-identical to amm_decompose + amm_approx_matmul of the same operands.
//
// Queue and dependencies.  The host writes the queue stage by stage (all KEYS tiles of every
// product, largest product first, then all REDUCE tiles, ...), which is a topological order of the
// tasks.  A CTA takes the next index with an atomic add; before running a task of stage s > 0 its
// thread 0 waits until the product's counter of stage s - 1 has reached that stage's tile count,
// and after the task (block barrier, fence) it increments the counter of stage s.  A task only
// waits for tasks that sit earlier in the queue and were therefore taken by running CTAs, so the
// waits end without any CTA needing to be co-resident with another.  Each wait is bounded (an
// iteration cap and a %globaltimer limit); a wait that runs out stores AMM_ERR_TIMEOUT and the
// product / stage it waited for in the control block, and every CTA stops at its next task.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstring>
#include <vector>

#include "../../include/amm.h"
#include "api_internal.h"
#include "common.cuh"
#include "cycle_kernels.cuh"
#include "kernels.h"
#include "persistent.h"
#include "trace.h"

namespace amm {

enum PqStage { PQ_KEYS = 0, PQ_REDUCE, PQ_SELECT, PQ_GATHER, PQ_COL, PQ_ROW, PQ_NSTAGE };
constexpr int PQ_RED_KEYS = 256;  // keys per REDUCE tile
constexpr int PQ_GATHER_U = 8;    // selected cycles per GATHER tile

struct PqItem {
  const float* A;
  const float* B;
  float* C;
  int64_t lda, ldb, ldc;
  int n, k, rp, nparts;
  float* part[2];         // key partials, nparts x n (A, B)
  double* key2[2];        // squared keys, n
  int32_t* sel[2];        // selections, k
  float* cyc[2];          // selected cycles, k x n
  unsigned char* insel;   // n flags: cycle of A kept
  int ntiles[PQ_NSTAGE];  // tiles per stage
};

struct PqTask {
  int item, stage, tile;
};

struct PqCtl {
  unsigned int head;  // next queue index
  int status;         // AMM_OK, or AMM_ERR_TIMEOUT once a wait ran out
  int item, stage;    // the product and the stage whose counter the failed wait read
};

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Thread 0: wait until *cnt >= need, the control block reports a failure, or the limit passes.
// Returns true when the dependency is met.
__device__ bool pq_wait(const int* cnt, int need, PqCtl* ctl, uint64_t limit_ns, int item, int stage) {
  if (ld_acquire(cnt) >= need) return true;
  const uint64_t t0 = globaltimer_ns();
  // iteration cap as a second bound: each pass sleeps at least ~100 ns and reads L2 twice
  const uint64_t cap = limit_ns / 100 + 100000;
  for (uint64_t it = 0; it < cap; ++it) {
    __nanosleep(100);
    if (ld_acquire(cnt) >= need) return true;
    if (ld_acquire(&ctl->status) != AMM_OK) return false;
    if (globaltimer_ns() - t0 > limit_ns) break;
  }
  if (atomicCAS(&ctl->status, AMM_OK, AMM_ERR_TIMEOUT) == AMM_OK) {
    ctl->item = item;
    ctl->stage = stage;
  }
  return false;
}

// KEYS: part[rb][j] for every cycle j of row block rb, the sums of cyc_keys_tile (the same FMA
// chain over the rows, in order) with all n / 256 cycle blocks of a thread interleaved, so that a
// thread has that many independent loads in flight per row.
AMM_DEV void pq_keys_tile(const float* __restrict__ A, int64_t lda, int n, int rp, float* __restrict__ part, int rb) {
  constexpr int G = PQ_MAX_N / 256;
  const int nb = (n + 255) / 256;
  const int r0 = rb * rp, r1 = min(n, r0 + rp);
  float s[G];
#pragma unroll
  for (int g = 0; g < G; ++g) s[g] = 0.f;
  for (int r = r0; r < r1; ++r) {
    const float* row = A + (int64_t)r * lda;
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int j = g * 256 + threadIdx.x;
      if (g < nb && j < n) {
        const float v = __ldg(row + cwrap<false>(r - j, n));
        s[g] = fmaf(v, v, s[g]);
      }
    }
  }
#pragma unroll
  for (int g = 0; g < G; ++g) {
    const int j = g * 256 + threadIdx.x;
    if (g < nb && j < n) part[(int64_t)rb * n + j] = s[g];
  }
}

// REDUCE: key2[t] for the 256 keys of block tb: thread (x, y) = (tid % 8, tid / 8) sums the
// partial rows y, y + 32, ... of key t0 + x in FP64, then row y = 0 adds the 32 sums in order (the
// order of amm_decompose's reduction).
AMM_DEV void pq_reduce_tile(const float* part, int nparts, int n, double* key2, int tb, double (*sm)[9]) {
  const int x = threadIdx.x & 7, y = threadIdx.x >> 3;
  for (int t0 = tb * PQ_RED_KEYS; t0 < min(n, (tb + 1) * PQ_RED_KEYS); t0 += 8) {
    const int t = t0 + x;
    double s = 0.0;
    if (t < n)
      for (int c = y; c < nparts; c += 32) s += (double)__ldcg(part + (int64_t)c * n + t);
    sm[y][x] = s;
    __syncthreads();
    if (y == 0 && t < n) {
      double v = 0.0;
      for (int yy = 0; yy < 32; ++yy) v += sm[yy][x];
      key2[t] = v;
    }
    __syncthreads();
  }
}

// SELECT: sel = the k largest keys, ordered by (key desc, index asc), by a bitonic sort of all n
// (key, index) pairs (P = next power of two >= n).  Keys are compared as the unsigned bit patterns
// of the doubles, as amm_decompose's radix selection compares them (the same order for every key,
// NaN included); the padding (bits 0, index INT_MAX) sorts after every real key.  insel (A only)
// is zeroed.
AMM_DEV void pq_select_tile(const double* key2, int n, int k, int32_t* sel, unsigned char* insel, unsigned char* smem) {
  int P = 1;
  while (P < n) P <<= 1;
  unsigned long long* sk = reinterpret_cast<unsigned long long*>(smem);
  int* si = reinterpret_cast<int*>(sk + P);
  for (int i = threadIdx.x; i < P; i += CYC_NT) {
    sk[i] = i < n ? (unsigned long long)__double_as_longlong(__ldcg(key2 + i)) : 0ull;
    si[i] = i < n ? i : INT_MAX;
  }
  if (insel)
    for (int i = threadIdx.x; i < n; i += CYC_NT) insel[i] = 0;
  __syncthreads();
  for (int size = 2; size <= P; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = threadIdx.x; i < P; i += CYC_NT) {
        const int q = i ^ stride;
        if (q > i) {
          const bool up = (i & size) == 0;  // this run ends up in (key desc, index asc) order
          const unsigned long long ki = sk[i], kq = sk[q];
          const int ii = si[i], iq = si[q];
          const bool i_first = (ki > kq) || (ki == kq && ii < iq);
          if (up ? !i_first : i_first) {
            sk[i] = kq;
            sk[q] = ki;
            si[i] = iq;
            si[q] = ii;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int u = threadIdx.x; u < k; u += CYC_NT) sel[u] = si[u];
}

AMM_DEV void pq_run(const PqItem& it, const PqTask& t, unsigned char* smem, double (*red)[9]) {
  const int n = it.n;
  const bool p2 = (n & (n - 1)) == 0;
  switch (t.stage) {
    case PQ_KEYS: {  // tile = operand * nparts + row block
      const int op = t.tile / it.nparts, rb = t.tile % it.nparts;
      const float* X = op ? it.B : it.A;
      const int64_t ld = op ? it.ldb : it.lda;
      pq_keys_tile(X, ld, n, it.rp, it.part[op], rb);
      break;
    }
    case PQ_REDUCE: {
      const int per = (n + PQ_RED_KEYS - 1) / PQ_RED_KEYS;
      const int op = t.tile / per;
      pq_reduce_tile(it.part[op], it.nparts, n, it.key2[op], t.tile % per, red);
      break;
    }
    case PQ_SELECT:
      pq_select_tile(it.key2[t.tile], n, it.k, it.sel[t.tile], t.tile == 0 ? it.insel : nullptr, smem);
      break;
    case PQ_GATHER: {
      const int per = (it.k + PQ_GATHER_U - 1) / PQ_GATHER_U;
      const int op = t.tile / per, u0 = (t.tile % per) * PQ_GATHER_U;
      const float* X = op ? it.B : it.A;
      const int64_t ld = op ? it.ldb : it.lda;
      for (int u = u0; u < min(it.k, u0 + PQ_GATHER_U); ++u)
        cyc_gather_tile<true>(X, ld, n, it.sel[op], it.cyc[op], it.insel, u, threadIdx.x, CYC_NT, op == 0);
      break;
    }
    case PQ_COL:
      if (p2) cyc_apply_col_tile<true, true>(it.B, it.ldb, n, it.sel[0], it.k, it.cyc[0], it.C, it.ldc, n, t.tile,
                                             reinterpret_cast<float4*>(smem));
      else cyc_apply_col_tile<false, true>(it.B, it.ldb, n, it.sel[0], it.k, it.cyc[0], it.C, it.ldc, n, t.tile,
                                           reinterpret_cast<float4*>(smem));
      break;
    default:
      if (p2) cyc_apply_row_tile<true, true>(it.A, it.lda, n, it.insel, it.sel[1], it.k, it.cyc[1], it.C, it.ldc, n,
                                             t.tile, reinterpret_cast<float*>(smem));
      else cyc_apply_row_tile<false, true>(it.A, it.lda, n, it.insel, it.sel[1], it.k, it.cyc[1], it.C, it.ldc, n,
                                           t.tile, reinterpret_cast<float*>(smem));
      break;
  }
}

// Three CTAs per SM (at most 85 registers a thread; shared memory 16 n + 4 k bytes each for n <= 4096):
// the gathers of the panel tiles are latency-bound, and three resident CTAs measured 16% faster than
// two on the 64 cycle-sparsifier products of the 256-product batch.
__global__ void __launch_bounds__(CYC_NT, 3) pq_kernel(const PqItem* __restrict__ items, const PqTask* __restrict__ queue,
                                                    int nq, int* __restrict__ done, PqCtl* __restrict__ ctl,
                                                    uint64_t limit_ns) {
  extern __shared__ __align__(16) unsigned char pq_smem[];
  __shared__ double red[32][9];
  __shared__ int s_idx, s_go;
  for (;;) {
    __syncthreads();  // the previous task's reads of shared memory are complete
    if (threadIdx.x == 0) {
      int go = ld_acquire(&ctl->status) == AMM_OK;
      const int i = go ? (int)atomicAdd(&ctl->head, 1u) : nq;
      if (i >= nq) go = 0;
      if (go) {
        const PqTask t = queue[i];
        if (t.stage > 0)
          go = pq_wait(done + t.item * PQ_NSTAGE + t.stage - 1, items[t.item].ntiles[t.stage - 1], ctl, limit_ns,
                       t.item, t.stage - 1);
      }
      s_idx = i;
      s_go = go;
    }
    __syncthreads();
    if (!s_go) return;
    const PqTask t = queue[s_idx];
    pq_run(items[t.item], t, pq_smem, red);
    __syncthreads();  // every thread's writes of this task precede the count
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(done + t.item * PQ_NSTAGE + t.stage, 1);
    }
  }
}

// ============================================================================ host side
struct PqPlan {
  unsigned char* arena = nullptr;  // every device buffer of the plan
  PqItem* d_items = nullptr;
  PqTask* d_queue = nullptr;
  int* d_done = nullptr;
  PqCtl* d_ctl = nullptr;
  size_t ctl_bytes = 0;  // counters + control block, zeroed before each launch
  int nitems = 0, nq = 0, grid = 0;
  size_t smem = 0;
  double work = 0.0;
};

bool pq_eligible(int method, int dtype, int64_t m, int64_t n, int64_t p, bool has_grad) {
  return method == AMM_SPARSE_CYCLE && dtype == AMM_F32 && !has_grad && m == n && p == n && n >= 16 &&
         n <= PQ_MAX_N && n % 4 == 0;
}

static size_t pq_smem_bytes(int n, int k) {
  int P = 1;
  while (P < n) P <<= 1;
  const size_t col = sizeof(float4) * (size_t)n + sizeof(int) * (size_t)k;
  const size_t row = sizeof(float) * CYC_RW * (size_t)n;
  const size_t sel = (sizeof(unsigned long long) + sizeof(int)) * (size_t)P;
  return std::max(col, std::max(row, sel));
}

cudaError_t pq_build(const std::vector<PqDesc>& in, PqPlan** out) {
  *out = nullptr;
  if (in.empty()) return cudaSuccess;
  // layout of the arena: every buffer 256-byte aligned (no cache line holds two buffers)
  auto al = [](size_t b) { return (b + 255) / 256 * 256; };
  size_t off = 0;
  std::vector<PqItem> items(in.size());
  std::vector<size_t> offs;
  const size_t items_off = off;
  off += al(sizeof(PqItem) * in.size());
  for (size_t i = 0; i < in.size(); ++i) {
    const PqDesc& d = in[i];
    PqItem& it = items[i];
    it.A = d.A;
    it.B = d.B;
    it.C = d.C;
    it.lda = d.lda;
    it.ldb = d.ldb;
    it.ldc = d.ldc;
    it.n = (int)d.n;
    it.k = (int)d.k;
    it.rp = cyc_rows_per_part(it.n);
    it.nparts = (it.n + it.rp - 1) / it.rp;
    for (int op = 0; op < 2; ++op) {
      offs.push_back(off);
      off += al(sizeof(float) * (size_t)it.nparts * it.n);
      offs.push_back(off);
      off += al(sizeof(double) * (size_t)it.n);
      offs.push_back(off);
      off += al(sizeof(int32_t) * (size_t)it.k);
      offs.push_back(off);
      off += al(sizeof(float) * (size_t)it.k * it.n);
    }
    offs.push_back(off);
    off += al((size_t)it.n);
    it.ntiles[PQ_KEYS] = 2 * it.nparts;
    it.ntiles[PQ_REDUCE] = 2 * ((it.n + PQ_RED_KEYS - 1) / PQ_RED_KEYS);
    it.ntiles[PQ_SELECT] = 2;
    it.ntiles[PQ_GATHER] = 2 * ((it.k + PQ_GATHER_U - 1) / PQ_GATHER_U);
    it.ntiles[PQ_COL] = (it.n + CYC_CW - 1) / CYC_CW;
    it.ntiles[PQ_ROW] = (it.n + CYC_RW - 1) / CYC_RW;
  }
  // queue: stage-major, products in descending order of work within a stage
  std::vector<int> order(in.size());
  for (size_t i = 0; i < in.size(); ++i) order[i] = (int)i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return (double)items[a].n * items[a].n * items[a].k > (double)items[b].n * items[b].n * items[b].k;
  });
  std::vector<PqTask> queue;
  for (int s = 0; s < PQ_NSTAGE; ++s)
    for (int i : order)
      for (int t = 0; t < items[i].ntiles[s]; ++t) queue.push_back(PqTask{i, s, t});
  const size_t queue_off = off;
  off += al(sizeof(PqTask) * queue.size());
  const size_t done_off = off;
  const size_t ctl_bytes = al(sizeof(int) * PQ_NSTAGE * in.size()) + al(sizeof(PqCtl));
  off += ctl_bytes;

  PqPlan* p = new PqPlan();
  cudaError_t e = cudaMalloc((void**)&p->arena, off);
  if (e != cudaSuccess) {
    delete p;
    return e;
  }
  size_t oi = 0;
  size_t smem = 0;
  for (size_t i = 0; i < in.size(); ++i) {
    PqItem& it = items[i];
    for (int op = 0; op < 2; ++op) {
      it.part[op] = (float*)(p->arena + offs[oi++]);
      it.key2[op] = (double*)(p->arena + offs[oi++]);
      it.sel[op] = (int32_t*)(p->arena + offs[oi++]);
      it.cyc[op] = (float*)(p->arena + offs[oi++]);
    }
    it.insel = p->arena + offs[oi++];
    smem = std::max(smem, pq_smem_bytes(it.n, it.k));
    p->work += 4.0 * it.k * (double)it.n * it.n;
  }
  p->d_items = (PqItem*)(p->arena + items_off);
  p->d_queue = (PqTask*)(p->arena + queue_off);
  p->d_done = (int*)(p->arena + done_off);
  p->d_ctl = (PqCtl*)(p->arena + done_off + al(sizeof(int) * PQ_NSTAGE * in.size()));
  p->ctl_bytes = ctl_bytes;
  p->nitems = (int)in.size();
  p->nq = (int)queue.size();
  p->smem = smem;
  e = cudaMemcpy(p->d_items, items.data(), sizeof(PqItem) * items.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(p->d_queue, queue.data(), sizeof(PqTask) * queue.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute((const void*)pq_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per_sm = 0, dev = 0, nsm = 0;
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pq_kernel, CYC_NT, smem);
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess && per_sm < 1) e = cudaErrorInvalidConfiguration;
  if (e != cudaSuccess) {
    cudaFree(p->arena);
    delete p;
    return e;
  }
  // every resident slot: the launch drains its queue at the whole GPU's rate, and as its CTAs
  // run out of tasks the SMs go to the kernels of the other items, already queued on their streams
  // (a grid cut to the products' share of the work would hold that share of the SMs to the end)
  p->grid = std::max(1, std::min(per_sm * nsm, p->nq));
  *out = p;
  return cudaSuccess;
}

cudaError_t pq_launch(PqPlan* p, cudaStream_t st, uint64_t limit_ns) {
  if (!p) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(p->d_done, 0, p->ctl_bytes, st);
  if (e != cudaSuccess) return e;
  AMM_TRACE_W("pq_cycle_batch", st, p->work, 0.0, nullptr);
  pq_kernel<<<p->grid, CYC_NT, p->smem, st>>>(p->d_items, p->d_queue, p->nq, p->d_done, p->d_ctl, limit_ns);
  return cudaGetLastError();
}

cudaError_t pq_status(PqPlan* p, int32_t* status, int32_t* item, int32_t* stage) {
  *status = AMM_OK;
  *item = *stage = -1;
  if (!p) return cudaSuccess;
  PqCtl c;
  cudaError_t e = cudaMemcpy(&c, p->d_ctl, sizeof(c), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return e;
  *status = c.status;
  if (c.status != AMM_OK) {
    *item = c.item;
    *stage = c.stage;
  }
  return cudaSuccess;
}


void pq_destroy(PqPlan* p) {
  if (!p) return;
  cudaFree(p->arena);
  delete p;
}

}  // namespace amm

// Test hook: one persistent launch (one CTA) over a queue whose only task waits for a stage that
// no task completes, so that its bounded wait runs out after limit_ns.  Writes the control block's
// status (AMM_ERR_TIMEOUT expected) and the product / stage the wait read.
extern "C" amm_status_t amm_debug_persistent_wait_timeout(int64_t limit_ns, void* stream, int32_t* status_out,
                                                          int32_t* stage_out) {
  using namespace amm;
  if (!status_out || !stage_out) return fail(AMM_ERR_INVALID_ARG, "amm_debug_persistent_wait_timeout: NULL output");
  if (limit_ns <= 0 || limit_ns > 5000000000LL)
    return fail(AMM_ERR_INVALID_ARG, "amm_debug_persistent_wait_timeout: limit_ns must be in (0, 5e9]");
  cudaStream_t st = (cudaStream_t)stream;
  PqItem it;
  std::memset(&it, 0, sizeof(it));
  it.n = 16;
  it.k = 1;
  it.ntiles[PQ_COL] = 1;  // the ROW task below waits for one COL tile; the queue holds none
  const PqTask task{0, PQ_ROW, 0};
  unsigned char* buf = nullptr;
  const size_t items_off = 0, queue_off = 256, done_off = 512, ctl_off = 768, bytes = 1024;
  cudaError_t e = cudaMalloc((void**)&buf, bytes);
  if (e != cudaSuccess) return cuda_fail(e, "amm_debug_persistent_wait_timeout: cudaMalloc");
  e = cudaMemsetAsync(buf, 0, bytes, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(buf + items_off, &it, sizeof(it), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(buf + queue_off, &task, sizeof(task), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    pq_kernel<<<1, CYC_NT, 0, st>>>((const PqItem*)(buf + items_off), (const PqTask*)(buf + queue_off), 1,
                                    (int*)(buf + done_off), (PqCtl*)(buf + ctl_off), (uint64_t)limit_ns);
    e = cudaGetLastError();
  }
  PqCtl c;
  std::memset(&c, 0, sizeof(c));
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaMemcpy(&c, buf + ctl_off, sizeof(c), cudaMemcpyDeviceToHost);
  cudaFree(buf);
  if (e != cudaSuccess) return cuda_fail(e, "amm_debug_persistent_wait_timeout");
  *status_out = c.status;
  *stage_out = c.stage;
  return AMM_OK;
}
