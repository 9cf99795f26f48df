// Tensor-core GEMM for the thin low-rank products (Alg. 1 and Section 2.2), sm_103a.
//
//   C[M x N] = alpha * A[M x K] * B[N x K]^T + beta * C        (A, B K-major: row-major along K)
//
// One 128 x BN output tile per CTA, BN = 128, or the smallest of 16 / 32 / 64 that covers N when
// N is that thin (the sketch and projection GEMMs of Alg. 1 have N = k): the MMAs, the B tiles and,
// in the TF32X3 mode, the hi / lo split of B then scale with k instead of a fixed 128.  K may be split over grid.z: every split stores its partial
// tile in a workspace, and a reduction kernel sums the partials in split order (compensated FP32)
// into C.  (Summing in the last CTA of each tile left one CTA per tile doing all the loads, which
// measured slower than spreading the sum over the whole GPU.)
// Warps 0-3 drain the accumulator from tensor memory, warp 4 drives TMA, warp 5 issues MMAs:
//   * TMA (cp.async.bulk.tensor.2d) loads 128-row x 128-byte boxes of A and B with the 128-byte
//     swizzle into a STAGES-deep ring, completion tracked by mbarrier transaction counts;
//   * one thread issues tcgen05.mma (cta_group::1, M = 128, N = 128) per 32-byte K slice, the
//     accumulator lives in 128 TMEM columns, tcgen05.commit releases each smem stage;
//   * the epilogue waits for the last commit, reads TMEM with tcgen05.ld.32x32b and stores
//     through a padded shared tile so that every warp store covers 128 contiguous bytes.
// Element modes:
//   BF16  kind::f16, BF16 inputs, FP32 accumulation (the BF16 precision mode);
//   TF32X3  FP32 inputs split in shared memory into hi = tf32(x) and lo = tf32(x - hi), both
//           rounded to nearest; kind::tf32 products hi*hi + hi*lo + lo*hi give products within
//           about 2^-21 relative (the lo*lo term and the rounding of lo are dropped).  The
//           small correction products accumulate in a second TMEM accumulator, and long K is
//           split into chains of at most UM_TF32_MAX_KB k-blocks whose partials are summed with
//           compensation, which bounds the rounding the tensor core's FP32 accumulation adds.
// Every mbarrier wait is bounded; a wait that gives up sets *err and the CTA drains and exits.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <type_traits>

#include "api_internal.h"
#include "common.cuh"
#include "kernels.h"
#include "trace.h"

namespace amm {

constexpr int UM_BM = 128;
constexpr int UM_THREADS = 192;
constexpr int UM_TF32_MAX_KB = 16;  // longest TF32X3 accumulation chain, in 32-wide k-blocks
constexpr int UM_CTA_FIXED_KB = 8;  // per-CTA set-up and epilogue cost, in k-blocks (split choice)
constexpr int UM_SHORT_KB = 4;      // k-blocks up to which a wide output takes the short ring
constexpr uint32_t UM_SPIN_LIMIT = 1u << 26;  // ~ seconds of polling, then give up

// ----------------------------------------------------------------------------- PTX wrappers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// bounded wait for the phase with the given parity; returns false if it gave up
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  for (uint32_t it = 0; it < UM_SPIN_LIMIT; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* tm, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          smem_u32(dst)),
      "l"(tm), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

// 64-bit shared-memory matrix descriptor (tcgen05): K-major, 128-byte swizzle, 8-row groups 1024 B apart
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);       // start address
  d |= (uint64_t)(16u >> 4) << 16;                // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024u >> 4) << 32;              // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;                         // descriptor version for tcgen05
  d |= (uint64_t)2 << 61;                         // 128-byte swizzle
  return d;
}

// instruction descriptor: D = F32, A/B format (1 = BF16, 2 = TF32), K-major A and B, N, M
__host__ __device__ constexpr uint32_t umma_idesc(uint32_t ab_format, int M, int N) {
  return (1u << 4) | (ab_format << 7) | (ab_format << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

template <bool TF32>
__device__ __forceinline__ void umma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
  if constexpr (TF32) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
  }
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// 16 consecutive accumulator columns of this warp's 32 TMEM lanes
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
      "[%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// 32 consecutive accumulator columns of this warp's 32 TMEM lanes
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// ----------------------------------------------------------------------------- the kernel
// Shared memory (1024-aligned): a ring of RAW stages {A tile, B tile} written by TMA; for TF32X3
// also a ring of SLOTS split slots {A hi, B hi, A lo, B lo} read by the MMAs; then barriers.
// BF16 tiles go from the TMA ring straight to the MMAs.  TF32X3 tiles are split into hi/lo by
// the four epilogue warps, which release the raw stage as soon as it is read, so TMA keeps
// RAW stages in flight while the MMAs work from the split ring.
// SHORT: a ring for products of at most UM_SHORT_KB k-blocks (two TMA stages, one split slot), so
// that two CTAs fit per SM and one CTA's prologue and epilogue overlap the other's work; used for
// the wide outputs of short contractions (the n x n product of two n x 2k factors).
template <bool TF32, int BN, bool SHORT = false>
struct UmmaCfg {
  static_assert(BN == 16 || BN == 32 || BN == 64 || BN == 128, "tile widths of the M = 128 MMA used here");
  static constexpr int ELEM = TF32 ? 4 : 2;
  static constexpr int BK = 128 / ELEM;                      // one 128-byte swizzle atom of K
  static constexpr int MMA_K = 32 / ELEM;                    // K per tcgen05.mma
  static constexpr int A_BYTES = UM_BM * 128;                // 16 KiB A tile
  static constexpr int B_BYTES = BN * 128;                   // BN rows of B (a multiple of 1024 bytes)
  // the thinnest tiles run two CTAs per SM (each CTA's prologue, pipeline fill and epilogue then
  // overlap the other's streaming), with the ring depth cut to fit: BN = 16 and 32 in both modes
  // (TF32X3 at BN = 32: three TMA stages and one split slot, 101.6 KB)
  static constexpr int CTAS = (SHORT || BN == 16 || BN == 32) ? 2 : 1;
  static constexpr int RAW = SHORT ? 2
                             : TF32 ? (BN == 128 ? 3 : BN == 16 ? 2 : BN == 32 ? 3 : 4)
                                    : (CTAS == 2 ? 5 : BN == 128 ? 5 : 7);  // TMA stages
  static constexpr int RAW_BYTES = A_BYTES + B_BYTES;        // A, B
  static constexpr int SLOTS = TF32 ? (SHORT || BN == 32 ? 1 : 2) : 0;  // split slots
  static constexpr int SLOT_BYTES = 2 * RAW_BYTES;           // A hi, B hi, A lo, B lo
  // accumulator columns (TF32X3: main + correction), a power of two >= 32 as tcgen05.alloc requires
  static constexpr uint32_t TMEM_COLS = (TF32 ? 2 * BN : BN) < 32 ? 32u : (uint32_t)(TF32 ? 2 * BN : BN);
  static constexpr size_t SMEM = 1024 + (size_t)RAW * RAW_BYTES + (size_t)SLOTS * SLOT_BYTES + 256;
  static_assert(SMEM * CTAS <= 232448, "dynamic shared memory per SM");
};

// Round to the nearest TF32 value (10 fraction bits, ties away from zero); Inf and NaN pass.
__device__ __forceinline__ float tf32_round(float x) {
  const uint32_t u = __float_as_uint(x);
  if ((u & 0x7F800000u) == 0x7F800000u) return x;
  return __uint_as_float((u + 0x1000u) & 0xFFFFE000u);
}

// Split raw x into hi = tf32(x) and lo = tf32(x - hi).  Both halves are rounded to nearest, so
// |x - hi - lo| <= 2^-22 |x| and the tensor core's operand truncation loses nothing.  The copy
// keeps byte offsets, so the 128-byte-swizzled layout of the TMA tile carries over.
__device__ __forceinline__ void split_tile(const float* raw, float* hi, float* lo, int nfloat, int tid, int nthr) {
  const float4* r4 = reinterpret_cast<const float4*>(raw);
  float4* h4 = reinterpret_cast<float4*>(hi);
  float4* l4 = reinterpret_cast<float4*>(lo);
#pragma unroll 4
  for (int i = tid; i < nfloat / 4; i += nthr) {
    float4 x = r4[i], h, l;
    h.x = tf32_round(x.x); l.x = tf32_round(x.x - h.x);
    h.y = tf32_round(x.y); l.y = tf32_round(x.y - h.y);
    h.z = tf32_round(x.z); l.z = tf32_round(x.z - h.z);
    h.w = tf32_round(x.w); l.w = tf32_round(x.w - h.w);
    h4[i] = h;
    l4[i] = l;
  }
}

// TRANS: the kernel computes C^T = B A^T (its M, N are the caller's N, M) and stores C itself:
// element (i, j) of its tile goes to C[j * ldc + i], so a warp's 32 lanes (consecutive i) write 128
// contiguous bytes per column j; split partials are kept in C's own [z][N][M] layout.
template <bool TF32, int BN, bool TRANS, bool SHORT = false>
__global__ void __launch_bounds__(UM_THREADS, UmmaCfg<TF32, BN, SHORT>::CTAS)
    umma_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int M, int N,
                     int K, float alpha, float beta, float* __restrict__ C, int64_t ldc, int per,
                     float* __restrict__ ws, int* __restrict__ err) {
  using Cfg = UmmaCfg<TF32, BN, SHORT>;
  constexpr int RAW = Cfg::RAW;
  constexpr int SLOTS = Cfg::SLOTS > 0 ? Cfg::SLOTS : 1;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* tiles = smem;                                           // raw ring
  unsigned char* slots = tiles + (size_t)RAW * Cfg::RAW_BYTES;          // split ring (TF32X3)
  uint64_t* full = reinterpret_cast<uint64_t*>(slots + (size_t)Cfg::SLOTS * Cfg::SLOT_BYTES);
  uint64_t* empty = full + RAW;
  uint64_t* sfull = empty + RAW;   // split slot written
  uint64_t* sempty = sfull + SLOTS;  // split slot consumed by the MMAs
  uint64_t* accum = sempty + SLOTS;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accum + 1);
  __shared__ int s_fail;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * UM_BM, n0 = blockIdx.x * BN;
  // split z takes a contiguous run of k-blocks (each CTA streams its row segments in order: DRAM
  // page locality; interleaving the splits measured 2x slower)
  const int kblocks = (K + Cfg::BK - 1) / Cfg::BK;
  const int kb0 = (int)blockIdx.z * per;  // the host makes every split non-empty
  const int nkb = min(per, kblocks - kb0);

  if (threadIdx.x == 0) {
    s_fail = 0;
    for (int s = 0; s < RAW; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], TF32 ? 128 : 1);  // TF32X3: the splitters release it; BF16: the MMA commit
    }
    for (int t = 0; t < SLOTS; ++t) {
      mbar_init(&sfull[t], 128);
      mbar_init(&sempty[t], 1);
    }
    mbar_init(accum, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  constexpr uint32_t TMEM_COLS = Cfg::TMEM_COLS;
  if (warp == 0) {  // TMEM: 128 lanes x BN FP32 columns per accumulator
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  bool ok = true;

  if (warp == 4) {
    // ---------------------------------------------------------------- TMA producer
    if (lane == 0) {
      for (int kb = 0; kb < nkb && ok; ++kb) {
        const int s = kb % RAW;
        const uint32_t ph = (kb / RAW) & 1;
        ok = mbar_wait(&empty[s], ph ^ 1);
        if (!ok) break;
        unsigned char* st = tiles + (size_t)s * Cfg::RAW_BYTES;
        mbar_expect_tx(&full[s], Cfg::A_BYTES + Cfg::B_BYTES);
        const int kx = (kb0 + kb) * Cfg::BK;
        tma_load_2d(st, &tmA, &full[s], kx, m0);
        tma_load_2d(st + Cfg::A_BYTES, &tmB, &full[s], kx, n0);
      }
      if (!ok) atomicExch(&s_fail, 1);
    }
  } else if (warp == 5) {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      constexpr uint32_t idesc = umma_idesc(TF32 ? 2u : 1u, UM_BM, BN);
      for (int kb = 0; kb < nkb && ok; ++kb) {
        unsigned char* st;
        if constexpr (TF32) {
          const int t = kb % SLOTS;
          ok = mbar_wait(&sfull[t], (kb / SLOTS) & 1);
          st = slots + (size_t)t * Cfg::SLOT_BYTES;
        } else {
          const int s = kb % RAW;
          ok = mbar_wait(&full[s], (kb / RAW) & 1);
          st = tiles + (size_t)s * Cfg::RAW_BYTES;
        }
        if (!ok) break;
        tc_fence_after();
        const uint32_t a_hi = smem_u32(st), b_hi = smem_u32(st + Cfg::A_BYTES);
        const uint32_t a_lo = smem_u32(st + Cfg::RAW_BYTES), b_lo = smem_u32(st + Cfg::RAW_BYTES + Cfg::A_BYTES);
#pragma unroll
        for (int k = 0; k < Cfg::BK / Cfg::MMA_K; ++k) {
          const uint32_t off = k * 32;  // 32-byte K slice inside the swizzle atom
          const uint32_t acc = (kb > 0 || k > 0) ? 1u : 0u;
          umma<TF32>(tmem, umma_desc(a_hi + off), umma_desc(b_hi + off), idesc, acc);
          if constexpr (TF32) {  // correction products into their own accumulator (columns BN..2 BN-1)
            umma<TF32>(tmem + (uint32_t)BN, umma_desc(a_hi + off), umma_desc(b_lo + off), idesc, acc);
            umma<TF32>(tmem + (uint32_t)BN, umma_desc(a_lo + off), umma_desc(b_hi + off), idesc, 1u);
          }
        }
        // the slot / stage is free once these MMAs have read it
        if constexpr (TF32) umma_commit(&sempty[kb % SLOTS]);
        else umma_commit(&empty[kb % RAW]);
      }
      umma_commit(accum);
      if (!ok) atomicExch(&s_fail, 1);
    }
  } else {
    // ---------------------------------------------------------------- warps 0-3
    if constexpr (TF32) {
      for (int kb = 0; kb < nkb && ok; ++kb) {
        const int s = kb % RAW, t = kb % SLOTS;
        ok = mbar_wait(&full[s], (kb / RAW) & 1);
        if (ok) ok = mbar_wait(&sempty[t], ((kb / SLOTS) & 1) ^ 1);
        if (!ok) break;
        const float* raw = reinterpret_cast<const float*>(tiles + (size_t)s * Cfg::RAW_BYTES);
        float* slot = reinterpret_cast<float*>(slots + (size_t)t * Cfg::SLOT_BYTES);
        constexpr int AF = Cfg::A_BYTES / 4, BF = Cfg::B_BYTES / 4, RF = Cfg::RAW_BYTES / 4;
        split_tile(raw, slot, slot + RF, AF, threadIdx.x, 128);                    // A -> A hi, A lo
        split_tile(raw + AF, slot + AF, slot + RF + AF, BF, threadIdx.x, 128);     // B -> B hi, B lo
        mbar_arrive(&empty[s]);                                                    // raw stage read
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> async proxy (MMA)
        mbar_arrive(&sfull[t]);
      }
    }
    if (ok) ok = mbar_wait(accum, 0);
    if (ok) {
      tc_fence_after();
      // Every MMA has completed (accum), so the stage buffers are free: each warp transposes its
      // 32 x 32 accumulator chunks through a padded shared tile and stores whole row segments
      // (lane = column), so every store instruction writes 128 contiguous bytes.  TRANS stores
      // straight from the registers (lane = row of the kernel's tile = column of C).
      float* stage = reinterpret_cast<float*>(tiles) + warp * (32 * 33);
      const int trow = m0 + warp * 32 + lane;
      const int col_base = n0 + lane;
      constexpr int CW = BN < 32 ? BN : 32;  // accumulator columns per TMEM load
      for (int c0 = 0; c0 < BN; c0 += CW) {
        float v[CW];
        const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
        if constexpr (CW == 16) tmem_ld16(ta, v);
        else tmem_ld32(ta, v);
        if constexpr (TF32) {
          float w[CW];
          if constexpr (CW == 16) tmem_ld16(ta + (uint32_t)BN, w);
          else tmem_ld32(ta + (uint32_t)BN, w);
#pragma unroll
          for (int j = 0; j < CW; ++j) v[j] += w[j];
        }
        if constexpr (TRANS) {
          if (trow < M) {
#pragma unroll
            for (int j = 0; j < CW; ++j) {
              const int col = n0 + c0 + j;
              if (col >= N) break;
              if (ws) {
                ws[((int64_t)blockIdx.z * N + col) * M + trow] = v[j];
              } else {
                float* d = C + (int64_t)col * ldc + trow;
                *d = (beta == 0.f) ? alpha * v[j] : fmaf(alpha, v[j], beta * *d);
              }
            }
          }
          continue;
        }
#pragma unroll
        for (int j = 0; j < CW; ++j) stage[lane * 33 + j] = v[j];
        __syncwarp();
        const int col = col_base + c0;
        if (lane < CW && col < N) {
          for (int r = 0; r < 32; ++r) {
            const int row = m0 + warp * 32 + r;
            if (row >= M) break;
            const float x = stage[r * 33 + lane];
            if (ws) {
              ws[((int64_t)blockIdx.z * M + row) * N + col] = x;
            } else {
              float* d = C + (int64_t)row * ldc + col;
              *d = (beta == 0.f) ? alpha * x : fmaf(alpha, x, beta * *d);
            }
          }
        }
        __syncwarp();
      }
    } else {
      atomicExch(&s_fail, 1);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
  }
  if (threadIdx.x == 0 && s_fail) atomicExch(err, 1);
}

// ----------------------------------------------------------------------------- host side
static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
static std::mutex g_encode_mu;

static cudaError_t get_encoder() {
  std::lock_guard<std::mutex> lk(g_encode_mu);
  if (g_encode) return cudaSuccess;
  cudaDriverEntryPointQueryResult q;
  void* fn = nullptr;
  cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
  if (e != cudaSuccess) return e;
  if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
  g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  return cudaSuccess;
}

// 2-D map over a row-major (rows x cols) matrix, box = box_rows rows x 128 bytes, 128-byte swizzle,
// out-of-range reads return zero (ragged M / N / K edges).
static cudaError_t make_map(CUtensorMap* tm, const void* base, bool tf32, int64_t rows, int64_t cols, int64_t ld,
                            int box_rows) {
  const int elem = tf32 ? 4 : 2;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * elem)};
  cuuint32_t box[2] = {(cuuint32_t)(128 / elem), (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = g_encode(tm, tf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                        const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// C = alpha * sum_z ws[z] + beta * C, four consecutive outputs per thread (all split partials of
// them in flight), summed in split order with Neumaier compensation (FP32)
__global__ void umma_splitk_reduce_kernel(int M, int N, int splits, const float* __restrict__ ws, float alpha,
                                          float beta, float* __restrict__ C, int64_t ldc) {
  const int64_t e0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4;
  const int64_t MN = (int64_t)M * N;
  if (e0 >= MN) return;
  float sum[4] = {0.f, 0.f, 0.f, 0.f}, comp[4] = {0.f, 0.f, 0.f, 0.f};
  const bool vec = (e0 + 4 <= MN) && (N % 4 == 0);
  for (int z = 0; z < splits; ++z) {
    const float* w = ws + (int64_t)z * MN + e0;
    float x[4];
    if (vec) {
      const float4 v = __ldcs(reinterpret_cast<const float4*>(w));
      x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j) x[j] = e0 + j < MN ? __ldcs(w + j) : 0.f;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float t = sum[j] + x[j];
      comp[j] += (fabsf(sum[j]) >= fabsf(x[j])) ? (sum[j] - t) + x[j] : (x[j] - t) + sum[j];
      sum[j] = t;
    }
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int64_t e = e0 + j;
    if (e >= MN) break;
    float* c = C + (e / N) * ldc + (e % N);
    const float v = sum[j] + comp[j];
    *c = (beta == 0.f) ? alpha * v : fmaf(alpha, v, beta * *c);
  }
}

// SM count of the current device, queried once per process (thread-safe static initialisation);
// 152, GB300's count, only if the query fails
int umma_num_sms() {
  static const int n = [] {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 152;
  }();
  return n;
}

// C = alpha A B^T + beta C with A (M x K, lda) and B (N x K, ldb) K-major; tf32 selects the
// FP32-input TF32X3 mode, otherwise inputs are BF16.  err: device int set to 1 if a wait gave up.
cudaError_t umma_gemm_tn(bool tf32, int M, int N, int K, float alpha, const void* A, int64_t lda, const void* B,
                         int64_t ldb, float beta, float* C, int64_t ldc, int* err, cudaStream_t st) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  const int elem = tf32 ? 4 : 2;
  if (((uintptr_t)A & 15) || ((uintptr_t)B & 15) || (lda * elem) % 16 || (ldb * elem) % 16 || K <= 0)
    return cudaErrorInvalidValue;
  cudaError_t e = get_encoder();
  if (e != cudaSuccess) return e;
  // a thin M with a wide N: compute C^T = B A^T so that the thin side is the tile width
  const bool trans = M <= 64 && N > 64;
  if (trans) {
    std::swap(M, N);
    std::swap(A, B);
    std::swap(lda, ldb);
  }
  // the narrowest tile that covers a thin N (one column of tiles), else 128 columns; a short K with
  // a wide output takes 64-column tiles on the two-CTA short ring
  const int bk0 = 128 / elem;
  const bool shortk = (K + bk0 - 1) / bk0 <= UM_SHORT_KB && N > 64 &&
                      (int64_t)((M + UM_BM - 1) / UM_BM) * ((N + 63) / 64) >= 4 * (int64_t)umma_num_sms();
  const int bn = shortk ? 64 : N <= 16 ? 16 : N <= 32 ? 32 : N <= 64 ? 64 : 128;
  CUtensorMap ta, tb;
  if ((e = make_map(&ta, A, tf32, M, K, lda, UM_BM)) != cudaSuccess) return e;
  if ((e = make_map(&tb, B, tf32, N, K, ldb, bn)) != cudaSuccess) return e;
  const int bk = 128 / elem;
  const int tiles = ((M + UM_BM - 1) / UM_BM) * ((N + bn - 1) / bn);
  const int kblocks = (K + bk - 1) / bk;
  // K splits: minimise waves x per-CTA time (chain of k-blocks + a fixed prologue / epilogue cost of
  // about UM_CTA_FIXED_KB k-blocks) + the partial sums, with TF32X3 chains of at most
  // UM_TF32_MAX_KB k-blocks (the tensor core's FP32 accumulation loses up to an ulp per MMA; longer
  // K is split and the partials are summed with compensation)
  const int nsm = umma_num_sms() * ((shortk || bn == 16 || bn == 32) ? 2 : 1);  // resident CTAs (UmmaCfg::CTAS)
  const int smin = tf32 ? std::max(1, (kblocks + UM_TF32_MAX_KB - 1) / UM_TF32_MAX_KB) : 1;
  const int smax = std::max(smin, std::min(32, kblocks / 2));
  int splits = smin;
  int64_t best = -1;
  for (int s = smin; s <= smax; ++s) {
    const int64_t waves = ((int64_t)tiles * s + nsm - 1) / nsm;
    const int64_t cost = waves * ((kblocks + s - 1) / s + UM_CTA_FIXED_KB) + (s > 1 ? s : 0);
    if (best < 0 || cost < best) {
      best = cost;
      splits = s;
    }
  }
  const int per = (kblocks + splits - 1) / splits;  // k-blocks per split
  splits = (kblocks + per - 1) / per;               // no empty split
  float* ws = nullptr;
  if (splits > 1) {
    e = dev_alloc((void**)&ws, sizeof(float) * (size_t)splits * M * N, st);
    if (e != cudaSuccess) return e;
  }
  dim3 grid((N + bn - 1) / bn, (M + UM_BM - 1) / UM_BM, splits);
  {
    AMM_TRACE_W(tf32 ? "umma_gemm_tf32x3" : "umma_gemm_bf16", st, 2.0 * M * N * (double)K,
                (double)elem * ((double)M * K + (double)N * K) + 4.0 * M * N, nullptr);
    auto launch = [&](auto tf32_c, auto bn_c, auto short_c) -> cudaError_t {
      constexpr bool T = decltype(tf32_c)::value;
      constexpr int BN = decltype(bn_c)::value;
      constexpr bool SH = decltype(short_c)::value;
      using Cfg = UmmaCfg<T, BN, SH>;
      static DeviceOnce once;
      const cudaError_t a = once([] {
        cudaError_t r = cudaFuncSetAttribute((const void*)umma_gemm_kernel<T, BN, false, SH>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM);
        if (r == cudaSuccess)
          r = cudaFuncSetAttribute((const void*)umma_gemm_kernel<T, BN, true, SH>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM);
        return r;
      });
      if (a != cudaSuccess) return a;
      if (trans)
        umma_gemm_kernel<T, BN, true, SH><<<grid, UM_THREADS, Cfg::SMEM, st>>>(ta, tb, M, N, K, alpha, beta, C, ldc,
                                                                              per, ws, err);
      else
        umma_gemm_kernel<T, BN, false, SH><<<grid, UM_THREADS, Cfg::SMEM, st>>>(ta, tb, M, N, K, alpha, beta, C, ldc,
                                                                               per, ws, err);
      return cudaSuccess;
    };
    using I16 = std::integral_constant<int, 16>;
    using I32 = std::integral_constant<int, 32>;
    using I64 = std::integral_constant<int, 64>;
    using I128 = std::integral_constant<int, 128>;
    using NO = std::false_type;
    cudaError_t la;
    if (tf32)
      la = shortk ? launch(std::true_type{}, I64{}, std::true_type{})
         : bn == 16 ? launch(std::true_type{}, I16{}, NO{}) : bn == 32 ? launch(std::true_type{}, I32{}, NO{})
         : bn == 64 ? launch(std::true_type{}, I64{}, NO{}) : launch(std::true_type{}, I128{}, NO{});
    else
      la = shortk ? launch(std::false_type{}, I64{}, std::true_type{})
         : bn == 16 ? launch(std::false_type{}, I16{}, NO{}) : bn == 32 ? launch(std::false_type{}, I32{}, NO{})
         : bn == 64 ? launch(std::false_type{}, I64{}, NO{}) : launch(std::false_type{}, I128{}, NO{});
    if (la != cudaSuccess) {
      dev_free(ws, st);
      return la;
    }
  }
  e = cudaGetLastError();
  if (e == cudaSuccess && splits > 1) {
    AMM_TRACE("umma_splitk_reduce", st);
    const int64_t quads = ((int64_t)M * N + 3) / 4;
    // partials are in C's layout: (caller's) M rows x N columns
    const int Mc = trans ? N : M, Nc = trans ? M : N;
    umma_splitk_reduce_kernel<<<(unsigned)((quads + 255) / 256), 256, 0, st>>>(Mc, Nc, splits, ws, alpha, beta, C,
                                                                               ldc);
    e = cudaGetLastError();
  }
  dev_free(ws, st);
  return e;
}

}  // namespace amm

// Test hook: C = alpha A B^T + beta C through the tensor-core GEMM (see amm.h).
extern "C" amm_status_t amm_debug_gemm_tn(int32_t mode, int64_t M, int64_t N, int64_t K, float alpha, const void* A,
                                          int64_t lda, const void* B, int64_t ldb, float beta, float* C, int64_t ldc,
                                          int32_t* dev_err, void* stream) {
  using namespace amm;
  if (!A || !B || !C || !dev_err) return fail(AMM_ERR_INVALID_ARG, "amm_debug_gemm_tn: NULL pointer");
  if (mode != 0 && mode != 1) return fail(AMM_ERR_INVALID_ARG, "amm_debug_gemm_tn: mode must be 0 (TF32X3) or 1 (BF16)");
  if (M <= 0 || N <= 0 || K <= 0 || lda < K || ldb < K || ldc < N)
    return fail(AMM_ERR_INVALID_ARG, "amm_debug_gemm_tn: bad sizes");
  cudaError_t e = umma_gemm_tn(mode == 0, (int)M, (int)N, (int)K, alpha, A, lda, B, ldb, beta, C, ldc, dev_err,
                               (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "amm_debug_gemm_tn");
  return AMM_OK;
}
