// Grouped GEMM engine on the 5th-generation tensor cores (tcgen05), BF16 operands, FP32
// accumulators in tensor memory.  Used by the BF16 batched form for every predictor GEMM.
//
// One CTA of 256 threads computes a 128-row x nt-column tile (nt a multiple of 64, <= 256) of
// problem z = blockIdx.z over that problem's whole K, in stages of 64 K:
//   * dense operands (weights, activations) arrive by TMA (cp.async.bulk.tensor) in the
//     128-byte-swizzled layout, one bulk copy per 64-wide box, counted on the stage's "full"
//     mbarrier; operands gathered from an embedding table (the context vectors X) are written
//     into the same layout by the threads, from a copy of the table in shared memory;
//   * one thread issues the tcgen05.mma instructions of a landed stage (M 128, N nt, K 16) and
//     commits them to the stage's "done" mbarrier, which frees the buffer for the TMA issued
//     stages - 1 iterations later;
//   * the epilogue reads the accumulator back with tcgen05.ld (warp w owns tensor-memory lanes
//     32w..32w+31, i.e. tile rows) and hands the op either 8 consecutive columns of a thread's
//     row or, staged through shared memory, one element per lane with the lanes of a warp on
//     consecutive columns of one row (for scattered atomics).
// Every mbarrier wait is bounded; on expiry the CTA sets kErrTimeout in the plan's error word,
// waits (bounded) for its bulk copies, frees its tensor memory and returns.
//
// Shared-memory operand layouts (each tile 1024-byte aligned), 128-byte swizzle: a 16-byte chunk
// c of a 128-byte row r sits at r*128 + ((c ^ (r % 8)) * 16).
//   K-major  (R x 64): row r = the 64 K values of M/N index r.  Descriptor: SBO 1024 (8 rows),
//            layout SWIZZLE_128B; the K=16 step j starts 32j bytes into the row.
//   MN-major (64 x R): R/64 boxes of 64 K-rows x 128 bytes (64 M/N values), 8 KB apart.
//            Descriptor: LBO 8192 (next box along M/N), SBO 1024 (next 8 K-rows); the K=16
//            step j starts 2048j bytes in.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>

#include "internal.h"

namespace pmklc {
namespace tc {

using bf16 = __nv_bfloat16;
constexpr int kRows = 128;             // MMA M: tile rows = tensor-memory lanes
constexpr int kBK = 64;                // BF16 K per pipeline stage (one 128-byte swizzle row)
constexpr int kRowBytes = 128;         // bytes of K per operand row and stage (64 BF16 or 128 E4M3)
constexpr int kThreads = 256;          // eight warps: warps w and w + 4 share tensor-memory lanes 32(w % 4)..
constexpr int kStages = 6;             // most stage buffers of a ring (a launch may use fewer)
constexpr long kSpinLimit = 1L << 24;  // mbarrier polls before a wait gives up
constexpr int kStagedPitch = 66;       // uint2 per staged row of a kEpi == 1 epilogue (64 columns + pad)
// bytes of stage buffers a kEpi == 1 epilogue stages its 64-column chunks through
constexpr size_t kStagedBytes = (size_t)kRows * kStagedPitch * 8;
constexpr int kFloatPitch = 68;        // floats per staged row of a kEpi == 2 epilogue

__device__ __forceinline__ uint32_t sa(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t desc_sw128(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long polls = kSpinLimit) {
  for (long it = 0; it < polls; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity));
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ void expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}

// TMA box loads into shared memory, completion counted on bar
__device__ __forceinline__ void tma2(uint32_t dst, const CUtensorMap *m, int c0, int c1, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(
          dst),
      "l"((uint64_t)m), "r"(c0), "r"(c1), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void tma3(uint32_t dst, const CUtensorMap *m, int c0, int c1, int c2, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(
          dst),
      "l"((uint64_t)m), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
      : "memory");
}

// A dense operand tile by TMA.  K-major: one box {64 K, R rows} at (k0, row0[, grp]).
// MN-major: R/64 boxes {64 M/N, 64 K} at (mn0 + 64j, kofs + k0[, grp]), 8 KB apart.
struct TmaOperand {
  const CUtensorMap *map;
  int rank;  // 2 or 3
  int grp;   // third coordinate (rank 3)
  int kofs;  // MN-major: first K row (a group's first lane in an activation map)
};
__device__ __forceinline__ void tma_k_tile(uint32_t dst, const TmaOperand &o, int k0, int row0, uint32_t bar) {
  if (o.rank == 3)
    tma3(dst, o.map, k0, row0, o.grp, bar);
  else
    tma2(dst, o.map, k0, row0, bar);
}
__device__ __forceinline__ void tma_mn_tile(uint32_t dst, const TmaOperand &o, int mn0, int R, int k0, uint32_t bar) {
  for (int j = 0; j < R / 64; ++j) {
    if (o.rank == 3)
      tma3(dst + j * 8192, o.map, mn0 + 64 * j, o.kofs + k0, o.grp, bar);
    else
      tma2(dst + j * 8192, o.map, mn0 + 64 * j, o.kofs + k0, bar);
  }
}

// Swizzled byte offsets of 16-byte chunk c (8 BF16) of K-major row r, and of the 8 M/N values
// n..n+7 (n % 8 == 0) at K-row k of an MN-major tile.
__device__ __forceinline__ uint32_t sw_k(int r, int c) { return (uint32_t)(r * 128 + ((c ^ (r & 7)) << 4)); }
__device__ __forceinline__ uint32_t sw_mn(int n, int k) {
  return (uint32_t)((n >> 6) * 8192 + k * 128 + ((((n & 63) >> 3) ^ (k & 7)) << 4));
}

// Op interface (device, const):
//   static constexpr bool kAMN, kBMN;         operand majors (A: M x K, B: N x K)
//   static constexpr bool kFP8;               E4M3 operands (kind::f8f6f4, K-major only, 128 K per
//                                             stage, K = 32 per MMA) instead of BF16 (kind::f16)
//   static constexpr bool kTail;              K rows past K(z) in the last stage must be zeroed
//                                             (the dense operands run on into other groups)
//   static constexpr int kGather;             0: both operands by TMA; 1: A gathered; 2: B gathered
//   bool active(z); int M(z), N(z), K(z);
//   void prepare(uint8_t *meta, z, m0);       every thread calls it before the first barrier:
//                                             per-tile data (row targets, context tokens, the
//                                             embedding table of a gathered operand)
//   TmaOperand tma_a(z), tma_b(z); int row_a(z, m0), row_b(z, n0): TMA row coordinates
//   G gather_ctx(const uint8_t *meta, z, mn0, R)   once per thread after the first barrier: a
//                                             value holding everything the thread's gathers read
//                                             (kept in registers: per-element work never reloads
//                                             the op's fields from the parameter space, which the
//                                             compiler must assume the tile stores may alias)
//   void G::gather(uint8_t *tile, int k0) const      the gathered operand of K block k0
//   E epi_ctx(const uint8_t *meta, z, m0, n0) likewise for the epilogue, with
//   static constexpr int kEpi;                0: void E::epilogue(m, rl, n, const float v[8]) per
//                                             row (8 columns n.., m < M);
//                                             1: uint2 E::stage(float v) applied by the row's thread,
//                                             then bool E::row_active(rl), uint32_t E::index(rl, n)
//                                             and void E::add(index, uint2 staged) per element (a
//                                             zero staged value adds nothing), the 32 lanes of a
//                                             warp on consecutive n of one row;
//                                             2: void E::chunk(const float *stg, c0), every thread,
//                                             after the 64 columns c0.. of all rows are staged as
//                                             FP32 (row r at stg + r * kFloatPitch)
//   static constexpr bool kFinish; void finish(uint8_t *meta, z): every thread, after the epilogue
//   int zb;                                   first problem of the launch (blockIdx.z + zb)
//   int *err();                               the error word
template <class Op>
__global__ void __launch_bounds__(kThreads, 1) gemm_kernel(const __grid_constant__ Op op, int nt_max, int tmem_cols,
                                                         int ns) {
  pdl_wait();
  pdl_trigger();
  const int z = blockIdx.z + op.zb;  // problem index (a launch may cover a subrange of the problems)
  if (!op.active(z)) return;
  const int M = op.M(z), N = op.N(z), K = op.K(z);
  const int m0 = blockIdx.x * kRows, n0 = blockIdx.y * nt_max;
  if (m0 >= M || n0 >= N) return;
  const int nt = min(nt_max, N - n0);  // MMA N of this tile (N and nt_max are multiples of 64)
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // dynamic shared memory: [alignment slack][stages x A tile][stages x B tile][meta]
  extern __shared__ uint8_t smem_raw[];
  const uint32_t base = (sa(smem_raw) + 1023) & ~1023u;
  uint8_t *gbase = smem_raw + (base - sa(smem_raw));
  static_assert(!Op::kFP8 || (!Op::kAMN && !Op::kBMN && !Op::kTail), "E4M3 operands are K-major");
  constexpr int BK = Op::kFP8 ? 2 * kBK : kBK;  // K elements per stage
  const uint32_t a_bytes = kRows * kRowBytes, b_bytes = nt_max * kRowBytes;
  const uint32_t sA = base, sB = base + ns * a_bytes;
  uint8_t *meta = gbase + ns * (a_bytes + b_bytes);
  __shared__ __align__(8) uint64_t full[kStages], done[kStages];
  __shared__ uint32_t tmem_base;
  op.prepare(meta, z, m0);
  if (tid == 0) {
    for (int s = 0; s < ns; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(sa(&full[s])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(sa(&done[s])));
    }
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(sa(&tmem_base)),
                 "r"(tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
  const uint32_t tmem = tmem_base;
  const auto gc = op.gather_ctx(meta, z, Op::kGather == 2 ? n0 : m0, Op::kGather == 2 ? nt : kRows);

  const int nk = max(1, (K + BK - 1) / BK);  // K = 0 still runs one all-zero stage
  const TmaOperand ta = op.tma_a(z), tb = op.tma_b(z);
  const int ra = op.row_a(z, m0), rb = op.row_b(z, n0);
  // bytes per stage: a K-major box is as high as the map's box (nt_max rows for B), MN-major
  // boxes are issued for this tile's nt columns only
  const uint32_t tx = (Op::kGather == 1 ? 0u : a_bytes) +
                      (Op::kGather == 2 ? 0u : (uint32_t)(Op::kBMN ? nt : nt_max) * kRowBytes);
  // fill stage s with K block kt: bulk copies by thread 0, the gathered operand by every thread
  auto issue = [&](int s, int kt) {
    const int k0 = kt * BK;
    if (tid == 0) {
      const uint32_t bar = sa(&full[s]);
      expect_tx(bar, tx);
      if (Op::kGather != 1) {
        if (Op::kAMN)
          tma_mn_tile(sA + s * a_bytes, ta, ra, kRows, k0, bar);
        else
          tma_k_tile(sA + s * a_bytes, ta, k0, ra, bar);
      }
      if (Op::kGather != 2) {
        if (Op::kBMN)
          tma_mn_tile(sB + s * b_bytes, tb, rb, nt, k0, bar);
        else
          tma_k_tile(sB + s * b_bytes, tb, k0, rb, bar);
      }
    }
    if (Op::kGather == 1) gc.gather(gbase + s * a_bytes, k0);
    if (Op::kGather == 2) gc.gather(gbase + ns * a_bytes + s * b_bytes, k0);
    if (Op::kGather) asm volatile("cp.async.commit_group;\n" ::);  // gathers copied from global memory
  };
  // zero the K rows r >= rows of a stage (MN-major operands of the last, partial K block)
  auto zero_tail = [&](int s, int rows) {
    const uint4 zz = make_uint4(0, 0, 0, 0);
    for (int i = tid; i < (kBK - rows) * 8; i += kThreads) {  // 8 chunks of 16 B per 128-byte row
      const int r = rows + (i >> 3), c = i & 7;
      if (Op::kAMN)
        for (int j = 0; j < kRows / 64; ++j)
          *reinterpret_cast<uint4 *>(gbase + s * a_bytes + j * 8192 + r * 128 + c * 16) = zz;
      if (Op::kBMN)
        for (int j = 0; j < nt / 64; ++j)
          *reinterpret_cast<uint4 *>(gbase + ns * a_bytes + s * b_bytes + j * 8192 + r * 128 + c * 16) = zz;
    }
  };

  // instruction descriptor: FP32 accumulator, A and B BF16 (format 1 of kind::f16) or E4M3 (format 0 of
  // kind::f8f6f4), operand majors, N = nt, M = 128
  const uint32_t fmt = Op::kFP8 ? 0u : 1u;
  const uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((Op::kAMN ? 1u : 0u) << 15) |
                         ((Op::kBMN ? 1u : 0u) << 16) | ((uint32_t)(nt >> 3) << 17) | ((uint32_t)(kRows >> 4) << 24);
  const uint32_t a_lbo = Op::kAMN ? 8192 : 16, a_step = Op::kAMN ? 2048 : 32;
  const uint32_t b_lbo = Op::kBMN ? 8192 : 16, b_step = Op::kBMN ? 2048 : 32;
  // Prefetch distance pf: K block kt + pf is staged while block kt is multiplied.  Its buffer was
  // last read by the MMAs of block kt + pf - ns, i.e. kt - 2 (ns >= 3), which were committed two
  // iterations earlier, so refilling it rarely waits on the tensor core; with ns = 2 the distance
  // is one block and the refill waits for block kt - 1.
  const int pf = ns >= 3 ? ns - 2 : 1;
  bool ok = true;
  for (int s = 0; s < pf; ++s) {
    if (s < nk)
      issue(s, s);
    else if (Op::kGather)
      asm volatile("cp.async.commit_group;\n" ::);
  }
  for (int kt = 0; kt < nk; ++kt) {
    const int s = kt % ns;
    const uint32_t par = (uint32_t)((kt / ns) & 1);
    const bool tail = Op::kTail && kt == nk - 1 && K - kt * BK < BK;
    if (Op::kGather || tail) {
      // a gathered stage kt is the oldest of the pf copy groups in flight
      if (Op::kGather) {
        switch (pf) {
          case 1: asm volatile("cp.async.wait_group 0;\n" ::); break;
          case 2: asm volatile("cp.async.wait_group 1;\n" ::); break;
          case 3: asm volatile("cp.async.wait_group 2;\n" ::); break;
          default: asm volatile("cp.async.wait_group 3;\n" ::); break;
        }
      }
      if (Op::kGather) {
        if (ok) ok = mbar_wait(sa(&full[s]), par);  // every thread waits at every stage: in step
      } else {
        // the tail of a TMA-only op: only thread 0 has waited on the earlier stages, so another
        // thread's parity wait here could see this buffer's previous phase (same parity) and pass
        // before the copy landed; thread 0 waits, and the barrier releases the others
        if (tid == 0 && ok) ok = mbar_wait(sa(&full[s]), par);
        __syncthreads();
      }
      if (tail && ok) zero_tail(s, max(0, K - kt * BK));
      asm volatile("fence.proxy.async.shared::cta;\n" ::);
      __syncthreads();
    } else if (tid == 0 && ok) {
      ok = mbar_wait(sa(&full[s]), par);
    }
    if (tid == 0 && ok) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
      for (int kk = 0; kk < 4; ++kk) {  // four MMAs of 32 bytes of K (K = 16 BF16 or 32 E4M3)
        const uint64_t da = desc_sw128(sA + s * a_bytes + kk * a_step, a_lbo, 1024);
        const uint64_t db = desc_sw128(sB + s * b_bytes + kk * b_step, b_lbo, 1024);
        const uint32_t accum = (kt > 0 || kk > 0) ? 1u : 0u;
        if constexpr (Op::kFP8)
          asm volatile(
              "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
              "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
              "l"(da), "l"(db), "r"(idesc), "r"(accum));
        else
          asm volatile(
              "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
              "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
              "l"(da), "l"(db), "r"(idesc), "r"(accum));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
          sa(&done[s])));
    }
    // stage K block kt + pf once the MMAs that last read its buffer (block kt + pf - ns) are done
    const int nxt = kt + pf, prev = nxt - ns;
    if (nxt < nk) {
      const bool need = Op::kGather != 0 || tid == 0;
      if (need && prev >= 0 && ok) ok = mbar_wait(sa(&done[prev % ns]), (uint32_t)((prev / ns) & 1));
      if (need && ok)
        issue(nxt % ns, nxt);
      else if (Op::kGather)
        asm volatile("cp.async.commit_group;\n" ::);
    } else if (Op::kGather) {
      asm volatile("cp.async.commit_group;\n" ::);  // one group per iteration keeps the wait count exact
    }
  }
  // the last commit covers every MMA of the tile
  if (tid == 0 && ok) ok = mbar_wait(sa(&done[(nk - 1) % ns]), (uint32_t)(((nk - 1) / ns) & 1));
  if (Op::kGather) asm volatile("cp.async.wait_group 0;\n" ::);
  if (!__syncthreads_and(ok)) {
    if (tid == 0) {
      atomicOr(op.err(), kErrTimeout);
      // let the bulk copies this CTA issued land before its shared memory is released: stage s
      // was last filled with K block last(s); waits on phases already completed return at once
      for (int s = 0; s < ns && s < nk; ++s) {
        const int last = ((nk - 1 - s) / ns) * ns + s;
        mbar_wait(sa(&full[s]), (uint32_t)((last / ns) & 1));
      }
    }
  } else {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
    const int quad = warp & 3, half = warp >> 2;  // tensor-memory lanes 32 quad.., column half
    const int rl = quad * 32 + lane;
    const auto ec = op.epi_ctx(meta, z, m0, n0);
    if constexpr (Op::kEpi == 0) {
      // per row: thread rl hands the op 8 consecutive columns of its row at a time, the two warps
      // of a lane quarter taking one half of the columns each
      const int m = m0 + rl;
      for (int c0 = half * (nt / 2); c0 < (half + 1) * (nt / 2); c0 += 16) {
        uint32_t v[16];
        const uint32_t taddr = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)c0;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::);
        if (m < M) {
          float f[16];
#pragma unroll
          for (int q = 0; q < 16; ++q) f[q] = __uint_as_float(v[q]);
          ec.epilogue(m, rl, n0 + c0, f);
          ec.epilogue(m, rl, n0 + c0 + 8, f + 8);
        }
      }
    } else if constexpr (Op::kEpi == 1) {
      // 64-column chunks staged through the (now idle) stage buffers: thread rl converts its half of
      // its row (E::stage, 16 independent values per tensor-memory load) and stores it to shared
      // memory, then warp w emits rows w, w + 8, ... with its lanes on consecutive columns, so the
      // global accesses of a warp touch one row
      uint2 *stg = reinterpret_cast<uint2 *>(gbase);
      constexpr int kPitch = kStagedPitch;  // the 16-byte stores of 8 threads hit distinct banks
      for (int c0 = 0; c0 < nt; c0 += 64) {
#pragma unroll
        for (int q = half * 32; q < half * 32 + 32; q += 16) {
          uint32_t v[16];
          const uint32_t taddr = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(c0 + q);
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
              : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
              : "r"(taddr));
          asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::);
          uint2 w[16];
#pragma unroll
          for (int i = 0; i < 16; ++i) w[i] = ec.stage(__uint_as_float(v[i]));
          uint4 *dst = reinterpret_cast<uint4 *>(stg + rl * kPitch + q);
#pragma unroll
          for (int i = 0; i < 8; ++i) dst[i] = make_uint4(w[2 * i].x, w[2 * i].y, w[2 * i + 1].x, w[2 * i + 1].y);
        }
        __syncthreads();
        // rows in batches of four: every load of a batch (staged values, destinations) is issued
        // before its first reduction, so the latencies overlap (8 warps per SM leave little else
        // to hide them)
        for (int r0 = warp; r0 < kRows; r0 += 4 * (kThreads / 32)) {
          uint2 v[4][2];
          uint32_t dst[4][2];
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            const int r = r0 + b * (kThreads / 32);
            const bool act = m0 + r < M && ec.row_active(r);
#pragma unroll
            for (int jj = 0; jj < 2; ++jj) {
              const int j = lane + 32 * jj, n = n0 + c0 + j;
              const bool in = act && n < N;
              v[b][jj] = in ? stg[r * kPitch + j] : make_uint2(0u, 0u);
              dst[b][jj] = in ? ec.index(r, n) : 0u;
            }
          }
#pragma unroll
          for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int jj = 0; jj < 2; ++jj) ec.add(dst[b][jj], v[b][jj]);
        }
        __syncthreads();
      }
    }
    if constexpr (Op::kEpi == 2) {
      // 64-column chunks staged as FP32 through the stage buffers, each followed by a pass of the
      // whole CTA over the staged chunk (E::chunk), between barriers
      float *stg = reinterpret_cast<float *>(gbase);
      for (int c0 = 0; c0 < nt; c0 += 64) {
#pragma unroll
        for (int q = half * 32; q < half * 32 + 32; q += 16) {
          uint32_t v[16];
          const uint32_t taddr = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(c0 + q);
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
              : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
              : "r"(taddr));
          asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::);
          float4 *dst = reinterpret_cast<float4 *>(stg + rl * kFloatPitch + q);
#pragma unroll
          for (int j = 0; j < 4; ++j)
            dst[j] = make_float4(__uint_as_float(v[4 * j]), __uint_as_float(v[4 * j + 1]),
                                 __uint_as_float(v[4 * j + 2]), __uint_as_float(v[4 * j + 3]));
        }
        __syncthreads();
        ec.chunk(stg, c0);
        __syncthreads();
      }
    }
    if (Op::kFinish) op.finish(meta, z);  // the op's CTA-wide step after the epilogue
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(tmem_cols));
}

inline int pow2_at_least(int x) {
  int c = 32;
  while (c < x) c <<= 1;
  return c;
}

// Tile plan for Z problems whose M, N and K are at most Mmax, Nmax (a multiple of 64) and Kmax,
// with meta_bytes of per-tile shared data: K blocks + 2 stage buffers (up to kStages) and
// the widest column tile (a multiple of 64, <= 256) that still gives at least one CTA per SM and
// fits the shared memory.  Tensor maps of K-major B operands use nt as their box height.
struct TilePlan {
  int nt, ns;
};
inline size_t smem_bytes(const TilePlan &t, size_t meta_bytes) {
  return 1024 + (size_t)t.ns * (kRows + t.nt) * kRowBytes + ((meta_bytes + 15) & ~(size_t)15);
}
inline TilePlan plan_tiles(int Mmax, int Nmax, int Kmax, int Z, size_t meta_bytes, bool split = true, int bk = kBK) {
  const int mt = (Mmax + kRows - 1) / kRows, nk = (Kmax + bk - 1) / bk;
  // K blocks + 2 buffers let every block be staged before the MMAs need it (prefetch ns - 2)
  TilePlan t{min(256, Nmax), max(2, min(kStages, nk + 2))};
  // (an op that gathers its A operand pays the gather once per column tile: split = false)
  while (split && t.nt > 64 && (t.nt / 2) % 64 == 0 && (long)mt * ((Nmax + t.nt - 1) / t.nt) * Z < 152L) t.nt /= 2;
  while (t.ns > 2 && smem_bytes(t, meta_bytes) > 220 * 1024) --t.ns;  // fewer buffers before narrower tiles
  while (t.nt > 64 && (t.nt / 2) % 64 == 0 && smem_bytes(t, meta_bytes) > 220 * 1024) t.nt /= 2;
  return t;
}

template <class Op>
void launch(const Op &op, int Mmax, int Nmax, int Z, const TilePlan &t, size_t meta_bytes, cudaStream_t st) {
  if (Mmax <= 0 || Nmax <= 0 || Z <= 0) return;
  const int smem = (int)smem_bytes(t, meta_bytes);
  // the opt-in limit covers static + dynamic shared memory; a failure stays recorded for the
  // caller's cudaGetLastError
  if (!smem_optin((const void *)gemm_kernel<Op>, smem)) return;
  dim3 grid((Mmax + kRows - 1) / kRows, (Nmax + t.nt - 1) / t.nt, Z);
  launch_pdl(gemm_kernel<Op>, grid, dim3(kThreads), (size_t)smem, st, op, t.nt, pow2_at_least(t.nt), t.ns);
}

}  // namespace tc
}  // namespace pmklc
