// Grouped GEMM engine on the 5th-generation tensor cores (tcgen05), BF16 operands, FP32
// accumulators in tensor memory.  Used by the BF16 batched form for every predictor GEMM.
//
// One CTA of 128 threads computes a 128-row x nt-column tile (nt a multiple of 16, <= 256) of
// problem z = blockIdx.z over that problem's whole K:
//   * both operands are staged into shared memory by cp.async, 16 bytes (8 BF16) per copy, in
//     the canonical no-swizzle layouts of 8-row x 16-byte core matrices.  An operand whose 8
//     contiguous elements run along K is "K-major", one whose 8 contiguous elements run along M
//     (or N) is "MN-major"; the op of each GEMM says which, so every operand is read in the
//     layout it already has in global memory (no transposes);
//   * stages of 64 K cycle through a ring; one elected thread issues the tcgen05.mma
//     instructions of a landed stage (M 128, N nt, K 16 each) and commits them to that stage's
//     mbarrier, which frees the buffer for the copy issued kStages - 1 stages later;
//   * the epilogue reads the accumulator back with tcgen05.ld: warp w owns tensor-memory lanes
//     32w..32w+31, i.e. tile rows, and hands the op 8 consecutive columns of one row at a time.
// Every mbarrier wait is bounded; on expiry the CTA sets kErrTimeout in the plan's error word,
// drains its own copies, frees its tensor memory and returns.
//
// Shared-memory layouts of one R x 64 stage (R rows along M or N, 64 along K), byte offsets:
//   K-major : core matrix (r/8, k/8) at (r/8)*1024 + (k/8)*128, its row r%8 at +16*(r%8);
//             descriptor LBO = 128 (next core matrix along K), SBO = 1024 (next along M/N)
//   MN-major: core matrix (r/8, k/8) at (r/8)*128 + (k/8)*16R, its row k%8 at +16*(k%8);
//             descriptor LBO = 16R (next core matrix along K), SBO = 128 (next along M/N)
#pragma once
#include <cuda_bf16.h>

#include "internal.h"

namespace pmklc {
namespace tc {

using bf16 = __nv_bfloat16;
constexpr int kRows = 128;             // MMA M: tile rows = tensor-memory lanes
constexpr int kBK = 64;                // K per pipeline stage
constexpr int kThreads = 128;          // four warps
constexpr long kSpinLimit = 1L << 24;  // mbarrier polls before a wait gives up

__device__ __forceinline__ uint32_t sa(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  // no swizzle, base offset 0, descriptor version 1
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

__device__ const uint4 kZero16 = {0u, 0u, 0u, 0u};  // source of zero-filled copies

// 16-byte async copy; a null source fills zeros
__device__ __forceinline__ void cp16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa(dst)), "l"(src ? src : &kZero16),
               "r"(src ? 16 : 0));
}

__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  for (long it = 0; it < kSpinLimit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(sa(bar)), "r"(parity));
    if (ok) return true;
  }
  return false;
}

// Staging of one R x 64 operand tile (R rows along M or N, a multiple of 16) by 128 threads.
// In both layouts a thread's position along K is fixed for the whole tile, so each routine forms
// the per-thread part of the address once and then steps over its R/16 rows:
//   K-major : thread covers k-chunk (tid >> 3) & 7 of rows (tid >> 6) * 8 + (tid & 7) + 16 i;
//             eight consecutive threads fill one 128-byte core matrix
//   MN-major: thread covers k = tid & 63 of row-chunks (tid >> 6) * 8 + 16 i
// rlim / klim are the valid extents of the tile (rows, and K from the stage start k0).

// K-major, each row a contiguous run along K: rowp(r) is row r's address at k = 0, or nullptr
template <class RowPtr>
__device__ __forceinline__ void stage_k_rows(uint8_t *dst, int R, int rlim, int k0, int klim, RowPtr rowp) {
  const int kj = (threadIdx.x >> 3) & 7, k = k0 + kj * 8;
  const bool kin = kj * 8 < klim;
  for (int r = (threadIdx.x >> 6) * 8 + (threadIdx.x & 7); r < R; r += 16) {
    const bf16 *p = (kin && r < rlim) ? rowp(r) : nullptr;
    cp16(dst + (r >> 3) * 1024 + kj * 128 + (r & 7) * 16, p ? p + k : nullptr);
  }
}

// K-major rows gathered from an embedding table: row r's K run is the concatenation of the
// E-wide embedding rows of its t context tokens tok[r * t + pos] (E % 8 == 0); rows with
// tpos[r] < 0 are zero
__device__ __forceinline__ void stage_k_gather(uint8_t *dst, int rlim, int k0, int klim, const long long *tpos,
                                               const uint16_t *tok, int t, int E, const bf16 *emb) {
  const int kj = (threadIdx.x >> 3) & 7, k = k0 + kj * 8;
  const bool kin = kj * 8 < klim;
  const int pos = kin ? k / E : 0, e = k - pos * E;
  for (int r = (threadIdx.x >> 6) * 8 + (threadIdx.x & 7); r < kRows; r += 16) {
    const bool ok = kin && r < rlim && tpos[r] >= 0;
    cp16(dst + (r >> 3) * 1024 + kj * 128 + (r & 7) * 16, ok ? emb + (size_t)tok[r * t + pos] * E + e : nullptr);
  }
}

// MN-major, each K row a contiguous run along M/N: kptr(k) is the address of K row k0 + k at
// the tile's first M/N index, or nullptr
template <class KPtr>
__device__ __forceinline__ void stage_mn_rows(uint8_t *dst, int R, int rlim, int klim, KPtr kptr) {
  const int k = threadIdx.x & 63;
  const bf16 *base = k < klim ? kptr(k) : nullptr;
  for (int r = (threadIdx.x >> 6) * 8; r < R; r += 16)
    cp16(dst + (r >> 3) * 128 + (k >> 3) * (R * 16) + (k & 7) * 16, (base && r < rlim) ? base + r : nullptr);
}

// MN-major rows gathered from an embedding table: K row k0 + k is lane k0 + k's context vector
// (concatenated embedding rows of tok[(k0 + k) * t + pos]); M/N index n0 + r is element r of it
__device__ __forceinline__ void stage_mn_gather(uint8_t *dst, int R, int rlim, int n0, int k0, int klim,
                                                const long long *tpos, const uint16_t *tok, int t, int E,
                                                const bf16 *emb) {
  const int k = threadIdx.x & 63;
  const bool ok = k < klim && tpos[k0 + k] >= 0;
  const uint16_t *tk = tok + (size_t)(k0 + k) * t;
  for (int r = (threadIdx.x >> 6) * 8; r < R; r += 16) {
    const bf16 *p = nullptr;
    if (ok && r < rlim) {
      const int i = n0 + r, pos = i / E;
      p = emb + (size_t)tk[pos] * E + (i - pos * E);
    }
    cp16(dst + (r >> 3) * 128 + (k >> 3) * (R * 16) + (k & 7) * 16, p);
  }
}

// Op interface (device, const):
//   static constexpr bool kAMN, kBMN;       operand majors (A: M x K, B: N x K)
//   bool active(z); int M(z), N(z), K(z);
//   void prepare(uint8_t *meta, z, m0);     every thread calls it before the first barrier: the
//                                           op's per-tile data (row targets, context tokens) go
//                                           to shared memory so that staging reads no global
//                                           memory to form an address
//   void stage_a(uint8_t *dst, const uint8_t *meta, z, m0, k0, rlim, klim);   128 x 64 A tile
//   void stage_b(uint8_t *dst, const uint8_t *meta, z, n0, k0, R, rlim, klim);  R x 64 B tile
//   void epilogue(const uint8_t *meta, z, m, rl, n, const float v[8]);   m < M, n + 7 < N
//   int *err();                             the error word
template <class Op>
__global__ void __launch_bounds__(kThreads) gemm_kernel(const Op op, int nt_max, int tmem_cols, int stages) {
  // dynamic shared memory: [stages x A tile][stages x B tile][op metadata]
  const int z = blockIdx.z;
  if (!op.active(z)) return;
  const int M = op.M(z), N = op.N(z), K = op.K(z);
  const int m0 = blockIdx.x * kRows, n0 = blockIdx.y * nt_max;
  if (m0 >= M || n0 >= N) return;
  const int nt = min(nt_max, (N - n0 + 15) & ~15);  // MMA N of this tile
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  extern __shared__ __align__(1024) uint8_t smem[];
  const int a_bytes = kRows * kBK * 2, b_bytes = nt_max * kBK * 2;
  uint8_t *sA = smem, *sB = smem + stages * a_bytes;
  uint8_t *meta = smem + stages * (a_bytes + b_bytes);
  __shared__ __align__(8) uint64_t mbar[4];
  __shared__ uint32_t tmem_base;
  op.prepare(meta, z, m0);
  if (tid == 0) {
    for (int s = 0; s < stages; ++s) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(sa(&mbar[s])));
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

  auto issue = [&](int s, int k0) {
    op.stage_a(sA + s * a_bytes, meta, z, m0, k0, M - m0, K - k0);
    op.stage_b(sB + s * b_bytes, meta, z, n0, k0, nt, N - n0, K - k0);
    asm volatile("cp.async.commit_group;\n" ::);
  };
  auto commit_empty = [] { asm volatile("cp.async.commit_group;\n" ::); };

  const int nk = max(1, (K + kBK - 1) / kBK);  // K = 0 still runs one all-zero stage
  // instruction descriptor: FP32 accumulator, BF16 A and B, operand majors, N = nt, M = 128
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((Op::kAMN ? 1u : 0u) << 15) |
                         ((Op::kBMN ? 1u : 0u) << 16) | ((uint32_t)(nt >> 3) << 17) | ((uint32_t)(kRows >> 4) << 24);
  const uint32_t a_lbo = Op::kAMN ? kRows * 16 : 128, a_sbo = Op::kAMN ? 128 : 1024, a_step = Op::kAMN ? kRows * 32 : 256;
  const uint32_t b_lbo = Op::kBMN ? nt * 16 : 128, b_sbo = Op::kBMN ? 128 : 1024, b_step = Op::kBMN ? nt * 32 : 256;
  bool ok = true;
  for (int s = 0; s < stages - 1; ++s) {
    if (s < nk)
      issue(s, s * kBK);
    else
      commit_empty();
  }
  for (int kt = 0; kt < nk; ++kt) {
    const int s = kt % stages;
    // all but the newest stages - 2 copy groups have landed: stage kt is in shared memory
    if (stages == 4)
      asm volatile("cp.async.wait_group 2;\n" ::);
    else
      asm volatile("cp.async.wait_group 1;\n" ::);
    asm volatile("fence.proxy.async.shared::cta;\n" ::);
    __syncthreads();
    if (tid == 0 && ok) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
      const uint32_t a0 = sa(sA + s * a_bytes), b0 = sa(sB + s * b_bytes);
      for (int kk = 0; kk < kBK / 16; ++kk) {
        const uint64_t da = smem_desc(a0 + kk * a_step, a_lbo, a_sbo);
        const uint64_t db = smem_desc(b0 + kk * b_step, b_lbo, b_sbo);
        const uint32_t accum = (kt > 0 || kk > 0) ? 1u : 0u;
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
            "l"(da), "l"(db), "r"(idesc), "r"(accum));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
          sa(&mbar[s])));
    }
    // the buffer refilled next held stage kt - 1: wait until its MMAs have read it
    const int nxt = kt + stages - 1;
    if (nxt < nk) {
      if (kt >= 1 && ok) ok = mbar_wait(&mbar[(kt - 1) % stages], (uint32_t)(((kt - 1) / stages) & 1));
      if (ok)
        issue(nxt % stages, nxt * kBK);
      else
        commit_empty();
    } else {
      commit_empty();
    }
  }
  // the last commit covers every MMA of the tile
  if (ok) ok = mbar_wait(&mbar[(nk - 1) % stages], (uint32_t)(((nk - 1) / stages) & 1));
  asm volatile("cp.async.wait_group 0;\n" ::);
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
  if (!__syncthreads_and(ok)) {
    if (tid == 0) atomicOr(op.err(), kErrTimeout);
  } else {
    const int rl = warp * 32 + lane, m = m0 + rl;
    for (int c0 = 0; c0 < nt; c0 += 16) {
      uint32_t v[16];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
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
        if (n0 + c0 < N) op.epilogue(meta, z, m, rl, n0 + c0, f);
        if (n0 + c0 + 8 < N) op.epilogue(meta, z, m, rl, n0 + c0 + 8, f + 8);
      }
    }
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

// Launch op over Z problems whose M and N are at most Mmax and Nmax, with meta_bytes of per-tile
// shared data.  The column tile is the widest multiple of 16 (<= 256) that still gives at least
// one CTA per SM.
template <class Op>
void launch(const Op &op, int Mmax, int Nmax, int Z, size_t meta_bytes, cudaStream_t st) {
  if (Mmax <= 0 || Nmax <= 0 || Z <= 0) return;
  const int mt = (Mmax + kRows - 1) / kRows;
  int nt = min(256, (Nmax + 15) & ~15);
  while (nt >= 64 && (nt / 2) % 16 == 0 && (long)mt * ((Nmax + nt - 1) / nt) * Z < 152L) nt /= 2;
  const int stages = 3;
  const int meta = (int)((meta_bytes + 15) & ~(size_t)15);
  // stay inside the opt-in shared memory per block (with room for the kernel's static variables)
  while (nt > 16 && (nt / 2) % 16 == 0 && stages * (kRows * kBK * 2 + nt * kBK * 2) + meta > 220 * 1024) nt /= 2;
  const int smem = stages * (kRows * kBK * 2 + nt * kBK * 2) + meta;
  static int configured = 0;  // per op type: the opt-in limit covers static + dynamic shared memory
  if (configured < smem) {
    if (cudaFuncSetAttribute(gemm_kernel<Op>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
      return;  // recorded for the caller's cudaGetLastError
    configured = smem;
  }
  dim3 grid(mt, (Nmax + nt - 1) / nt, Z);
  gemm_kernel<Op><<<grid, kThreads, smem, st>>>(op, nt, pow2_at_least(nt), stages);
}

}  // namespace tc
}  // namespace pmklc
