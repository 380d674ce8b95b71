// BF16 batched form on tcgen05: the six GEMMs of one global step of every group's predictors
// (paper §2 steps 3-4, the MLP of the measured configurations), on the engine of tcgemm.cuh.
//
//   forward   h  = relu(X W1 + b1)    X gathered from the embedding rows of the context tokens
//             L  = h W2 + b2          dynamic model (z < G) and static model (z >= G) in one launch
//   backward  dh = (dz W2^T) * [h > 0]
//             dW2 = h^T dz,  dX = dh W1^T (scattered into the embedding rows),  dW1 = X^T dh
//             db2 = sum of dz, db1 = sum of dh over the predicted rows (fixed-order column sums)
// The weight-gradient epilogues store the gradient; the streaming optimiser of predictor.cu then
// updates every parameter (spread over all SMs at full occupancy it outruns an optimiser applied
// in these epilogues, whose four-to-eight warps per SM keep too few accesses in flight).
//
// Operand majors follow the stored layouts, so every dense operand is one TMA box per stage:
// W1 is stored transposed (W1t[h][i]: K-major for the hidden layer, MN-major for dX), W2 as
// [h][a] (MN-major for the logits, K-major for dh), activations as [lane row][feature] (K-major
// where rows are lanes, MN-major where the GEMM reduces over lanes).  The context vectors X are
// gathered from the embedding table (copied to shared memory when it fits).  The lanes a group
// predicts at a step are a prefix of its lanes (lanes differ by at most one token), so the
// lane-reducing GEMMs run over that prefix and zero the rows past it in their last K stage.
#include <cudaTypedefs.h>
#include <cuda_fp8.h>

#include <mutex>

#include "tcgemm.cuh"

namespace pmklc {

namespace {

using tc::bf16;

constexpr size_t kTableMax = 48 * 1024;  // largest embedding table copied to shared memory
constexpr size_t kAccMax = 96 * 1024;    // largest fixed-point gradient table summed in shared memory

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

// Per-tile shared data ("meta").  Row tiles (rows = lanes): [target of each of the 128 rows]
// [their t context tokens][embedding table].  Lane reductions: [target of every lane][their
// context tokens][embedding table].
struct MetaLayout {
  int nrows;   // 128 for row tiles, Mmax for lane reductions
  int t;       // context tokens per row kept (0: none)
  int table;   // bytes of embedding table kept (0: none)
  __host__ __device__ size_t tok_off() const { return align16((size_t)nrows * 8); }
  __host__ __device__ size_t tab_off() const { return tok_off() + align16((size_t)nrows * t * 2); }
  __host__ __device__ size_t bytes() const { return tab_off() + (size_t)table; }
};

struct TBase {
  static constexpr bool kFinish = false;
  static constexpr bool kFP8 = false;
  Plan p;
  int T;
  MetaLayout ml;
  __device__ void finish(uint8_t *, int) const {}
  __device__ void epilogue(const uint8_t *, int, int, int, int, const float *) const {}
  __device__ bool row_active(const uint8_t *, int, int, int) const { return false; }
  __device__ void emit(const uint8_t *, int, int, int, int, float) const {}
  __device__ int *err() const { return p.err; }
  __device__ int nrows(int g) const { return p.grp_lane_off[g + 1] - p.grp_lane_off[g]; }
  __device__ int row(int g, int r) const { return p.grp_lane_off[g] + r; }
  __device__ long long target_pos(int g, int r) const {
    const int rw = row(g, r);
    if (!row_pred(p, T, rw, g)) return -1;
    return p.lane_tok[rw] + (T - p.grp_start[g]);
  }
  __device__ int npred(int g) const { return live_lanes(p, g, T - p.grp_start[g]); }
  __device__ const bf16 *wb(int g) const { return p.wbf + (size_t)g * p.P; }
  __device__ const long long *tp(const uint8_t *meta) const { return reinterpret_cast<const long long *>(meta); }
  __device__ const uint16_t *tk(const uint8_t *meta) const {
    return reinterpret_cast<const uint16_t *>(meta + ml.tok_off());
  }
  __device__ const bf16 *table(const uint8_t *meta) const {
    return reinterpret_cast<const bf16 *>(meta + ml.tab_off());
  }
  // targets of rows r0 .. r0 + n - 1 of group g (-1 past the group or for rows that predict
  // nothing), their t context tokens and the embedding table emb (A x E) if ml.table.  The table
  // arrives by one bulk copy that overlaps the target and token loads.
  __device__ void fill(uint8_t *meta, const MetaLayout &ml, int g, int r0, int n, const void *emb, int bytes) const {
    __shared__ __align__(8) uint64_t tbar;
    long long *tpw = reinterpret_cast<long long *>(meta);
    const bool copy = emb != nullptr && bytes > 0 && ml.table >= bytes;
    if (copy && threadIdx.x == 0) {
      const uint32_t bar = tc::sa(&tbar);
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar));
      asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
      tc::expect_tx(bar, (uint32_t)bytes);
      asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                       tc::sa(meta + ml.tab_off())),
                   "l"(emb), "r"(bytes), "r"(bar)
                   : "memory");
    }
    const int L = nrows(g);
    for (int i = threadIdx.x; i < n; i += tc::kThreads) tpw[i] = r0 + i < L ? target_pos(g, r0 + i) : -1;
    __syncthreads();
    if (ml.t > 0) {
      uint16_t *tkw = reinterpret_cast<uint16_t *>(meta + ml.tok_off());
      const int t = ml.t, total = n * t;
      for (int i0 = 0; i0 < total; i0 += 16 * tc::kThreads) {  // sixteen loads in flight per thread
        uint16_t v[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int i = i0 + q * tc::kThreads + threadIdx.x;
          v[q] = 0;
          if (i < total) {
            const int r = i / t;
            const long long b = tpw[r];
            if (b >= 0) v[q] = p.tokens[b - t + (i - r * t)];
          }
        }
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int i = i0 + q * tc::kThreads + threadIdx.x;
          if (i < total) tkw[i] = v[q];
        }
      }
    }
    if (copy && !tc::mbar_wait(tc::sa(&tbar), 0) && threadIdx.x == 0) atomicOr(p.err, kErrTimeout);
  }
};

// 16 bytes from the shared-memory table or, without one, an async copy from global memory
__device__ __forceinline__ void put16(uint8_t *dst, const bf16 *tab_s, const bf16 *tab_g, size_t off) {
  if (tab_s) {
    *reinterpret_cast<uint4 *>(dst) = *reinterpret_cast<const uint4 *>(tab_s + off);
  } else {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(tc::sa(dst)), "l"(tab_g + off));
  }
}
__device__ __forceinline__ void zero16(uint8_t *dst) { *reinterpret_cast<uint4 *>(dst) = make_uint4(0, 0, 0, 0); }

// z < G: dynamic model of group z; z >= G: static model on group z - G's rows
struct TwoModels : TBase {
  __device__ bool stat(int z) const { return z >= p.G; }
  __device__ int grp(int z) const { return stat(z) ? z - p.G : z; }
  __device__ const Dims &d(int z) const { return stat(z) ? p.st : p.dm; }
  __device__ const bf16 *w(int z) const { return stat(z) ? p.static_bf : wb(grp(z)); }
  __device__ const float *w32(int z) const { return stat(z) ? p.static_params : p.params + (size_t)grp(z) * p.P; }
  __device__ bool active(int z) const { return group_trains(p, T, grp(z)); }
};

__device__ __forceinline__ uint4 pack8(const float *x) {
  uint32_t w[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    __nv_bfloat162 h = __floats2bfloat162_rn(x[2 * q], x[2 * q + 1]);
    w[q] = *reinterpret_cast<uint32_t *>(&h);
  }
  return make_uint4(w[0], w[1], w[2], w[3]);
}

__device__ __forceinline__ void store8(float *dst, const float *v) {
  reinterpret_cast<float4 *>(dst)[0] = make_float4(v[0], v[1], v[2], v[3]);
  reinterpret_cast<float4 *>(dst)[1] = make_float4(v[4], v[5], v[6], v[7]);
}

constexpr tc::TmaOperand kNoTma = {nullptr, 2, 0, 0};

// h = relu(X W1 + b1): A = X gathered (K-major), B = W1t by TMA (K-major)
struct HiddenT : TwoModels {
  static constexpr bool kAMN = false, kBMN = false, kTail = false;
  static constexpr int kEpi = 0;
  static constexpr int kGather = 1;
  CUtensorMap w1[2];  // W1t of the dynamic models (3-D, per group) and of the static model
  int table[2];       // embedding table kept in shared memory (dynamic, static)
  __device__ int M(int z) const { return nrows(grp(z)); }
  __device__ int N(int z) const { return d(z).H; }
  __device__ int K(int z) const { return d(z).K1(); }
  __device__ void prepare(uint8_t *meta, int z, int m0) const {
    MetaLayout l = ml;
    l.t = d(z).t;
    l.table = table[stat(z)] ? d(z).A * d(z).E * 2 : 0;
    fill(meta, l, grp(z), m0, tc::kRows, w(z) + d(z).off_emb(), d(z).A * d(z).E * 2);
  }
  __device__ tc::TmaOperand tma_a(int) const { return kNoTma; }
  __device__ tc::TmaOperand tma_b(int z) const { return {&w1[stat(z)], stat(z) ? 2 : 3, grp(z), 0}; }
  __device__ int row_a(int, int) const { return 0; }
  __device__ int row_b(int, int n0) const { return n0; }
  // thread: 16-byte chunk c = tid % 8 of rows tid / 8 + 32 i; the 4 table reads are in flight together
  __device__ void gather(uint8_t *tile, const uint8_t *meta, int z, int, int k0, int) const {
    const Dims &D = d(z);
    MetaLayout l = ml;
    l.t = D.t;
    const long long *tpv = reinterpret_cast<const long long *>(meta);
    const uint16_t *tkv = reinterpret_cast<const uint16_t *>(meta + l.tok_off());
    const bf16 *tab_s = table[stat(z)] ? reinterpret_cast<const bf16 *>(meta + l.tab_off()) : nullptr;
    const bf16 *tab_g = w(z) + D.off_emb();
    const int c = threadIdx.x & 7, k = k0 + 8 * c, r0 = threadIdx.x >> 3;
    const bool kin = k < D.K1();
    const int pos = kin ? k / D.E : 0, e = k - pos * D.E;
    constexpr int kPer = tc::kRows * 8 / tc::kThreads, kStep = tc::kThreads / 8;
    int off[kPer];
    bool ok[kPer];
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
      const int r = r0 + kStep * i;
      ok[i] = kin && tpv[r] >= 0;
      off[i] = ok[i] ? (int)tkv[r * D.t + pos] * D.E + e : 0;
    }
    if (tab_s) {
      uint4 v[kPer];
#pragma unroll
      for (int i = 0; i < kPer; ++i)
        v[i] = ok[i] ? *reinterpret_cast<const uint4 *>(tab_s + off[i]) : make_uint4(0, 0, 0, 0);
#pragma unroll
      for (int i = 0; i < kPer; ++i) *reinterpret_cast<uint4 *>(tile + tc::sw_k(r0 + kStep * i, c)) = v[i];
    } else {
#pragma unroll
      for (int i = 0; i < kPer; ++i) {
        uint8_t *dst = tile + tc::sw_k(r0 + kStep * i, c);
        if (ok[i])
          put16(dst, nullptr, tab_g, (size_t)off[i]);
        else
          zero16(dst);
      }
    }
  }
  __device__ void epilogue(const uint8_t *meta, int z, int m, int rl, int n, const float *v) const {
    if (tp(meta)[rl] < 0) return;
    const Dims &D = d(z);
    const float *b1 = w32(z) + D.off_b1() + n;
    float x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = fmaxf(v[j] + b1[j], 0.f);
    *reinterpret_cast<uint4 *>((stat(z) ? p.hs_b : p.hd_b) + (size_t)row(grp(z), m) * D.H + n) = pack8(x);
  }
};

// L = h W2 + b2: A = h by TMA (K-major), B = W2[h][a] by TMA (MN-major)
struct LogitsT : TwoModels {
  static constexpr bool kAMN = false, kBMN = true, kTail = false;
  static constexpr int kEpi = 0;
  static constexpr int kGather = 0;
  CUtensorMap h[2], w2[2];
  __device__ int M(int z) const { return nrows(grp(z)); }
  __device__ int N(int z) const { return d(z).A; }
  __device__ int K(int z) const { return d(z).H; }
  __device__ void prepare(uint8_t *meta, int z, int m0) const { fill(meta, ml, grp(z), m0, tc::kRows, nullptr, 0); }
  __device__ tc::TmaOperand tma_a(int z) const { return {&h[stat(z)], 2, 0, 0}; }
  __device__ tc::TmaOperand tma_b(int z) const { return {&w2[stat(z)], stat(z) ? 2 : 3, grp(z), 0}; }
  __device__ int row_a(int z, int m0) const { return row(grp(z), m0); }
  __device__ int row_b(int, int n0) const { return n0; }
  __device__ void gather(uint8_t *, const uint8_t *, int, int, int, int) const {}
  __device__ void epilogue(const uint8_t *meta, int z, int m, int rl, int n, const float *v) const {
    if (tp(meta)[rl] < 0) return;
    const Dims &D = d(z);
    const float *b2 = w32(z) + D.off_b2() + n;
    float x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = v[j] + b2[j];
    store8((stat(z) ? p.zu : p.zm) + (size_t)row(grp(z), m) * D.A + n, x);
  }
};

// dh = (dz W2^T) * [h > 0]: A = dz by TMA (K-major), B = W2[h][a] as N = h, K = a (K-major)
struct DhT : TBase {
  static constexpr bool kAMN = false, kBMN = false, kTail = false;
  static constexpr int kEpi = 0;
  static constexpr int kGather = 0;
  CUtensorMap dz, w2;
  __device__ bool active(int z) const { return group_trains(p, T, z); }
  __device__ int M(int z) const { return nrows(z); }
  __device__ int N(int) const { return p.dm.H; }
  __device__ int K(int) const { return p.dm.A; }
  __device__ void prepare(uint8_t *meta, int z, int m0) const { fill(meta, ml, z, m0, tc::kRows, nullptr, 0); }
  __device__ tc::TmaOperand tma_a(int) const { return {&dz, 2, 0, 0}; }
  __device__ tc::TmaOperand tma_b(int z) const { return {&w2, 3, z, 0}; }
  __device__ int row_a(int z, int m0) const { return row(z, m0); }
  __device__ int row_b(int, int n0) const { return n0; }
  __device__ void gather(uint8_t *, const uint8_t *, int, int, int, int) const {}
  __device__ void epilogue(const uint8_t *meta, int z, int m, int rl, int n, const float *v) const {
    const size_t i = (size_t)row(z, m) * p.dm.H + n;
    const bool ok = tp(meta)[rl] >= 0;  // zeros where nothing is predicted
    uint4 hw = *reinterpret_cast<const uint4 *>(p.hd_b + i);
    const bf16 *hv = reinterpret_cast<const bf16 *>(&hw);
    float x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = (ok && __bfloat162float(hv[j]) > 0.f) ? v[j] : 0.f;
    *reinterpret_cast<uint4 *>(p.dh_b + i) = pack8(x);
  }
};

// dW2 = h^T dz over the predicted lanes: M = H, N = A, K = lanes; both operands MN-major by TMA
struct DW2T : TBase {
  static constexpr bool kAMN = true, kBMN = true, kTail = true;
  static constexpr int kEpi = 0;
  static constexpr int kGather = 0;
  CUtensorMap h, dz;
  __device__ bool active(int z) const { return group_trains(p, T, z); }
  __device__ int M(int) const { return p.dm.H; }
  __device__ int N(int) const { return p.dm.A; }
  __device__ int K(int z) const { return npred(z); }
  __device__ void prepare(uint8_t *, int, int) const {}
  __device__ tc::TmaOperand tma_a(int z) const { return {&h, 2, 0, p.grp_lane_off[z]}; }
  __device__ tc::TmaOperand tma_b(int z) const { return {&dz, 2, 0, p.grp_lane_off[z]}; }
  __device__ int row_a(int, int m0) const { return m0; }
  __device__ int row_b(int, int n0) const { return n0; }
  __device__ void gather(uint8_t *, const uint8_t *, int, int, int, int) const {}
  __device__ void epilogue(const uint8_t *, int z, int h_, int, int n, const float *v) const {
    store8(p.grad + (size_t)z * p.P + p.dm.off_w2() + (size_t)h_ * p.dm.A + n, v);
  }
};

// dX = dh W1^T scattered into the embedding rows as fixed-point integers (order-free sums, so the
// result does not depend on scheduling): A = dh by TMA (K-major), B = W1t[h][i] as N = i, K = h
// by TMA (MN-major).  The lanes of a warp add consecutive elements of one embedding row.  Where
// the group's fixed-point table (A x E x 8 bytes) fits in shared memory, the CTA first sums its
// tile there and then adds each non-zero entry to global memory once, so a token that appears at
// several (lane, position) pairs of the tile costs one global atomic per element instead of one
// per pair.  A 64-bit shared-memory sum is kept as two 32-bit words updated by native 32-bit
// atomics: the low word first, then the high word plus the carry out of the low word (the number
// of wraps of the low word does not depend on the order of the adds, so the sum is exact).
struct DXT : TBase {
  static constexpr bool kAMN = false, kBMN = true, kTail = false;
  static constexpr int kEpi = 1;
  static constexpr int kGather = 0;
  static constexpr bool kFinish = true;
  CUtensorMap dh, w1;
  int sacc;    // sum the tile in shared memory (ml.table bytes: low words [A*E] then high words [A*E])
  int eshift;  // log2 E when E is a power of two, else -1
  __device__ bool active(int z) const { return group_trains(p, T, z); }
  __device__ int M(int z) const { return nrows(z); }
  __device__ int N(int) const { return p.dm.K1(); }
  __device__ int K(int) const { return p.dm.H; }
  __device__ uint32_t *lo_s(const uint8_t *meta) const {
    return reinterpret_cast<uint32_t *>(const_cast<uint8_t *>(meta) + ml.tab_off());
  }
  __device__ void prepare(uint8_t *meta, int z, int m0) const {
    MetaLayout l = ml;
    l.table = 0;  // the accumulator region is not an embedding copy
    fill(meta, l, z, m0, tc::kRows, nullptr, 0);
    if (sacc) {
      uint4 *a = reinterpret_cast<uint4 *>(lo_s(meta));
      for (int i = threadIdx.x; i < p.dm.A * p.dm.E / 2; i += tc::kThreads) a[i] = make_uint4(0, 0, 0, 0);
    }
  }
  __device__ tc::TmaOperand tma_a(int) const { return {&dh, 2, 0, 0}; }
  __device__ tc::TmaOperand tma_b(int z) const { return {&w1, 3, z, 0}; }
  __device__ int row_a(int z, int m0) const { return row(z, m0); }
  __device__ int row_b(int, int n0) const { return n0; }
  __device__ void gather(uint8_t *, const uint8_t *, int, int, int, int) const {}
  __device__ bool row_active(const uint8_t *meta, int, int, int rl) const { return tp(meta)[rl] >= 0; }
  __device__ void emit(const uint8_t *meta, int z, int, int rl, int n, float v) const {
    const int pos = eshift >= 0 ? n >> eshift : n / p.dm.E;
    const uint32_t i = (uint32_t)tk(meta)[rl * p.dm.t + pos] * (uint32_t)p.dm.E + (uint32_t)(n - pos * p.dm.E);
    const long long q = fix40(v);
    if (q == 0) return;
    if (sacc) {
      uint32_t *lo = lo_s(meta);
      const uint32_t ql = (uint32_t)(unsigned long long)q, qh = (uint32_t)((unsigned long long)q >> 32);
      const uint32_t old = atomicAdd(lo + i, ql);
      const uint32_t up = qh + (old + ql < old ? 1u : 0u);  // high part plus the carry out of the low word
      if (up) atomicAdd(lo + p.dm.A * p.dm.E + i, up);
    } else {
      atomicAdd(reinterpret_cast<unsigned long long *>(p.demb_acc) + (size_t)z * p.dm.A * p.dm.E + i,
                (unsigned long long)q);
    }
  }
  // every thread, after the epilogue's last barrier: the non-zero sums of the tile to global memory
  __device__ void finish(uint8_t *meta, int z) const {
    if (!sacc) return;
    const uint32_t *lo = lo_s(meta), *hi = lo + p.dm.A * p.dm.E;
    unsigned long long *dst = reinterpret_cast<unsigned long long *>(p.demb_acc) + (size_t)z * p.dm.A * p.dm.E;
    for (int i = threadIdx.x; i < p.dm.A * p.dm.E; i += tc::kThreads) {
      const unsigned long long q = ((unsigned long long)hi[i] << 32) | lo[i];
      if (q) atomicAdd(dst + i, q);
    }
  }
};

// dW1 (stored transposed: dW1t[h][i] = sum over predicted lanes of dh[m][h] X[m][i]): M = H,
// N = t*E, K = lanes; A = dh by TMA (MN-major), B = X gathered (MN-major)
struct DW1T : TBase {
  static constexpr bool kAMN = true, kBMN = true, kTail = true;
  static constexpr int kEpi = 0;
  static constexpr int kGather = 2;
  CUtensorMap dh;
  int table;
  __device__ bool active(int z) const { return group_trains(p, T, z); }
  __device__ int M(int) const { return p.dm.H; }
  __device__ int N(int) const { return p.dm.K1(); }
  __device__ int K(int z) const { return npred(z); }
  __device__ void prepare(uint8_t *meta, int z, int) const {
    fill(meta, ml, z, 0, npred(z), wb(z) + p.dm.off_emb(), p.dm.A * p.dm.E * 2);
  }
  __device__ tc::TmaOperand tma_a(int z) const { return {&dh, 2, 0, p.grp_lane_off[z]}; }
  __device__ tc::TmaOperand tma_b(int) const { return kNoTma; }
  __device__ int row_a(int, int m0) const { return m0; }
  __device__ int row_b(int, int) const { return 0; }
  // chunk idx = 16 bytes at column n = 8 (idx % (R/8)) of K row idx / (R/8); consecutive threads
  // take consecutive chunks of a row, four per thread in flight
  __device__ void gather(uint8_t *tile, const uint8_t *meta, int z, int n0, int k0, int R) const {
    const Dims &D = p.dm;
    const long long *tpv = tp(meta);
    const uint16_t *tkv = tk(meta);
    const bf16 *tab_s = table ? this->table_ptr(meta) : nullptr;
    const bf16 *tab_g = wb(z) + D.off_emb();
    const int K = npred(z), cpr = R / 8, total = cpr * tc::kBK;
    for (int i0 = 0; i0 < total; i0 += 4 * tc::kThreads) {
      int off[4], dsto[4];
      bool ok[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int idx = i0 + j * tc::kThreads + threadIdx.x;
        const int n = (idx % cpr) * 8, k = idx / cpr, m = k0 + k;
        dsto[j] = idx < total ? (int)tc::sw_mn(n, k) : -1;
        ok[j] = idx < total && m < K && tpv[m] >= 0;
        const int i = n0 + n, pos = i / D.E;
        off[j] = ok[j] ? (int)tkv[m * D.t + pos] * D.E + (i - pos * D.E) : 0;
      }
      if (tab_s) {
        uint4 v[4];
#pragma unroll
        for (int j = 0; j < 4; ++j)
          v[j] = ok[j] ? *reinterpret_cast<const uint4 *>(tab_s + off[j]) : make_uint4(0, 0, 0, 0);
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (dsto[j] >= 0) *reinterpret_cast<uint4 *>(tile + dsto[j]) = v[j];
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          if (dsto[j] < 0) continue;
          if (ok[j])
            put16(tile + dsto[j], nullptr, tab_g, (size_t)off[j]);
          else
            zero16(tile + dsto[j]);
        }
      }
    }
  }
  __device__ const bf16 *table_ptr(const uint8_t *meta) const { return TBase::table(meta); }
  __device__ void epilogue(const uint8_t *, int z, int h_, int, int n, const float *v) const {
    store8(p.grad + (size_t)z * p.P + p.dm.off_w1() + (size_t)h_ * p.dm.K1() + n, v);
  }
};

// ---- the frozen static model in FP8 (E4M3): hidden layer and logits on kind::f8f6f4 ----
// h = relu((X_q W1_q) c1[h] + b1) in FP32, X_q gathered from the E4M3 embedding codes (16 codes per
// 16-byte chunk; E % 16 == 0), W1_q = the W1t codes by TMA (K-major).  The epilogue also raises the
// row's largest activation (float bits: h >= 0, so integer order is float order).
struct HiddenF8 : TBase {
  static constexpr bool kAMN = false, kBMN = false, kTail = false, kFP8 = true;
  static constexpr int kEpi = 0;
  static constexpr int kGather = 1;
  CUtensorMap w1;  // W1t codes [H][t*E], box {128, nt}
  int table;       // E4M3 embedding table kept in shared memory
  __device__ bool active(int z) const { return group_trains(p, T, z); }
  __device__ int M(int z) const { return nrows(z); }
  __device__ int N(int) const { return p.st.H; }
  __device__ int K(int) const { return p.st.K1(); }
  __device__ void prepare(uint8_t *meta, int z, int m0) const {
    MetaLayout l = ml;
    l.table = table ? p.st.A * p.st.E : 0;
    fill(meta, l, z, m0, tc::kRows, p.st8, p.st.A * p.st.E);
  }
  __device__ tc::TmaOperand tma_a(int) const { return kNoTma; }
  __device__ tc::TmaOperand tma_b(int) const { return {&w1, 2, 0, 0}; }
  __device__ int row_a(int, int) const { return 0; }
  __device__ int row_b(int, int n0) const { return n0; }
  // thread: 16-byte chunk c = tid % 8 (16 codes) of rows tid / 8 + 32 i
  __device__ void gather(uint8_t *tile, const uint8_t *meta, int, int, int k0, int) const {
    const Dims &D = p.st;
    const long long *tpv = tp(meta);
    const uint16_t *tkv = tk(meta);
    const uint8_t *tab_s = table ? meta + ml.tab_off() : nullptr;
    const int c = threadIdx.x & 7, k = k0 + 16 * c, r0 = threadIdx.x >> 3;
    const bool kin = k < D.K1();
    const int pos = kin ? k / D.E : 0, e = k - pos * D.E;
    constexpr int kPer = tc::kRows * 8 / tc::kThreads, kStep = tc::kThreads / 8;
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
      const int r = r0 + kStep * i;
      uint8_t *dst = tile + tc::sw_k(r, c);
      const bool ok = kin && tpv[r] >= 0;
      const int off = ok ? (int)tkv[r * D.t + pos] * D.E + e : 0;
      if (!ok)
        zero16(dst);
      else if (tab_s)
        *reinterpret_cast<uint4 *>(dst) = *reinterpret_cast<const uint4 *>(tab_s + off);
      else
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(tc::sa(dst)), "l"(p.st8 + off));
    }
  }
  __device__ void epilogue(const uint8_t *meta, int z, int m, int rl, int n, const float *v) const {
    if (tp(meta)[rl] < 0) return;
    const float *c1 = p.st8_c1 + n, *b1 = p.static_params + p.st.off_b1() + n;
    const int rw = row(z, m);
    float x[8], mx = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const float a = fmaf(v[j], c1[j], b1[j]);
      x[j] = a > 0.f ? a : 0.f;  // +0 below zero (its bits must order as a float)
      mx = fmaxf(mx, x[j]);
    }
    store8(p.hs + (size_t)rw * p.st.H + n, x);
    atomicMax(p.hs_rowmax + rw, __float_as_uint(mx));
  }
};

// L = (h_q W2_q) s_r s_w2[a] + b2: A = the row's activations coded as E4M3 with the row scale
// s_r = max h / 448 (gathered from the FP32 h), B = the transposed W2 codes [A][H] by TMA (K-major).
struct LogitsF8 : TBase {
  static constexpr bool kAMN = false, kBMN = false, kTail = false, kFP8 = true;
  static constexpr int kEpi = 0;
  static constexpr int kGather = 1;
  CUtensorMap w2;  // W2t codes [A][H], box {128, nt}
  __device__ bool active(int z) const { return group_trains(p, T, z); }
  __device__ int M(int z) const { return nrows(z); }
  __device__ int N(int) const { return p.st.A; }
  __device__ int K(int) const { return p.st.H; }
  // meta: targets | (no tokens) | per row: s_r and 448 / max h (0 for an all-zero row)
  __device__ float *rs(const uint8_t *meta) const {
    return reinterpret_cast<float *>(const_cast<uint8_t *>(meta) + ml.tab_off());
  }
  __device__ void prepare(uint8_t *meta, int z, int m0) const {
    fill(meta, ml, z, m0, tc::kRows, nullptr, 0);
    float *r = rs(meta);
    for (int i = threadIdx.x; i < tc::kRows; i += tc::kThreads) {
      const int m = m0 + i;
      const float mx = m < nrows(z) ? __uint_as_float(p.hs_rowmax[row(z, m)]) : 0.f;
      r[2 * i] = mx > 0.f ? __fdiv_rn(mx, 448.f) : 1.f;
      r[2 * i + 1] = mx > 0.f ? __fdiv_rn(448.f, mx) : 0.f;
    }
  }
  __device__ tc::TmaOperand tma_a(int) const { return kNoTma; }
  __device__ tc::TmaOperand tma_b(int) const { return {&w2, 2, 0, 0}; }
  __device__ int row_a(int, int) const { return 0; }
  __device__ int row_b(int, int n0) const { return n0; }
  // thread: 16-byte chunk c = tid % 8 (16 activations) of rows tid / 8 + 32 i
  __device__ void gather(uint8_t *tile, const uint8_t *meta, int z, int m0, int k0, int) const {
    const int H = p.st.H;
    const long long *tpv = tp(meta);
    const float *r = rs(meta);
    const int c = threadIdx.x & 7, k = k0 + 16 * c, r0 = threadIdx.x >> 3;
    constexpr int kPer = tc::kRows * 8 / tc::kThreads, kStep = tc::kThreads / 8;
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
      const int rl = r0 + kStep * i;
      uint4 out = make_uint4(0, 0, 0, 0);
      if (k < H && tpv[rl] >= 0) {  // H % 16 == 0: a chunk is all in or all out
        const float inv = r[2 * rl + 1];
        const float4 *src = reinterpret_cast<const float4 *>(p.hs + (size_t)row(z, m0 + rl) * H + k);
        uint32_t w[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float4 f = src[q];
          const __nv_fp8x4_e4m3 x(make_float4(f.x * inv, f.y * inv, f.z * inv, f.w * inv));
          w[q] = *reinterpret_cast<const uint32_t *>(&x);
        }
        out = make_uint4(w[0], w[1], w[2], w[3]);
      }
      *reinterpret_cast<uint4 *>(tile + tc::sw_k(rl, c)) = out;
    }
  }
  __device__ void epilogue(const uint8_t *meta, int z, int m, int rl, int n, const float *v) const {
    if (tp(meta)[rl] < 0) return;
    const float sr = rs(meta)[2 * rl];
    const float *s2 = p.st8_s2 + n, *b2 = p.static_params + p.st.off_b2() + n;
    float x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = fmaf(v[j], __fmul_rn(sr, s2[j]), b2[j]);
    store8(p.zu + (size_t)row(z, m) * p.st.A + n, x);
  }
};

// db1 = sum of dh, db2 = sum of dz over the predicted rows of each group (the predicted lanes are
// a prefix of the group's lanes).  Block: 16 chunks of 8 columns x 16 row slices; slice y adds
// rows y, y + 16, ... in order (16-byte loads), then slice 0 adds the 16 partial sums in order,
// so the result does not depend on scheduling.
constexpr int kBiasChunks = 16, kBiasSlices = 16;
__global__ void __launch_bounds__(kBiasChunks * kBiasSlices) bias_grad_kernel(Plan p, int T) {
  __shared__ float part[kBiasSlices][kBiasChunks * 8 + 4];
  const int g = blockIdx.y;
  if (!group_trains(p, T, g)) return;
  const int H = p.dm.H, A = p.dm.A;
  const int cx = threadIdx.x % kBiasChunks, y = threadIdx.x / kBiasChunks;
  const int c = (blockIdx.x * kBiasChunks + cx) * 8;  // first of 8 columns (H and A are multiples of 8)
  const bool in = c < H + A, is1 = c < H;
  const int w = is1 ? H : A, cc = is1 ? c : c - H;
  const bf16 *src = is1 ? p.dh_b : p.dz_b;
  const int r0 = p.grp_lane_off[g], n = live_lanes(p, g, T - p.grp_start[g]);
  float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  if (in) {
#pragma unroll 4
    for (int r = y; r < n; r += kBiasSlices) {
      const uint4 v = *reinterpret_cast<const uint4 *>(src + (size_t)(r0 + r) * w + cc);
      const bf16 *b = reinterpret_cast<const bf16 *>(&v);
#pragma unroll
      for (int q = 0; q < 8; ++q) s[q] += __bfloat162float(b[q]);
    }
  }
#pragma unroll
  for (int q = 0; q < 8; ++q) part[y][cx * 8 + q] = s[q];
  __syncthreads();
  if (threadIdx.x < kBiasChunks * 8) {
    const int col = blockIdx.x * kBiasChunks * 8 + threadIdx.x;
    if (col < H + A) {
      float t = 0.f;
      for (int yy = 0; yy < kBiasSlices; ++yy) t += part[yy][threadIdx.x];
      const bool b1 = col < H;
      p.grad[(size_t)g * p.P + (b1 ? p.dm.off_b1() + col : p.dm.off_b2() + (col - H))] = t;
    }
  }
}


// ---- host: tensor maps -----------------------------------------------------------------

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  }();
  return fn;
}

// BF16 (or, with u8, E4M3 code) tensor map with 128-byte swizzle: dims[0] innermost (elements),
// strides in bytes for the outer dimensions, box {128 bytes of elements, box1}
bool make_map(CUtensorMap *m, const void *ptr, int rank, const uint64_t *dims, const uint64_t *strides, int box1,
              bool u8 = false) {
  auto fn = encode_fn();
  if (!fn || !ptr) return false;
  cuuint64_t d[3], s[2];
  cuuint32_t box[3] = {u8 ? 128u : 64u, (cuuint32_t)box1, 1}, es[3] = {1, 1, 1};
  for (int i = 0; i < rank; ++i) d[i] = dims[i];
  for (int i = 0; i + 1 < rank; ++i) s[i] = strides[i];
  return fn(m, u8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, (cuuint32_t)rank,
            const_cast<void *>(ptr), d, s, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Everything the six launches of a plan need: tile widths, shared data sizes and tensor maps.
struct TcSetup {
  // key: the plan's buffers and shapes
  const void *wbf, *static_bf, *hd_b, *hs_b, *dz_b, *dh_b, *st8;
  int G, NL, Mmax, use_static;
  Dims dm, st;
  size_t P;
  bool ok;
  tc::TilePlan t_h, t_l, t_dh, t_w2, t_dx, t_w1, t_h8, t_l8;
  MetaLayout ml_h, ml_l, ml_dh, ml_w2, ml_dx, ml_w1, ml_h8, ml_l8;
  int table_h[2], table_w1, sacc_dx, table_h8;
  CUtensorMap w1k[2], w1mn, w2mn[2], w2k, hk[2], dzk, dhk, hmn, dzmn, dhmn, w1_8, w2_8;
};

bool same_key(const TcSetup &a, const Plan &p) {
  auto dims_eq = [](const Dims &x, const Dims &y) { return x.A == y.A && x.E == y.E && x.t == y.t && x.H == y.H; };
  return a.wbf == p.wbf && a.static_bf == p.static_bf && a.hd_b == p.hd_b && a.hs_b == p.hs_b && a.dz_b == p.dz_b &&
         a.dh_b == p.dh_b && a.st8 == p.st8 && a.G == p.G && a.NL == p.NL && a.Mmax == p.Mmax &&
         a.use_static == p.use_static &&
         dims_eq(a.dm, p.dm) && (!p.use_static || dims_eq(a.st, p.st)) && a.P == p.P;
}

bool shapes_ok(const Plan &p) {
  auto ok = [](const Dims &d) { return d.E % 8 == 0 && d.H % 64 == 0 && d.A % 64 == 0 && d.K1() % 64 == 0; };
  // the FP8 static model: 16 E4M3 codes per gathered chunk never straddle two embedding rows
  const bool f8 = p.st8 == nullptr || p.st.E % 16 == 0;
  return p.G > 0 && p.NL > 0 && p.Mmax > 0 && ok(p.dm) && p.P % 8 == 0 && (!p.use_static || ok(p.st)) && f8;
}

bool build(TcSetup &S, const Plan &p) {
  S.wbf = p.wbf, S.static_bf = p.static_bf, S.hd_b = p.hd_b, S.hs_b = p.hs_b, S.dz_b = p.dz_b, S.dh_b = p.dh_b;
  S.st8 = p.st8;
  S.G = p.G, S.NL = p.NL, S.Mmax = p.Mmax, S.use_static = p.use_static, S.dm = p.dm, S.st = p.st, S.P = p.P;
  S.ok = false;
  if (!shapes_ok(p) || !encode_fn()) return false;
  const Dims &D = p.dm, &Sd = p.st;
  const int Z = p.use_static ? 2 * p.G : p.G;
  const int tmax = p.use_static ? max(D.t, Sd.t) : D.t;
  const size_t limit = 220 * 1024;
  // embedding tables kept in shared memory where they fit
  S.table_h[0] = (size_t)D.A * D.E * 2 <= kTableMax;
  S.table_h[1] = p.use_static && (size_t)Sd.A * Sd.E * 2 <= kTableMax;
  S.table_w1 = S.table_h[0];
  S.ml_h = {tc::kRows, tmax, (int)max(S.table_h[0] ? (size_t)D.A * D.E * 2 : 0,
                                       S.table_h[1] ? (size_t)Sd.A * Sd.E * 2 : 0)};
  S.ml_l = S.ml_dh = {tc::kRows, 0, 0};
  S.ml_w2 = {0, 0, 0};
  S.sacc_dx = (size_t)D.A * D.E * 8 <= kAccMax;
  S.ml_dx = {tc::kRows, D.t, S.sacc_dx ? D.A * D.E * 8 : 0};
  S.ml_w1 = {p.Mmax, D.t, S.table_w1 ? D.A * D.E * 2 : 0};
  const int Hmax = p.use_static ? max(D.H, Sd.H) : D.H, K1max = p.use_static ? max(D.K1(), Sd.K1()) : D.K1();
  S.t_h = tc::plan_tiles(p.Mmax, Hmax, K1max, Z, S.ml_h.bytes(), false);
  S.t_l = tc::plan_tiles(p.Mmax, D.A, Hmax, Z, S.ml_l.bytes());
  S.t_dh = tc::plan_tiles(p.Mmax, D.H, D.A, p.G, S.ml_dh.bytes());
  S.t_w2 = tc::plan_tiles(D.H, D.A, p.Mmax, p.G, S.ml_w2.bytes());
  S.t_dx = tc::plan_tiles(p.Mmax, D.K1(), D.H, p.G, S.ml_dx.bytes());
  S.t_w1 = tc::plan_tiles(D.H, D.K1(), p.Mmax, p.G, S.ml_w1.bytes());
  for (const auto &pr : {std::make_pair(S.t_h, S.ml_h.bytes()), std::make_pair(S.t_l, S.ml_l.bytes()),
                         std::make_pair(S.t_dh, S.ml_dh.bytes()), std::make_pair(S.t_w2, S.ml_w2.bytes()),
                         std::make_pair(S.t_dx, S.ml_dx.bytes()), std::make_pair(S.t_w1, S.ml_w1.bytes())})
    if (tc::smem_bytes(pr.first, pr.second) > limit) return false;
  // per-group weights: [G][P] BF16 with W1t [H][t*E] and W2 [H][A] inside
  const uint64_t gs = (uint64_t)p.P * 2;
  bool ok = true;
  {
    const uint64_t d[3] = {(uint64_t)D.K1(), (uint64_t)D.H, (uint64_t)p.G}, s[2] = {(uint64_t)D.K1() * 2, gs};
    ok &= make_map(&S.w1k[0], p.wbf + D.off_w1(), 3, d, s, S.t_h.nt);
    ok &= make_map(&S.w1mn, p.wbf + D.off_w1(), 3, d, s, 64);
  }
  {
    const uint64_t d[3] = {(uint64_t)D.A, (uint64_t)D.H, (uint64_t)p.G}, s[2] = {(uint64_t)D.A * 2, gs};
    ok &= make_map(&S.w2mn[0], p.wbf + D.off_w2(), 3, d, s, 64);
    ok &= make_map(&S.w2k, p.wbf + D.off_w2(), 3, d, s, S.t_dh.nt);
  }
  auto act = [&](CUtensorMap *m, const void *ptr, int width, int box1) {
    const uint64_t d[2] = {(uint64_t)width, (uint64_t)p.NL}, s[1] = {(uint64_t)width * 2};
    return make_map(m, ptr, 2, d, s, box1);
  };
  ok &= act(&S.hk[0], p.hd_b, D.H, tc::kRows);
  ok &= act(&S.dzk, p.dz_b, D.A, tc::kRows);
  ok &= act(&S.dhk, p.dh_b, D.H, tc::kRows);
  ok &= act(&S.hmn, p.hd_b, D.H, 64);
  ok &= act(&S.dzmn, p.dz_b, D.A, 64);
  ok &= act(&S.dhmn, p.dh_b, D.H, 64);
  const bool f8 = p.use_static && p.st8 != nullptr;
  if (f8) {  // the static model in E4M3: its own tiles (128 K per stage) and code maps
    S.table_h8 = (size_t)Sd.A * Sd.E <= kTableMax;
    S.ml_h8 = {tc::kRows, Sd.t, S.table_h8 ? Sd.A * Sd.E : 0};
    S.ml_l8 = {tc::kRows, 0, tc::kRows * 8};
    S.t_h8 = tc::plan_tiles(p.Mmax, Sd.H, Sd.K1(), p.G, S.ml_h8.bytes(), false, 2 * tc::kBK);
    S.t_l8 = tc::plan_tiles(p.Mmax, Sd.A, Sd.H, p.G, S.ml_l8.bytes(), false, 2 * tc::kBK);
    if (tc::smem_bytes(S.t_h8, S.ml_h8.bytes()) > limit || tc::smem_bytes(S.t_l8, S.ml_l8.bytes()) > limit)
      return false;
    const uint8_t *w1c = p.st8 + (size_t)Sd.A * Sd.E, *w2c = w1c + (size_t)Sd.H * Sd.K1();
    const uint64_t d1[2] = {(uint64_t)Sd.K1(), (uint64_t)Sd.H}, s1[1] = {(uint64_t)Sd.K1()};
    ok &= make_map(&S.w1_8, w1c, 2, d1, s1, S.t_h8.nt, true);
    const uint64_t d2[2] = {(uint64_t)Sd.H, (uint64_t)Sd.A}, s2[1] = {(uint64_t)Sd.H};
    ok &= make_map(&S.w2_8, w2c, 2, d2, s2, S.t_l8.nt, true);
  }
  if (p.use_static && !f8) {
    const uint64_t d1[2] = {(uint64_t)Sd.K1(), (uint64_t)Sd.H}, s1[1] = {(uint64_t)Sd.K1() * 2};
    ok &= make_map(&S.w1k[1], p.static_bf + Sd.off_w1(), 2, d1, s1, S.t_h.nt);
    const uint64_t d2[2] = {(uint64_t)Sd.A, (uint64_t)Sd.H}, s2[1] = {(uint64_t)Sd.A * 2};
    ok &= make_map(&S.w2mn[1], p.static_bf + Sd.off_w2(), 2, d2, s2, 64);
    ok &= act(&S.hk[1], p.hs_b, Sd.H, tc::kRows);
  } else {
    S.w1k[1] = S.w1k[0], S.w2mn[1] = S.w2mn[0], S.hk[1] = S.hk[0];
  }
  S.ok = ok;
  return ok;
}

std::mutex g_tc_mu;
TcSetup g_tc;  // the last plan's setup (runs reuse their buffers for every step)
bool g_tc_valid = false;

bool get_setup(const Plan &p, TcSetup &out) {
  std::lock_guard<std::mutex> lk(g_tc_mu);
  if (!g_tc_valid || !same_key(g_tc, p)) {
    build(g_tc, p);
    g_tc_valid = true;
  }
  out = g_tc;
  return out.ok;
}

}  // namespace

bool tc_supported(const Plan &p) {
  if (!shapes_ok(p)) return false;
  TcSetup S;
  return get_setup(p, S);
}

void launch_forward_tc(const Plan &p, int T, cudaStream_t st) {
  TcSetup S;
  if (!get_setup(p, S)) return;
  const double R = prof_work().pred_rows;
  const bool f8 = p.use_static && p.st8 != nullptr;  // static model on its own E4M3 launches
  const int Z = p.use_static && !f8 ? 2 * p.G : p.G;
  if (f8) {
    {
      ProfScope ps("fwd_hidden_static_fp8", 2.0 * R * p.st.K1() * p.st.H, 0, st);
      HiddenF8 op;
      op.p = p, op.T = T, op.ml = S.ml_h8, op.w1 = S.w1_8, op.table = S.table_h8;
      tc::launch(op, p.Mmax, p.st.H, p.G, S.t_h8, S.ml_h8.bytes(), st);
    }
    ProfScope ps("fwd_logits_static_fp8", 2.0 * R * p.st.H * p.st.A, 0, st);
    LogitsF8 op;
    op.p = p, op.T = T, op.ml = S.ml_l8, op.w2 = S.w2_8;
    tc::launch(op, p.Mmax, p.st.A, p.G, S.t_l8, S.ml_l8.bytes(), st);
  }
  {
    double fl = 2.0 * R * p.dm.K1() * p.dm.H + (p.use_static && !f8 ? 2.0 * R * p.st.K1() * p.st.H : 0.0);
    ProfScope ps("fwd_hidden_bf16", fl, 0, st);
    HiddenT op;
    op.p = p, op.T = T, op.ml = S.ml_h, op.w1[0] = S.w1k[0], op.w1[1] = S.w1k[1];
    op.table[0] = S.table_h[0], op.table[1] = S.table_h[1];
    tc::launch(op, p.Mmax, p.use_static ? max(p.dm.H, p.st.H) : p.dm.H, Z, S.t_h, S.ml_h.bytes(), st);
  }
  double fl = 2.0 * R * p.dm.H * p.dm.A + (p.use_static && !f8 ? 2.0 * R * p.st.H * p.st.A : 0.0);
  ProfScope ps("fwd_logits_bf16", fl, 0, st);
  LogitsT op;
  op.p = p, op.T = T, op.ml = S.ml_l, op.h[0] = S.hk[0], op.h[1] = S.hk[1], op.w2[0] = S.w2mn[0], op.w2[1] = S.w2mn[1];
  tc::launch(op, p.Mmax, p.dm.A, Z, S.t_l, S.ml_l.bytes(), st);
}

void launch_backward_tc(const Plan &p, int T, cudaStream_t st, const StepStreams *ss) {
  TcSetup S;
  if (!get_setup(p, S)) return;
  const double R = prof_work().pred_rows;
  const Dims &D = p.dm;
  {
    ProfScope ps("bwd_dh_bf16", 2.0 * R * D.A * D.H, 0, st);
    DhT op;
    op.p = p, op.T = T, op.ml = S.ml_dh, op.dz = S.dzk, op.w2 = S.w2k;
    tc::launch(op, p.Mmax, D.H, p.G, S.t_dh, S.ml_dh.bytes(), st);
  }
  // dW2 (+ bias sums), dX and dW1 only read dh, dz, h and the weights
  // and write disjoint buffers: with auxiliary streams they run side by side
  cudaStream_t s1 = st, s2 = st;
  if (ss) {
    cudaEventRecord(ss->fork, st);
    cudaStreamWaitEvent(ss->aux[0], ss->fork, 0);
    cudaStreamWaitEvent(ss->aux[1], ss->fork, 0);
    s1 = ss->aux[0], s2 = ss->aux[1];
  }
  {
    ProfScope ps("bwd_dx_bf16", 2.0 * R * D.K1() * D.H, 0, s2);
    DXT op;
    op.p = p, op.T = T, op.ml = S.ml_dx, op.dh = S.dhk, op.w1 = S.w1mn, op.sacc = S.sacc_dx;
    op.eshift = (D.E & (D.E - 1)) == 0 ? __builtin_ctz((unsigned)D.E) : -1;
    tc::launch(op, p.Mmax, D.K1(), p.G, S.t_dx, S.ml_dx.bytes(), s2);
  }
  {
    ProfScope ps("bwd_dw2_bf16", 2.0 * R * D.A * D.H, 0, s1);
    DW2T op;
    op.p = p, op.T = T, op.ml = S.ml_w2, op.h = S.hmn, op.dz = S.dzmn;
    tc::launch(op, D.H, D.A, p.G, S.t_w2, S.ml_w2.bytes(), s1);
    bias_grad_kernel<<<dim3((D.H + D.A + 8 * kBiasChunks - 1) / (8 * kBiasChunks), p.G), kBiasChunks * kBiasSlices, 0,
                       s1>>>(p, T);
  }
  {
    ProfScope ps("bwd_dw1_bf16", 2.0 * R * D.K1() * D.H, 0, st);
    DW1T op;
    op.p = p, op.T = T, op.ml = S.ml_w1, op.dh = S.dhmn, op.table = S.table_w1;
    tc::launch(op, D.H, D.K1(), p.G, S.t_w1, S.ml_w1.bytes(), st);
  }
  if (ss) {
    cudaEventRecord(ss->join[0], s1);
    cudaEventRecord(ss->join[1], s2);
    cudaStreamWaitEvent(st, ss->join[0], 0);
    cudaStreamWaitEvent(st, ss->join[1], 0);
  }
}

}  // namespace pmklc
