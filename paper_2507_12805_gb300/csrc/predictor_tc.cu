// BF16 batched form on tcgen05: the six GEMMs of one global step of every group's predictors
// (paper §2 steps 3-4, the MLP of the measured configurations), on the engine of tcgemm.cuh.
//
//   forward   h  = relu(X W1 + b1)    X gathered from the embedding rows of the context tokens
//             L  = h W2 + b2          dynamic model (z < G) and static model (z >= G) in one launch
//   backward  dh = (dz W2^T) * [h > 0]
//             dW2 = h^T dz,  dX = dh W1^T (summed into the embedding rows),  dW1 = X^T dh
//             db2 = sum of dz, db1 = sum of dh over the predicted rows (fixed-order column sums)
// With enough weight-gradient tiles to keep every SM streaming optimiser state (p.fused_w), Adam
// on W1 and W2 runs in the epilogues of their gradient GEMMs; otherwise those epilogues store the
// gradient and the streaming optimiser of predictor.cu updates every parameter.  The embedding
// and biases always go through the streaming optimiser.  With overlap-masked coding the logits
// layer and dh run over each row's coded slice only (slice.cu).
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

struct NoGather {
  __device__ void gather(uint8_t *, int) const {}
};

struct TBase {
  static constexpr bool kFinish = false;
  static constexpr bool kFP8 = false;
  Plan p;
  int T;
  MetaLayout ml;
  int zb = 0;
  __device__ void finish(uint8_t *, int) const {}
  __device__ NoGather gather_ctx(const uint8_t *, int, int, int) const { return {}; }
  __device__ int *err() const { return p.err; }
  __device__ int nrows(int g) const { return p.grp_lane_off[g + 1] - p.grp_lane_off[g]; }
  __device__ int row(int g, int r) const { return p.grp_lane_off[g] + r; }
  __device__ long long target_pos(int g, int r) const {
    const int rw = row(g, r);
    if (!row_pred(p, T, rw, g)) return -1;
    return p.lane_tok[rw] + (T - p.grp_start[g]);
  }
  __device__ int npred(int g) const { return live_lanes(p, g, T - p.grp_start[g]); }
  // Columns [lo, hi) of the logits the mixer reads for the row whose target is at tpos: with
  // overlap masking the slice of 4^s tokens that agree with the previous token (a predicted row's
  // token has index >= t_eff >= 1 in its lane), else all A.  A kEpi == 0 thread owns one tile row,
  // rl = 32 (warp % 4) + lane.
  __device__ void logit_cols(long long tpos, int A, int &lo, int &hi) const {
    lo = 0, hi = A;
    if (p.ov_w > 0 && tpos >= 1) {
      lo = ((int)p.tokens[tpos - 1] % p.ov_mod) * p.ov_w;
      hi = lo + p.ov_w;
    }
  }
  __device__ static int epi_row() { return ((threadIdx.x >> 5) & 3) * 32 + (threadIdx.x & 31); }
  __device__ const bf16 *wb(int g) const { return p.wbf + (size_t)g * p.P; }
  __device__ const long long *tp(const uint8_t *meta) const { return reinterpret_cast<const long long *>(meta); }
  __device__ const uint16_t *tk(const uint8_t *meta) const {
    return reinterpret_cast<const uint16_t *>(meta + ml.tok_off());
  }
  // targets of rows r0 .. r0 + n - 1 of group g (-1 past the group or for rows that predict
  // nothing), their t context tokens and the embedding table emb (A x E) if ml.table.  The table
  // arrives by one bulk copy that overlaps the target and token loads.
  __device__ void fill(uint8_t *meta, const MetaLayout &ml_, int g, int r0, int n, const void *emb, int bytes) const {
    __shared__ __align__(8) uint64_t tbar;
    const MetaLayout l = ml_;
    long long *tpw = reinterpret_cast<long long *>(meta);
    const bool copy = emb != nullptr && bytes > 0 && l.table >= bytes;
    if (copy && threadIdx.x == 0) {
      const uint32_t bar = tc::sa(&tbar);
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar));
      asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
      tc::expect_tx(bar, (uint32_t)bytes);
      asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                       tc::sa(meta + l.tab_off())),
                   "l"(emb), "r"(bytes), "r"(bar)
                   : "memory");
    }
    const int L = nrows(g);
    for (int i = threadIdx.x; i < n; i += tc::kThreads) tpw[i] = r0 + i < L ? target_pos(g, r0 + i) : -1;
    __syncthreads();
    if (l.t > 0) {
      uint16_t *tkw = reinterpret_cast<uint16_t *>(meta + l.tok_off());
      const uint16_t *tokens = p.tokens;
      const int t = l.t, total = n * t;
      for (int i0 = 0; i0 < total; i0 += 16 * tc::kThreads) {  // sixteen loads in flight per thread
        uint16_t v[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int i = i0 + q * tc::kThreads + threadIdx.x;
          v[q] = 0;
          if (i < total) {
            const int r = i / t;
            const long long b = tpw[r];
            if (b >= 0) v[q] = tokens[b - t + (i - r * t)];
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

__device__ __forceinline__ void zero16(uint8_t *dst) { *reinterpret_cast<uint4 *>(dst) = make_uint4(0, 0, 0, 0); }

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
constexpr int kRowsPerThread = tc::kRows * 8 / tc::kThreads;  // K-major gathers: rows a thread fills
constexpr int kRowStep = tc::kThreads / 8;                     // ... 32 apart, one 16-byte chunk each

// Gather of a K-major operand from an embedding table: thread (chunk c = tid % 8, rows tid / 8 +
// 32 i) fills 16-byte chunk c of its rows with the embedding codes of the context token at the
// chunk's position (bytes per element eb: 2 for BF16, 1 for E4M3; E * eb a multiple of 16).
struct EmbGather {
  const uint8_t *tab_s;  // table in shared memory, else nullptr
  const uint8_t *tab_g;  // table in global memory
  const uint16_t *tk;    // context tokens of the tile's rows (t per row)
  int E, t, K1, eb;
  int c;
  int tokrow[kRowsPerThread];  // row r * t, or -1 for rows that predict nothing
  __device__ void gather(uint8_t *tile, int k0) const {
    const int per = 16 / eb, k = k0 + per * c;
    const bool kin = k < K1;
    const int pos = kin ? k / E : 0, e = k - pos * E;
    int off[kRowsPerThread];
    bool ok[kRowsPerThread];
#pragma unroll
    for (int i = 0; i < kRowsPerThread; ++i) {
      ok[i] = kin && tokrow[i] >= 0;
      off[i] = ok[i] ? ((int)tk[tokrow[i] + pos] * E + e) * eb : 0;
    }
    const int r0 = threadIdx.x >> 3;
    if (tab_s) {
      uint4 v[kRowsPerThread];
#pragma unroll
      for (int i = 0; i < kRowsPerThread; ++i)
        v[i] = ok[i] ? *reinterpret_cast<const uint4 *>(tab_s + off[i]) : make_uint4(0, 0, 0, 0);
#pragma unroll
      for (int i = 0; i < kRowsPerThread; ++i) *reinterpret_cast<uint4 *>(tile + tc::sw_k(r0 + kRowStep * i, c)) = v[i];
    } else {
#pragma unroll
      for (int i = 0; i < kRowsPerThread; ++i) {
        uint8_t *dst = tile + tc::sw_k(r0 + kRowStep * i, c);
        if (ok[i])
          asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(tc::sa(dst)), "l"(tab_g + off[i]));
        else
          zero16(dst);
      }
    }
  }
};

__device__ __forceinline__ EmbGather emb_gather(const uint8_t *meta, const MetaLayout &ml, const Dims &D,
                                                const void *tab_g, bool in_smem, int eb) {
  EmbGather g;
  g.tab_s = in_smem ? meta + ml.tab_off() : nullptr;
  g.tab_g = reinterpret_cast<const uint8_t *>(tab_g);
  g.tk = reinterpret_cast<const uint16_t *>(meta + ml.tok_off());
  g.E = D.E, g.t = D.t, g.K1 = D.K1(), g.eb = eb;
  g.c = threadIdx.x & 7;
  const long long *tpv = reinterpret_cast<const long long *>(meta);
  const int r0 = threadIdx.x >> 3;
#pragma unroll
  for (int i = 0; i < kRowsPerThread; ++i) {
    const int r = r0 + kRowStep * i;
    g.tokrow[i] = tpv[r] >= 0 ? r * D.t : -1;
  }
  return g;
}

// z < G: dynamic model of group z; z >= G: static model on group z - G's rows
struct TwoModels : TBase {
  __device__ bool stat(int z) const { return z >= p.G; }
  __device__ int grp(int z) const { return stat(z) ? z - p.G : z; }
  __device__ Dims d(int z) const { return stat(z) ? p.st : p.dm; }
  __device__ const bf16 *w(int z) const { return stat(z) ? p.static_bf : wb(grp(z)); }
  __device__ const float *w32(int z) const { return stat(z) ? p.static_params : p.params + (size_t)grp(z) * p.P; }
  __device__ bool active(int z) const { return group_trains(p, T, grp(z)); }
};

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
  __device__ MetaLayout lay(int z) const {
    MetaLayout l = ml;
    l.t = d(z).t;
    l.table = table[stat(z)] ? d(z).A * d(z).E * 2 : 0;
    return l;
  }
  __device__ void prepare(uint8_t *meta, int z, int m0) const {
    const Dims D = d(z);
    fill(meta, lay(z), grp(z), m0, tc::kRows, w(z) + D.off_emb(), D.A * D.E * 2);
  }
  __device__ tc::TmaOperand tma_a(int) const { return kNoTma; }
  __device__ tc::TmaOperand tma_b(int z) const { return {&w1[stat(z)], stat(z) ? 2 : 3, grp(z), 0}; }
  __device__ int row_a(int, int) const { return 0; }
  __device__ int row_b(int, int n0) const { return n0; }
  __device__ EmbGather gather_ctx(const uint8_t *meta, int z, int, int) const {
    const Dims D = d(z);
    return emb_gather(meta, lay(z), D, w(z) + D.off_emb(), table[stat(z)] != 0, 2);
  }
  struct Epi {
    const long long *tp;
    const float *b1;
    bf16 *out;  // row 0 of the group
    int H;
    __device__ void epilogue(int m, int rl, int n, const float *v) const {
      if (tp[rl] < 0) return;
      float x[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) x[j] = fmaxf(v[j] + b1[n + j], 0.f);
      *reinterpret_cast<uint4 *>(out + (size_t)m * H + n) = pack8(x);
    }
  };
  __device__ Epi epi_ctx(const uint8_t *meta, int z, int, int) const {
    const Dims D = d(z);
    return {tp(meta), w32(z) + D.off_b1(), (stat(z) ? p.hs_b : p.hd_b) + (size_t)row(grp(z), 0) * D.H, D.H};
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
  struct Epi {
    const long long *tp;
    const float *b2;
    float *out;
    int A;
    int lo, hi;  // the columns the mixer reads for this thread's row (the coded slice)
    __device__ void epilogue(int m, int rl, int n, const float *v) const {
      if (tp[rl] < 0 || n + 8 <= lo || n >= hi) return;
      float x[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) x[j] = v[j] + b2[n + j];
      store8(out + (size_t)m * A + n, x);
    }
  };
  __device__ Epi epi_ctx(const uint8_t *meta, int z, int, int) const {
    const Dims D = d(z);
    Epi e{tp(meta), w32(z) + D.off_b2(), (stat(z) ? p.zu : p.zm) + (size_t)row(grp(z), 0) * D.A, D.A, 0, 0};
    const long long t = e.tp[epi_row()];
    if (t >= 0) logit_cols(t, D.A, e.lo, e.hi);
    return e;
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
  struct Epi {
    const long long *tp;
    const bf16 *h;
    bf16 *dh;
    int H;
    __device__ void epilogue(int m, int rl, int n, const float *v) const {
      const size_t i = (size_t)m * H + n;
      const bool ok = tp[rl] >= 0;  // zeros where nothing is predicted
      const uint4 hw = *reinterpret_cast<const uint4 *>(h + i);
      const bf16 *hv = reinterpret_cast<const bf16 *>(&hw);
      float x[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) x[j] = (ok && __bfloat162float(hv[j]) > 0.f) ? v[j] : 0.f;
      *reinterpret_cast<uint4 *>(dh + i) = pack8(x);
    }
  };
  __device__ Epi epi_ctx(const uint8_t *meta, int z, int, int) const {
    const size_t r0 = (size_t)row(z, 0) * p.dm.H;
    return {tp(meta), p.hd_b + r0, p.dh_b + r0, p.dm.H};
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
  struct Epi {
    float *g;  // the group's dW2
    int A;
    __device__ void epilogue(int h_, int, int n, const float *v) const { store8(g + (size_t)h_ * A + n, v); }
  };
  __device__ Epi epi_ctx(const uint8_t *, int z, int, int) const {
    return {p.grad + (size_t)z * p.P + p.dm.off_w2(), p.dm.A};
  }
};

// dX = dh W1^T scattered into the embedding rows as fixed-point integers (order-free sums, so the
// result does not depend on scheduling): A = dh by TMA (K-major), B = W1t[h][i] as N = i, K = h
// by TMA (MN-major).  The lanes of a warp add consecutive elements of one embedding row.  Where
// the group's fixed-point table fits in shared memory, the CTA first sums its tile there and then
// adds each non-zero entry to global memory once, so a token that appears at several (lane,
// position) pairs of the tile costs one global atomic per element instead of one per pair.  In
// shared memory a 64-bit value q is held as a 22-bit low part (q mod 2^22, unsigned) and a 32-bit
// high part (q >> 22, signed), each summed by a fire-and-forget 32-bit atomic add: an address
// receives at most 128 rows x 8 positions = 1024 adds per tile, so the low sum stays below 2^32,
// and the high sum is exact (modulo 2^32) for tile sums below 2^13 in magnitude; the two
// recombine as high * 2^22 + low.
struct DXT : TBase {
  static constexpr bool kAMN = false, kBMN = true, kTail = false;
  static constexpr int kEpi = 1;
  static constexpr int kGather = 0;
  static constexpr bool kFinish = true;
  CUtensorMap dh, w1;
  int eshift;  // log2 E when E is a power of two, else -1
  __device__ bool active(int z) const { return group_trains(p, T, z); }
  __device__ int M(int z) const { return nrows(z); }
  __device__ int N(int) const { return p.dm.K1(); }
  __device__ int K(int) const { return p.dm.H; }
  // the tile's sums (ml.table bytes: low parts [A*E] then high parts [A*E])
  __device__ uint32_t *lo_s(const uint8_t *meta) const {
    return reinterpret_cast<uint32_t *>(const_cast<uint8_t *>(meta) + ml.tab_off());
  }
  __device__ void prepare(uint8_t *meta, int z, int m0) const {
    MetaLayout l = ml;
    l.table = 0;  // the accumulator region is not an embedding copy
    fill(meta, l, z, m0, tc::kRows, nullptr, 0);
    uint4 *a = reinterpret_cast<uint4 *>(lo_s(meta));
    const int n4 = p.dm.A * p.dm.E / 2;
    for (int i = threadIdx.x; i < n4; i += tc::kThreads) a[i] = make_uint4(0, 0, 0, 0);
  }
  __device__ tc::TmaOperand tma_a(int) const { return {&dh, 2, 0, 0}; }
  __device__ tc::TmaOperand tma_b(int z) const { return {&w1, 3, z, 0}; }
  __device__ int row_a(int z, int m0) const { return row(z, m0); }
  __device__ int row_b(int, int n0) const { return n0; }
  struct Epi {
    const long long *tp;
    const uint16_t *tk;
    uint32_t *lo;  // shared-memory sums
    int E, t, AE, eshift;
    __device__ bool row_active(int rl) const { return tp[rl] >= 0; }
    // fixed point v 2^40 as (low 22 bits, the rest)
    __device__ uint2 stage(float v) const { return fix40_split22(v); }
    // table entry of column n of tile row rl: its context token's row, embedding offset
    __device__ uint32_t index(int rl, int n) const {
      const int pos = eshift >= 0 ? n >> eshift : n / E;
      return (uint32_t)tk[rl * t + pos] * (uint32_t)E + (uint32_t)(n - pos * E);
    }
    __device__ void add(uint32_t i, uint2 s) const {
      if (s.x) atomicAdd(lo + i, s.x);  // results unused: reductions, no return
      if (s.y) atomicAdd(reinterpret_cast<int *>(lo) + AE + i, (int)s.y);
    }
  };
  __device__ Epi epi_ctx(const uint8_t *meta, int, int, int) const {
    return {tp(meta), tk(meta), lo_s(meta), p.dm.E, p.dm.t, p.dm.A * p.dm.E, eshift};
  }
  // every thread, after the epilogue's last barrier: the non-zero sums of the tile to global memory
  __device__ void finish(uint8_t *meta, int z) const {
    const int AE = p.dm.A * p.dm.E;
    const uint32_t *lo = lo_s(meta);
    const int *hi = reinterpret_cast<const int *>(lo) + AE;
    unsigned long long *dst = reinterpret_cast<unsigned long long *>(p.demb_acc) + (size_t)z * AE;
    for (int i = threadIdx.x; i < AE; i += tc::kThreads) {
      const long long q = (long long)hi[i] * (1ll << 22) + (long long)lo[i];
      if (q) atomicAdd(dst + i, (unsigned long long)q);
    }
  }
};

// dX = dh W1^T stored per lane row (FP32, t*E columns) for groups whose embedding gradient table
// is too large to sum in shared memory; emb_grad_kernel then sums the rows into the table.  The
// tile leaves tensor memory through the stage buffers 64 columns at a time and each warp writes
// whole 256-byte row segments.
struct DXRowsT : TBase {
  static constexpr bool kAMN = false, kBMN = true, kTail = false;
  static constexpr int kEpi = 2;
  static constexpr int kGather = 0;
  CUtensorMap dh, w1;
  __device__ bool active(int z) const { return group_trains(p, T, z); }
  __device__ int M(int z) const { return nrows(z); }
  __device__ int N(int) const { return p.dm.K1(); }
  __device__ int K(int) const { return p.dm.H; }
  __device__ void prepare(uint8_t *meta, int z, int m0) const { fill(meta, ml, z, m0, tc::kRows, nullptr, 0); }
  __device__ tc::TmaOperand tma_a(int) const { return {&dh, 2, 0, 0}; }
  __device__ tc::TmaOperand tma_b(int z) const { return {&w1, 3, z, 0}; }
  __device__ int row_a(int z, int m0) const { return row(z, m0); }
  __device__ int row_b(int, int n0) const { return n0; }
  struct Epi {
    const long long *tp;
    float *out;  // row m0 of the tile, column n0
    int K1;
    __device__ void chunk(const float *stg, int c0) const {
      const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
      for (int r = warp; r < tc::kRows; r += tc::kThreads / 32) {
        if (tp[r] < 0) continue;  // rows that predict nothing are never read
        const float2 v = *reinterpret_cast<const float2 *>(stg + r * tc::kFloatPitch + 2 * lane);
        *reinterpret_cast<float2 *>(out + (size_t)r * K1 + c0 + 2 * lane) = v;
      }
    }
  };
  __device__ Epi epi_ctx(const uint8_t *meta, int z, int m0, int n0) const {
    return {tp(meta), p.dx_rows + (size_t)row(z, m0) * p.dm.K1() + n0, p.dm.K1()};
  }
};

// The embedding gradient of every training group from its stored dX rows, in two kernels.
// emb_bin_kernel (one CTA per group) lists the group's (row, context position) pairs of predicted
// rows by range of R table rows ("bins"): entry = pair index << 12 | token - bin R, bin offsets per
// group.  emb_grad_kernel (CTA (bin, group)) adds the E values of its bin's pairs into its R table
// rows, kept in shared memory in the 2^40 fixed point of the other dX forms as a low unsigned word
// and a high signed word whose carry is taken from the value the low word's atomic add returns:
// every add is exact modulo 2^64, so neither the order of the bin's entries nor that of the adds
// matters, and the sums equal those of the forms that add in global memory.  The sums go to the
// embedding part of the group's gradient as FP32 (one rounding), where the streaming optimiser
// reads them.
constexpr int kEmbThreads = 512;
constexpr int kEmbTableBytes = 64 * 1024;  // two CTAs per SM
constexpr int kEmbMaxBins = 256;
constexpr int kEmbPairBits = 20;           // pair index bits of an entry (token offset: the low 12)

__host__ __device__ inline int emb_range(int E) { return kEmbTableBytes / (8 * E); }

__device__ __forceinline__ void emb_add(uint32_t *lo, int *hi, int i, long long q) {
  const uint32_t ql = (uint32_t)(unsigned long long)q;
  const uint32_t old = atomicAdd(lo + i, ql);
  const int qh = (int)(q >> 32) + (old + ql < old ? 1 : 0);  // the low word's carry
  if (qh) atomicAdd(hi + i, qh);
}

__global__ void __launch_bounds__(kEmbThreads) emb_bin_kernel(Plan p, int T, int range, int nbins) {
  pdl_wait();
  pdl_trigger();
  __shared__ int cnt[kEmbMaxBins], cur[kEmbMaxBins];
  const int g = blockIdx.x;
  if (!group_trains(p, T, g)) return;  // the same for the whole CTA
  const int t = p.dm.t, r0 = p.grp_lane_off[g], rows = p.grp_lane_off[g + 1] - r0;
  const long long j = T - p.grp_start[g];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  uint32_t *out = p.emb_pairs + (size_t)r0 * t;
  for (int b = tid; b < nbins; b += kEmbThreads) cnt[b] = 0;
  __syncthreads();
  // two walks over the pairs, a warp per row, its lanes on the row's positions: count, then place
  for (int walk = 0; walk < 2; ++walk) {
    for (int r = warp; r < rows; r += kEmbThreads / 32) {
      const int rw = r0 + r;
      if (!row_pred(p, T, rw, g)) continue;  // the same for the whole warp
      const long long b0 = p.lane_tok[rw] + j - t;
      for (int pos0 = 0; pos0 < t; pos0 += 32) {
        const int pos = pos0 + lane;
        const bool in = pos < t;
        const int a = in ? p.tokens[b0 + pos] : 0, bin = in ? a / range : -1;
        const unsigned act = __ballot_sync(0xffffffffu, in);
        if (!in) continue;
        const unsigned same = __match_any_sync(act, bin);
        const int leader = __ffs(same) - 1, rank = __popc(same & ((1u << lane) - 1u));
        if (walk == 0) {
          if (lane == leader) atomicAdd(&cnt[bin], __popc(same));
        } else {
          int slot = 0;
          if (lane == leader) slot = atomicAdd(&cur[bin], __popc(same));
          slot = __shfl_sync(same, slot, leader) + rank;
          out[slot] = ((uint32_t)(r * t + pos) << 12) | (uint32_t)(a - bin * range);
        }
      }
    }
    __syncthreads();
    if (walk == 0 && tid == 0) {  // bin offsets within the group's entries
      int* off = p.emb_bin_off + (size_t)g * (nbins + 1);
      int o = 0;
      for (int b = 0; b < nbins; ++b) off[b] = o, cur[b] = o, o += cnt[b];
      off[nbins] = o;
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kEmbThreads, 2) emb_grad_kernel(Plan p, int T, int range, int nbins) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ __align__(16) uint8_t emb_smem[];
  const int g = blockIdx.y;
  if (!group_trains(p, T, g)) return;  // the same for the whole CTA
  const int E = p.dm.E, t = p.dm.t, K1 = t * E;
  const int a0 = blockIdx.x * range, na = min(range, p.dm.A - a0);
  if (na <= 0) return;
  const int tid = threadIdx.x, n = na * E, cpp = E >> 3;  // 8-value chunks per pair
  uint32_t *lo = reinterpret_cast<uint32_t *>(emb_smem);
  int *hi = reinterpret_cast<int *>(lo + n);
  for (int i = tid; i < n; i += kEmbThreads) lo[i] = 0u, hi[i] = 0;
  const int r0 = p.grp_lane_off[g];
  const int *off = p.emb_bin_off + (size_t)g * (nbins + 1);
  const int e0 = off[blockIdx.x], items = (off[blockIdx.x + 1] - e0) * cpp;
  const uint32_t *ent = p.emb_pairs + (size_t)r0 * t + e0;
  const float *dx = p.dx_rows + (size_t)r0 * K1;
  __syncthreads();
  for (int it0 = 0; it0 < items; it0 += 2 * kEmbThreads) {
    float x[2][8];
    int dst[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {  // both items' loads before any add
      const int it = it0 + u * kEmbThreads + tid;
      dst[u] = -1;
      if (it < items) {
        const int m = it / cpp, c = it - m * cpp;
        const uint32_t en = ent[m];
        const int i = (int)(en >> 12), r = i / t;
        const float4 *src = reinterpret_cast<const float4 *>(dx + (size_t)r * K1 + (i - r * t) * E + 8 * c);
        const float4 v0 = src[0], v1 = src[1];
        x[u][0] = v0.x, x[u][1] = v0.y, x[u][2] = v0.z, x[u][3] = v0.w;
        x[u][4] = v1.x, x[u][5] = v1.y, x[u][6] = v1.z, x[u][7] = v1.w;
        dst[u] = (int)(en & 0xFFFu) * E + 8 * c;
      }
    }
#pragma unroll
    for (int u = 0; u < 2; ++u)
      if (dst[u] >= 0)
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const long long v = fix40(x[u][q]);
          if (v) emb_add(lo, hi, dst[u] + q, v);
        }
  }
  __syncthreads();
  float *gr = p.grad + (size_t)g * p.P + p.dm.off_emb() + (size_t)a0 * E;
  for (int i = tid; i < n; i += kEmbThreads)
    gr[i] = unfix40((long long)(((unsigned long long)(uint32_t)hi[i] << 32) | lo[i]));
}

// dX = dh W1^T summed into the embedding rows without atomics (groups whose table A x E fits in
// 32 KB of FP32 and E divides 64): the tile is staged out of tensor memory 64 columns at a time
// and warp w owns the table rows of the tokens a with a % 8 == w; each warp walks the chunk's
// (row, position) pairs in order and adds the E values of every pair of one of its tokens to
// that token's row, lane e on element e, so every table element is summed by one lane in a
// fixed order.  The CTA's table goes to its own partial (row tile bx, column tile by) and the
// optimiser sums a group's partials in order: the result does not depend on scheduling.
struct DXOwnT : TBase {
  static constexpr bool kAMN = false, kBMN = true, kTail = false;
  static constexpr int kEpi = 2;
  static constexpr int kGather = 0;
  static constexpr bool kFinish = true;
  CUtensorMap dh, w1;
  int qshift;  // log2 of the positions per 64-column chunk (64 / E)
  __device__ bool active(int z) const { return group_trains(p, T, z); }
  __device__ int M(int z) const { return nrows(z); }
  __device__ int N(int) const { return p.dm.K1(); }
  __device__ int K(int) const { return p.dm.H; }
  __device__ float *tab(const uint8_t *meta) const {
    return reinterpret_cast<float *>(const_cast<uint8_t *>(meta) + ml.tab_off());
  }
  __device__ void prepare(uint8_t *meta, int z, int m0) const {
    MetaLayout l = ml;
    l.table = 0;  // the table region is not an embedding copy
    fill(meta, l, z, m0, tc::kRows, nullptr, 0);
    float4 *t4 = reinterpret_cast<float4 *>(tab(meta));
    const int n4 = p.dm.A * p.dm.E / 4;
    for (int i = threadIdx.x; i < n4; i += tc::kThreads) t4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  __device__ tc::TmaOperand tma_a(int) const { return {&dh, 2, 0, 0}; }
  __device__ tc::TmaOperand tma_b(int z) const { return {&w1, 3, z, 0}; }
  __device__ int row_a(int z, int m0) const { return row(z, m0); }
  __device__ int row_b(int, int n0) const { return n0; }
  struct Epi {
    const long long *tp;
    const uint16_t *tk;
    float *tab;
    int E, t, n0, qshift;
    __device__ void chunk(const float *stg, int c0) const {
      const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
      const int p0 = (n0 + c0) / E, q = 1 << qshift, npairs = tc::kRows << qshift;
      for (int i0 = 0; i0 < npairs; i0 += 32) {
        const int i = i0 + lane, r = i >> qshift, ps = p0 + (i & (q - 1));
        int tok = -1;
        if (i < npairs && ps < t && tp[r] >= 0) tok = tk[r * t + ps];
        unsigned mine = __ballot_sync(0xffffffffu, tok >= 0 && (tok & 7) == warp);
        // matches four at a time, in pair order: every load of the batch first, a token met twice
        // in the batch chained in registers (same order as one at a time), one store per token
        while (mine) {
          int tb[4];
          const float *src[4];
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            tb[k] = -1;
            src[k] = stg;
            if (mine) {
              const int b = __ffs(mine) - 1;
              mine &= mine - 1;
              tb[k] = __shfl_sync(0xffffffffu, tok, b);
              const int ib = i0 + b;
              src[k] = stg + (ib >> qshift) * tc::kFloatPitch + (ib & (q - 1)) * E;
            }
          }
          for (int e = lane; e < E; e += 32) {
            float v[4], d[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              v[k] = tb[k] >= 0 ? src[k][e] : 0.f;
              d[k] = tb[k] >= 0 ? tab[tb[k] * E + e] : 0.f;
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              if (tb[k] < 0) continue;
              bool first = true;  // the batch's first match of this token carries the running sum
#pragma unroll
              for (int j = 0; j < k; ++j)
                if (tb[j] == tb[k]) first = false;
              if (!first) continue;
              float acc = d[k] + v[k];
#pragma unroll
              for (int j = k + 1; j < 4; ++j)
                if (tb[j] == tb[k]) acc += v[j];
              tab[tb[k] * E + e] = acc;
            }
          }
        }
      }
    }
  };
  __device__ Epi epi_ctx(const uint8_t *meta, int, int, int n0) const {
    return {tp(meta), tk(meta), tab(meta), p.dm.E, p.dm.t, n0, qshift};
  }
  // every thread, after the last chunk's barrier: the CTA's table to its partial
  __device__ void finish(uint8_t *meta, int z) const {
    const int AE = p.dm.A * p.dm.E;
    const float4 *src = reinterpret_cast<const float4 *>(tab(meta));
    float4 *dst = reinterpret_cast<float4 *>(p.demb_part + ((size_t)z * p.dx_np + blockIdx.x * p.dx_ct + blockIdx.y) * AE);
    for (int i = threadIdx.x; i < AE / 4; i += tc::kThreads) dst[i] = src[i];
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
  // The MN-major X tile of K block k0: chunk idx = 16 bytes at column n = 8 (idx % cpr) of lane
  // row idx / cpr (cpr = R / 8 chunks per K row).  Where cpr divides the thread count a thread
  // keeps one column n (one context position and embedding offset) and steps over lane rows;
  // otherwise (general) every chunk computes its own column.
  struct Gather {
    const bf16 *tab_s, *tab_g;
    const uint16_t *tk;
    const long long *tp;
    int K, t, E, pos, e, n, kfirst, kstep, nper;
    int general, cpr, n0;
    __device__ void gather(uint8_t *tile, int k0) const {
      if (general) {
        const int total = cpr * tc::kBK;
        for (int i0 = 0; i0 < total; i0 += 4 * tc::kThreads) {
          int off[4], dsto[4];
          bool ok[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int idx = i0 + j * tc::kThreads + threadIdx.x;
            const int nn = (idx % cpr) * 8, k = idx / cpr, m = k0 + k;
            dsto[j] = idx < total ? (int)tc::sw_mn(nn, k) : -1;
            ok[j] = idx < total && m < K && tp[m] >= 0;
            const int i = n0 + nn, ps = i / E;
            off[j] = ok[j] ? (int)tk[m * t + ps] * E + (i - ps * E) : 0;
          }
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            if (dsto[j] < 0) continue;
            uint8_t *dst = tile + dsto[j];
            if (!ok[j])
              zero16(dst);
            else if (tab_s)
              *reinterpret_cast<uint4 *>(dst) = *reinterpret_cast<const uint4 *>(tab_s + off[j]);
            else
              asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(tc::sa(dst)), "l"(tab_g + off[j]));
          }
        }
        return;
      }
      for (int j0 = 0; j0 < nper; j0 += 4) {
        int off[4], kk[4];
        bool ok[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          kk[j] = kfirst + (j0 + j) * kstep;
          const int m = k0 + kk[j];
          ok[j] = j0 + j < nper && m < K && tp[m] >= 0;
          off[j] = ok[j] ? (int)tk[m * t + pos] * E + e : 0;
        }
        if (tab_s) {
          uint4 v[4];
#pragma unroll
          for (int j = 0; j < 4; ++j)
            v[j] = ok[j] ? *reinterpret_cast<const uint4 *>(tab_s + off[j]) : make_uint4(0, 0, 0, 0);
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if (j0 + j < nper) *reinterpret_cast<uint4 *>(tile + tc::sw_mn(n, kk[j])) = v[j];
        } else {
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            if (j0 + j >= nper) continue;
            uint8_t *dst = tile + tc::sw_mn(n, kk[j]);
            if (ok[j])
              asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(tc::sa(dst)), "l"(tab_g + off[j]));
            else
              zero16(dst);
          }
        }
      }
    }
  };
  __device__ Gather gather_ctx(const uint8_t *meta, int z, int n0, int R) const {
    Gather g;
    g.tab_s = table ? reinterpret_cast<const bf16 *>(meta + ml.tab_off()) : nullptr;
    g.tab_g = wb(z) + p.dm.off_emb();
    g.tk = tk(meta);
    g.tp = tp(meta);
    g.K = npred(z), g.t = p.dm.t, g.E = p.dm.E;
    const int cpr = R / 8;
    g.general = tc::kThreads % cpr != 0;
    g.cpr = cpr, g.n0 = n0;
    g.n = (threadIdx.x % cpr) * 8;
    g.pos = (n0 + g.n) / g.E, g.e = n0 + g.n - g.pos * g.E;
    g.kfirst = threadIdx.x / cpr;
    g.kstep = tc::kThreads / cpr;
    g.nper = tc::kBK / g.kstep;
    return g;
  }
  struct Epi {
    float *g;  // the group's dW1t
    int K1;
    __device__ void epilogue(int h_, int, int n, const float *v) const { store8(g + (size_t)h_ * K1 + n, v); }
  };
  __device__ Epi epi_ctx(const uint8_t *, int z, int, int) const {
    return {p.grad + (size_t)z * p.P + p.dm.off_w1(), p.dm.K1()};
  }
};

// ---- Adam in the epilogue of a weight-gradient GEMM (p.fused_w) ----
// The 64-column chunks of the tile's FP32 gradient are staged in shared memory (kEpi 2); the whole
// CTA then streams the chunk's master weights and moments with 16-byte accesses (16 threads per
// row of the matrix, so a warp touches two 256-byte row segments), every load of a batch of four
// float4 groups issued before its first store, applies the optimiser rule of the streaming
// optimiser (adam_n, explicitly rounded: the same bits) and rewrites w, m, v and the BF16 copy.
// The gradient of W1 and W2 never reaches global memory.  Every element of the matrix belongs to
// exactly one tile, so each parameter is updated once per step.
struct AdamEpi {
  float *w, *m, *v;  // element (0, 0) of the group's matrix in each array (row pitch ld)
  bf16 *wb;
  int ld, rows, cols, m0, n0;
  float lr, bc1, bc2;
  bool adam;
  __device__ void chunk(const float *stg, int c0) const {
    constexpr int kPer = tc::kRows * 16 / tc::kThreads;  // float4 groups of the chunk per thread
    constexpr int kBatch = 4;
#pragma unroll 1
    for (int b = 0; b < kPer; b += kBatch) {
      float t[kBatch][4], mm[kBatch][4], vv[kBatch][4], g[kBatch][4];
      size_t idx[kBatch];
      bool ok[kBatch];
#pragma unroll
      for (int q = 0; q < kBatch; ++q) {
        const int f = threadIdx.x + (b + q) * tc::kThreads, r = f >> 4, c4 = (f & 15) * 4;
        const int row = m0 + r, col = n0 + c0 + c4;
        ok[q] = row < rows && col < cols;  // cols is a multiple of 64: a float4 is all in or all out
        idx[q] = ok[q] ? (size_t)row * ld + col : 0;
        if (ok[q]) {
          const float4 a = *reinterpret_cast<const float4 *>(w + idx[q]);
          t[q][0] = a.x, t[q][1] = a.y, t[q][2] = a.z, t[q][3] = a.w;
          if (adam) {
            const float4 b4 = *reinterpret_cast<const float4 *>(m + idx[q]);
            const float4 c = *reinterpret_cast<const float4 *>(v + idx[q]);
            mm[q][0] = b4.x, mm[q][1] = b4.y, mm[q][2] = b4.z, mm[q][3] = b4.w;
            vv[q][0] = c.x, vv[q][1] = c.y, vv[q][2] = c.z, vv[q][3] = c.w;
          }
          const float4 gs = *reinterpret_cast<const float4 *>(stg + r * tc::kFloatPitch + c4);
          g[q][0] = gs.x, g[q][1] = gs.y, g[q][2] = gs.z, g[q][3] = gs.w;
        }
      }
#pragma unroll
      for (int q = 0; q < kBatch; ++q) {
        if (!ok[q]) continue;
        adam_n<4>(t[q], mm[q], vv[q], g[q], lr, bc1, bc2, adam);
        *reinterpret_cast<float4 *>(w + idx[q]) = make_float4(t[q][0], t[q][1], t[q][2], t[q][3]);
        if (adam) {
          *reinterpret_cast<float4 *>(m + idx[q]) = make_float4(mm[q][0], mm[q][1], mm[q][2], mm[q][3]);
          *reinterpret_cast<float4 *>(v + idx[q]) = make_float4(vv[q][0], vv[q][1], vv[q][2], vv[q][3]);
        }
        __nv_bfloat162 lo = __floats2bfloat162_rn(t[q][0], t[q][1]), hi = __floats2bfloat162_rn(t[q][2], t[q][3]);
        *reinterpret_cast<uint2 *>(wb + idx[q]) =
            make_uint2(*reinterpret_cast<uint32_t *>(&lo), *reinterpret_cast<uint32_t *>(&hi));
      }
    }
  }
};

__device__ __forceinline__ AdamEpi adam_epi(const Plan &p, int T, int g, size_t off, int rows, int cols, int m0,
                                            int n0) {
  const int tau = group_tau(p, T, g);
  const size_t base = (size_t)g * p.P + off;
  return {p.params + base, p.m + base, p.v + base, p.wbf + base, cols, rows, cols, m0, n0,
          p.lr, p.bc1[tau], p.bc2[tau], p.optimizer == PMKLC_ADAM};
}

// dW2 with the update of W2 in its epilogue
struct DW2F : DW2T {
  static constexpr int kEpi = 2;
  __device__ AdamEpi epi_ctx(const uint8_t *, int z, int m0, int n0) const {
    return adam_epi(p, T, z, p.dm.off_w2(), p.dm.H, p.dm.A, m0, n0);
  }
};

// dW1 with the update of W1 (stored transposed, W1t[h][i]) in its epilogue
struct DW1F : DW1T {
  static constexpr int kEpi = 2;
  __device__ AdamEpi epi_ctx(const uint8_t *, int z, int m0, int n0) const {
    return adam_epi(p, T, z, p.dm.off_w1(), p.dm.H, p.dm.K1(), m0, n0);
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
  __device__ MetaLayout lay() const {
    MetaLayout l = ml;
    l.table = table ? p.st.A * p.st.E : 0;
    return l;
  }
  __device__ void prepare(uint8_t *meta, int z, int m0) const {
    fill(meta, lay(), z, m0, tc::kRows, p.st8, p.st.A * p.st.E);
  }
  __device__ tc::TmaOperand tma_a(int) const { return kNoTma; }
  __device__ tc::TmaOperand tma_b(int) const { return {&w1, 2, 0, 0}; }
  __device__ int row_a(int, int) const { return 0; }
  __device__ int row_b(int, int n0) const { return n0; }
  __device__ EmbGather gather_ctx(const uint8_t *meta, int, int, int) const {
    return emb_gather(meta, lay(), p.st, p.st8, table != 0, 1);
  }
  struct Epi {
    const long long *tp;
    const float *c1, *b1;
    float *hs;       // row 0 of the group (FP32 h for the E4M3 logits layer)
    unsigned *rmax;  // row 0 of the group
    bf16 *hb;        // row 0 of the group (BF16 h for the BF16 logits layer), else nullptr
    int H;
    __device__ void epilogue(int m, int rl, int n, const float *v) const {
      if (tp[rl] < 0) return;
      float x[8], mx = 0.f;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const float a = fmaf(v[j], c1[n + j], b1[n + j]);
        x[j] = a > 0.f ? a : 0.f;  // +0 below zero (its bits must order as a float)
        mx = fmaxf(mx, x[j]);
      }
      if (hb) {
        *reinterpret_cast<uint4 *>(hb + (size_t)m * H + n) = pack8(x);
        return;
      }
      store8(hs + (size_t)m * H + n, x);
      atomicMax(rmax + m, __float_as_uint(mx));
    }
  };
  __device__ Epi epi_ctx(const uint8_t *meta, int z, int, int) const {
    const int r0 = row(z, 0);
    if (p.precision == PMKLC_BF16_FP8HIDDEN)
      return {tp(meta), p.st8_c1, p.static_params + p.st.off_b1(), nullptr, nullptr,
              p.hs_b + (size_t)r0 * p.st.H, p.st.H};
    return {tp(meta), p.st8_c1, p.static_params + p.st.off_b1(), p.hs + (size_t)r0 * p.st.H, p.hs_rowmax + r0,
            nullptr, p.st.H};
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
    const int L = nrows(z), r0 = row(z, m0);
    const unsigned *rmax = p.hs_rowmax;
    for (int i = threadIdx.x; i < tc::kRows; i += tc::kThreads) {
      const float mx = m0 + i < L ? __uint_as_float(rmax[r0 + i]) : 0.f;
      r[2 * i] = mx > 0.f ? __fdiv_rn(mx, 448.f) : 1.f;
      r[2 * i + 1] = mx > 0.f ? __fdiv_rn(448.f, mx) : 0.f;
    }
  }
  __device__ tc::TmaOperand tma_a(int) const { return kNoTma; }
  __device__ tc::TmaOperand tma_b(int) const { return {&w2, 2, 0, 0}; }
  __device__ int row_a(int, int) const { return 0; }
  __device__ int row_b(int, int n0) const { return n0; }
  // thread: 16-byte chunk c = tid % 8 (16 activations) of rows tid / 8 + 32 i
  struct Gather {
    const float *src[kRowsPerThread];  // the row's FP32 activations, nullptr for rows that predict nothing
    float inv[kRowsPerThread];
    int H, c;
    __device__ void gather(uint8_t *tile, int k0) const {
      const int k = k0 + 16 * c, r0 = threadIdx.x >> 3;
#pragma unroll
      for (int i = 0; i < kRowsPerThread; ++i) {
        uint4 out = make_uint4(0, 0, 0, 0);
        if (k < H && src[i]) {  // H % 16 == 0: a chunk is all in or all out
          const float4 *s4 = reinterpret_cast<const float4 *>(src[i] + k);
          uint32_t w[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const float4 f = s4[q];
            const __nv_fp8x4_e4m3 x(make_float4(f.x * inv[i], f.y * inv[i], f.z * inv[i], f.w * inv[i]));
            w[q] = *reinterpret_cast<const uint32_t *>(&x);
          }
          out = make_uint4(w[0], w[1], w[2], w[3]);
        }
        *reinterpret_cast<uint4 *>(tile + tc::sw_k(r0 + kRowStep * i, c)) = out;
      }
    }
  };
  __device__ Gather gather_ctx(const uint8_t *meta, int z, int m0, int) const {
    Gather g;
    g.H = p.st.H, g.c = threadIdx.x & 7;
    const long long *tpv = tp(meta);
    const float *r = rs(meta);
    const int r0 = threadIdx.x >> 3;
#pragma unroll
    for (int i = 0; i < kRowsPerThread; ++i) {
      const int rl = r0 + kRowStep * i;
      g.src[i] = tpv[rl] >= 0 ? p.hs + (size_t)row(z, m0 + rl) * g.H : nullptr;
      g.inv[i] = r[2 * rl + 1];
    }
    return g;
  }
  struct Epi {
    const long long *tp;
    const float *rs, *s2, *b2;
    float *zu;  // row 0 of the group
    int A;
    int lo, hi;  // the columns the mixer reads for this thread's row (the coded slice)
    __device__ void epilogue(int m, int rl, int n, const float *v) const {
      if (tp[rl] < 0 || n + 8 <= lo || n >= hi) return;
      const float sr = rs[2 * rl];
      float x[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) x[j] = fmaf(v[j], __fmul_rn(sr, s2[n + j]), b2[n + j]);
      store8(zu + (size_t)m * A + n, x);
    }
  };
  __device__ Epi epi_ctx(const uint8_t *meta, int z, int, int) const {
    Epi e{tp(meta), rs(meta), p.st8_s2, p.static_params + p.st.off_b2(), p.zu + (size_t)row(z, 0) * p.st.A,
          p.st.A, 0, 0};
    const long long t = e.tp[epi_row()];
    if (t >= 0) logit_cols(t, p.st.A, e.lo, e.hi);
    return e;
  }
};

// db1 = sum of dh, db2 = sum of dz over the predicted rows of each group (the predicted lanes are
// a prefix of the group's lanes).  Block: 16 chunks of 8 columns x 16 row slices; slice y adds
// rows y, y + 16, ... in order (16-byte loads), then slice 0 adds the 16 partial sums in order,
// so the result does not depend on scheduling.
constexpr int kBiasChunks = 16, kBiasSlices = 16;
__global__ void __launch_bounds__(kBiasChunks * kBiasSlices) bias_grad_kernel(Plan p, int T) {
  pdl_wait();
  pdl_trigger();
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
  tc::TilePlan t_h, t_l, t_dh, t_w2, t_dx, t_w1, t_h8, t_l8, t_w2f, t_w1f;
  int tile_cap = 0;
  MetaLayout ml_h, ml_l, ml_dh, ml_w2, ml_dx, ml_w1, ml_h8, ml_l8;
  int table_h[2], table_w1, sacc_dx, table_h8, dx_owner, dx_rows, emb_range, emb_bins;
  CUtensorMap w1k[2], w1mn, w2mn[2], w2k, hk[2], dzk, dhk, hmn, dzmn, dhmn, w1_8, w2_8;
};

bool same_key(const TcSetup &a, const Plan &p) {
  auto dims_eq = [](const Dims &x, const Dims &y) { return x.A == y.A && x.E == y.E && x.t == y.t && x.H == y.H; };
  return a.wbf == p.wbf && a.static_bf == p.static_bf && a.hd_b == p.hd_b && a.hs_b == p.hs_b && a.dz_b == p.dz_b &&
         a.dh_b == p.dh_b && a.st8 == p.st8 && a.G == p.G && a.NL == p.NL && a.Mmax == p.Mmax &&
         a.use_static == p.use_static &&
         dims_eq(a.dm, p.dm) && (!p.use_static || dims_eq(a.st, p.st)) && a.P == p.P && a.tile_cap == p.tile_cap;
}

// dX by owner warps: the group's FP32 table fits in 32 KB and E divides the 64-column chunks
bool dx_owner_rule(const Plan &p) {
  const Dims &D = p.dm;
  return D.E >= 8 && 64 % D.E == 0 && (size_t)D.A * D.E * 4 <= 32 * 1024;
}
int dx_owner_nt(const Plan &p) { return p.dm.K1() >= 128 ? 128 : 64; }

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
  S.tile_cap = p.tile_cap;
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
  // a kernel variant may cap the row GEMMs' column tiles (more, narrower CTAs; the reduction over
  // K of every output element is unchanged, so the results are the same)
  auto capped = [&](tc::TilePlan t) {
    while (p.tile_cap >= 64 && t.nt > p.tile_cap && (t.nt / 2) % 64 == 0) t.nt /= 2;
    return t;
  };
  S.t_h = capped(tc::plan_tiles(p.Mmax, Hmax, K1max, Z, S.ml_h.bytes(), false));
  S.t_l = capped(tc::plan_tiles(p.Mmax, D.A, Hmax, Z, S.ml_l.bytes()));
  S.t_dh = capped(tc::plan_tiles(p.Mmax, D.H, D.A, p.G, S.ml_dh.bytes()));
  S.t_w2 = tc::plan_tiles(D.H, D.A, p.Mmax, p.G, S.ml_w2.bytes());
  S.t_dx = capped(tc::plan_tiles(p.Mmax, D.K1(), D.H, p.G, S.ml_dx.bytes()));
  if (S.sacc_dx && S.t_dx.nt > 8 * D.E) S.sacc_dx = 0;  // over 8 positions per tile the 22-bit low sums could overflow
  S.dx_owner = dx_owner_rule(p);
  S.dx_rows = !S.dx_owner && !S.sacc_dx;
  S.emb_range = S.emb_bins = 0;
  if (S.dx_owner) {  // 128-column tiles, two stage buffers: two CTAs per SM
    S.ml_dx = {tc::kRows, D.t, D.A * D.E * 4};
    S.t_dx = {dx_owner_nt(p), 2};
    if ((size_t)S.t_dx.ns * (tc::kRows + S.t_dx.nt) * tc::kRowBytes < (size_t)tc::kRows * tc::kFloatPitch * 4)
      return false;
  } else if (S.dx_rows) {  // dX rows stored, then summed per range of table rows (emb_grad_kernel)
    S.ml_dx = {tc::kRows, 0, 0};
    S.t_dx = capped(tc::plan_tiles(p.Mmax, D.K1(), D.H, p.G, S.ml_dx.bytes()));
    // the staged epilogue's 128 x kFloatPitch floats fit in the stage buffers
    while ((size_t)S.t_dx.ns * (tc::kRows + S.t_dx.nt) * tc::kRowBytes < (size_t)tc::kRows * tc::kFloatPitch * 4)
      ++S.t_dx.ns;
    if (S.t_dx.ns > tc::kStages) return false;
    S.emb_range = emb_range(D.E);
    S.emb_bins = S.emb_range > 0 ? (D.A + S.emb_range - 1) / S.emb_range : 0;
    // entries hold a pair index in 20 bits and a token offset in 12
    if (S.emb_range < 1 || S.emb_range > 4096 || S.emb_bins > kEmbMaxBins ||
        (long long)p.Mmax * D.t >= (1LL << kEmbPairBits))
      return false;
  } else {
    // the staged epilogue needs kStagedBytes of stage buffers (checked against the limit below)
    while ((size_t)S.t_dx.ns * (tc::kRows + S.t_dx.nt) * tc::kRowBytes < tc::kStagedBytes) ++S.t_dx.ns;
    if (S.t_dx.ns > tc::kStages) return false;
  }
  S.t_w1 = tc::plan_tiles(D.H, D.K1(), p.Mmax, p.G, S.ml_w1.bytes());
  // with the optimiser in their epilogues (p.fused_w) the weight-gradient GEMMs are bound by the
  // stream of optimiser state: 128-column tiles and two stage buffers (their K, the predicted lanes,
  // is a few 64-row blocks), so two CTAs share an SM and one's epilogue overlaps the other's MMAs;
  // the staged epilogue's 128 x kFloatPitch floats fit in the two buffers
  S.t_w2f = {min(128, D.A), 2};
  S.t_w1f = {min(128, D.K1()), 2};
  for (const auto &pr : {std::make_pair(S.t_h, S.ml_h.bytes()), std::make_pair(S.t_l, S.ml_l.bytes()),
                         std::make_pair(S.t_dh, S.ml_dh.bytes()), std::make_pair(S.t_w2, S.ml_w2.bytes()),
                         std::make_pair(S.t_dx, S.ml_dx.bytes()), std::make_pair(S.t_w1, S.ml_w1.bytes()),
                         std::make_pair(S.t_w2f, S.ml_w2.bytes()), std::make_pair(S.t_w1f, S.ml_w1.bytes())})
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
  // the BF16 static model, or the BF16 logits layer of the FP8-hidden form (its W1 map unused)
  if (p.use_static && (!f8 || p.precision == PMKLC_BF16_FP8HIDDEN)) {
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

int dx_partials(const Plan &p, int *ct) {
  *ct = 0;
  if (!dx_owner_rule(p) || !tc_supported(p)) return 0;
  *ct = (p.dm.K1() + dx_owner_nt(p) - 1) / dx_owner_nt(p);
  return ((p.Mmax + tc::kRows - 1) / tc::kRows) * *ct;
}

bool tc_supported(const Plan &p) {
  if (!shapes_ok(p)) return false;
  TcSetup S;
  return get_setup(p, S);
}

bool dx_rows_rule(const Plan &p) { return dx_rows_bins(p) > 0; }

int dx_rows_bins(const Plan &p) {
  if (!shapes_ok(p)) return 0;
  TcSetup S;
  return get_setup(p, S) && S.dx_rows ? S.emb_bins : 0;
}

namespace {
// The bounded-wait path of every kernel here, on its own: one thread waits, at most `polls` polls,
// on an mbarrier that expects one arrival which never comes, gives up and reports kErrTimeout in
// the error word, exactly as a GEMM whose copies never land would.
__global__ void wait_selftest_kernel(long polls, int *err) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(tc::sa(&bar)));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
  }
  __syncthreads();
  if (threadIdx.x == 0 && !tc::mbar_wait(tc::sa(&bar), 0, polls)) atomicOr(err, kErrTimeout);
}
}  // namespace

void launch_forward_tc(const Plan &p, int T, cudaStream_t st, int which) {
  TcSetup S;
  if (!get_setup(p, S)) return;
  const double R = prof_work().pred_rows;
  const bool stat = p.use_static && (which & kFwdStatic), dyn = (which & kFwdDynamic) != 0;
  const bool f8 = p.use_static && p.st8 != nullptr;  // static model on its own E4M3 launches
  const bool f8_logits = f8 && p.precision != PMKLC_BF16_FP8HIDDEN;  // its logits layer in E4M3 too
  if (stat && f8) {
    ProfScope ps("fwd_hidden_static_fp8", 2.0 * R * p.st.K1() * p.st.H, 0, st);
    HiddenF8 op;
    op.p = p, op.T = T, op.ml = S.ml_h8, op.w1 = S.w1_8, op.table = S.table_h8;
    tc::launch(op, p.Mmax, p.st.H, p.G, S.t_h8, S.ml_h8.bytes(), st);
  }
  if (stat && f8_logits) {
    ProfScope ps("fwd_logits_static_fp8", 2.0 * R * p.st.H * p.st.A, 0, st);
    LogitsF8 op;
    op.p = p, op.T = T, op.ml = S.ml_l8, op.w2 = S.w2_8;
    tc::launch(op, p.Mmax, p.st.A, p.G, S.t_l8, S.ml_l8.bytes(), st);
  }
  // BF16 problems: z < G dynamic models, z >= G the static model; one launch covers [zb, zb + Z).
  // The static hidden layer runs here in the BF16 form, its logits layer in the BF16 and the
  // FP8-hidden forms (after HiddenF8 wrote its BF16 h)
  const bool s_hid = stat && !f8 && !p.st_gru, s_log = stat && !f8_logits;
  if (stat && p.st_gru) launch_bigru_static(p, T, st);  // the BiGRU static predictor's h
  if (dyn || s_hid) {
    const int zb = dyn ? 0 : p.G, Z = (dyn ? p.G : 0) + (s_hid ? p.G : 0);
    const char *hname = dyn && s_hid ? "fwd_hidden_bf16" : dyn ? "fwd_hidden_dyn_bf16" : "fwd_hidden_static_bf16";
    double fl = (dyn ? 2.0 * R * p.dm.K1() * p.dm.H : 0.0) + (s_hid ? 2.0 * R * p.st.K1() * p.st.H : 0.0);
    ProfScope ps(hname, fl, 0, st);
    HiddenT op;
    op.p = p, op.T = T, op.ml = S.ml_h, op.w1[0] = S.w1k[0], op.w1[1] = S.w1k[1], op.zb = zb;
    op.table[0] = S.table_h[0], op.table[1] = S.table_h[1];
    tc::launch(op, p.Mmax, p.use_static ? max(p.dm.H, p.st.H) : p.dm.H, Z, S.t_h, S.ml_h.bytes(), st);
  }
  if (dyn || s_log) {
    const int zb = dyn ? 0 : p.G, Z = (dyn ? p.G : 0) + (s_log ? p.G : 0);
    const char *lname = dyn && s_log ? "fwd_logits_bf16" : dyn ? "fwd_logits_dyn_bf16" : "fwd_logits_static_bf16";
    double fl = (dyn ? 2.0 * R * p.dm.H * p.dm.A : 0.0) + (s_log ? 2.0 * R * p.st.H * p.st.A : 0.0);
    if (slice_rule(p)) {  // only each row's coded slice: bound by reading W2 (BF16)
      const double sfl = (dyn ? 2.0 * R * p.dm.H * p.ov_w : 0.0) + (s_log ? 2.0 * R * p.st.H * p.ov_w : 0.0);
      const double sb = (dyn ? prof_work().train_groups * 2.0 * p.dm.H * p.dm.A : 0.0) +
                        (s_log ? 2.0 * p.st.H * p.st.A : 0.0);
      ProfScope ps(dyn && s_log ? "fwd_logits_slice" : dyn ? "fwd_logits_slice_dyn" : "fwd_logits_slice_static", sfl,
                   sb, st);
      launch_slice_logits(p, T, st, zb, Z);
      return;
    }
    ProfScope ps(lname, fl, 0, st);
    LogitsT op;
    op.p = p, op.T = T, op.ml = S.ml_l, op.h[0] = S.hk[0], op.h[1] = S.hk[1], op.w2[0] = S.w2mn[0],
    op.w2[1] = S.w2mn[1];
    op.zb = zb;
    tc::launch(op, p.Mmax, p.dm.A, Z, S.t_l, S.ml_l.bytes(), st);
  }
}

void launch_backward_tc(const Plan &p, int T, cudaStream_t st, const StepStreams *ss) {
  TcSetup S;
  if (!get_setup(p, S)) return;
  const double R = prof_work().pred_rows;
  const Dims &D = p.dm;
  // dW2 reads only h and dz: with auxiliary streams it starts beside dh; dX and dW1 follow dh side
  // by side, and the bias sums (db1 needs dh) follow both dW2 and dh.  With the optimiser in the
  // dW epilogues (p.fused_w) W2 may change only once dh has read it and W1 once dX has: dW2 then
  // follows dh, and dW1 follows dX on dX's stream.
  cudaStream_t s1 = st, s2 = st;
  if (ss) {
    cudaEventRecord(ss->fork, st);
    cudaStreamWaitEvent(ss->aux[0], ss->fork, 0);
    s1 = ss->aux[0], s2 = ss->aux[1];
  }
  // Adam bytes of a fused update: read w, m, v, write w, m, v and the BF16 copy
  const double tg = prof_work().train_groups, adam_b = p.optimizer == PMKLC_ADAM ? 26.0 : 10.0;
  if (!p.fused_w) {
    ProfScope ps("bwd_dw2_bf16", 2.0 * R * D.A * D.H, 0, s1);
    DW2T op;
    op.p = p, op.T = T, op.ml = S.ml_w2, op.h = S.hmn, op.dz = S.dzmn;
    tc::launch(op, D.H, D.A, p.G, S.t_w2, S.ml_w2.bytes(), s1);
  }
  if (slice_rule(p)) {  // only each row's coded slice: bound by reading W2 (BF16)
    ProfScope ps("bwd_dh_slice", 2.0 * R * p.ov_w * D.H, tg * 2.0 * D.H * D.A, st);
    launch_slice_dh(p, T, st);
  } else {
    ProfScope ps("bwd_dh_bf16", 2.0 * R * D.A * D.H, 0, st);
    DhT op;
    op.p = p, op.T = T, op.ml = S.ml_dh, op.dz = S.dzk, op.w2 = S.w2k;
    tc::launch(op, p.Mmax, D.H, p.G, S.t_dh, S.ml_dh.bytes(), st);
  }
  if (ss) {
    cudaEventRecord(ss->fork, st);  // dh done
    cudaStreamWaitEvent(ss->aux[1], ss->fork, 0);
    cudaStreamWaitEvent(ss->aux[0], ss->fork, 0);
  }
  launch_pdl(bias_grad_kernel, dim3((D.H + D.A + 8 * kBiasChunks - 1) / (8 * kBiasChunks), p.G),
             dim3(kBiasChunks * kBiasSlices), 0, s1, p, T);
  if (p.fused_w) {
    ProfScope ps("bwd_dw2_adam_bf16", 2.0 * R * D.A * D.H, tg * adam_b * D.H * D.A, s1);
    DW2F op;
    op.p = p, op.T = T, op.ml = S.ml_w2, op.h = S.hmn, op.dz = S.dzmn;
    tc::launch(op, D.H, D.A, p.G, S.t_w2f, S.ml_w2.bytes(), s1);
  }
  if (S.dx_owner) {
    ProfScope ps("bwd_dx_bf16", 2.0 * R * D.K1() * D.H, 0, s2);
    DXOwnT op;
    op.p = p, op.T = T, op.ml = S.ml_dx, op.dh = S.dhk, op.w1 = S.w1mn;
    op.qshift = __builtin_ctz((unsigned)(64 / D.E));
    tc::launch(op, p.Mmax, D.K1(), p.G, S.t_dx, S.ml_dx.bytes(), s2);
  } else if (S.dx_rows) {
    {  // bytes: the context tokens read, one 4-byte entry per pair written
      ProfScope ps("bwd_emb_bin", 0, R * D.t * 6.0, s2);
      launch_pdl(emb_bin_kernel, dim3(p.G), dim3(kEmbThreads), 0, s2, p, T, S.emb_range, S.emb_bins);
    }
    {
      ProfScope ps("bwd_dx_bf16", 2.0 * R * D.K1() * D.H, 0, s2);
      DXRowsT op;
      op.p = p, op.T = T, op.ml = S.ml_dx, op.dh = S.dhk, op.w1 = S.w1mn;
      tc::launch(op, p.Mmax, D.K1(), p.G, S.t_dx, S.ml_dx.bytes(), s2);
    }
    // bytes: the predicted rows' dX read (t E FP32 each), every training group's table written
    ProfScope ps("bwd_emb_grad", 0, R * D.K1() * 4.0 + tg * D.A * D.E * 4.0, s2);
    const int smem = min(S.emb_range, D.A) * D.E * 8;
    if (smem_optin((const void *)emb_grad_kernel, smem))
      launch_pdl(emb_grad_kernel, dim3(S.emb_bins, p.G), dim3(kEmbThreads), smem, s2, p, T, S.emb_range,
                 S.emb_bins);
  } else {
    ProfScope ps("bwd_dx_bf16", 2.0 * R * D.K1() * D.H, 0, s2);
    DXT op;
    op.p = p, op.T = T, op.ml = S.ml_dx, op.dh = S.dhk, op.w1 = S.w1mn;
    op.eshift = (D.E & (D.E - 1)) == 0 ? __builtin_ctz((unsigned)D.E) : -1;
    tc::launch(op, p.Mmax, D.K1(), p.G, S.t_dx, S.ml_dx.bytes(), s2);
  }
  if (p.fused_w) {
    ProfScope ps("bwd_dw1_adam_bf16", 2.0 * R * D.K1() * D.H, tg * adam_b * D.H * D.K1(), s2);
    DW1F op;
    op.p = p, op.T = T, op.ml = S.ml_w1, op.dh = S.dhmn, op.table = S.table_w1;
    tc::launch(op, D.H, D.K1(), p.G, S.t_w1f, S.ml_w1.bytes(), s2);
  } else {
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

extern "C" int pmklc_wait_selftest(uint64_t polls, void *stream) {
  using namespace pmklc;
  if (polls == 0 || polls > (1ull << 30)) return PMKLC_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  int *d_err = nullptr;
  PMKLC_CUDA_TRY(cudaMallocAsync((void **)&d_err, sizeof(int), st));
  cudaMemsetAsync(d_err, 0, sizeof(int), st);
  wait_selftest_kernel<<<1, 32, 0, st>>>((long)polls, d_err);
  int h = 0;
  cudaMemcpyAsync(&h, d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
  cudaFreeAsync(d_err, st);
  PMKLC_CUDA_TRY(cudaGetLastError());
  PMKLC_CUDA_TRY(cudaStreamSynchronize(st));
  return (h & kErrTimeout) ? PMKLC_ETIMEOUT : PMKLC_OK;
}
