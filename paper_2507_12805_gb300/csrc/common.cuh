// Shared device-side definitions of libpmklc (sm_103a).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "pmklc.h"

namespace pmklc {

constexpr int kTotalBits = 24;             // frequency tables sum to 2^24 (the quantiser's total)
constexpr uint32_t kTotal = 1u << kTotalBits;

// K-slices of the BF16 hidden-layer GEMM (split-K; the slices are summed in a fixed order)
constexpr int kHiddenSplit = 4;

enum GroupMode : int { kEncode = 0, kDecode = 1, kReplay = 2 };

// Error word bits written by kernels (host turns them into PMKLC_E* codes).
enum ErrBits : int { kErrBadBase = 1, kErrOverflow = 2, kErrCorrupt = 4, kErrTimeout = 8 };

// Dimensions of one MLP predictor: alphabet A = 4^k, embedding E, context t, hidden H.
struct Dims {
  int A, E, t, H;
  __host__ __device__ int K1() const { return t * E; }
  __host__ __device__ size_t off_emb() const { return 0; }
  __host__ __device__ size_t off_w1() const { return (size_t)A * E; }
  __host__ __device__ size_t off_b1() const { return off_w1() + (size_t)t * E * H; }
  __host__ __device__ size_t off_w2() const { return off_b1() + H; }
  __host__ __device__ size_t off_b2() const { return off_w2() + (size_t)H * A; }
  __host__ __device__ size_t count() const { return off_b2() + A; }
};

// Per-lane range-coder states (byte-oriented range coder, 56-bit window).
struct EncState {
  unsigned long long low, range;
  uint32_t cache, pending, pos, has_cache;
};
struct DecState {
  unsigned long long code, range;
  uint32_t pos, pad;
};

// Everything the per-step kernels of one run need (device pointers + sizes).
struct Plan {
  int G;             // groups (= blocks)
  int NL;            // lanes (= rows of every per-step GEMM)
  int Mmax;          // largest number of lanes in a group
  int t_eff;         // uniform-coded prefix length per lane
  int ov_w, ov_mod;  // overlap-masked coding (s < k): slice width 4^s and 4^(k-s); 0 = whole alphabet
  int use_static;
  int optimizer;     // PMKLC_ADAM / PMKLC_SGD
  float lr;
  Dims dm, st;
  size_t P;          // dm.count()
  // schedule (per group)
  const int *grp_start, *grp_steps, *grp_lane_off, *grp_base, *grp_extra, *grp_mode, *grp_tau0;
  // lanes
  const long long *lane_tok;   // absolute token index of the lane's first token
  const int *lane_len, *lane_grp;
  uint16_t *tokens;
  // model state
  float *params, *m, *v, *grad, *alpha, *alpha_m, *alpha_v;
  const float *static_params;
  // BiGRU static predictor (§4.2.2 / §4.2.3): its FP32 parameters (nullptr: the static model is an
  // MLP), GRU width per direction and layer count, and with two layers a scratch for the first
  // layer's outputs (st.t x 2 gru_hg x NL).  Its Linear layer writes the static h (st.H = 128
  // columns); static_params then holds an MLP-layout block whose W2, b2 are the Dense layer's
  // W4, b4, so the static logits run on the MLP's logits kernels.
  const float *st_gru;
  int gru_hg, gru_layers;
  float *gru_y;
  __nv_bfloat16 *wbf;               // BF16 copy of every group's parameters (BF16 form), G x P
  const __nv_bfloat16 *static_bf;   // BF16 copy of the static parameters (BF16 form)
  // FP8 static form (PMKLC_BF16_FP8STATIC with a static model; else nullptr): E4M3 codes
  // [Emb A x E][W1t H x tE][W2t A x H], the hidden scales c1[h] = s_emb s_w1[h], the logit scales
  // s_w2[a], and per lane row the largest static hidden activation of the step (float bits,
  // raised by integer atomicMax; reset by the mixer once the logits are formed)
  const uint8_t *st8;
  const float *st8_c1, *st8_s2;
  unsigned *hs_rowmax;
  int precision;                    // PMKLC_FP32_PLAIN / PMKLC_BF16_BATCHED / PMKLC_BF16_FP8STATIC
  const float *bc1, *bc2;      // Adam bias corrections 1 - beta^tau, indexed by tau
  int tile_cap;                // 0, or the widest column tile of the row GEMMs (hidden, logits, dh, dX)
  int fused_w;                 // 1: W1 and W2 are updated in the epilogues of their gradient GEMMs
                               // (BF16 forms on the tcgen05 engine; no stored gradient for them)
  // activations (NL rows)
  float *hd, *hs, *zm, *zu, *dz, *dh, *dalpha_row, *dalpha_grp;
  float *out_P;                // optional: mixed probabilities of predicted rows (tests)
  __nv_bfloat16 *hd_b, *hs_b, *dz_b, *dh_b;  // BF16 activations of the BF16 form (else nullptr)
  float *hpart;                // split-K partial sums of the hidden layer (BF16 form, mma.sync engine)
  long long *demb_acc;         // fixed-point embedding gradient accumulators, G x A x E (else nullptr)
  // BF16 form on tcgen05 with tables too large for shared memory: dX of every lane row (NL x t*E
  // FP32), summed per group into the embedding gradient (grad's embedding part) by a kernel that
  // owns a range of table rows; nullptr otherwise
  float *dx_rows;
  uint32_t *emb_pairs;  // with dx_rows: every predicted row's (row, position) pairs by bin (NL x t)
  int *emb_bin_off;     // with dx_rows: per group, the bins' first entries and the total
  // BF16 form with small tables: per group, dx_np partial FP32 tables (A x E) of the dX tiles
  // (row tile bx, column tile by at partial bx * dx_ct + by), summed by the optimiser in that
  // order; nullptr: the fixed-point accumulators above
  float *demb_part;
  int dx_np, dx_ct;
  // coders
  EncState *enc;
  DecState *dec;
  uint8_t *lane_buf;           // encode: output bytes; decode: input bytes
  const unsigned long long *lane_buf_off;
  const uint32_t *lane_buf_cap;  // encode: capacity; decode: payload length
  int *err;
};

// The count model's per-run state (its lanes are the network's lanes).
struct CountPlan {
  int m, s, k;               // order, (s,k)
  const int *grp_cmode;      // per group: 0 off, 1 encode, 2 decode
  uint32_t *table;           // G x 4^m x 4 counts
  uint32_t *ctx;             // per lane: context (previous m bases)
  EncState *enc;
  DecState *dec;
  uint8_t *buf;              // per-lane payload bytes (output when encoding, input when decoding)
  const unsigned long long *buf_off;
  const uint32_t *buf_cap;   // capacity when encoding, payload length when decoding
};

__device__ __forceinline__ int row_local_step(const Plan &p, int T, int g) { return T - p.grp_start[g]; }

// Number of lanes of group g still live at local step j (lanes differ by at most one token).
__device__ __forceinline__ int live_lanes(const Plan &p, int g, int j) {
  int M = p.grp_lane_off[g + 1] - p.grp_lane_off[g];
  int base = p.grp_base[g];
  return j < base ? M : (j == base ? p.grp_extra[g] : 0);
}

// A lane is predicted (and trained on) at step T iff its local step j has t_eff <= j < len.
__device__ __forceinline__ bool row_pred(const Plan &p, int T, int r, int g) {
  int j = T - p.grp_start[g];
  return j >= p.t_eff && j < p.lane_len[r];
}

// Group g trains at step T iff some lane predicts: t_eff <= j < steps.
__device__ __forceinline__ bool group_trains(const Plan &p, int T, int g) {
  int j = T - p.grp_start[g];
  return j >= p.t_eff && j < p.grp_steps[g];
}

// d loss / d alpha of group g: the predicted rows' contributions, summed by one warp in a fixed
// order (each lane takes rows lane, lane+32, ... in turn, then a butterfly whose lane-0 value is
// broadcast).  All 32 lanes must call it.
__device__ __forceinline__ float alpha_grad(const Plan &p, int T, int g) {
  const int lane = threadIdx.x & 31;
  float s = 0.f;
  for (int r = p.grp_lane_off[g] + lane; r < p.grp_lane_off[g + 1]; r += 32)
    if (row_pred(p, T, r, g)) s += p.dalpha_row[r];
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return __shfl_sync(0xffffffffu, s, 0);
}

// One optimiser step of n parameters (paper §2 step 4; Adam with beta 0.9 / 0.999, eps 1e-8 and
// bias corrections bc1 = 1 - 0.9^tau, bc2 = 1 - 0.999^tau, else plain SGD), in registers.
template <int n>
__device__ __forceinline__ void adam_n(float *t, float *m, float *v, const float *g, float lr, float bc1, float bc2,
                                       bool adam) {
  // every operation rounded explicitly (no contraction left to the compiler), so each kernel that
  // applies the rule - the streaming optimiser or a gradient GEMM's epilogue - gets the same bits
#pragma unroll
  for (int e = 0; e < n; ++e) {
    if (adam) {
      m[e] = __fadd_rn(__fmul_rn(0.9f, m[e]), __fmul_rn(0.1f, g[e]));
      v[e] = __fadd_rn(__fmul_rn(0.999f, v[e]), __fmul_rn(__fmul_rn(0.001f, g[e]), g[e]));
      const float den = __fadd_rn(__fsqrt_rn(__fdiv_rn(v[e], bc2)), 1e-8f);
      t[e] = __fsub_rn(t[e], __fdiv_rn(__fmul_rn(lr, __fdiv_rn(m[e], bc1)), den));
    } else {
      t[e] = __fsub_rn(t[e], __fmul_rn(lr, g[e]));
    }
  }
}

// Update count tau of group g at global step T (1-based).
__device__ __forceinline__ int group_tau(const Plan &p, int T, int g) {
  return p.grp_tau0[g] + (T - p.grp_start[g] - p.t_eff) + 1;
}

// Fixed point scale of the embedding gradient accumulators (integer adds are order-free,
// so the sum is deterministic; resolution 2^-40, range +-2^23).
constexpr double kEmbFix = 1099511627776.0;  // 2^40

// v * 2^40 rounded to the nearest integer (ties to even), saturated to the int64 range (NaN -> 0),
// in integer arithmetic: the product is exact in binary floating point, so this equals the
// conversion of the exact product; no FP64 instruction is issued (GB300 has little FP64 rate).
__device__ __forceinline__ long long fix40(float v) {
  const uint32_t b = __float_as_uint(v);
  const int e = (int)((b >> 23) & 0xFFu);
  const bool neg = (b >> 31) != 0;
  if (e == 0xFF) return (b & 0x7FFFFFu) ? 0ll : (neg ? (long long)(1ull << 63) : (long long)((1ull << 63) - 1));
  if (e == 0) return 0ll;  // subnormal: |v| 2^40 < 2^-86
  const unsigned long long m = (unsigned long long)((b & 0x7FFFFFu) | 0x800000u);
  const int sh = e - 110;  // v 2^40 = m 2^(e - 150 + 40)
  unsigned long long q;
  if (sh >= 40) {  // |v| 2^40 >= 2^63
    return neg ? (long long)(1ull << 63) : (long long)((1ull << 63) - 1);
  } else if (sh >= 0) {
    q = m << sh;
  } else if (sh < -24) {
    q = 0;  // below one half (m < 2^24)
  } else {
    const int r = -sh;
    q = m >> r;
    const unsigned long long rem = m & ((1ull << r) - 1), half = 1ull << (r - 1);
    if (rem > half || (rem == half && (q & 1ull))) ++q;
  }
  return neg ? -(long long)q : (long long)q;
}

// The same fixed-point value q = rint(v 2^40) split as (q mod 2^22, floor(q / 2^22)), branch-free
// in FP32 on |v|: x = |v| 2^18 is exact, f = floor(x) and x - f are exact (x - f = x below 1,
// Sterbenz's lemma above), and rint((x - f) 2^22) = q - f 2^22 because f 2^22 is an even integer
// (ties to even are unaffected); a negative v negates the pair (rint is odd).  Exact for
// |v| < 2^13 (the high part then fits in 32 bits); beyond that the high part saturates.
__device__ __forceinline__ uint2 fix40_split22(float v) {
  const float x = __fmul_rn(fabsf(v), 262144.f);  // 2^18
  const float f = floorf(x);
  const float l = rintf(__fmul_rn(__fsub_rn(x, f), 4194304.f));  // in [0, 2^22]
  const bool carry = l == 4194304.f;
  const uint32_t lo = carry ? 0u : (uint32_t)l;
  const int hi = __float2int_rz(f) + (carry ? 1 : 0);
  if (!signbit(v)) return make_uint2(lo, (uint32_t)hi);
  return make_uint2(lo ? 4194304u - lo : 0u, (uint32_t)(lo ? -hi - 1 : -hi));
}

// q * 2^-40 rounded once to the nearest float (ties to even), in integer arithmetic.
__device__ __forceinline__ float unfix40(long long q) {
  if (q == 0) return 0.f;
  const bool neg = q < 0;
  unsigned long long u = neg ? 0ull - (unsigned long long)q : (unsigned long long)q;
  const int top = 63 - __clzll((long long)u);  // index of the leading one
  int sh = 0;
  if (top > 23) {
    sh = top - 23;
    const unsigned long long rem = u & ((1ull << sh) - 1), half = 1ull << (sh - 1);
    u >>= sh;
    if (rem > half || (rem == half && (u & 1ull))) ++u;  // may reach 2^24: still exact below
  }
  const float mag = __uint2float_rn((uint32_t)u) * __int_as_float((127 + sh - 40) << 23);
  return neg ? -mag : mag;
}

}  // namespace pmklc

namespace pmklc {
// Programmatic dependent launch: a kernel launched by launch_pdl may be scheduled while the previous
// kernel of its stream is still running.  Every such kernel calls pdl_wait() first, before any early
// exit (it returns once the previous kernel has completed and its writes are visible, so a kernel's
// completion still implies its predecessor's), then pdl_trigger() to let its own successor be
// scheduled early.  Launched the ordinary way, both are no-ops.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args &&...args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<Args &&>(args)...);
}
}  // namespace pmklc

#define PMKLC_CUDA_TRY(expr)                   \
  do {                                         \
    cudaError_t e_ = (expr);                   \
    if (e_ != cudaSuccess) return PMKLC_ECUDA; \
  } while (0)
