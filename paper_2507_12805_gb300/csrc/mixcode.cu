// Probability Mixer (Eq. 1) + softmax + integer CDF + range coding, one warp
// per lane row, and the cross-entropy gradient the Backward Controller needs
// (Eq. 2).
//
// Per predicted row:  z_a = alpha*L^u_a + (1-alpha)*L^m_a     (Eq. 1, S = (1,0,1))
//                     P_a = exp(z_a - max) * (1/sum)            (softmax)
//                     freq_a = 1 + floor(P_a * (2^24 - A)), remainder to the first maximum
// then the lane's token is range coded with (cum, freq) (or decoded from it)
// and dL^m = (1-alpha)(P - onehot)/n, dalpha_row = sum (P - onehot)/n (L^u - L^m).
//
// Determinism (encoder and decoder must build identical tables): every value
// is recomputed from the same inputs with the same instructions in every pass;
// all floating-point operations of the table are explicit round-to-nearest
// intrinsics (no contraction); each lane owns a contiguous chunk of the
// alphabet, reduces it sequentially, and warp results are combined in a fixed
// butterfly order and then broadcast from lane 0, so every lane holds the same
// value.  No float atomics.
#include "internal.h"
#include "rangecoder.cuh"

namespace pmklc {

namespace {

constexpr unsigned kFull = 0xffffffffu;

struct RowView {
  const float *zu, *zm;  // zu unused when !use_static
  float alpha, oma;
  int use_static;
  __device__ __forceinline__ float z(int a) const {
    return use_static ? __fadd_rn(__fmul_rn(alpha, zu[a]), __fmul_rn(oma, zm[a])) : __fmul_rn(oma, zm[a]);
  }
};

__device__ __forceinline__ uint32_t qfreq(float P, float scale) { return 1u + (uint32_t)floorf(__fmul_rn(P, scale)); }

// Alphabet chunk of a lane: [a0, a0 + n)
__device__ __forceinline__ void lane_chunk(int A, int lane, int &a0, int &n) {
  if (A >= 32) {
    n = A >> 5;
    a0 = lane * n;
  } else {
    n = lane < A ? 1 : 0;
    a0 = lane;
  }
}

struct RowTable {
  float mx, inv;
  uint32_t argmax;  // first index of maximal freq
  int rem;          // 2^24 - sum(freq before the remainder)
  uint32_t cbase;   // exclusive prefix of this lane's chunk (incl. remainder)
  uint32_t csum;    // this lane's chunk sum (incl. remainder)
  __device__ __forceinline__ float prob(const RowView &v, int a) const {
    return __fmul_rn(__expf(__fsub_rn(v.z(a), mx)), inv);
  }
  __device__ __forceinline__ uint32_t freq(const RowView &v, int a, float scale) const {
    uint32_t f = qfreq(prob(v, a), scale);
    return a == (int)argmax ? (uint32_t)((int)f + rem) : f;
  }
};

// Warp-cooperative distribution and frequency table of one row (all lanes call it).
__device__ __forceinline__ void row_table(const RowView &v, int A, RowTable &t) {
  const int lane = threadIdx.x & 31;
  int a0, n;
  lane_chunk(A, lane, a0, n);
  const float scale = (float)(kTotal - (uint32_t)A);
  // max
  float mx = -INFINITY;
  for (int i = 0; i < n; ++i) mx = fmaxf(mx, v.z(a0 + i));
  for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(kFull, mx, o));
  t.mx = mx;
  // sum of exponentials: chunk in order, butterfly, lane 0's value broadcast
  float s = 0.f;
  for (int i = 0; i < n; ++i) s = __fadd_rn(s, __expf(__fsub_rn(v.z(a0 + i), mx)));
  for (int o = 16; o; o >>= 1) s = __fadd_rn(s, __shfl_xor_sync(kFull, s, o));
  s = __shfl_sync(kFull, s, 0);
  t.inv = __frcp_rn(s);
  // frequencies before the remainder: sum and first maximum
  uint32_t fs = 0, fmx = 0, amx = 0xffffffffu;
  t.argmax = 0xffffffffu;
  t.rem = 0;
  for (int i = 0; i < n; ++i) {
    uint32_t f = qfreq(t.prob(v, a0 + i), scale);
    fs += f;
    if (f > fmx) {
      fmx = f;
      amx = a0 + i;
    }
  }
  uint32_t tot = fs;
  for (int o = 16; o; o >>= 1) {
    tot += __shfl_xor_sync(kFull, tot, o);
    uint32_t of = __shfl_xor_sync(kFull, fmx, o), oa = __shfl_xor_sync(kFull, amx, o);
    if (of > fmx || (of == fmx && oa < amx)) {
      fmx = of;
      amx = oa;
    }
  }
  t.argmax = amx;
  t.rem = (int)(kTotal - tot);
  // chunk sums with the remainder, exclusive scan over lanes
  uint32_t cs = fs + ((amx >= (uint32_t)a0 && amx < (uint32_t)(a0 + n)) ? (uint32_t)t.rem : 0u);
  uint32_t inc = cs;
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(kFull, inc, o);
    if (lane >= o) inc += y;
  }
  t.csum = cs;
  t.cbase = inc - cs;
}

// (cum, freq) of symbol e, gathered at lane 0 (all lanes call it).
__device__ __forceinline__ void symbol_interval(const RowView &v, int A, const RowTable &t, int e, uint32_t &cum,
                                                uint32_t &freq) {
  const int lane = threadIdx.x & 31;
  int a0, n;
  lane_chunk(A, lane, a0, n);
  const float scale = (float)(kTotal - (uint32_t)A);
  uint32_t c = 0, f = 0;
  int owner = A >= 32 ? e / (A >> 5) : e;
  if (lane == owner) {
    c = t.cbase;
    for (int a = a0; a < e; ++a) c += t.freq(v, a, scale);
    f = t.freq(v, e, scale);
  }
  cum = __shfl_sync(kFull, c, owner);
  freq = __shfl_sync(kFull, f, owner);
}

// Symbol whose interval contains target value x (all lanes call it; result on all lanes).
__device__ __forceinline__ int symbol_of(const RowView &v, int A, const RowTable &t, uint32_t x, uint32_t &cum,
                                         uint32_t &freq) {
  const int lane = threadIdx.x & 31;
  int a0, n;
  lane_chunk(A, lane, a0, n);
  const float scale = (float)(kTotal - (uint32_t)A);
  bool mine = n > 0 && x >= t.cbase && x - t.cbase < t.csum;
  unsigned bal = __ballot_sync(kFull, mine);
  int owner = bal ? __ffs(bal) - 1 : 0;
  int sym = 0;
  uint32_t c = 0, f = 0;
  if (lane == owner) {
    c = t.cbase;
    sym = a0 + n - 1;
    for (int a = a0; a < a0 + n; ++a) {
      uint32_t fa = t.freq(v, a, scale);
      if (x < c + fa) {
        sym = a;
        f = fa;
        break;
      }
      c += fa;
    }
    if (f == 0) f = t.freq(v, sym, scale);  // corrupt input: clamp into the last symbol
  }
  sym = __shfl_sync(kFull, sym, owner);
  cum = __shfl_sync(kFull, c, owner);
  freq = __shfl_sync(kFull, f, owner);
  return sym;
}

// ---- register-resident rows (A = 32 NR, NR = 2, 8, 32) ----
// Lane owns symbols [NR lane, NR lane + NR).  The row's logits are read once with vector loads
// and every exponential, probability and frequency is computed once and kept in registers; the
// operations and their order are those of the generic path above, so both give identical tables.
template <int NR>
struct RegRow {
  static constexpr bool kKeep = NR <= 8;  // raw logits kept for the gradient pass
  float u[kKeep ? NR : 1], m[kKeep ? NR : 1];
  float ex[NR];    // exp(z - max)
  uint32_t f[NR];  // final frequencies (remainder included)
  float inv;
  uint32_t cbase, csum;
};

template <int NR>
__device__ __forceinline__ void load_chunk(const float *src, float (&x)[NR]) {
  if constexpr (NR % 4 == 0) {
#pragma unroll
    for (int q = 0; q < NR / 4; ++q) {
      const float4 w = reinterpret_cast<const float4 *>(src)[q];
      x[4 * q] = w.x, x[4 * q + 1] = w.y, x[4 * q + 2] = w.z, x[4 * q + 3] = w.w;
    }
  } else {
#pragma unroll
    for (int q = 0; q < NR / 2; ++q) {
      const float2 w = reinterpret_cast<const float2 *>(src)[q];
      x[2 * q] = w.x, x[2 * q + 1] = w.y;
    }
  }
}

template <int NR>
__device__ __forceinline__ void reg_table(const RowView &v, int lane, RegRow<NR> &R) {
  const int a0 = lane * NR;
  float uu[NR], mm[NR], z[NR];
  load_chunk<NR>(v.zm + a0, mm);
  if (v.use_static) {
    load_chunk<NR>(v.zu + a0, uu);
  } else {
#pragma unroll
    for (int i = 0; i < NR; ++i) uu[i] = 0.f;
  }
  float mx = -INFINITY;
#pragma unroll
  for (int i = 0; i < NR; ++i) {
    z[i] = v.use_static ? __fadd_rn(__fmul_rn(v.alpha, uu[i]), __fmul_rn(v.oma, mm[i])) : __fmul_rn(v.oma, mm[i]);
    mx = fmaxf(mx, z[i]);
    if constexpr (RegRow<NR>::kKeep) R.u[i] = uu[i], R.m[i] = mm[i];
  }
  for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(kFull, mx, o));
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < NR; ++i) {
    R.ex[i] = __expf(__fsub_rn(z[i], mx));
    s = __fadd_rn(s, R.ex[i]);
  }
  for (int o = 16; o; o >>= 1) s = __fadd_rn(s, __shfl_xor_sync(kFull, s, o));
  s = __shfl_sync(kFull, s, 0);
  R.inv = __frcp_rn(s);
  const float scale = (float)(kTotal - (uint32_t)(32 * NR));
  uint32_t fs = 0, fmx = 0, amx = 0xffffffffu;
#pragma unroll
  for (int i = 0; i < NR; ++i) {
    R.f[i] = qfreq(__fmul_rn(R.ex[i], R.inv), scale);
    fs += R.f[i];
    if (R.f[i] > fmx) {
      fmx = R.f[i];
      amx = a0 + i;
    }
  }
  uint32_t tot = fs;
  for (int o = 16; o; o >>= 1) {
    tot += __shfl_xor_sync(kFull, tot, o);
    uint32_t of = __shfl_xor_sync(kFull, fmx, o), oa = __shfl_xor_sync(kFull, amx, o);
    if (of > fmx || (of == fmx && oa < amx)) {
      fmx = of;
      amx = oa;
    }
  }
  const int rem = (int)(kTotal - tot);
  const bool here = amx >= (uint32_t)a0 && amx < (uint32_t)(a0 + NR);
#pragma unroll
  for (int i = 0; i < NR; ++i)
    if (here && amx == (uint32_t)(a0 + i)) R.f[i] = (uint32_t)((int)R.f[i] + rem);
  const uint32_t cs = fs + (here ? (uint32_t)rem : 0u);
  uint32_t inc = cs;
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(kFull, inc, o);
    if (lane >= o) inc += y;
  }
  R.csum = cs;
  R.cbase = inc - cs;
}

// (cum, freq) of symbol e on every lane
template <int NR>
__device__ __forceinline__ void reg_interval(const RegRow<NR> &R, int e, uint32_t &cum, uint32_t &freq) {
  const int owner = e / NR, idx = e - owner * NR;
  uint32_t c = R.cbase, fr = 0;
#pragma unroll
  for (int i = 0; i < NR; ++i) {
    if (i < idx) c += R.f[i];
    if (i == idx) fr = R.f[i];
  }
  cum = __shfl_sync(kFull, c, owner);
  freq = __shfl_sync(kFull, fr, owner);
}

// symbol whose interval holds x, on every lane (every lane scans its own chunk; the owner's
// result is broadcast)
template <int NR>
__device__ __forceinline__ int reg_symbol(const RegRow<NR> &R, int lane, uint32_t x, uint32_t &cum,
                                          uint32_t &freq) {
  const bool mine = x >= R.cbase && x - R.cbase < R.csum;
  const unsigned bal = __ballot_sync(kFull, mine);
  const int owner = bal ? __ffs(bal) - 1 : 0;
  uint32_t c = R.cbase, fr = 0;
  int sym = NR - 1;
  bool found = false;
#pragma unroll
  for (int i = 0; i < NR; ++i) {
    if (!found) {
      if (x < c + R.f[i]) {
        sym = i;
        fr = R.f[i];
        found = true;
      } else {
        c += R.f[i];
      }
    }
  }
  if (!found) fr = R.f[NR - 1];  // corrupt input: clamp into the last symbol
  sym = __shfl_sync(kFull, lane * NR + sym, owner);
  cum = __shfl_sync(kFull, c, owner);
  freq = __shfl_sync(kFull, fr, owner);
  return sym;
}

template <int NR>
__global__ void __launch_bounds__(256) mixcode_kernel(Plan p, int T) {
  pdl_wait();
  pdl_trigger();
  const int lane = threadIdx.x & 31;
  const int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (r >= p.NL) return;
  if (p.hs_rowmax && lane == 0) p.hs_rowmax[r] = 0u;  // the FP8 static logits of this step are formed
  const int g = p.lane_grp[r];
  const int j = T - p.grp_start[g];
  if (j < 0 || j >= p.lane_len[r]) return;
  const int mode = p.grp_mode[g];
  const int A = p.dm.A;
  const long long tpos = p.lane_tok[r] + j;
  uint8_t *buf = p.lane_buf + p.lane_buf_off[r];
  const uint32_t cap = p.lane_buf_cap[r];
  // the symbols coded over: the whole alphabet, or with overlap masking (j >= 1) the W = 4^s
  // tokens [base, base + W) that agree with token j - 1 on their k - s shared digits
  int base = 0, W = A;
  if (p.ov_w > 0 && j > 0) {
    W = p.ov_w;
    base = ((int)p.tokens[tpos - 1] % p.ov_mod) * W;
  }
  if (j < p.t_eff) {  // uniform distribution for the first t symbols (§2)
    if (lane == 0 && mode != kReplay) {
      const uint32_t u = kTotal / (uint32_t)W;
      if (mode == kEncode) {
        EncState s = p.enc[r];
        uint32_t e = (uint32_t)((int)p.tokens[tpos] - base);
        enc_code24(s, e * u, u, buf, cap, p.err);
        p.enc[r] = s;
      } else {
        DecState s = p.dec[r];
        unsigned long long rr;
        uint32_t x = dec_target24(s, rr);
        uint32_t e = x / u;
        dec_consume(s, rr, e * u, u, buf, cap);
        p.dec[r] = s;
        p.tokens[tpos] = (uint16_t)(base + (int)e);
      }
    }
    return;
  }
  const float alpha = p.alpha[g];
  const size_t ro = (size_t)r * A + base;  // the slice's first element in the row-major [NL][A] buffers
  RowView v{p.zu + ro, p.zm + ro, alpha, __fsub_rn(1.f, alpha), p.use_static};
  const int n_pred = live_lanes(p, g, j);
  const float inv_n = 1.f / (float)n_pred;
  float *outP = p.out_P ? p.out_P + ro : nullptr;
  float da = 0.f;
  if (W < A) {
    // outside the slice the gradient is zero.  The row's dz starts at zero (set once per run) and
    // only slices are ever written, so the previous step's slice (the one of token j - 1, if that
    // token was predicted) is the only non-zero part left to clear.
    if (j - 1 >= p.t_eff) {
      const int pbase = ((int)p.tokens[tpos - 2] % p.ov_mod) * W;
      if (pbase != base)
        for (int a = pbase + lane; a < pbase + W; a += 32) {
          if (p.dz_b)
            p.dz_b[(size_t)r * A + a] = __float2bfloat16_rn(0.f);
          else
            p.dz[(size_t)r * A + a] = 0.f;
        }
    }
    if (p.out_P)
      for (int a = lane; a < A; a += 32)
        if (a < base || a >= base + W) p.out_P[(size_t)r * A + a] = 0.f;
  }
  if constexpr (NR > 0) {
    RegRow<NR> R;
    reg_table<NR>(v, lane, R);
    int e;
    if (mode == kDecode) {
      DecState s;
      unsigned long long rr = 0;
      uint32_t x = 0;
      if (lane == 0) {
        s = p.dec[r];
        x = dec_target24(s, rr);
      }
      x = __shfl_sync(kFull, x, 0);
      uint32_t cum, freq;
      e = reg_symbol<NR>(R, lane, x, cum, freq);
      if (lane == 0) {
        dec_consume(s, rr, cum, freq, buf, cap);
        p.dec[r] = s;
        p.tokens[tpos] = (uint16_t)(base + e);
      }
    } else {
      e = (int)p.tokens[tpos] - base;
      if (mode == kEncode) {
        uint32_t cum, freq;
        reg_interval<NR>(R, e, cum, freq);
        if (lane == 0) {
          EncState s = p.enc[r];
          enc_code24(s, cum, freq, buf, cap, p.err);
          p.enc[r] = s;
        }
      }
    }
    // Backward Controller inputs (Eq. 2): the lane's chunk in registers, stored with vector writes
    const int a0 = lane * NR;
    float dv[NR], uu[NR], mm[NR];
    if constexpr (RegRow<NR>::kKeep) {
#pragma unroll
      for (int i = 0; i < NR; ++i) uu[i] = R.u[i], mm[i] = R.m[i];
    } else {
      load_chunk<NR>(v.zm + a0, mm);
      if (p.use_static) load_chunk<NR>(v.zu + a0, uu);
    }
#pragma unroll
    for (int i = 0; i < NR; ++i) {
      const float P = __fmul_rn(R.ex[i], R.inv);
      if (outP) outP[a0 + i] = P;
      const float d = (P - (a0 + i == e ? 1.f : 0.f)) * inv_n;
      dv[i] = v.oma * d;
      const float diff = p.use_static ? uu[i] - mm[i] : -mm[i];
      da = fmaf(d, diff, da);
    }
    if (p.dz_b) {
#pragma unroll
      for (int q = 0; q < NR / 2; ++q) {
        __nv_bfloat162 h = __floats2bfloat162_rn(dv[2 * q], dv[2 * q + 1]);
        reinterpret_cast<__nv_bfloat162 *>(p.dz_b + ro + a0)[q] = h;
      }
    } else {
#pragma unroll
      for (int q = 0; q < NR / 2; ++q)
        reinterpret_cast<float2 *>(p.dz + ro + a0)[q] = make_float2(dv[2 * q], dv[2 * q + 1]);
    }
  } else {
    RowTable t;
    row_table(v, W, t);
    int e;
    if (mode == kDecode) {
      DecState s;
      unsigned long long rr = 0;
      uint32_t x = 0;
      if (lane == 0) {
        s = p.dec[r];
        x = dec_target24(s, rr);
      }
      x = __shfl_sync(kFull, x, 0);
      uint32_t cum, freq;
      e = symbol_of(v, W, t, x, cum, freq);
      if (lane == 0) {
        dec_consume(s, rr, cum, freq, buf, cap);
        p.dec[r] = s;
        p.tokens[tpos] = (uint16_t)(base + e);
      }
    } else {
      e = (int)p.tokens[tpos] - base;
      if (mode == kEncode) {
        uint32_t cum, freq;
        symbol_interval(v, W, t, e, cum, freq);
        if (lane == 0) {
          EncState s = p.enc[r];
          enc_code24(s, cum, freq, buf, cap, p.err);
          p.enc[r] = s;
        }
      }
    }
    // Backward Controller inputs: mean cross entropy over the group's predicted lanes
    int a0, n;
    lane_chunk(W, lane, a0, n);
    float *dz = p.dz + ro;
    __nv_bfloat16 *dzb = p.dz_b ? p.dz_b + ro : nullptr;
    for (int a = a0; a < a0 + n; ++a) {
      float P = t.prob(v, a);
      if (outP) outP[a] = P;
      float d = (P - (a == e ? 1.f : 0.f)) * inv_n;
      if (dzb)
        dzb[a] = __float2bfloat16_rn(v.oma * d);
      else
        dz[a] = v.oma * d;
      float diff = p.use_static ? v.zu[a] - v.zm[a] : -v.zm[a];
      da = fmaf(d, diff, da);
    }
  }
  for (int o = 16; o; o >>= 1) da += __shfl_xor_sync(kFull, da, o);
  if (lane == 0) p.dalpha_row[r] = da;
}

__global__ void coder_init_kernel(Plan p, int encode) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= p.NL) return;
  if (encode) {
    EncState s;
    enc_init(s);
    p.enc[r] = s;
  } else {
    DecState s;
    dec_init(s, p.lane_buf + p.lane_buf_off[r], p.lane_buf_cap[r]);
    p.dec[r] = s;
  }
}

__global__ void coder_finish_kernel(Plan p, uint32_t *lane_len) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= p.NL) return;
  EncState s = p.enc[r];
  lane_len[r] = enc_finish(s, p.lane_buf + p.lane_buf_off[r], p.lane_buf_cap[r], p.err);
  p.enc[r] = s;
}

// ---- standalone kernels for the single-step entry points ----

__global__ void quantize_kernel(const float *P, int rows, int A, uint32_t *freq) {
  const int lane = threadIdx.x & 31;
  const int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (r >= rows) return;
  // a RowTable whose probabilities are given directly
  const float *pr = P + (size_t)r * A;
  const float scale = (float)(kTotal - (uint32_t)A);
  int a0, n;
  lane_chunk(A, lane, a0, n);
  uint32_t fs = 0, fmx = 0, amx = 0xffffffffu;
  for (int i = 0; i < n; ++i) {
    uint32_t f = qfreq(pr[a0 + i], scale);
    fs += f;
    if (f > fmx) {
      fmx = f;
      amx = a0 + i;
    }
  }
  uint32_t tot = fs;
  for (int o = 16; o; o >>= 1) {
    tot += __shfl_xor_sync(kFull, tot, o);
    uint32_t of = __shfl_xor_sync(kFull, fmx, o), oa = __shfl_xor_sync(kFull, amx, o);
    if (of > fmx || (of == fmx && oa < amx)) {
      fmx = of;
      amx = oa;
    }
  }
  int rem = (int)(kTotal - tot);
  for (int i = 0; i < n; ++i) {
    int a = a0 + i;
    uint32_t f = qfreq(pr[a], scale);
    freq[(size_t)r * A + a] = a == (int)amx ? (uint32_t)((int)f + rem) : f;
  }
}

__global__ void mix_quantize_kernel(const float *Lu, const float *Lm, int rows, int A, float alpha, int use_static,
                                    float *P, uint32_t *freq) {
  const int lane = threadIdx.x & 31;
  const int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (r >= rows) return;
  RowView v{Lu ? Lu + (size_t)r * A : nullptr, Lm + (size_t)r * A, alpha, __fsub_rn(1.f, alpha), use_static};
  RowTable t;
  row_table(v, A, t);
  const float scale = (float)(kTotal - (uint32_t)A);
  int a0, n;
  lane_chunk(A, lane, a0, n);
  for (int a = a0; a < a0 + n; ++a) {
    P[(size_t)r * A + a] = t.prob(v, a);
    freq[(size_t)r * A + a] = t.freq(v, a, scale);
  }
}

__global__ void range_encode_kernel(const uint32_t *freq, const uint16_t *sym, int n_streams, int L, int A,
                                    uint8_t *out, uint32_t cap, uint32_t *len, int *err) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_streams) return;
  EncState s;
  enc_init(s);
  uint8_t *o = out + (size_t)i * cap;
  for (int j = 0; j < L; ++j) {
    const uint32_t *f = freq + ((size_t)i * L + j) * A;
    const int e = sym[(size_t)i * L + j];
    // a caller's symbol or table the coder cannot take (symbol outside the alphabet, frequency 0,
    // interval past the 2^24 total) ends the stream with an error instead of looping or reading on
    if (e >= A) {
      atomicOr(err, kErrCorrupt);
      break;
    }
    unsigned long long cum = 0;
    for (int a = 0; a < e; ++a) cum += f[a];
    if (f[e] == 0 || cum + f[e] > kTotal) {
      atomicOr(err, kErrCorrupt);
      break;
    }
    enc_code24(s, (uint32_t)cum, f[e], o, cap, err);
  }
  len[i] = enc_finish(s, o, cap, err);
}

__global__ void range_decode_kernel(const uint32_t *freq, const uint8_t *in, const uint32_t *len, int n_streams,
                                    int L, int A, uint32_t cap, uint16_t *sym, int *err) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_streams) return;
  DecState s;
  const uint8_t *b = in + (size_t)i * cap;
  const uint32_t n_in = len[i] < cap ? len[i] : cap;  // never past the stream's own cap bytes
  dec_init(s, b, n_in);
  for (int j = 0; j < L; ++j) {
    const uint32_t *f = freq + ((size_t)i * L + j) * A;
    unsigned long long rr;
    uint32_t x = dec_target24(s, rr);
    unsigned long long cum = 0;
    int e = -1;
    for (int a = 0; a < A; ++a) {
      if (x < cum + f[a]) {
        e = a;
        break;
      }
      cum += f[a];
    }
    // a table whose entries end below the target or run past the 2^24 total cannot be decoded
    if (e < 0 || cum + f[e] > kTotal) {
      atomicOr(err, kErrCorrupt);
      break;
    }
    dec_consume(s, rr, (uint32_t)cum, f[e], b, n_in);
    sym[(size_t)i * L + j] = (uint16_t)e;
  }
}

}  // namespace

void launch_mixcode(const Plan &p, int T, cudaStream_t st) {
  if (p.NL <= 0) return;
  // reads L^u and L^m over the coded symbols (8 bytes each) and writes the whole row of dL^m
  const double wc = p.ov_w > 0 ? p.ov_w : p.dm.A;
  ProfScope ps("mix_cdf_code", 0, prof_work().pred_rows * (8.0 * wc + 4.0 * p.dm.A), st);
  const unsigned grid = (unsigned)((p.NL * 32 + 255) / 256);
  // every predicted row is coded over W symbols (the slice with overlap masking)
  switch (p.ov_w > 0 ? p.ov_w : p.dm.A) {  // register-resident rows where a lane's chunk fits in registers
    case 64: launch_pdl(mixcode_kernel<2>, dim3(grid), dim3(256), 0, st, p, T); break;
    case 256: launch_pdl(mixcode_kernel<8>, dim3(grid), dim3(256), 0, st, p, T); break;
    case 1024: launch_pdl(mixcode_kernel<32>, dim3(grid), dim3(256), 0, st, p, T); break;
    default: launch_pdl(mixcode_kernel<0>, dim3(grid), dim3(256), 0, st, p, T); break;
  }
}

void launch_coder_init(const Plan &p, int encode, cudaStream_t st) {
  if (p.NL <= 0) return;
  coder_init_kernel<<<(p.NL + 127) / 128, 128, 0, st>>>(p, encode);
}

void launch_coder_finish(const Plan &p, uint32_t *d_lane_len, cudaStream_t st) {
  if (p.NL <= 0) return;
  coder_finish_kernel<<<(p.NL + 127) / 128, 128, 0, st>>>(p, d_lane_len);
}

}  // namespace pmklc

using namespace pmklc;

static bool pow4(uint32_t A) { return A >= 4 && A <= 65536 && (A & (A - 1)) == 0 && (__builtin_ctz(A) % 2 == 0); }

// rows of the per-row entry points: one warp per row, warp indices in 32 bits
constexpr size_t kMaxRows = size_t(1) << 26;

extern "C" int pmklc_quantize(const float *d_P, size_t rows, uint32_t A, uint32_t *d_freq, void *stream) {
  if (!pow4(A) || rows > kMaxRows || (rows && (!d_P || !d_freq))) return PMKLC_EINVAL;
  if (rows == 0) return PMKLC_OK;
  cudaStream_t st = (cudaStream_t)stream;
  quantize_kernel<<<(unsigned)((rows * 32 + 255) / 256), 256, 0, st>>>(d_P, (int)rows, (int)A, d_freq);
  PMKLC_CUDA_TRY(cudaGetLastError());
  PMKLC_CUDA_TRY(cudaStreamSynchronize(st));
  return PMKLC_OK;
}

extern "C" int pmklc_mix_quantize(const float *d_Lu, const float *d_Lm, size_t rows, uint32_t A, float alpha,
                                  uint32_t use_static, float *d_P, uint32_t *d_freq, void *stream) {
  if (!pow4(A) || rows > kMaxRows || (rows && (!d_Lm || !d_P || !d_freq || (use_static && !d_Lu))))
    return PMKLC_EINVAL;
  if (rows == 0) return PMKLC_OK;
  cudaStream_t st = (cudaStream_t)stream;
  mix_quantize_kernel<<<(unsigned)((rows * 32 + 255) / 256), 256, 0, st>>>(d_Lu, d_Lm, (int)rows, (int)A, alpha,
                                                                             (int)(use_static != 0), d_P, d_freq);
  PMKLC_CUDA_TRY(cudaGetLastError());
  PMKLC_CUDA_TRY(cudaStreamSynchronize(st));
  return PMKLC_OK;
}

extern "C" int pmklc_range_encode(const uint32_t *d_freq, const uint16_t *d_sym, uint32_t n_streams, uint32_t L,
                                  uint32_t A, uint8_t *d_out, uint32_t cap, uint32_t *d_len, void *stream) {
  if (!pow4(A) || !d_len || n_streams > INT32_MAX || L > INT32_MAX || (n_streams && (!d_out || (L && (!d_freq || !d_sym)))))
    return PMKLC_EINVAL;
  if (n_streams == 0) return PMKLC_OK;
  cudaStream_t st = (cudaStream_t)stream;
  int *d_err = nullptr;
  PMKLC_CUDA_TRY(cudaMallocAsync((void **)&d_err, sizeof(int), st));
  cudaMemsetAsync(d_err, 0, sizeof(int), st);
  range_encode_kernel<<<(n_streams + 63) / 64, 64, 0, st>>>(d_freq, d_sym, (int)n_streams, (int)L, (int)A, d_out, cap,
                                                            d_len, d_err);
  int h = 0;
  cudaMemcpyAsync(&h, d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
  cudaFreeAsync(d_err, st);
  PMKLC_CUDA_TRY(cudaGetLastError());
  PMKLC_CUDA_TRY(cudaStreamSynchronize(st));
  return (h & kErrCorrupt) ? PMKLC_EINVAL : h ? PMKLC_ENOSPC : PMKLC_OK;
}

extern "C" int pmklc_range_decode(const uint32_t *d_freq, const uint8_t *d_in, const uint32_t *d_len,
                                  uint32_t n_streams, uint32_t L, uint32_t A, uint32_t cap, uint16_t *d_sym,
                                  void *stream) {
  if (!pow4(A) || n_streams > INT32_MAX || L > INT32_MAX ||
      (n_streams && (!d_in || !d_len || (L && (!d_freq || !d_sym)))))
    return PMKLC_EINVAL;
  if (n_streams == 0) return PMKLC_OK;
  cudaStream_t st = (cudaStream_t)stream;
  int *d_err = nullptr;
  PMKLC_CUDA_TRY(cudaMallocAsync((void **)&d_err, sizeof(int), st));
  cudaMemsetAsync(d_err, 0, sizeof(int), st);
  range_decode_kernel<<<(n_streams + 63) / 64, 64, 0, st>>>(d_freq, d_in, d_len, (int)n_streams, (int)L, (int)A, cap,
                                                            d_sym, d_err);
  int h = 0;
  cudaMemcpyAsync(&h, d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
  cudaFreeAsync(d_err, st);
  PMKLC_CUDA_TRY(cudaGetLastError());
  PMKLC_CUDA_TRY(cudaStreamSynchronize(st));
  return h ? PMKLC_EINVAL : PMKLC_OK;
}
