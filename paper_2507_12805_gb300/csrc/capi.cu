// Host orchestration and the C ABI of libpmklc (include/pmklc.h).
//
// Compression follows the paper's loop (§2 steps (1)-(4)) organised as in §4:
// blocks from the Data Chunker (§4.3) are tokenised by GskE (§4.1); each block
// gets its own dynamic model and its tokens are split into lanes that advance
// in lockstep (the batch size bs of §5.1.4); every global step runs, for all
// blocks at once, the predictor forward, the Eq. (1) mixer + CDF + range
// coder, and the Backward Controller's update (Eq. 2); Step-wise Model
// Passing (§4.3, Fig. 5) copies a parent's state into a child at the child's
// start step.  The count model judges every block.  The host builds the lane
// tables and the schedule, launches the per-step kernels, and assembles the
// container.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <new>
#include <type_traits>
#include <vector>

#include "internal.h"

namespace pmklc {

namespace {

thread_local pmklc_stats g_stats;

// ---------------------------------------------------------------- utilities

struct Arena {  // stream-ordered device allocations, released together
  cudaStream_t st;
  std::vector<void *> ptrs;
  bool failed = false;
  explicit Arena(cudaStream_t s) : st(s) {}
  template <class T>
  T *alloc(size_t n) {
    void *p = nullptr;
    size_t bytes = (n ? n : 1) * sizeof(T);
    bytes = (bytes + 255) & ~(size_t)255;
    if (cudaMallocAsync(&p, bytes, st) != cudaSuccess) {
      failed = true;
      return nullptr;
    }
    ptrs.push_back(p);
    return (T *)p;
  }
  template <class T>
  T *upload(const std::vector<T> &v) {
    T *d = alloc<T>(v.size());
    if (d && !v.empty()) cudaMemcpyAsync(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st);
    return d;
  }
  ~Arena() {
    for (void *p : ptrs) cudaFreeAsync(p, st);
  }
};

uint64_t sm64_draw(uint64_t seed, uint64_t i) {  // splitmix64 output i of the stream seeded with `seed`
  uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Seeded initial parameters (counter-based splitmix64): w = (2u - 2^24) 2^-24, value = w * bound (float32 RN).
void init_params(const Dims &d, uint64_t seed, std::vector<float> &out) {
  out.assign(d.count(), 0.f);
  auto fill = [&](size_t lo, size_t hi, float bound) {
    for (size_t i = lo; i < hi; ++i) {
      int64_t u = (int64_t)(sm64_draw(seed, i) >> 40);
      float w = (float)(2 * u - (1 << 24)) * (1.0f / 16777216.0f);
      volatile float v = w * bound;  // one IEEE product, no contraction
      out[i] = v;
    }
  };
  fill(d.off_emb(), d.off_w1(), 1.0f);
  fill(d.off_w1(), d.off_b1(), 1.0f / sqrtf((float)(d.t * d.E)));
  fill(d.off_w2(), d.off_b2(), 1.0f / sqrtf((float)d.H));
}

uint64_t fnv1a(const void *p, size_t n) {
  const uint8_t *b = (const uint8_t *)p;
  uint64_t h = 0xCBF29CE484222325ull;
  for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 0x100000001B3ull;
  return h;
}

long long n_tokens_of(long long n, int s, int k) { return n < k ? 0 : (n - k) / s + 1; }
long long tail_len_of(long long n, int s, int k) {
  long long l = n_tokens_of(n, s, k);
  return l == 0 ? n : n - ((l - 1) * s + k);
}

void put_varint(std::vector<uint8_t> &o, uint64_t x) {
  while (true) {
    uint8_t b = x & 0x7F;
    x >>= 7;
    if (x) {
      o.push_back(b | 0x80);
    } else {
      o.push_back(b);
      return;
    }
  }
}
size_t varint_len(uint64_t x) {
  size_t n = 1;
  while (x >>= 7) ++n;
  return n;
}
bool get_varint(const uint8_t *buf, size_t len, size_t &pos, uint64_t &x) {
  x = 0;
  for (int shift = 0; shift < 64; shift += 7) {
    if (pos >= len) return false;
    uint8_t b = buf[pos++];
    x |= (uint64_t)(b & 0x7F) << shift;
    if (!(b & 0x80)) return true;
  }
  return false;
}

template <class T>
void put_le(std::vector<uint8_t> &o, T v) {
  uint8_t b[sizeof(T)];
  memcpy(b, &v, sizeof(T));  // both supported hosts (x86-64, aarch64) are little-endian
  o.insert(o.end(), b, b + sizeof(T));
}
template <class T>
T get_le(const uint8_t *p) {
  T v;
  memcpy(&v, p, sizeof(T));
  return v;
}

constexpr size_t kHeader = 80;
constexpr uint8_t kVersion = 1;
// Each block is one model group; the GEMMs run the groups of both models (static and dynamic)
// along the grid's z dimension and the per-group kernels along y, both limited to 65,535.
constexpr uint32_t kMaxGroups = 32767;
constexpr uint8_t kPrivateFlag = 8;  // container flags bit 3: a static private model is stored

// ---------------------------------------------------------------- configuration

struct Cfg {
  int s, k, use_static, precision, optimizer, smp_mode, count_order, fallback;
  Dims dm, st;
  int lanes;
  int lane_tokens;  // 0: every block gets min(lanes, l) lanes; else min(lanes, l, ceil(l / lane_tokens))
  float lr, alpha0, smp_f;
  uint64_t seed;
  int mask = 0;                        // overlap-masked coding (s < k)
  int update_path = PMKLC_UPDATE_AUTO;  // where W1 and W2 are updated (the same bytes either way)
  int gemm_tiles = 0;                   // row GEMMs' column-tile cap: 0 default, 1 128, 2 64 (same bytes)
  int priv = 0, priv_epochs = 1;      // Model Selector: static private model (0 off, 1 on, 2 auto)
  unsigned long long priv_bases = 0;  // bases of the input's head its pre-training reads (0 = all)
  unsigned long long priv_threshold = 0;  // the selector's input size in bases (0 = 5e8, the paper's 500 MB)
  // static predictor architecture: 0 the MLP (st its shape); 1 or 2 a BiGRU static predictor of
  // that many layers (§4.2.3 SPrM, §4.2.2 SPuM), GRU width gru_hg, st = (A, E, t, 128) the shape
  // of its Dense layer run as an MLP logits layer
  int st_arch = 0, gru_hg = 0;
  int A() const { return 1 << (2 * k); }
  // FP32 parameters of the static model as the caller passes it
  size_t static_count() const { return st_arch ? gru_offsets(A(), st.E, gru_hg, st_arch).count : st.count(); }
  int t_eff() const { return std::max(dm.t, use_static ? st.t : 0); }
};

// the BF16 batched forms (the static model in BF16 or in FP8)
bool bf_form(int precision) {
  return precision == PMKLC_BF16_BATCHED || precision == PMKLC_BF16_FP8STATIC || precision == PMKLC_BF16_FP8HIDDEN;
}
// the forms whose static model runs (at least partly) in E4M3 on the tcgen05 engine
bool f8_form(int precision) { return precision == PMKLC_BF16_FP8STATIC || precision == PMKLC_BF16_FP8HIDDEN; }

int check_cfg(const pmklc_model_cfg *c, Cfg &o) {
  if (!c || c->struct_size != sizeof(pmklc_model_cfg)) return PMKLC_EINVAL;
  if (c->s < 1 || c->s > c->k || c->k > 8) return PMKLC_EINVAL;
  if (c->emb_d < 1 || c->ctx_d < 1 || c->hid_d < 1 || c->emb_d > 4096 || c->ctx_d > 4096 || c->hid_d > 65535)
    return PMKLC_EINVAL;
  if (c->use_static && (c->emb_s < 1 || c->ctx_s < 1 || c->hid_s < 1 || c->emb_s > 4096 || c->ctx_s > 4096 ||
                        c->hid_s > 65535 || !c->static_weights))
    return PMKLC_EINVAL;
  if (c->precision > PMKLC_BF16_FP8HIDDEN) return PMKLC_EINVAL;
  if (c->optimizer > PMKLC_SGD || c->smp_mode > PMKLC_SMP_TREE || c->count_order > 7) return PMKLC_EINVAL;
  if (!(c->lr > 0.f) || !isfinite(c->lr) || !isfinite(c->alpha_init)) return PMKLC_EINVAL;
  if (!(c->smp_fraction >= 0.f && c->smp_fraction <= 1.f)) return PMKLC_EINVAL;
  if (c->lanes_per_block > (1u << 20) || c->fallback > 2) return PMKLC_EINVAL;
  if (c->overlap_mask > 1 || c->update_path > PMKLC_UPDATE_FUSED || c->gemm_tiles > 2) return PMKLC_EINVAL;
  if (c->private_model > 2 || c->private_epochs > kMaxGroups) return PMKLC_EINVAL;
  // a BiGRU static predictor: frozen, so never pre-trained as a private model here; FP32 or BF16
  if (c->static_arch > 2 ||
      (c->static_arch && (!c->use_static || c->private_model || c->precision > PMKLC_BF16_BATCHED ||
                          !gru_shape_ok((int)c->k, (int)c->emb_s, (int)c->ctx_s, (int)c->hid_s, (int)c->static_arch))))
    return PMKLC_EINVAL;
  if (c->private_model && (c->emb_s < 1 || c->ctx_s < 1 || c->hid_s < 1 || c->emb_s > 4096 || c->ctx_s > 4096 ||
                           c->hid_s > 65535))
    return PMKLC_EINVAL;
  o.s = (int)c->s;
  o.k = (int)c->k;
  o.use_static = c->use_static ? 1 : 0;
  o.precision = (int)c->precision;
  o.optimizer = (int)c->optimizer;
  o.smp_mode = (int)c->smp_mode;
  o.count_order = (int)c->count_order;
  o.fallback = (int)c->fallback;
  int A = 1 << (2 * c->k);
  o.dm = Dims{A, (int)c->emb_d, (int)c->ctx_d, (int)c->hid_d};
  o.st = o.use_static || c->private_model ? Dims{A, (int)c->emb_s, (int)c->ctx_s, (int)c->hid_s} : Dims{A, 0, 0, 0};
  o.st_arch = (int)c->static_arch;
  if (o.st_arch) {
    o.gru_hg = (int)c->hid_s;
    o.st.H = kGruDense;
  }
  o.priv = (int)c->private_model;
  o.priv_epochs = c->private_epochs ? (int)c->private_epochs : 1;
  o.priv_bases = c->private_bases;
  o.priv_threshold = c->private_threshold;
  o.mask = (int)c->overlap_mask;
  o.update_path = (int)c->update_path;
  o.gemm_tiles = (int)c->gemm_tiles;
  o.lanes = c->lanes_per_block ? (int)c->lanes_per_block : 64;
  o.lane_tokens = (int)c->lane_tokens;
  o.lr = c->lr;
  o.alpha0 = c->alpha_init;
  o.smp_f = c->smp_fraction;
  o.seed = c->seed;
  return PMKLC_OK;
}

// ---------------------------------------------------------------- lanes + schedule

struct Layout {
  int G = 0, NL = 0, Mmax = 0;
  std::vector<long long> base_off, tok_off;  // G+1
  std::vector<int> lane_off, base_len, extra, steps;
  std::vector<long long> lane_tok;
  std::vector<int> lane_len, lane_grp;
  long long n_tok = 0;
};

long long lanes_of(long long l, int M, int lane_tokens) {
  if (l == 0) return 0;
  long long m = std::min<long long>(M, l);
  if (lane_tokens > 0) m = std::min(m, std::max(1LL, (l + lane_tokens - 1) / lane_tokens));
  return m;
}

// Limits of one call's layout, checked on the host before anything is allocated: at most 2^24
// lanes in all (grids count lanes x 32 threads in 32 bits), lanes x hidden width below 2^31 (the
// BF16 hidden reduction walks rows x H with a 32-bit index), at most 2^27 tokens per lane (a lane's
// byte capacities are 32-bit: 3 per token for the network, 2 per base for the count model) and at
// most 2^30 steps in the schedule (placed as make_schedule places the groups).
constexpr long long kMaxLanes = 1LL << 24, kMaxLaneTokens = 1LL << 27, kMaxSteps = 1LL << 30;

bool layout_fits(const std::vector<unsigned long long> &lens, const Cfg &c, int smp_mode, float f32) {
  if (lens.size() > kMaxGroups) return false;
  const double f = (double)f32;
  long long lanes = 0, mx = 0;
  std::vector<long long> steps(lens.size(), 0);
  for (size_t g = 0; g < lens.size(); ++g) {
    if (lens[g] > (1ull << 56)) return false;
    const long long l = n_tokens_of((long long)lens[g], c.s, c.k), Mb = lanes_of(l, c.lanes, c.lane_tokens);
    if (Mb > 0) steps[g] = (l + Mb - 1) / Mb;
    if (steps[g] > kMaxLaneTokens) return false;
    lanes += Mb;
    mx = std::max(mx, steps[g]);
  }
  const long long hmax = std::max(c.dm.H, c.use_static || c.priv ? c.st.H : 0);
  if (lanes > kMaxLanes || lanes * hmax >= (1LL << 31)) return false;
  long long T = 0, start = 0;
  const long long D = (long long)ceil(f * (double)mx);
  for (size_t g = 0; g < lens.size(); ++g) {
    if (smp_mode == PMKLC_SMP_CHAIN && g > 0) start += (long long)ceil(f * (double)steps[g - 1]);
    if (smp_mode == PMKLC_SMP_TREE) start = g ? (long long)(64 - __builtin_clzll((unsigned long long)g)) * D : 0;
    T = std::max(T, start + steps[g]);
  }
  return T <= kMaxSteps;
}

void make_layout(const std::vector<unsigned long long> &lens, int s, int k, int M, int lane_tokens, Layout &L) {
  L.G = (int)lens.size();
  L.base_off.assign(L.G + 1, 0);
  L.tok_off.assign(L.G + 1, 0);
  L.lane_off.assign(L.G + 1, 0);
  L.base_len.assign(L.G, 0);
  L.extra.assign(L.G, 0);
  L.steps.assign(L.G, 0);
  for (int g = 0; g < L.G; ++g) {
    long long n = (long long)lens[g];
    long long l = n_tokens_of(n, s, k);
    L.base_off[g + 1] = L.base_off[g] + n;
    L.tok_off[g + 1] = L.tok_off[g] + l;
    int Mb = (int)lanes_of(l, M, lane_tokens);
    L.lane_off[g + 1] = L.lane_off[g] + Mb;
    if (Mb > 0) {
      long long base = l / Mb, extra = l % Mb;
      L.base_len[g] = (int)base;
      L.extra[g] = (int)extra;
      L.steps[g] = (int)(base + (extra > 0));
      for (int r = 0; r < Mb; ++r) {
        L.lane_tok.push_back(L.tok_off[g] + r * base + std::min<long long>(r, extra));
        L.lane_len.push_back((int)(base + (r < extra)));
        L.lane_grp.push_back(g);
      }
    }
    L.Mmax = std::max(L.Mmax, Mb);
  }
  L.NL = L.lane_off[L.G];
  L.n_tok = L.tok_off[L.G];
}

struct Schedule {
  std::vector<int> start, parent, tau0;
  int T_total = 0, max_tau = 0;
  std::vector<std::vector<int>> pairs_at;  // T -> flattened (child, parent) pairs
};

void make_schedule(const Layout &L, int mode, float f32, int t_eff, Schedule &S) {
  int G = L.G;
  double f = (double)f32;
  S.start.assign(G, 0);
  S.parent.assign(G, -1);
  S.tau0.assign(G, 0);
  if (G > 0 && mode == PMKLC_SMP_CHAIN) {
    for (int g = 1; g < G; ++g) {
      S.parent[g] = g - 1;
      S.start[g] = S.start[g - 1] + (int)ceil(f * L.steps[g - 1]);
    }
  } else if (G > 0 && mode == PMKLC_SMP_TREE) {
    int mx = *std::max_element(L.steps.begin(), L.steps.end());
    int D = (int)ceil(f * mx);
    for (int g = 1; g < G; ++g) {
      int lvl = 32 - __builtin_clz((unsigned)g);
      S.parent[g] = g - (1 << (lvl - 1));
      S.start[g] = lvl * D;
    }
  }
  S.T_total = 0;
  S.max_tau = 0;
  for (int g = 0; g < G; ++g) {
    int p = S.parent[g];
    if (p >= 0) {
      int ran = std::min(S.start[g] - S.start[p], L.steps[p]);
      S.tau0[g] = S.tau0[p] + std::max(0, ran - t_eff);
    }
    S.T_total = std::max(S.T_total, S.start[g] + L.steps[g]);
    S.max_tau = std::max(S.max_tau, S.tau0[g] + std::max(0, L.steps[g] - t_eff));
  }
  // Hand-overs happen at the child's start step (children starting at 0 already hold the
  // init, which is what their parent holds then).  Copies of one step run in parallel, so a
  // parent that itself receives a copy at the same step is replaced by its own source.
  S.pairs_at.assign(S.T_total + 1, {});
  for (int g = 0; g < G; ++g)
    if (S.parent[g] >= 0 && S.start[g] > 0 && S.start[g] <= S.T_total) {
      int src = S.parent[g];
      while (S.parent[src] >= 0 && S.start[src] == S.start[g]) src = S.parent[src];
      S.pairs_at[S.start[g]].push_back(g);
      S.pairs_at[S.start[g]].push_back(src);
    }
}

// ---------------------------------------------------------------- device run

struct Run {
  Plan p{};
  Layout L;
  Schedule S;
  Cfg c;
  int *d_pairs = nullptr;
  std::vector<int> pair_off;  // T -> offset (pairs) into d_pairs
  uint64_t launches = 0;
  bool net = true;            // run the network (false: count model only)
  const float *init_host = nullptr;  // initial parameters of every group (default: the seeded init)
  CountPlan cp{};
  std::vector<int> cmode;     // per group: count model 0 off, 1 encode, 2 decode
};

// Count-model state of a run: one table per group, per-lane contexts and coder states.
// buf/buf_off/buf_cap are set by the caller.
int setup_count(Arena &ar, Run &R) {
  const Layout &L = R.L;
  CountPlan &c = R.cp;
  c.m = R.c.count_order;
  c.s = R.c.s;
  c.k = R.c.k;
  c.grp_cmode = ar.upload(R.cmode);
  size_t tab = ((size_t)std::max(L.G, 1) << (2 * c.m)) * 4;
  c.table = ar.alloc<uint32_t>(tab);
  c.ctx = ar.alloc<uint32_t>(std::max(L.NL, 1));
  c.enc = ar.alloc<EncState>(std::max(L.NL, 1));
  c.dec = ar.alloc<DecState>(std::max(L.NL, 1));
  if (ar.failed) return PMKLC_ENOMEM;
  cudaMemsetAsync(c.table, 0, tab * sizeof(uint32_t), ar.st);
  return PMKLC_OK;
}

// Allocates the model state, activations and tables of a run.  lane_buf / caps / enc / dec are set by the caller.
int setup_run(Arena &ar, Run &R, const std::vector<int> &grp_mode, const float *d_static) {
  const Cfg &c = R.c;
  const Layout &L = R.L;
  Plan &p = R.p;
  p.G = L.G;
  p.NL = L.NL;
  p.Mmax = L.Mmax;
  p.t_eff = c.t_eff();
  p.ov_w = c.mask && c.s < c.k ? 1 << (2 * c.s) : 0;
  p.ov_mod = c.mask && c.s < c.k ? 1 << (2 * (c.k - c.s)) : 0;
  p.use_static = c.use_static;
  p.optimizer = c.optimizer;
  p.lr = c.lr;
  p.dm = c.dm;
  p.st = c.st;
  p.P = c.dm.count();
  size_t G = (size_t)std::max(L.G, 1), NL = (size_t)std::max(L.NL, 1);
  p.grp_start = ar.upload(R.S.start);
  p.grp_steps = ar.upload(L.steps);
  p.grp_lane_off = ar.upload(L.lane_off);
  p.grp_base = ar.upload(L.base_len);
  p.grp_extra = ar.upload(L.extra);
  p.grp_mode = ar.upload(grp_mode);
  p.grp_tau0 = ar.upload(R.S.tau0);
  p.lane_tok = ar.upload(L.lane_tok);
  p.lane_len = ar.upload(L.lane_len);
  p.lane_grp = ar.upload(L.lane_grp);
  p.params = ar.alloc<float>(G * p.P);
  p.m = ar.alloc<float>(G * p.P);
  p.v = ar.alloc<float>(G * p.P);
  p.grad = ar.alloc<float>(G * p.P);
  p.alpha = ar.alloc<float>(G);
  p.alpha_m = ar.alloc<float>(G);
  p.alpha_v = ar.alloc<float>(G);
  p.dalpha_grp = ar.alloc<float>(G);
  p.static_params = d_static;
  p.st_gru = nullptr;
  p.gru_hg = p.gru_layers = 0;
  p.gru_y = nullptr;
  if (c.st_arch && c.use_static && d_static) {
    // the BiGRU static predictor forms the static h itself; its Dense layer (W4, b4) runs as the
    // logits layer of an MLP-layout block of shape st = (A, E, t, 128), the rest of it zero and
    // never read
    float *blk = ar.alloc<float>(c.st.count());
    float *y = c.st_arch == 2 ? ar.alloc<float>((size_t)c.st.t * 2 * c.gru_hg * NL) : nullptr;
    if (ar.failed) return PMKLC_ENOMEM;
    const GruOff o = gru_offsets(c.A(), c.st.E, c.gru_hg, c.st_arch);
    cudaMemsetAsync(blk, 0, sizeof(float) * c.st.count(), ar.st);
    cudaMemcpyAsync(blk + c.st.off_w2(), d_static + o.w4, sizeof(float) * (size_t)kGruDense * c.A(),
                    cudaMemcpyDeviceToDevice, ar.st);
    cudaMemcpyAsync(blk + c.st.off_b2(), d_static + o.b4, sizeof(float) * (size_t)c.A(), cudaMemcpyDeviceToDevice,
                    ar.st);
    p.st_gru = d_static;
    p.gru_hg = c.gru_hg;
    p.gru_layers = c.st_arch;
    p.gru_y = y;
    p.static_params = blk;
    d_static = blk;  // the BF16 copy below is the block's
  }
  p.precision = c.precision;
  p.wbf = nullptr;
  p.static_bf = nullptr;
  p.st8 = nullptr;
  p.st8_c1 = p.st8_s2 = nullptr;
  p.hs_rowmax = nullptr;
  if (bf_form(c.precision)) {
    p.wbf = ar.alloc<__nv_bfloat16>(G * p.P);
    if (c.use_static && d_static && f8_form(c.precision)) {
      // the frozen static model in E4M3 with per-channel scales (fp8static.cu); the FP8-hidden
      // form keeps a BF16 copy for its logits layer instead of the FP8 activations' row maxima
      const bool hidden_only = c.precision == PMKLC_BF16_FP8HIDDEN;
      uint8_t *codes = ar.alloc<uint8_t>(fp8_code_bytes(c.st));
      float *scales = ar.alloc<float>(fp8_scale_count(c.st));
      float *c1 = ar.alloc<float>(c.st.H);
      unsigned *rmax = hidden_only ? nullptr : ar.alloc<unsigned>(NL);
      __nv_bfloat16 *sb = hidden_only ? ar.alloc<__nv_bfloat16>(c.st.count()) : nullptr;
      if (ar.failed) return PMKLC_ENOMEM;
      launch_quantize_fp8(d_static, c.st, codes, scales, ar.st);
      launch_fp8_hidden_scale(scales, c.st, c1, ar.st);
      if (rmax) cudaMemsetAsync(rmax, 0, sizeof(unsigned) * NL, ar.st);
      if (sb) launch_to_bf16(d_static, sb, c.st.count(), ar.st);
      p.st8 = codes;
      p.st8_c1 = c1;
      p.st8_s2 = scales + 1 + c.st.H;
      p.hs_rowmax = rmax;
      p.static_bf = sb;
    } else if (c.use_static && d_static) {
      __nv_bfloat16 *sb = ar.alloc<__nv_bfloat16>(c.st.count());
      if (sb) launch_to_bf16(d_static, sb, c.st.count(), ar.st);
      p.static_bf = sb;
    }
  }
  int A = c.A();
  p.hd = ar.alloc<float>(NL * c.dm.H);
  p.hs = c.use_static ? ar.alloc<float>(NL * c.st.H) : nullptr;
  p.zm = ar.alloc<float>(NL * A);
  p.zu = c.use_static ? ar.alloc<float>(NL * A) : nullptr;
  p.dz = ar.alloc<float>(NL * A);
  p.dh = ar.alloc<float>(NL * c.dm.H);
  p.dalpha_row = ar.alloc<float>(NL);
  p.out_P = nullptr;
  p.hd_b = p.hs_b = p.dz_b = p.dh_b = nullptr;
  p.hpart = nullptr;
  if (bf_form(c.precision)) {
    int hmax = std::max(c.dm.H, c.use_static ? c.st.H : 0);
    p.hpart = ar.alloc<float>((size_t)2 * kHiddenSplit * NL * hmax);  // 2 models x K-slices
    p.hd_b = ar.alloc<__nv_bfloat16>(NL * c.dm.H);
    p.hs_b = c.use_static ? ar.alloc<__nv_bfloat16>(NL * c.st.H) : nullptr;
    p.dz_b = ar.alloc<__nv_bfloat16>(NL * A);
    p.dh_b = ar.alloc<__nv_bfloat16>(NL * c.dm.H);
  }
  p.demb_acc = nullptr;
  p.dx_rows = nullptr;
  p.emb_pairs = nullptr;
  p.emb_bin_off = nullptr;
  p.err = ar.alloc<int>(1);
  std::vector<float> bc1(R.S.max_tau + 2), bc2(R.S.max_tau + 2);
  for (size_t t = 0; t < bc1.size(); ++t) {
    bc1[t] = (float)(1.0 - pow(0.9, (double)t));
    bc2[t] = (float)(1.0 - pow(0.999, (double)t));
  }
  p.bc1 = ar.upload(bc1);
  p.bc2 = ar.upload(bc2);
  // SMP hand-over pairs by start step
  std::vector<int> flat;
  R.pair_off.assign(R.S.T_total + 2, 0);
  for (int T = 0; T <= R.S.T_total; ++T) {
    R.pair_off[T] = (int)flat.size() / 2;
    flat.insert(flat.end(), R.S.pairs_at[T].begin(), R.S.pairs_at[T].end());
  }
  R.pair_off[R.S.T_total + 1] = (int)flat.size() / 2;
  R.d_pairs = ar.upload(flat);
  if (ar.failed) return PMKLC_ENOMEM;
  // the FP8 static model runs on the tcgen05 engine only (no mma.sync form of it)
  if (p.st8 && !tc_supported(p)) return PMKLC_EINVAL;
  // BF16 forms with small embedding tables: per-tile FP32 partials of the embedding gradient
  p.demb_part = nullptr;
  p.dx_np = p.dx_ct = 0;
  if (bf_form(c.precision)) {
    int ct = 0;
    const int np = dx_partials(p, &ct);
    if (np > 0) {
      p.demb_part = ar.alloc<float>(G * (size_t)np * A * c.dm.E);
      if (ar.failed) return PMKLC_ENOMEM;
      p.dx_np = np, p.dx_ct = ct;
    } else if (const int nb = dx_rows_bins(p)) {  // large tables on tcgen05: dX rows, summed per range of table rows
      p.dx_rows = ar.alloc<float>(NL * (size_t)c.dm.K1());
      p.emb_pairs = ar.alloc<uint32_t>(NL * (size_t)c.dm.t);
      p.emb_bin_off = ar.alloc<int>(G * (size_t)(nb + 1));
      if (ar.failed) return PMKLC_ENOMEM;
    }
  }
  // the other forms add the embedding gradient into fixed-point accumulators (zeroed below)
  if (!p.demb_part && !p.dx_rows) {
    p.demb_acc = ar.alloc<long long>(G * A * c.dm.E);
    if (ar.failed) return PMKLC_ENOMEM;
  }
  p.tile_cap = c.gemm_tiles == 1 ? 128 : c.gemm_tiles == 2 ? 64 : 0;
  // BF16 forms on the tcgen05 engine update W1 and W2 in their gradient GEMMs' epilogues when those
  // GEMMs have enough tiles to keep every SM streaming optimiser state (at least 8 of dW2's
  // 128 x 128 tiles per SM); with fewer, the full-grid streaming optimiser is faster.  Both apply the
  // same explicitly rounded rule to the same FP32 gradients: the results are identical either way.
  const long long w2_tiles = (long long)L.G * ((c.dm.H + 127) / 128) * ((c.dm.A + 127) / 128);
  const bool fuse = c.update_path == PMKLC_UPDATE_FUSED || (c.update_path == PMKLC_UPDATE_AUTO && w2_tiles >= 8LL * 152);
  p.fused_w = bf_form(c.precision) && fuse && tc_supported(p) ? 1 : 0;
  if (p.demb_acc) cudaMemsetAsync(p.demb_acc, 0, sizeof(long long) * G * A * c.dm.E, ar.st);
  // the mixer writes a row's dz only inside the coded slice (overlap masking) and clears the
  // previous one, so every row starts at zero
  if (p.dz_b)
    cudaMemsetAsync(p.dz_b, 0, sizeof(__nv_bfloat16) * NL * A, ar.st);
  else
    cudaMemsetAsync(p.dz, 0, sizeof(float) * NL * A, ar.st);
  cudaMemsetAsync(p.err, 0, sizeof(int), ar.st);
  std::vector<float> init;
  if (R.init_host)
    init.assign(R.init_host, R.init_host + c.dm.count());
  else
    init_params(c.dm, c.seed, init);
  float *d_init = ar.upload(init);
  if (ar.failed) return PMKLC_ENOMEM;
  launch_init_groups(p, d_init, c.alpha0, ar.st);
  if (p.wbf) launch_to_bf16(p.params, p.wbf, G * p.P, ar.st);
  return PMKLC_OK;
}

// The lockstep loop over global steps.
void run_steps(Run &R, const std::vector<int> &grp_mode, cudaStream_t st) {
  const Layout &L = R.L;
  const Schedule &S = R.S;
  const int t_eff = R.p.t_eff;
  // auxiliary streams: the count model beside the network's forward, the three gradient GEMMs side
  // by side, and (BF16 forms) the static model's forward of step T + 1 beside the backward and the
  // optimiser of step T (it reads only tokens decoded by step T), joined by events before the
  // kernels that read their results
  StepStreams ss;
  bool use_ss = !prof_enabled();
  for (auto &a : ss.aux) use_ss = use_ss && cudaStreamCreateWithFlags(&a, cudaStreamNonBlocking) == cudaSuccess;
  for (cudaEvent_t *e : {&ss.fork, &ss.join[0], &ss.join[1], &ss.count_done, &ss.mix_done, &ss.static_done})
    use_ss = use_ss && cudaEventCreateWithFlags(e, cudaEventDisableTiming) == cudaSuccess;
  if (!use_ss) cudaGetLastError();  // fall back to the caller's stream alone
  // per global step: does any group predict (and so run the network's forward)?
  std::vector<char> pred_at(S.T_total + 1, 0);
  for (int g = 0; g < L.G; ++g)
    for (int j = t_eff; j < L.steps[g]; ++j) pred_at[S.start[g] + j] = 1;
  // rows predicted and groups trained at a global step (the profiler's work figures)
  auto work_at = [&](int T) {
    StepWork w{0.0, 0.0};
    for (int g = 0; g < L.G; ++g) {
      const int j = T - S.start[g];
      if (j < t_eff || j >= L.steps[g]) continue;
      const int M = L.lane_off[g + 1] - L.lane_off[g];
      w.pred_rows += j < L.base_len[g] ? M : (j == L.base_len[g] ? L.extra[g] : 0);
      w.train_groups += 1;
    }
    return w;
  };
  const bool bf = bf_form(R.p.precision);
  // kernels of one backward + update: dh, the bias sums, dW2, dX (+ the embedding sum of stored dX
  // rows, listed first by table-row range), dW1 and the optimiser on tcgen05; dh, dW2, dX, dW1 and
  // the optimiser otherwise
  const int bwd_launches = bf && tc_supported(R.p) ? (R.p.dx_rows ? 8 : 6) : 5;
  const bool split_static = R.net && use_ss && bf && R.p.use_static && tc_supported(R.p);
  int static_for = -1;  // the step whose static forward is already queued on ss.aux[2]
  for (int T = 0; T < S.T_total; ++T) {
    int np = R.pair_off[T + 1] - R.pair_off[T];
    if (np > 0) {
      launch_smp_copy(R.p, R.d_pairs + 2 * R.pair_off[T], np, st);
      R.launches++;
    }
    bool any_pred = false, any_code = false, any_count = false;
    for (int g = 0; g < L.G; ++g) {
      int j = T - S.start[g];
      if (j < 0 || j >= L.steps[g]) continue;
      if (j >= t_eff) any_pred = true;
      if (grp_mode[g] != kReplay) any_code = true;
      if (!R.cmode.empty() && R.cmode[g]) any_count = true;
    }
    const StepWork w = work_at(T);
    prof_step(T, w);
    const bool net = R.net && (any_pred || any_code);
    if (any_count) {
      // a count-decoded token is the network's target at this step: joined before the mixer
      cudaStream_t cs = st;
      if (use_ss && net) {
        cudaEventRecord(ss.fork, st);
        cudaStreamWaitEvent(ss.aux[0], ss.fork, 0);
        cs = ss.aux[0];
      }
      launch_count_step(R.p, R.cp, T, cs);
      if (cs != st) cudaEventRecord(ss.count_done, cs);
      R.launches++;
    }
    if (!R.net) continue;
    if (any_pred) {
      if (split_static) {
        if (static_for != T) {  // not queued by the previous step (the first predicting step)
          cudaEventRecord(ss.fork, st);
          cudaStreamWaitEvent(ss.aux[2], ss.fork, 0);
          launch_forward_bf16(R.p, T, ss.aux[2], kFwdStatic);
          cudaEventRecord(ss.static_done, ss.aux[2]);
          R.launches += 2;
        }
        launch_forward_bf16(R.p, T, st, kFwdDynamic);
        cudaStreamWaitEvent(st, ss.static_done, 0);
        R.launches += 2;
      } else if (bf) {
        launch_forward_bf16(R.p, T, st);
        R.launches += 2;
      } else {
        launch_forward(R.p, T, st);
        R.launches += R.c.use_static ? 4 : 2;
      }
    }
    if (any_count && use_ss && net) cudaStreamWaitEvent(st, ss.count_done, 0);
    if (any_pred || any_code) {
      launch_mixcode(R.p, T, st);
      R.launches++;
    }
    // static forward of the next step (BF16 forms): its contexts are decoded by now and the mixer
    // has read this step's static logits; queued once this step's gradient GEMMs are done, so it
    // shares the SMs with the HBM-bound optimiser rather than with the latency-bound GEMMs
    auto queue_static_next = [&]() {
      if (!(split_static && T + 1 < S.T_total && pred_at[T + 1])) return;
      cudaEventRecord(ss.mix_done, st);
      cudaStreamWaitEvent(ss.aux[2], ss.mix_done, 0);
      prof_step(T + 1, work_at(T + 1));
      launch_forward_bf16(R.p, T + 1, ss.aux[2], kFwdStatic);
      prof_step(T, w);
      cudaEventRecord(ss.static_done, ss.aux[2]);
      static_for = T + 1;
      R.launches += 2;
    };
    if (any_pred) {
      if (bf) {
        launch_backward_bf16(R.p, T, st, use_ss ? &ss : nullptr);
        queue_static_next();
        launch_update(R.p, T, st);
      } else {
        launch_backward_update(R.p, T, st);
      }
      R.launches += bwd_launches;
    } else {
      queue_static_next();
    }
  }
  prof_stop_sampling();
  if (use_ss)
    for (auto &a : ss.aux) cudaStreamSynchronize(a);
  for (auto &a : ss.aux)
    if (use_ss) cudaStreamDestroy(a);
  if (use_ss)
    for (cudaEvent_t e : {ss.fork, ss.join[0], ss.join[1], ss.count_done, ss.mix_done, ss.static_done})
      cudaEventDestroy(e);
}

__global__ void gather_kernel(const unsigned long long *seg, int n_seg, const uint8_t *src0, const uint8_t *src1,
                              uint8_t *dst) {
  int q = blockIdx.x;
  if (q >= n_seg) return;
  unsigned long long so = seg[4 * q], dof = seg[4 * q + 1], len = seg[4 * q + 2], which = seg[4 * q + 3];
  const uint8_t *s = (which ? src1 : src0) + so;
  for (unsigned long long i = threadIdx.x; i < len; i += blockDim.x) dst[dof + i] = s[i];
}

__global__ void check_tokens_kernel(const uint16_t *tok, long long n, int A, int *err) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  bool bad = i < n && tok[i] >= A;
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(err, kErrCorrupt);
}

int err_to_rc(int e) {
  if (e & kErrBadBase) return PMKLC_EINVAL;
  if (e & kErrCorrupt) return PMKLC_ECORRUPT;
  if (e & kErrTimeout) return PMKLC_ETIMEOUT;
  if (e & kErrOverflow) return PMKLC_ENOSPC;
  return PMKLC_OK;
}

// The Model Selector (§4.2.1): the static private model for inputs above 500 MB (5e8 bases), or
// above the configured threshold
bool private_selected(const Cfg &c, unsigned long long n) {
  return c.priv == 1 || (c.priv == 2 && n > (c.priv_threshold ? c.priv_threshold : 500000000ull));
}

// float32 rounded to the nearest BF16 (ties to even), as float32
float bf16_round_host(float x) {
  uint32_t u;
  memcpy(&u, &x, 4);
  u = (u + 0x7FFFu + ((u >> 16) & 1u)) & 0xFFFF0000u;
  float y;
  memcpy(&y, &u, 4);
  return y;
}

size_t bound_of(const std::vector<unsigned long long> &lens, const Cfg &c) {
  size_t b = kHeader;
  unsigned long long n_all = 0;
  for (unsigned long long n : lens) n_all += n;
  if (private_selected(c, n_all)) b += 2 * c.st.count();  // the stored private model, BF16
  for (unsigned long long n : lens) {
    long long l = n_tokens_of((long long)n, c.s, c.k);
    long long Mb = lanes_of(l, c.lanes, c.lane_tokens);
    // a lane's stream: the network's at most 3 bytes per token + 8 (24-bit totals); the count
    // model's at most 2 bytes per base + 8 (totals below 2^13), which only the count-only form
    // (fallback 2) stores unconditionally; the judge keeps it only when it is the smaller
    size_t stream = (size_t)l * 3 + (size_t)Mb * 8;
    if (c.fallback == 2)
      stream = 2 * ((size_t)c.k * Mb + (size_t)c.s * (size_t)(l - Mb)) + (size_t)Mb * 8;
    b += 10 + 1 + 2 + (size_t)Mb * 10 + stream;
  }
  return b;
}

// ---------------------------------------------------------------- pre-training

// The dynamic-model loop over device bases without coding (the pre-training of a static model,
// §4(b)): the n bases are tokenised and cut into c.lanes lanes; `epochs` passes are consecutive
// groups chained with f = 1, each continuing from the previous one's state; the last state's
// parameters go to out (host).  init: the starting parameters (host), else the seeded init.
// Without a static model Eq. (1) forms the logits (1 - alpha) L^m, and alpha trains with the
// weights: only the product is determined, and the pair drifts along (alpha, L^m) -> (alpha',
// L^m (1 - alpha) / (1 - alpha')).  So the final (1 - alpha) goes into the returned logits layer
// (W2 and b2, in FP32): the returned predictor alone computes the logits the training fitted.
// alpha starts at c.alpha0 from the seeded init, and at 0 from a given predictor (init), whose
// logits the training then starts from as they are.
int train_dev(const Cfg &c, const uint8_t *d_seq, size_t n, uint32_t epochs, const float *init, float *out,
              cudaStream_t st) {
  if (c.use_static || !out || (n && !d_seq) || epochs < 1 || epochs > kMaxGroups) return PMKLC_EINVAL;
  Run R;
  R.c = c;
  if (init) R.c.alpha0 = 0.f;
  R.init_host = init;
  std::vector<unsigned long long> lens(epochs, (unsigned long long)n);
  if (!layout_fits(lens, c, PMKLC_SMP_CHAIN, 1.0f)) return PMKLC_EINVAL;
  make_layout(lens, c.s, c.k, c.lanes, c.lane_tokens, R.L);
  make_schedule(R.L, PMKLC_SMP_CHAIN, 1.0f, c.t_eff(), R.S);
  Arena ar(st);
  uint16_t *d_tokens = ar.alloc<uint16_t>(R.L.n_tok);
  if (ar.failed) return PMKLC_ENOMEM;
  // every epoch reads the same bases: tokenised once as one block, copied to the other epochs
  const std::vector<long long> one_off = {0, (long long)n}, tok_one = {0, R.L.tok_off[1]};
  const std::vector<int> one_cta = tokenize_ctas(one_off);
  long long *d_one_off = ar.upload(one_off);
  long long *d_tok_one = ar.upload(tok_one);
  int *d_one_cta = ar.upload(one_cta);
  std::vector<int> grp_mode(R.L.G, kReplay);
  R.p.tokens = d_tokens;
  R.p.lane_buf = nullptr;
  std::vector<unsigned long long> zoff(std::max(R.L.NL, 1), 0);
  std::vector<uint32_t> zcap(std::max(R.L.NL, 1), 0);
  R.p.lane_buf_off = ar.upload(zoff);
  R.p.lane_buf_cap = ar.upload(zcap);
  if (ar.failed) return PMKLC_ENOMEM;
  int rc = setup_run(ar, R, grp_mode, nullptr);
  if (rc) return rc;
  launch_validate_tokenize(d_seq, n, d_one_off, d_tok_one, d_one_cta, 1, one_cta[1], c.s, c.k, d_tokens, R.p.err,
                           st);
  for (int g = 1; g < R.L.G; ++g)  // identical tokens for every epoch
    cudaMemcpyAsync(d_tokens + R.L.tok_off[g], d_tokens, sizeof(uint16_t) * (size_t)R.L.tok_off[1],
                    cudaMemcpyDeviceToDevice, st);
  run_steps(R, grp_mode, st);
  int h_err = 0;
  float alpha = 0.f;
  cudaMemcpyAsync(&h_err, R.p.err, sizeof(int), cudaMemcpyDeviceToHost, st);
  const int last = R.L.G - 1;
  cudaMemcpyAsync(out, R.p.params + (size_t)last * R.p.P, sizeof(float) * R.p.P, cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(&alpha, R.p.alpha + last, sizeof(float), cudaMemcpyDeviceToHost, st);
  PMKLC_CUDA_TRY(cudaStreamSynchronize(st));
  PMKLC_CUDA_TRY(cudaGetLastError());
  if (h_err) return err_to_rc(h_err);
  const float keep = 1.f - alpha;
  for (size_t i = c.dm.off_w2(); i < c.dm.count(); ++i) out[i] *= keep;
  return PMKLC_OK;
}

// The static private model of a compression (§4.2.3): a model of the static shape pre-trained on
// the input's head, starting from the public static model when one is given (the two share
// structure and parameters), else from the seeded init; returned rounded to BF16.
int pretrain_private(const Cfg &c, const pmklc_model_cfg *cfg, const uint8_t *d_seq, size_t n, cudaStream_t st,
                     std::vector<float> &w) {
  Cfg tc = c;
  tc.use_static = 0, tc.priv = 0, tc.fallback = 0;
  tc.dm = c.st;
  const size_t n_train = c.priv_bases ? (size_t)std::min<unsigned long long>(c.priv_bases, n) : n;
  std::vector<float> init;
  if (c.use_static)
    init.assign(cfg->static_weights, cfg->static_weights + c.st.count());
  else
    init_params(c.st, c.seed, init);
  w.assign(c.st.count(), 0.f);
  int rc = train_dev(tc, d_seq, n_train, (uint32_t)c.priv_epochs, init.data(), w.data(), st);
  if (rc) return rc;
  for (float &x : w) x = bf16_round_host(x);
  return PMKLC_OK;
}

// ---------------------------------------------------------------- compress

int compress_dev_impl(const uint8_t *d_seq, size_t n, const uint64_t *block_lens, size_t n_blocks,
                      const pmklc_model_cfg *cfg, cudaStream_t st, uint8_t *d_out, size_t out_cap, size_t *out_len) {
  auto t0 = std::chrono::steady_clock::now();
  Run R;
  int rc = check_cfg(cfg, R.c);
  if (rc) return rc;
  const Cfg &c = R.c;
  if ((n && !d_seq) || (n_blocks && !block_lens) || !out_len || !d_out) return PMKLC_EINVAL;
  if (n_blocks > kMaxGroups) return PMKLC_EINVAL;
  std::vector<unsigned long long> lens(block_lens, block_lens + n_blocks);
  unsigned long long sum = 0;
  for (auto x : lens) sum += x;
  if (sum != n || !layout_fits(lens, c, c.smp_mode, c.smp_f)) return PMKLC_EINVAL;
  if (out_cap < bound_of(lens, c)) return PMKLC_ENOSPC;
  // Model Selector (§4.2.1): a static private model (§4.2.3) pre-trained on the input takes the
  // static slot of Eq. (1); its BF16 values are what both sides use
  std::vector<float> priv_w;
  const bool priv = private_selected(c, n);
  if (priv) {
    rc = pretrain_private(c, cfg, d_seq, n, st, priv_w);
    if (rc) return rc;
    R.c.use_static = 1;
  }
  make_layout(lens, c.s, c.k, c.lanes, c.lane_tokens, R.L);
  make_schedule(R.L, c.smp_mode, c.smp_f, c.t_eff(), R.S);
  const Layout &L = R.L;
  Arena ar(st);
  // static weights
  const float *d_static = nullptr;
  uint64_t shash = 0;
  if (c.use_static) {
    size_t cnt = c.static_count();
    const float *sw = priv ? priv_w.data() : cfg->static_weights;
    shash = fnv1a(sw, cnt * sizeof(float));
    float *d = ar.alloc<float>(cnt);
    if (!d) return PMKLC_ENOMEM;
    cudaMemcpyAsync(d, sw, cnt * sizeof(float), cudaMemcpyHostToDevice, st);
    d_static = d;
  }
  std::vector<int> grp_mode(L.G, kEncode);
  long long *d_base_off = ar.upload(L.base_off);
  long long *d_tok_off = ar.upload(L.tok_off);
  const std::vector<int> tok_cta = tokenize_ctas(L.base_off);
  int *d_tok_cta = ar.upload(tok_cta);
  uint16_t *d_tokens = ar.alloc<uint16_t>(L.n_tok);
  uint8_t *d_tail = ar.alloc<uint8_t>((size_t)L.G * 8);
  // lane output buffers: cap = 3 len + 8 (at most 3 byte shifts per symbol + flush)
  std::vector<unsigned long long> lane_off(L.NL + 1, 0);
  std::vector<uint32_t> lane_cap(L.NL);
  for (int r = 0; r < L.NL; ++r) {
    lane_cap[r] = (uint32_t)(3ull * L.lane_len[r] + 8);
    lane_off[r + 1] = lane_off[r] + ((lane_cap[r] + 15) & ~15u);
  }
  uint8_t *d_lane_buf = ar.alloc<uint8_t>(lane_off[L.NL]);
  R.p.lane_buf = d_lane_buf;
  R.p.lane_buf_off = ar.upload(lane_off);
  R.p.lane_buf_cap = ar.upload(lane_cap);
  R.p.enc = ar.alloc<EncState>(L.NL);
  R.p.dec = nullptr;
  R.p.tokens = d_tokens;
  uint32_t *d_lane_len = ar.alloc<uint32_t>(L.NL);
  if (ar.failed) return PMKLC_ENOMEM;
  rc = setup_run(ar, R, grp_mode, d_static);
  if (rc) return rc;
  prof_step(0, StepWork{0.0, 0.0});
  {
    ProfScope ps("validate_tokenize", 0, 1.0 * n + 2.0 * L.n_tok, st);
    launch_validate_tokenize(d_seq, n, d_base_off, d_tok_off, d_tok_cta, L.G, tok_cta[L.G], c.s, c.k, d_tokens,
                             R.p.err, st);
  }
  launch_tails(d_seq, d_base_off, d_tok_off, L.G, c.s, c.k, d_tail, st);
  // count model (judge / fallback): same lanes, coded inside the same steps
  R.net = c.fallback != 2;
  std::vector<unsigned long long> cnt_off(L.NL + 1, 0);
  std::vector<uint32_t> cnt_len(L.NL, 0);
  uint8_t *d_cnt_buf = nullptr;
  uint32_t *d_cnt_len = nullptr;
  if (c.fallback) {
    if (L.Mmax > 1024) return PMKLC_EINVAL;
    R.cmode.assign(L.G, 1);
    std::vector<uint32_t> cap(L.NL);
    for (int r = 0; r < L.NL; ++r) {  // at most 15 bits per base
      cap[r] = (uint32_t)(2ull * (c.k + (unsigned long long)c.s * (L.lane_len[r] - 1)) + 8);
      cnt_off[r + 1] = cnt_off[r] + ((cap[r] + 15) & ~15u);
    }
    if (setup_count(ar, R)) return PMKLC_ENOMEM;
    d_cnt_buf = ar.alloc<uint8_t>(cnt_off[L.NL]);
    R.cp.buf = d_cnt_buf;
    R.cp.buf_off = ar.upload(cnt_off);
    R.cp.buf_cap = ar.upload(cap);
    d_cnt_len = ar.alloc<uint32_t>(L.NL);
    if (ar.failed) return PMKLC_ENOMEM;
    launch_count_init(R.p, R.cp, 1, st);
  }
  if (R.net) launch_coder_init(R.p, 1, st);
  run_steps(R, grp_mode, st);
  if (R.net) launch_coder_finish(R.p, d_lane_len, st);
  if (c.fallback) launch_count_finish(R.p, R.cp, d_cnt_len, st);
  // results to the host
  std::vector<uint32_t> lane_len(L.NL, 0);
  std::vector<uint8_t> tails((size_t)L.G * 8);
  int h_err = 0;
  if (L.NL && R.net) cudaMemcpyAsync(lane_len.data(), d_lane_len, sizeof(uint32_t) * L.NL, cudaMemcpyDeviceToHost, st);
  if (L.NL && d_cnt_len)
    cudaMemcpyAsync(cnt_len.data(), d_cnt_len, sizeof(uint32_t) * L.NL, cudaMemcpyDeviceToHost, st);
  if (L.G) cudaMemcpyAsync(tails.data(), d_tail, tails.size(), cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(&h_err, R.p.err, sizeof(int), cudaMemcpyDeviceToHost, st);
  PMKLC_CUDA_TRY(cudaStreamSynchronize(st));
  PMKLC_CUDA_TRY(cudaGetLastError());
  if (h_err) return err_to_rc(h_err);
  uint32_t crc = 0;
  rc = crc32_device(d_seq, n, &crc, st);
  if (rc) return rc;
  // container
  std::vector<uint8_t> H;
  H.reserve(kHeader + (size_t)L.G * 16 + (size_t)L.NL * 3);
  H.insert(H.end(), {'P', 'M', 'K', 'L'});
  uint8_t flags = (uint8_t)((c.use_static ? 1 : 0) | (c.fallback << 1) | (priv ? kPrivateFlag : 0) | (c.st_arch << 4));
  uint8_t b8[8] = {kVersion, (uint8_t)c.s, (uint8_t)c.k, flags, (uint8_t)c.precision, (uint8_t)c.optimizer,
                   (uint8_t)c.smp_mode, (uint8_t)c.count_order};
  H.insert(H.end(), b8, b8 + 8);
  put_le<uint16_t>(H, (uint16_t)c.dm.E);
  put_le<uint16_t>(H, (uint16_t)c.dm.t);
  put_le<uint16_t>(H, (uint16_t)c.dm.H);
  put_le<uint16_t>(H, (uint16_t)(c.use_static ? c.st.E : 0));
  put_le<uint16_t>(H, (uint16_t)(c.use_static ? c.st.t : 0));
  put_le<uint16_t>(H, (uint16_t)(c.use_static ? (c.st_arch ? c.gru_hg : c.st.H) : 0));  // BiGRU: its GRU width
  put_le<uint32_t>(H, (uint32_t)c.lanes);
  put_le<float>(H, c.lr);
  put_le<float>(H, c.alpha0);
  put_le<float>(H, c.smp_f);
  put_le<uint64_t>(H, c.seed);
  put_le<uint64_t>(H, shash);
  put_le<uint64_t>(H, (uint64_t)n);
  put_le<uint32_t>(H, (uint32_t)n_blocks);
  put_le<uint32_t>(H, crc);
  // variant: bit 0 overlap-masked coding; bits 8-9 the GEMM tile variant and bits 10-11 the update
  // path (kernel choices that leave every byte unchanged, kept so decoding runs the same kernels)
  put_le<uint32_t>(H, (c.mask ? 1u : 0u) | ((uint32_t)c.gemm_tiles << 8) | ((uint32_t)c.update_path << 10));
  put_le<uint32_t>(H, (uint32_t)c.lane_tokens);
  std::vector<unsigned long long> seg;  // (src, dst-relative, len, which)
  unsigned long long pay = 0;
  uint64_t n_net = 0, n_cnt = 0, net_bytes = 0, cnt_bytes = 0;
  for (int g = 0; g < L.G; ++g) {
    long long tl = tail_len_of((long long)lens[g], c.s, c.k);
    size_t tbytes = (size_t)(tl * 2 + 7) / 8;
    size_t net_cost = 0, cnt_cost = 0;
    for (int r = L.lane_off[g]; r < L.lane_off[g + 1]; ++r) {
      net_cost += lane_len[r] + varint_len(lane_len[r]);
      cnt_cost += cnt_len[r] + varint_len(cnt_len[r]);
    }
    bool use_cnt = c.fallback == 2 || (c.fallback == 1 && cnt_cost < net_cost);
    net_bytes += c.fallback == 2 ? 0 : net_cost;
    cnt_bytes += c.fallback == 0 ? 0 : cnt_cost;
    put_varint(H, lens[g]);
    H.push_back(use_cnt ? 1 : 0);
    uint8_t tb[2] = {0, 0};
    for (long long i = 0; i < tl; ++i) tb[i >> 2] |= (uint8_t)(tails[(size_t)g * 8 + i] << (2 * (i & 3)));
    H.insert(H.end(), tb, tb + tbytes);
    for (int r = L.lane_off[g]; r < L.lane_off[g + 1]; ++r) {
      uint32_t ln = use_cnt ? cnt_len[r] : lane_len[r];
      put_varint(H, ln);
      if (ln) seg.insert(seg.end(), {use_cnt ? cnt_off[r] : lane_off[r], pay, ln, use_cnt ? 1ull : 0ull});
      pay += ln;
    }
    (use_cnt ? n_cnt : n_net)++;
  }
  for (float x : priv_w) {  // the private model's BF16 bits follow the block records
    uint32_t u;
    memcpy(&u, &x, 4);
    put_le<uint16_t>(H, (uint16_t)(u >> 16));
  }
  size_t total = H.size() + pay;
  if (total > out_cap) return PMKLC_ENOSPC;
  for (size_t q = 0; q < seg.size(); q += 4) seg[q + 1] += H.size();
  cudaMemcpyAsync(d_out, H.data(), H.size(), cudaMemcpyHostToDevice, st);
  int n_seg = (int)(seg.size() / 4);
  if (n_seg) {
    unsigned long long *d_seg = ar.upload(seg);
    if (!d_seg) return PMKLC_ENOMEM;
    gather_kernel<<<n_seg, 128, 0, st>>>(d_seg, n_seg, d_lane_buf, d_cnt_buf, d_out);
  }
  PMKLC_CUDA_TRY(cudaStreamSynchronize(st));
  PMKLC_CUDA_TRY(cudaGetLastError());
  *out_len = total;
  g_stats.net_blocks = n_net;
  g_stats.count_blocks = n_cnt;
  g_stats.net_bytes = net_bytes;
  g_stats.count_bytes = cnt_bytes;
  g_stats.global_steps = (uint64_t)R.S.T_total;
  g_stats.kernel_launches = R.launches;
  g_stats.ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return PMKLC_OK;
}

// ---------------------------------------------------------------- decompress

struct Parsed {
  Cfg c;
  uint64_t shash = 0, n = 0;
  uint32_t n_blocks = 0, crc = 0;
  std::vector<unsigned long long> lens;
  std::vector<int> mode;                 // per block
  std::vector<uint8_t> tails;            // per block x 8 codes
  std::vector<std::vector<uint64_t>> sizes;  // per block: lane sizes or {count size}
  size_t header_len = 0;
  unsigned long long payload = 0;
  bool priv = false;            // a static private model is stored after the block records
  std::vector<float> priv_w;    // its values (BF16, widened)
};

int parse_fixed(const uint8_t *h, size_t len, Parsed &P) {
  if (len < kHeader || memcmp(h, "PMKL", 4) != 0 || h[4] != kVersion) return PMKLC_ECORRUPT;
  Cfg &c = P.c;
  c.s = h[5];
  c.k = h[6];
  c.use_static = h[7] & 1;
  c.precision = h[8];
  c.optimizer = h[9];
  c.smp_mode = h[10];
  c.count_order = h[11];
  c.fallback = (h[7] >> 1) & 3;
  P.priv = (h[7] & kPrivateFlag) != 0;
  if (P.priv && !c.use_static) return PMKLC_ECORRUPT;  // the private model takes the static slot
  c.st_arch = (h[7] >> 4) & 3;  // flags bits 4-5: the BiGRU static predictor's layers (0: the MLP)
  if ((h[7] & 0xC0) || c.st_arch == 3 || (c.st_arch && (!c.use_static || P.priv || h[8] > PMKLC_BF16_BATCHED)))
    return PMKLC_ECORRUPT;
  if (c.s < 1 || c.s > c.k || c.k > 8 || c.optimizer > 1 || c.smp_mode > 2 || c.count_order > 7 ||
      c.fallback > 2 || c.precision > PMKLC_BF16_FP8HIDDEN)
    return PMKLC_ECORRUPT;
  int A = 1 << (2 * c.k);
  c.dm = Dims{A, get_le<uint16_t>(h + 12), get_le<uint16_t>(h + 14), get_le<uint16_t>(h + 16)};
  c.st = Dims{A, get_le<uint16_t>(h + 18), get_le<uint16_t>(h + 20), get_le<uint16_t>(h + 22)};
  // the limits compression accepts (check_cfg): a header beyond them was not written by it, and
  // widths above 4096 would overflow the 32-bit row width t x E
  if (c.dm.E < 1 || c.dm.t < 1 || c.dm.H < 1 || c.dm.E > 4096 || c.dm.t > 4096) return PMKLC_ECORRUPT;
  if (c.use_static && (c.st.E < 1 || c.st.t < 1 || c.st.H < 1 || c.st.E > 4096 || c.st.t > 4096))
    return PMKLC_ECORRUPT;
  if (c.st_arch) {
    if (!gru_shape_ok(c.k, c.st.E, c.st.t, c.st.H, c.st_arch)) return PMKLC_ECORRUPT;
    c.gru_hg = c.st.H;
    c.st.H = kGruDense;
  }
  c.lanes = (int)get_le<uint32_t>(h + 24);
  if (c.lanes < 1 || c.lanes > (1 << 20)) return PMKLC_ECORRUPT;
  c.lr = get_le<float>(h + 28);
  c.alpha0 = get_le<float>(h + 32);
  c.smp_f = get_le<float>(h + 36);
  c.seed = get_le<uint64_t>(h + 40);
  P.shash = get_le<uint64_t>(h + 48);
  P.n = get_le<uint64_t>(h + 56);
  P.n_blocks = get_le<uint32_t>(h + 64);
  if (P.n_blocks > kMaxGroups) return PMKLC_ECORRUPT;
  P.crc = get_le<uint32_t>(h + 68);
  const uint32_t variant = get_le<uint32_t>(h + 72);
  c.mask = (int)(variant & 1u);
  c.gemm_tiles = (int)((variant >> 8) & 3u);
  c.update_path = (int)((variant >> 10) & 3u);
  if ((variant & ~0xF01u) || c.gemm_tiles > 2 || c.update_path > PMKLC_UPDATE_FUSED) return PMKLC_ECORRUPT;
  c.lane_tokens = (int)get_le<uint32_t>(h + 76);
  if (c.lane_tokens < 0) return PMKLC_ECORRUPT;
  if (!(c.smp_f >= 0.f && c.smp_f <= 1.f) || !(c.lr > 0.f) || !isfinite(c.lr) || !isfinite(c.alpha0))
    return PMKLC_ECORRUPT;
  if (P.n > (1ull << 56)) return PMKLC_ECORRUPT;  // keeps every length sum below 2^63
  return PMKLC_OK;
}

int parse_records(const uint8_t *h, size_t len, size_t in_len, Parsed &P) {
  const Cfg &c = P.c;
  size_t pos = kHeader;
  // a block record takes at least two bytes (its length and its mode): a count the input cannot
  // hold is corrupt, and is refused before any per-block allocation
  if (in_len < kHeader || P.n_blocks > (in_len - kHeader) / 2) return PMKLC_ECORRUPT;
  P.lens.resize(P.n_blocks);
  P.mode.resize(P.n_blocks);
  P.tails.assign((size_t)P.n_blocks * 8, 0);
  P.sizes.assign(P.n_blocks, {});
  unsigned long long sum = 0, pay = 0;
  for (uint32_t b = 0; b < P.n_blocks; ++b) {
    uint64_t nb;
    if (!get_varint(h, len, pos, nb) || nb > P.n - sum) return PMKLC_ECORRUPT;
    P.lens[b] = nb;
    sum += nb;
    if (pos >= len) return PMKLC_ECORRUPT;
    int mode = h[pos++];
    P.mode[b] = mode;
    if (mode > 1 || (mode == 0 && c.fallback == 2)) return PMKLC_ECORRUPT;
    long long tl = tail_len_of((long long)nb, c.s, c.k);
    size_t tbytes = (size_t)(tl * 2 + 7) / 8;
    if (pos + tbytes > len) return PMKLC_ECORRUPT;
    for (long long i = 0; i < tl; ++i) P.tails[(size_t)b * 8 + i] = (h[pos + (i >> 2)] >> (2 * (i & 3))) & 3;
    pos += tbytes;
    long long l = n_tokens_of((long long)nb, c.s, c.k);
    long long Mb = lanes_of(l, c.lanes, c.lane_tokens);
    for (long long r = 0; r < Mb; ++r) {
      uint64_t x;
      if (!get_varint(h, len, pos, x) || x > 0xFFFFFFFFull) return PMKLC_ECORRUPT;
      P.sizes[b].push_back(x);
      pay += x;
    }
  }
  if (sum != P.n || !layout_fits(P.lens, c, c.smp_mode, c.smp_f)) return PMKLC_ECORRUPT;
  if (P.priv) {  // the private model's BF16 values, checked against the header's hash
    const size_t cnt = c.st.count();
    if (pos > len || cnt > (len - pos) / 2) return PMKLC_ECORRUPT;
    P.priv_w.resize(cnt);
    for (size_t i = 0; i < cnt; ++i) {
      const uint32_t u = ((uint32_t)h[pos + 2 * i] | (uint32_t)h[pos + 2 * i + 1] << 8) << 16;
      memcpy(&P.priv_w[i], &u, 4);
    }
    pos += 2 * cnt;
    if (fnv1a(P.priv_w.data(), cnt * sizeof(float)) != P.shash) return PMKLC_ECORRUPT;
  }
  P.header_len = pos;
  P.payload = pay;
  if (pos + pay != in_len) return PMKLC_ECORRUPT;
  return PMKLC_OK;
}

int decompress_dev_impl(const uint8_t *d_in, size_t in_len, const float *static_weights, size_t static_count,
                        cudaStream_t st, uint8_t *d_seq, size_t seq_cap, size_t *n_out,
                        std::vector<unsigned long long> *lens_out) {
  auto t0 = std::chrono::steady_clock::now();
  if (!d_in || !n_out || in_len < kHeader) return in_len < kHeader ? PMKLC_ECORRUPT : PMKLC_EINVAL;
  Parsed P;
  std::vector<uint8_t> h(kHeader);
  PMKLC_CUDA_TRY(cudaMemcpyAsync(h.data(), d_in, kHeader, cudaMemcpyDeviceToHost, st));
  PMKLC_CUDA_TRY(cudaStreamSynchronize(st));
  int rc = parse_fixed(h.data(), kHeader, P);
  if (rc) return rc;
  // the block records end within n_blocks x (23 + 10 x lanes) bytes of the fixed header
  const size_t per_block = 23 + 10 * (size_t)P.c.lanes;
  size_t hl = in_len;
  if (P.n_blocks <= (in_len - kHeader) / per_block) {
    hl = std::min(in_len, kHeader + P.n_blocks * per_block);
    const size_t model = P.priv ? 2 * P.c.st.count() : 0;  // and the stored private model
    hl = model > in_len - hl ? in_len : hl + model;
  }
  h.resize(hl);
  PMKLC_CUDA_TRY(cudaMemcpyAsync(h.data(), d_in, hl, cudaMemcpyDeviceToHost, st));
  PMKLC_CUDA_TRY(cudaStreamSynchronize(st));
  rc = parse_records(h.data(), hl, in_len, P);
  if (rc) return rc;
  if (lens_out) *lens_out = P.lens;
  *n_out = (size_t)P.n;
  if (P.n > seq_cap || (P.n && !d_seq)) return PMKLC_ENOSPC;
  Run R;
  R.c = P.c;
  const Cfg &c = R.c;
  if (P.priv) {  // the container's own private model (any given static model is not used)
    static_weights = P.priv_w.data();
    static_count = P.priv_w.size();
  } else if (c.use_static) {
    if (!static_weights || static_count != c.static_count()) return PMKLC_EMODEL;
    if (fnv1a(static_weights, static_count * sizeof(float)) != P.shash) return PMKLC_EMODEL;
  }
  make_layout(P.lens, c.s, c.k, c.lanes, c.lane_tokens, R.L);
  make_schedule(R.L, c.smp_mode, c.smp_f, c.t_eff(), R.S);
  const Layout &L = R.L;
  Arena ar(st);
  const float *d_static = nullptr;
  if (c.use_static) {
    float *d = ar.alloc<float>(static_count);
    if (!d) return PMKLC_ENOMEM;
    cudaMemcpyAsync(d, static_weights, static_count * sizeof(float), cudaMemcpyHostToDevice, st);
    d_static = d;
  }
  std::vector<int> grp_mode(L.G), all_sel(L.G, 1);
  R.net = c.fallback != 2;
  R.cmode.assign(L.G, 0);
  bool any_cnt = false;
  for (int g = 0; g < L.G; ++g) {
    grp_mode[g] = P.mode[g] == 0 ? kDecode : kReplay;
    R.cmode[g] = P.mode[g] == 1 ? 2 : 0;
    any_cnt |= P.mode[g] == 1;
  }
  if (any_cnt && L.Mmax > 1024) return PMKLC_ECORRUPT;
  // every lane's payload (network or count model) at its offset from the payload start
  const uint8_t *d_pay = d_in + P.header_len;
  std::vector<unsigned long long> lane_off(std::max(L.NL, 1), 0);
  std::vector<uint32_t> lane_cap(std::max(L.NL, 1), 0);
  unsigned long long pos = 0;
  for (int g = 0; g < L.G; ++g)
    for (int r = L.lane_off[g], q = 0; r < L.lane_off[g + 1]; ++r, ++q) {
      lane_off[r] = pos;
      lane_cap[r] = (uint32_t)P.sizes[g][q];
      pos += P.sizes[g][q];
    }
  long long *d_base_off = ar.upload(L.base_off);
  long long *d_tok_off = ar.upload(L.tok_off);
  uint16_t *d_tokens = ar.alloc<uint16_t>(L.n_tok);
  uint8_t *d_tail = ar.upload(P.tails);
  int *d_all_sel = ar.upload(all_sel);
  R.p.lane_buf = const_cast<uint8_t *>(d_pay);
  R.p.lane_buf_off = ar.upload(lane_off);
  R.p.lane_buf_cap = ar.upload(lane_cap);
  R.p.enc = nullptr;
  R.p.dec = ar.alloc<DecState>(L.NL);
  R.p.tokens = d_tokens;
  if (ar.failed) return PMKLC_ENOMEM;
  rc = setup_run(ar, R, grp_mode, d_static);
  if (rc) return rc;
  if (any_cnt) {
    if (setup_count(ar, R)) return PMKLC_ENOMEM;
    R.cp.buf = const_cast<uint8_t *>(d_pay);
    R.cp.buf_off = R.p.lane_buf_off;
    R.cp.buf_cap = R.p.lane_buf_cap;
    launch_count_init(R.p, R.cp, 0, st);
  }
  if (R.net) launch_coder_init(R.p, 0, st);
  run_steps(R, grp_mode, st);
  launch_detokenize(d_tokens, d_tail, d_base_off, d_tok_off, d_all_sel, L.G, (long long)P.n, c.s, c.k, d_seq,
                    R.p.err, st);
  int h_err = 0;
  cudaMemcpyAsync(&h_err, R.p.err, sizeof(int), cudaMemcpyDeviceToHost, st);
  PMKLC_CUDA_TRY(cudaStreamSynchronize(st));
  PMKLC_CUDA_TRY(cudaGetLastError());
  if (h_err) return (h_err & kErrBadBase) ? PMKLC_ECORRUPT : err_to_rc(h_err);
  uint32_t crc = 0;
  rc = crc32_device(d_seq, (size_t)P.n, &crc, st);
  if (rc) return rc;
  if (crc != P.crc) return PMKLC_ECORRUPT;
  g_stats.net_bytes = g_stats.count_bytes = 0;  // a decompression codes nothing
  g_stats.global_steps = (uint64_t)R.S.T_total;
  g_stats.kernel_launches = R.launches;
  g_stats.ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return PMKLC_OK;
}

}  // namespace
}  // namespace pmklc

using namespace pmklc;

// Every C++ exception stops at the C boundary: a host allocation that fails (std::bad_alloc)
// becomes ENOMEM, anything else EINVAL (size_t results: 0).  Work already queued on the stream
// completes and the arena's stream-ordered frees follow it.
template <class R, class F>
R guarded(F &&f) {
  try {
    return f();
  } catch (const std::bad_alloc &) {
    return std::is_same<R, size_t>::value ? (R)0 : (R)PMKLC_ENOMEM;
  } catch (...) {
    return std::is_same<R, size_t>::value ? (R)0 : (R)PMKLC_EINVAL;
  }
}

extern "C" {

int pmklc_abi_version(void) { return PMKLC_ABI_VERSION; }

const char *pmklc_strerror(int rc) {
  switch (rc) {
    case PMKLC_OK: return "ok";
    case PMKLC_EINVAL: return "invalid argument";
    case PMKLC_ENOMEM: return "out of memory";
    case PMKLC_ECUDA: return "CUDA error";
    case PMKLC_ECORRUPT: return "corrupt compressed stream";
    case PMKLC_EMODEL: return "static model mismatch";
    case PMKLC_ETIMEOUT: return "device wait timed out";
    case PMKLC_ENOSPC: return "output buffer too small";
  }
  return "unknown error";
}

void pmklc_free(void *p) { free(p); }

// the widths a configuration accepts (check_cfg)
static bool widths_ok(uint32_t k, uint32_t emb, uint32_t ctx, uint32_t hid) {
  return k >= 1 && k <= 8 && emb >= 1 && emb <= 4096 && ctx >= 1 && ctx <= 4096 && hid >= 1 && hid <= 65535;
}

size_t pmklc_model_count(uint32_t k, uint32_t emb, uint32_t ctx, uint32_t hid) {
  if (!widths_ok(k, emb, ctx, hid)) return 0;
  Dims d{1 << (2 * (int)k), (int)emb, (int)ctx, (int)hid};
  return d.count();
}

void pmklc_default_cfg(pmklc_model_cfg *c, uint32_t s, uint32_t k, uint32_t emb, uint32_t ctx, uint32_t hid) {
  if (!c) return;
  memset(c, 0, sizeof(*c));
  c->struct_size = sizeof(*c);
  c->s = s;
  c->k = k;
  c->emb_d = emb;
  c->ctx_d = ctx;
  c->hid_d = hid;
  c->lanes_per_block = 64;
  c->precision = PMKLC_FP32_PLAIN;
  c->optimizer = PMKLC_ADAM;
  c->lr = 1e-3f;
  c->alpha_init = 0.5f;
  c->smp_mode = PMKLC_SMP_TREE;
  c->smp_fraction = 0.05f;
  c->count_order = 6;
  c->fallback = 1;
  c->seed = 42;
}

size_t pmklc_compress_bound(size_t n, const uint64_t *block_lens, size_t n_blocks, const pmklc_model_cfg *cfg) {
  return guarded<size_t>([&]() -> size_t {
    Cfg c;
    if (check_cfg(cfg, c) || (n_blocks && !block_lens) || n_blocks > kMaxGroups) return 0;
    std::vector<unsigned long long> lens(block_lens, block_lens + n_blocks);
    (void)n;
    if (!layout_fits(lens, c, c.smp_mode, c.smp_f)) return 0;
    return bound_of(lens, c);
  });
}

int pmklc_compress_dev(const uint8_t *d_seq, size_t n, const uint64_t *block_lens, size_t n_blocks,
                       const pmklc_model_cfg *cfg, void *stream, uint8_t *d_out, size_t out_cap, size_t *out_len) {
  return guarded<int>([&]() -> int {
    return compress_dev_impl(d_seq, n, block_lens, n_blocks, cfg, (cudaStream_t)stream, d_out, out_cap, out_len);
  });
}

int pmklc_autotune_lanes(const uint8_t *d_seq, size_t n, const uint64_t *block_lens, size_t n_blocks,
                         size_t sample_blocks, pmklc_model_cfg *cfg, const uint32_t *candidates, size_t n_candidates,
                         float max_rel_size, void *stream, uint64_t *sizes, float *ms) {
  return guarded<int>([&]() -> int {
    if (!cfg || !candidates || n_candidates == 0 || (n_blocks && !block_lens) || !(max_rel_size >= 0.f))
      return PMKLC_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    size_t nb = std::min(n_blocks, std::max<size_t>(sample_blocks, 1));
    size_t ns = 0;
    for (size_t b = 0; b < nb; ++b) ns += block_lens[b];
    if (ns > n) return PMKLC_EINVAL;
    pmklc_model_cfg trial = *cfg;
    size_t cap = 0;
    for (size_t i = 0; i < n_candidates; ++i) {
      trial.lanes_per_block = candidates[i];
      cap = std::max(cap, pmklc_compress_bound(ns, block_lens, nb, &trial));
    }
    if (cap == 0) return PMKLC_EINVAL;
    uint8_t *d_out = nullptr;
    PMKLC_CUDA_TRY(cudaMallocAsync((void **)&d_out, cap, st));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int rc = PMKLC_OK, best = -1;
    std::vector<uint64_t> sz(n_candidates, 0);
    std::vector<float> tm(n_candidates, 0.f);
    for (size_t i = 0; i < n_candidates && rc == PMKLC_OK; ++i) {
      trial.lanes_per_block = candidates[i];
      size_t len = 0;
      rc = compress_dev_impl(d_seq, ns, block_lens, nb, &trial, st, d_out, cap, &len);  // warm-up
      if (rc) break;
      cudaEventRecord(e0, st);
      rc = compress_dev_impl(d_seq, ns, block_lens, nb, &trial, st, d_out, cap, &len);
      cudaEventRecord(e1, st);
      cudaEventSynchronize(e1);
      cudaEventElapsedTime(&tm[i], e0, e1);
      sz[i] = len;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFreeAsync(d_out, st);
    cudaStreamSynchronize(st);
    if (rc) return rc;
    for (size_t i = 0; i < n_candidates; ++i) {
      bool ok = (double)sz[i] <= (double)sz[0] * (1.0 + (double)max_rel_size);
      if (ok && (best < 0 || tm[i] < tm[best])) best = (int)i;
    }
    cfg->lanes_per_block = candidates[best < 0 ? 0 : best];
    for (size_t i = 0; i < n_candidates; ++i) {
      if (sizes) sizes[i] = sz[i];
      if (ms) ms[i] = tm[i];
    }
    return PMKLC_OK;
  });
}

int pmklc_autotune_variant(const uint8_t *d_seq, size_t n, const uint64_t *block_lens, size_t n_blocks,
                           uint64_t head_bases, pmklc_model_cfg *cfg, const uint32_t *variants, size_t n_variants,
                           void *stream, float *ms) {
  return guarded<int>([&]() -> int {
    if (!cfg || !variants || n_variants == 0 || n_blocks == 0 || !block_lens || head_bases == 0 || (n && !d_seq))
      return PMKLC_EINVAL;
    for (size_t i = 0; i < n_variants; ++i)
      if ((variants[i] & 3u) > 2 || ((variants[i] >> 2) & 3u) > PMKLC_UPDATE_FUSED || variants[i] > 15u)
        return PMKLC_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    // the heads of every block, gathered into one device buffer (one copy per block)
    std::vector<uint64_t> heads(n_blocks);
    unsigned long long sum = 0, off = 0;
    for (size_t b = 0; b < n_blocks; ++b) {
      heads[b] = std::min<uint64_t>(block_lens[b], head_bases);
      sum += heads[b];
      off += block_lens[b];
    }
    if (off != n) return PMKLC_EINVAL;
    pmklc_model_cfg trial = *cfg;
    const size_t cap = pmklc_compress_bound(sum, heads.data(), n_blocks, &trial);
    if (cap == 0) return PMKLC_EINVAL;
    uint8_t *d_heads = nullptr, *d_out = nullptr;
    PMKLC_CUDA_TRY(cudaMallocAsync((void **)&d_heads, std::max<size_t>(sum, 1), st));
    if (cudaMallocAsync((void **)&d_out, cap, st) != cudaSuccess) {
      cudaFreeAsync(d_heads, st);
      return PMKLC_ENOMEM;
    }
    off = 0;
    unsigned long long dst = 0;
    for (size_t b = 0; b < n_blocks; ++b) {
      if (heads[b]) cudaMemcpyAsync(d_heads + dst, d_seq + off, heads[b], cudaMemcpyDeviceToDevice, st);
      dst += heads[b];
      off += block_lens[b];
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int rc = PMKLC_OK, best = -1;
    std::vector<float> tm(n_variants, 0.f);
    for (size_t i = 0; i < n_variants && rc == PMKLC_OK; ++i) {
      trial.gemm_tiles = variants[i] & 3u;
      trial.update_path = (variants[i] >> 2) & 3u;
      size_t len = 0;
      rc = compress_dev_impl(d_heads, sum, heads.data(), n_blocks, &trial, st, d_out, cap, &len);  // warm-up
      if (rc) break;
      cudaEventRecord(e0, st);
      rc = compress_dev_impl(d_heads, sum, heads.data(), n_blocks, &trial, st, d_out, cap, &len);
      cudaEventRecord(e1, st);
      cudaEventSynchronize(e1);
      cudaEventElapsedTime(&tm[i], e0, e1);
      if (best < 0 || tm[i] < tm[best]) best = (int)i;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFreeAsync(d_out, st);
    cudaFreeAsync(d_heads, st);
    cudaStreamSynchronize(st);
    if (rc) return rc;
    cfg->gemm_tiles = variants[best] & 3u;
    cfg->update_path = (variants[best] >> 2) & 3u;
    if (ms)
      for (size_t i = 0; i < n_variants; ++i) ms[i] = tm[i];
    return PMKLC_OK;
  });
}

int pmklc_decompress_dev(const uint8_t *d_in, size_t in_len, const float *static_weights, size_t static_count,
                         void *stream, uint8_t *d_seq, size_t seq_cap, size_t *n) {
  return guarded<int>([&]() -> int {
    return decompress_dev_impl(d_in, in_len, static_weights, static_count, (cudaStream_t)stream, d_seq, seq_cap, n,
                               nullptr);
  });
}

int pmklc_compress(const uint8_t *seq, size_t n, const uint64_t *block_lens, size_t n_blocks,
                   const pmklc_model_cfg *cfg, void *stream, uint8_t **out, size_t *out_len) {
  return guarded<int>([&]() -> int {
    if (!out || !out_len || (n && !seq)) return PMKLC_EINVAL;
    *out = nullptr;
    *out_len = 0;
    size_t cap = pmklc_compress_bound(n, block_lens, n_blocks, cfg);
    if (cap == 0) return PMKLC_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    uint8_t *d_seq = nullptr, *d_out = nullptr;
    PMKLC_CUDA_TRY(cudaMallocAsync((void **)&d_seq, n ? n : 1, st));
    if (cudaMallocAsync((void **)&d_out, cap, st) != cudaSuccess) {
      cudaFreeAsync(d_seq, st);
      return PMKLC_ENOMEM;
    }
    if (n) cudaMemcpyAsync(d_seq, seq, n, cudaMemcpyHostToDevice, st);
    size_t len = 0;
    int rc = compress_dev_impl(d_seq, n, block_lens, n_blocks, cfg, st, d_out, cap, &len);
    uint8_t *h = nullptr;
    if (rc == PMKLC_OK) {
      h = (uint8_t *)malloc(len ? len : 1);
      if (!h) rc = PMKLC_ENOMEM;
      else if (cudaMemcpyAsync(h, d_out, len, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
               cudaStreamSynchronize(st) != cudaSuccess)
        rc = PMKLC_ECUDA;
    }
    cudaFreeAsync(d_seq, st);
    cudaFreeAsync(d_out, st);
    if (rc) {
      free(h);
      return rc;
    }
    *out = h;
    *out_len = len;
    return PMKLC_OK;
  });
}

int pmklc_decompress(const uint8_t *in, size_t in_len, const float *static_weights, size_t static_count,
                     void *stream, uint8_t **seq, size_t *n, uint64_t **block_lens, size_t *n_blocks) {
  return guarded<int>([&]() -> int {
    if (!in || !seq || !n) return PMKLC_EINVAL;
    *seq = nullptr;
    *n = 0;
    if (in_len < kHeader) return PMKLC_ECORRUPT;
    cudaStream_t st = (cudaStream_t)stream;
    Parsed P;
    int rc = parse_fixed(in, in_len, P);
    if (!rc) rc = parse_records(in, in_len, in_len, P);  // the whole container is on the host
    if (rc) return rc;
    uint8_t *d_in = nullptr, *d_seq = nullptr;
    PMKLC_CUDA_TRY(cudaMallocAsync((void **)&d_in, in_len, st));
    if (cudaMallocAsync((void **)&d_seq, P.n ? P.n : 1, st) != cudaSuccess) {
      cudaFreeAsync(d_in, st);
      return PMKLC_ENOMEM;
    }
    cudaMemcpyAsync(d_in, in, in_len, cudaMemcpyHostToDevice, st);
    size_t nn = 0;
    std::vector<unsigned long long> lens;
    rc = decompress_dev_impl(d_in, in_len, static_weights, static_count, st, d_seq, P.n, &nn, &lens);
    uint8_t *h = nullptr;
    if (rc == PMKLC_OK) {
      h = (uint8_t *)malloc(nn ? nn : 1);
      if (!h) rc = PMKLC_ENOMEM;
      else if (cudaMemcpyAsync(h, d_seq, nn, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
               cudaStreamSynchronize(st) != cudaSuccess)
        rc = PMKLC_ECUDA;
    }
    cudaFreeAsync(d_in, st);
    cudaFreeAsync(d_seq, st);
    if (rc) {
      free(h);
      return rc;
    }
    if (block_lens && n_blocks) {
      uint64_t *bl = (uint64_t *)malloc(sizeof(uint64_t) * (lens.size() ? lens.size() : 1));
      if (!bl) {
        free(h);
        return PMKLC_ENOMEM;
      }
      for (size_t i = 0; i < lens.size(); ++i) bl[i] = lens[i];
      *block_lens = bl;
      *n_blocks = lens.size();
    }
    *seq = h;
    *n = nn;
    return PMKLC_OK;
  });
}

int pmklc_train_model(const uint8_t *seq, size_t n, const pmklc_model_cfg *cfg, uint32_t epochs, void *stream,
                      float *out) {
  return guarded<int>([&]() -> int {
    Cfg c;
    int rc = check_cfg(cfg, c);
    if (rc) return rc;
    if (c.use_static || !out || (n && !seq) || epochs < 1 || epochs > kMaxGroups) return PMKLC_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    Arena ar(st);
    uint8_t *d_seq = ar.alloc<uint8_t>(n);
    if (ar.failed) return PMKLC_ENOMEM;
    cudaMemcpyAsync(d_seq, seq, n, cudaMemcpyHostToDevice, st);
    return train_dev(c, d_seq, n, epochs, nullptr, out, st);
  });
}

int pmklc_init_model(uint32_t k, uint32_t emb, uint32_t ctx, uint32_t hid, uint64_t seed, float *out) {
  return guarded<int>([&]() -> int {
    if (!widths_ok(k, emb, ctx, hid) || !out) return PMKLC_EINVAL;
    Dims d{1 << (2 * (int)k), (int)emb, (int)ctx, (int)hid};
    std::vector<float> v;
    init_params(d, seed, v);
    memcpy(out, v.data(), v.size() * sizeof(float));
    return PMKLC_OK;
  });
}

int pmklc_last_stats(pmklc_stats *st) {
  if (!st) return PMKLC_EINVAL;
  *st = g_stats;
  return PMKLC_OK;
}

int pmklc_crc32(const uint8_t *d_data, size_t n, uint32_t *crc, void *stream) {
  if (!crc || (n && !d_data)) return PMKLC_EINVAL;
  return crc32_device(d_data, n, crc, (cudaStream_t)stream);
}

int pmklc_tokenize(const uint8_t *d_seq, size_t n, uint32_t s, uint32_t k, uint16_t *d_tokens, uint8_t *d_tail,
                   size_t *n_tokens, void *stream) {
  return guarded<int>([&]() -> int {
    if (s < 1 || s > k || k > 8 || !n_tokens || (n && !d_seq) || n > (size_t(1) << 56)) return PMKLC_EINVAL;
    long long l = n_tokens_of((long long)n, (int)s, (int)k);
    if ((l && !d_tokens) || (!d_tail && tail_len_of((long long)n, (int)s, (int)k))) return PMKLC_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    Arena ar(st);
    std::vector<long long> boff = {0, (long long)n}, toff = {0, l};
    const std::vector<int> cta = tokenize_ctas(boff);
    long long *d_boff = ar.upload(boff), *d_toff = ar.upload(toff);
    int *d_cta = ar.upload(cta);
    int *d_err = ar.alloc<int>(1);
    uint8_t *d_t8 = ar.alloc<uint8_t>(8);
    if (ar.failed) return PMKLC_ENOMEM;
    cudaMemsetAsync(d_err, 0, sizeof(int), st);
    launch_validate_tokenize(d_seq, n, d_boff, d_toff, d_cta, 1, cta[1], (int)s, (int)k, d_tokens, d_err, st);
    launch_tails(d_seq, d_boff, d_toff, 1, (int)s, (int)k, d_t8, st);
    long long tl = tail_len_of((long long)n, (int)s, (int)k);
    if (tl) cudaMemcpyAsync(d_tail, d_t8, (size_t)tl, cudaMemcpyDeviceToDevice, st);
    int h_err = 0;
    cudaMemcpyAsync(&h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
    PMKLC_CUDA_TRY(cudaStreamSynchronize(st));
    PMKLC_CUDA_TRY(cudaGetLastError());
    *n_tokens = (size_t)l;
    return h_err ? PMKLC_EINVAL : PMKLC_OK;
  });
}

// Single-step form of the hot loop: G groups of M lanes whose token sequences are
// [context (t_eff tokens), target]; one global step at T = t_eff runs the same kernels.
static int one_step(const Cfg &c, uint32_t G, uint32_t M, float *d_params, float *d_m, float *d_v, float *d_alpha,
                    float *d_alpha_m, float *d_alpha_v, const float *d_static, const uint16_t *d_ctx,
                    const uint16_t *d_target, uint32_t tau, float *d_P, float *d_grad, float *d_dalpha,
                    float *d_logits_only, cudaStream_t st) {
  const int te = c.t_eff();
  Run R;
  R.c = c;
  Layout &L = R.L;
  L.G = (int)G;
  L.NL = (int)(G * M);
  L.Mmax = (int)M;
  L.base_off.assign(G + 1, 0);
  L.tok_off.assign(G + 1, 0);
  L.lane_off.assign(G + 1, 0);
  L.base_len.assign(G, te + 1);
  L.extra.assign(G, 0);
  L.steps.assign(G, te + 1);
  for (uint32_t g = 0; g < G; ++g) {
    L.lane_off[g + 1] = (int)((g + 1) * M);
    for (uint32_t r = 0; r < M; ++r) {
      L.lane_tok.push_back((long long)(g * M + r) * (te + 1));
      L.lane_len.push_back(te + 1);
      L.lane_grp.push_back((int)g);
    }
  }
  L.n_tok = (long long)G * M * (te + 1);
  R.S.start.assign(G, 0);
  R.S.parent.assign(G, -1);
  R.S.tau0.assign(G, (int)tau - 1);
  R.S.T_total = te + 1;
  R.S.max_tau = (int)tau;
  R.S.pairs_at.assign(R.S.T_total + 1, {});
  Arena ar(st);
  uint16_t *d_tok = ar.alloc<uint16_t>(L.n_tok);
  if (ar.failed) return PMKLC_ENOMEM;
  size_t rows = (size_t)G * M;
  cudaMemcpy2DAsync(d_tok, (te + 1) * sizeof(uint16_t), d_ctx, te * sizeof(uint16_t), te * sizeof(uint16_t), rows,
                    cudaMemcpyDeviceToDevice, st);
  if (d_target)
    cudaMemcpy2DAsync(d_tok + te, (te + 1) * sizeof(uint16_t), d_target, sizeof(uint16_t), sizeof(uint16_t), rows,
                      cudaMemcpyDeviceToDevice, st);
  // caller-provided tokens index the embedding tables: reject any >= 4^k before use
  int *d_chk = ar.alloc<int>(1);
  if (!d_chk) return PMKLC_ENOMEM;
  cudaMemsetAsync(d_chk, 0, sizeof(int), st);
  if (!d_target) cudaMemsetAsync(d_tok, 0, sizeof(uint16_t) * L.n_tok, st), cudaMemcpy2DAsync(
      d_tok, (te + 1) * sizeof(uint16_t), d_ctx, te * sizeof(uint16_t), te * sizeof(uint16_t), rows,
      cudaMemcpyDeviceToDevice, st);
  check_tokens_kernel<<<(unsigned)((L.n_tok + 255) / 256), 256, 0, st>>>(d_tok, L.n_tok, c.A(), d_chk);
  int h_chk = 0;
  cudaMemcpyAsync(&h_chk, d_chk, sizeof(int), cudaMemcpyDeviceToHost, st);
  PMKLC_CUDA_TRY(cudaStreamSynchronize(st));
  if (h_chk) return PMKLC_EINVAL;
  std::vector<int> mode(G, kReplay);
  R.p.tokens = d_tok;
  R.p.lane_buf = nullptr;
  R.p.lane_buf_off = nullptr;
  R.p.lane_buf_cap = nullptr;
  int rc = setup_run(ar, R, mode, d_static);
  if (d_grad) R.p.fused_w = 0;  // the gradient is wanted: stored by the GEMMs, applied by the optimiser
  if (rc) return rc;
  // use the caller's state in place of the seeded init
  R.p.params = d_params;
  R.p.m = d_m;
  R.p.v = d_v;
  R.p.alpha = d_alpha;
  R.p.alpha_m = d_alpha_m;
  R.p.alpha_v = d_alpha_v;
  const int T = te;
  const bool bf = bf_form(c.precision);
  prof_step(0, StepWork{(double)rows, (double)G});  // sampled when profiling is enabled
  if (bf) launch_to_bf16(d_params, R.p.wbf, (size_t)G * R.p.P, st);
  if (d_logits_only) {
    if (bf)
      launch_forward_bf16(R.p, T, st);
    else
      launch_forward(R.p, T, st);
    // the FP8 form returns the static model's logits (pmklc_predict runs the model as the static one)
    const float *src = f8_form(c.precision) ? R.p.zu : R.p.zm;
    cudaMemcpyAsync(d_logits_only, src, sizeof(float) * rows * c.A(), cudaMemcpyDeviceToDevice, st);
  } else if (bf) {
    std::vector<unsigned long long> off(rows, 0);
    std::vector<uint32_t> cap(rows, 0);
    R.p.lane_buf_off = ar.upload(off);
    R.p.lane_buf_cap = ar.upload(cap);
    R.p.lane_buf = ar.alloc<uint8_t>(16);
    R.p.out_P = d_P;
    if (ar.failed) return PMKLC_ENOMEM;
    launch_forward_bf16(R.p, T, st);
    launch_mixcode(R.p, T, st);
    launch_backward_bf16(R.p, T, st);
    if (d_grad) launch_export_grad(R.p, d_grad, st);
    launch_update(R.p, T, st);  // also forms dalpha of every group
    if (d_dalpha) cudaMemcpyAsync(d_dalpha, R.p.dalpha_grp, sizeof(float) * G, cudaMemcpyDeviceToDevice, st);
    prof_stop_sampling();
  } else {
    std::vector<unsigned long long> off(rows, 0);
    std::vector<uint32_t> cap(rows, 0);
    R.p.lane_buf_off = ar.upload(off);
    R.p.lane_buf_cap = ar.upload(cap);
    R.p.lane_buf = ar.alloc<uint8_t>(16);
    R.p.out_P = d_P;
    if (ar.failed) return PMKLC_ENOMEM;
    launch_forward(R.p, T, st);
    launch_mixcode(R.p, T, st);
    launch_backward(R.p, T, st);
    if (d_grad) launch_export_grad(R.p, d_grad, st);
    launch_update(R.p, T, st);  // also forms dalpha of every group
    if (d_dalpha) cudaMemcpyAsync(d_dalpha, R.p.dalpha_grp, sizeof(float) * G, cudaMemcpyDeviceToDevice, st);
  }
  prof_stop_sampling();
  int h_err = 0;
  cudaMemcpyAsync(&h_err, R.p.err, sizeof(int), cudaMemcpyDeviceToHost, st);
  PMKLC_CUDA_TRY(cudaStreamSynchronize(st));
  PMKLC_CUDA_TRY(cudaGetLastError());
  return h_err ? err_to_rc(h_err) : PMKLC_OK;
}

int pmklc_predict(const float *d_params, uint32_t k, uint32_t E, uint32_t t, uint32_t H, const uint16_t *d_ctx,
                  size_t rows, uint32_t precision, float *d_logits, void *stream) {
  return guarded<int>([&]() -> int {
    if (k < 1 || k > 8 || !E || !t || !H || precision > PMKLC_BF16_FP8HIDDEN ||
        (rows && (!d_params || !d_ctx || !d_logits)))
      return PMKLC_EINVAL;
    if (rows == 0) return PMKLC_OK;
    // the rows are the lanes of one group: the same limits as a compression's layout
    if (rows > (size_t)kMaxLanes || (long long)rows * (long long)H >= (1LL << 31)) return PMKLC_EINVAL;
    pmklc_model_cfg mc;
    pmklc_default_cfg(&mc, 1, k, E, t, H);
    mc.precision = precision;
    if (f8_form((int)precision)) {  // the model runs as the frozen static predictor in its FP8 form
      mc.use_static = 1;
      mc.emb_s = E, mc.ctx_s = t, mc.hid_s = H;
      mc.static_weights = d_params;  // only checked non-null
    }
    Cfg c;
    int rc = check_cfg(&mc, c);
    if (rc) return rc;
    if (f8_form((int)precision))
      return one_step(c, 1, (uint32_t)rows, const_cast<float *>(d_params), nullptr, nullptr, nullptr, nullptr, nullptr,
                      d_params, d_ctx, nullptr, 1, nullptr, nullptr, nullptr, d_logits, (cudaStream_t)stream);
    // a throw-away copy of the parameters: the forward never writes them, but the plan wants a mutable pointer
    return one_step(c, 1, (uint32_t)rows, const_cast<float *>(d_params), nullptr, nullptr, nullptr, nullptr, nullptr,
                    nullptr, d_ctx, nullptr, 1, nullptr, nullptr, nullptr, d_logits, (cudaStream_t)stream);
  });
}

int pmklc_train_step(const pmklc_model_cfg *cfg, uint32_t G, uint32_t M, float *d_params, float *d_m, float *d_v,
                     float *d_alpha, float *d_alpha_m, float *d_alpha_v, const float *d_static, const uint16_t *d_ctx,
                     const uint16_t *d_target, uint32_t tau, float *d_P, float *d_grad, float *d_dalpha,
                     void *stream) {
  return guarded<int>([&]() -> int {
    Cfg c;
    pmklc_model_cfg tmp;
    if (!cfg) return PMKLC_EINVAL;
    tmp = *cfg;
    if (tmp.use_static && !tmp.static_weights) tmp.static_weights = (const float *)d_static;  // only checked non-null
    int rc = check_cfg(&tmp, c);
    if (rc) return rc;
    if (c.st_arch) return PMKLC_EINVAL;  // the step entry points take an MLP static model
    const long long hmax = std::max(c.dm.H, c.use_static ? c.st.H : 0);
    if ((long long)G * M > kMaxLanes || (long long)G * M * hmax >= (1LL << 31)) return PMKLC_EINVAL;
    if (!G || G > kMaxGroups || !M || tau < 1 || !d_params || !d_m || !d_v || !d_alpha || !d_alpha_m || !d_alpha_v || !d_ctx ||
        !d_target || (c.use_static && !d_static))
      return PMKLC_EINVAL;
    return one_step(c, G, M, d_params, d_m, d_v, d_alpha, d_alpha_m, d_alpha_v, d_static, d_ctx, d_target, tau, d_P,
                    d_grad, d_dalpha, nullptr, (cudaStream_t)stream);
  });
}

}  // extern "C"
