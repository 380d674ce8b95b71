// BF16 batched form on tcgen05: the six GEMMs of one global step of every group's predictors
// (paper §2 steps 3-4, the MLP of the measured configurations), on the engine of tcgemm.cuh.
//
//   forward   h  = relu(X W1 + b1)    X gathered from the embedding rows of the context tokens
//             L  = h W2 + b2          dynamic model (z < G) and static model (z >= G) in one launch
//   backward  dh = (dz W2^T) * [h > 0]
//             dW2 = h^T dz,  dX = dh W1^T (scattered into the embedding rows),  dW1 = X^T dh
//             db2 = sum of dz, db1 = sum of dh over the predicted rows (fixed-order column sums)
// after which the streaming optimiser (predictor.cu) updates every parameter and refreshes the
// BF16 copy.
//
// Operand majors follow the stored layouts: W1 is stored transposed (W1t[h][i], K-major for the
// hidden layer), W2 as [h][a]; activations are [row][feature].  The weight-gradient GEMMs reduce
// over lanes, so both their operands are MN-major.
#include "tcgemm.cuh"

namespace pmklc {

namespace {

using tc::bf16;

// Per-tile shared data.  Row-tiled GEMMs (rows = lanes): the target position of each of the 128
// tile rows (-1: no prediction) and, when the op gathers embeddings, each row's t context tokens.
// Lane-reducing GEMMs (K = lanes): the target position of every lane of the group and, for dW1,
// its context tokens.
constexpr int kRowMetaTok = tc::kRows * 8;  // byte offset of the token block in a row-tile meta
__host__ __device__ inline size_t row_meta_bytes(int t) { return kRowMetaTok + (size_t)tc::kRows * t * 2; }
__host__ __device__ inline size_t lane_meta_bytes(int lanes, int t) { return (size_t)lanes * 8 + (size_t)lanes * t * 2; }

struct TBase {
  Plan p;
  int T;
  __device__ int *err() const { return p.err; }
  __device__ int nrows(int g) const { return p.grp_lane_off[g + 1] - p.grp_lane_off[g]; }
  __device__ int row(int g, int r) const { return p.grp_lane_off[g] + r; }
  __device__ long long target_pos(int g, int r) const {
    const int rw = row(g, r);
    if (!row_pred(p, T, rw, g)) return -1;
    return p.lane_tok[rw] + (T - p.grp_start[g]);
  }
  __device__ const bf16 *wb(int g) const { return p.wbf + (size_t)g * p.P; }
  // row-tile meta of group g's rows m0..m0+127, with t context tokens per row (t = 0: none)
  __device__ void prep_rows(uint8_t *meta, int g, int m0, int t) const {
    long long *tp = reinterpret_cast<long long *>(meta);
    for (int i = threadIdx.x; i < tc::kRows; i += tc::kThreads) {
      const int r = m0 + i;
      tp[i] = r < nrows(g) ? target_pos(g, r) : -1;
    }
    if (t <= 0) return;
    __syncthreads();
    uint16_t *tk = reinterpret_cast<uint16_t *>(meta + kRowMetaTok);
    for (int i = threadIdx.x; i < tc::kRows * t; i += tc::kThreads) {
      const int r = i / t, j = i - r * t;
      const long long b = tp[r];
      tk[i] = b >= 0 ? p.tokens[b - t + j] : 0;
    }
  }
  __device__ static long long row_target(const uint8_t *meta, int rl) {
    return reinterpret_cast<const long long *>(meta)[rl];
  }
  __device__ static int row_token(const uint8_t *meta, int rl, int t, int pos) {
    return reinterpret_cast<const uint16_t *>(meta + kRowMetaTok)[rl * t + pos];
  }
  // lane meta of every lane of group g, with t context tokens per lane (t = 0: none)
  __device__ void prep_lanes(uint8_t *meta, int g, int t) const {
    const int L = nrows(g);
    long long *tp = reinterpret_cast<long long *>(meta);
    for (int i = threadIdx.x; i < L; i += tc::kThreads) tp[i] = target_pos(g, i);
    if (t <= 0) return;
    __syncthreads();
    uint16_t *tk = reinterpret_cast<uint16_t *>(meta + (size_t)p.Mmax * 8);
    for (int i = threadIdx.x; i < L * t; i += tc::kThreads) {
      const int r = i / t, j = i - r * t;
      const long long b = tp[r];
      tk[i] = b >= 0 ? p.tokens[b - t + j] : 0;
    }
  }
  __device__ static long long lane_target(const uint8_t *meta, int m) {
    return reinterpret_cast<const long long *>(meta)[m];
  }
  __device__ int lane_token(const uint8_t *meta, int m, int t, int pos) const {
    return reinterpret_cast<const uint16_t *>(meta + (size_t)p.Mmax * 8)[m * t + pos];
  }
};

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

// h = relu(X W1 + b1): A = X (gathered, K-major), B = W1t (K-major)
struct HiddenT : TwoModels {
  static constexpr bool kAMN = false, kBMN = false;
  __device__ int M(int z) const { return nrows(grp(z)); }
  __device__ int N(int z) const { return d(z).H; }
  __device__ int K(int z) const { return d(z).K1(); }
  __device__ void prepare(uint8_t *meta, int z, int m0) const { prep_rows(meta, grp(z), m0, d(z).t); }
  __device__ void stage_a(uint8_t *dst, const uint8_t *meta, int z, int, int k0, int rlim, int klim) const {
    const Dims &D = d(z);
    tc::stage_k_gather(dst, rlim, k0, klim, reinterpret_cast<const long long *>(meta),
                       reinterpret_cast<const uint16_t *>(meta + kRowMetaTok), D.t, D.E, w(z) + D.off_emb());
  }
  __device__ void stage_b(uint8_t *dst, const uint8_t *, int z, int n0, int k0, int R, int rlim, int klim) const {
    const Dims &D = d(z);
    const bf16 *w1t = w(z) + D.off_w1() + (size_t)n0 * D.K1();
    const int K1 = D.K1();
    tc::stage_k_rows(dst, R, rlim, k0, klim, [&](int r) { return w1t + (size_t)r * K1; });
  }
  __device__ void epilogue(const uint8_t *meta, int z, int m, int rl, int n, const float *v) const {
    if (row_target(meta, rl) < 0) return;
    const Dims &D = d(z);
    const float *b1 = w32(z) + D.off_b1() + n;
    float x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = fmaxf(v[j] + b1[j], 0.f);
    *reinterpret_cast<uint4 *>((stat(z) ? p.hs_b : p.hd_b) + (size_t)row(grp(z), m) * D.H + n) = pack8(x);
  }
};

// L = h W2 + b2: A = h (K-major), B = W2[h][a] (MN-major)
struct LogitsT : TwoModels {
  static constexpr bool kAMN = false, kBMN = true;
  __device__ int M(int z) const { return nrows(grp(z)); }
  __device__ int N(int z) const { return d(z).A; }
  __device__ int K(int z) const { return d(z).H; }
  __device__ void prepare(uint8_t *meta, int z, int m0) const { prep_rows(meta, grp(z), m0, 0); }
  __device__ void stage_a(uint8_t *dst, const uint8_t *meta, int z, int m0, int k0, int rlim, int klim) const {
    const int g = grp(z), H = d(z).H;
    const bf16 *h = (stat(z) ? p.hs_b : p.hd_b) + (size_t)row(g, m0) * H;
    tc::stage_k_rows(dst, tc::kRows, rlim, k0, klim, [&](int r) -> const bf16 * {
      return row_target(meta, r) < 0 ? nullptr : h + (size_t)r * H;
    });
  }
  __device__ void stage_b(uint8_t *dst, const uint8_t *, int z, int n0, int k0, int R, int rlim, int klim) const {
    const Dims &D = d(z);
    const bf16 *w2 = w(z) + D.off_w2() + (size_t)k0 * D.A + n0;
    const int A = D.A;
    tc::stage_mn_rows(dst, R, rlim, klim, [&](int k) { return w2 + (size_t)k * A; });
  }
  __device__ void epilogue(const uint8_t *meta, int z, int m, int rl, int n, const float *v) const {
    if (row_target(meta, rl) < 0) return;
    const Dims &D = d(z);
    const float *b2 = w32(z) + D.off_b2() + n;
    float x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = v[j] + b2[j];
    store8((stat(z) ? p.zu : p.zm) + (size_t)row(grp(z), m) * D.A + n, x);
  }
};

// dh = (dz W2^T) * [h > 0]: A = dz (K-major), B = W2[h][a] read as N = h, K = a (K-major)
struct DhT : TBase {
  static constexpr bool kAMN = false, kBMN = false;
  __device__ bool active(int z) const { return group_trains(p, T, z); }
  __device__ int M(int z) const { return nrows(z); }
  __device__ int N(int) const { return p.dm.H; }
  __device__ int K(int) const { return p.dm.A; }
  __device__ void prepare(uint8_t *meta, int z, int m0) const { prep_rows(meta, z, m0, 0); }
  __device__ void stage_a(uint8_t *dst, const uint8_t *meta, int z, int m0, int k0, int rlim, int klim) const {
    const int A = p.dm.A;
    const bf16 *dz = p.dz_b + (size_t)row(z, m0) * A;
    tc::stage_k_rows(dst, tc::kRows, rlim, k0, klim, [&](int r) -> const bf16 * {
      return row_target(meta, r) < 0 ? nullptr : dz + (size_t)r * A;
    });
  }
  __device__ void stage_b(uint8_t *dst, const uint8_t *, int z, int n0, int k0, int R, int rlim, int klim) const {
    const int A = p.dm.A;
    const bf16 *w2 = wb(z) + p.dm.off_w2() + (size_t)n0 * A;
    tc::stage_k_rows(dst, R, rlim, k0, klim, [&](int r) { return w2 + (size_t)r * A; });
  }
  __device__ void epilogue(const uint8_t *meta, int z, int m, int rl, int n, const float *v) const {
    const size_t i = (size_t)row(z, m) * p.dm.H + n;
    const bool ok = row_target(meta, rl) >= 0;
    uint4 hw = *reinterpret_cast<const uint4 *>(p.hd_b + i);
    const bf16 *h = reinterpret_cast<const bf16 *>(&hw);
    float x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = (ok && __bfloat162float(h[j]) > 0.f) ? v[j] : 0.f;
    *reinterpret_cast<uint4 *>(p.dh_b + i) = pack8(x);
  }
};

// dW2 = h^T dz over the lanes: M = H, N = A, K = lanes; both operands MN-major
struct DW2T : TBase {
  static constexpr bool kAMN = true, kBMN = true;
  __device__ bool active(int z) const { return group_trains(p, T, z); }
  __device__ int M(int) const { return p.dm.H; }
  __device__ int N(int) const { return p.dm.A; }
  __device__ int K(int z) const { return nrows(z); }
  __device__ void prepare(uint8_t *meta, int z, int) const { prep_lanes(meta, z, 0); }
  __device__ void stage_a(uint8_t *dst, const uint8_t *meta, int z, int m0, int k0, int rlim, int klim) const {
    const int H = p.dm.H;
    tc::stage_mn_rows(dst, tc::kRows, rlim, klim, [&](int k) -> const bf16 * {
      return lane_target(meta, k0 + k) < 0 ? nullptr : p.hd_b + (size_t)row(z, k0 + k) * H + m0;
    });
  }
  __device__ void stage_b(uint8_t *dst, const uint8_t *meta, int z, int n0, int k0, int R, int rlim, int klim) const {
    const int A = p.dm.A;
    tc::stage_mn_rows(dst, R, rlim, klim, [&](int k) -> const bf16 * {
      return lane_target(meta, k0 + k) < 0 ? nullptr : p.dz_b + (size_t)row(z, k0 + k) * A + n0;
    });
  }
  __device__ void epilogue(const uint8_t *, int z, int h, int, int n, const float *v) const {
    store8(p.grad + (size_t)z * p.P + p.dm.off_w2() + (size_t)h * p.dm.A + n, v);
  }
};

// dX = dh W1^T scattered into the embedding rows (fixed-point atomics): A = dh (K-major),
// B = W1t[h][i] read as N = i, K = h (MN-major)
struct DXT : TBase {
  static constexpr bool kAMN = false, kBMN = true;
  __device__ bool active(int z) const { return group_trains(p, T, z); }
  __device__ int M(int z) const { return nrows(z); }
  __device__ int N(int) const { return p.dm.K1(); }
  __device__ int K(int) const { return p.dm.H; }
  __device__ void prepare(uint8_t *meta, int z, int m0) const { prep_rows(meta, z, m0, p.dm.t); }
  __device__ void stage_a(uint8_t *dst, const uint8_t *meta, int z, int m0, int k0, int rlim, int klim) const {
    const int H = p.dm.H;
    const bf16 *dh = p.dh_b + (size_t)row(z, m0) * H;
    tc::stage_k_rows(dst, tc::kRows, rlim, k0, klim, [&](int r) -> const bf16 * {
      return row_target(meta, r) < 0 ? nullptr : dh + (size_t)r * H;
    });
  }
  __device__ void stage_b(uint8_t *dst, const uint8_t *, int z, int n0, int k0, int R, int rlim, int klim) const {
    const int K1 = p.dm.K1();
    const bf16 *w1t = wb(z) + p.dm.off_w1() + (size_t)k0 * K1 + n0;
    tc::stage_mn_rows(dst, R, rlim, klim, [&](int k) { return w1t + (size_t)k * K1; });
  }
  __device__ void epilogue(const uint8_t *meta, int z, int, int rl, int n, const float *v) const {
    if (row_target(meta, rl) < 0) return;
    const int pos = n / p.dm.E, e = n - pos * p.dm.E;  // 8 columns stay inside one embedding row
    const int tok = row_token(meta, rl, p.dm.t, pos);
    unsigned long long *acc =
        reinterpret_cast<unsigned long long *>(p.demb_acc + ((size_t)z * p.dm.A + tok) * p.dm.E + e);
#pragma unroll
    for (int j = 0; j < 8; ++j) atomicAdd(acc + j, (unsigned long long)__double2ll_rn((double)v[j] * kEmbFix));
  }
};

// dW1 (stored transposed: dW1t[h][i] = sum over lanes of dh[m][h] X[m][i]): M = H, N = t*E,
// K = lanes; both operands MN-major
struct DW1T : TBase {
  static constexpr bool kAMN = true, kBMN = true;
  __device__ bool active(int z) const { return group_trains(p, T, z); }
  __device__ int M(int) const { return p.dm.H; }
  __device__ int N(int) const { return p.dm.K1(); }
  __device__ int K(int z) const { return nrows(z); }
  __device__ void prepare(uint8_t *meta, int z, int) const { prep_lanes(meta, z, p.dm.t); }
  __device__ void stage_a(uint8_t *dst, const uint8_t *meta, int z, int m0, int k0, int rlim, int klim) const {
    const int H = p.dm.H;
    tc::stage_mn_rows(dst, tc::kRows, rlim, klim, [&](int k) -> const bf16 * {
      return lane_target(meta, k0 + k) < 0 ? nullptr : p.dh_b + (size_t)row(z, k0 + k) * H + m0;
    });
  }
  __device__ void stage_b(uint8_t *dst, const uint8_t *meta, int z, int n0, int k0, int R, int rlim, int klim) const {
    tc::stage_mn_gather(dst, R, rlim, n0, k0, klim, reinterpret_cast<const long long *>(meta),
                        reinterpret_cast<const uint16_t *>(meta + (size_t)p.Mmax * 8), p.dm.t, p.dm.E,
                        wb(z) + p.dm.off_emb());
  }
  __device__ void epilogue(const uint8_t *, int z, int h, int, int n, const float *v) const {
    store8(p.grad + (size_t)z * p.P + p.dm.off_w1() + (size_t)h * p.dm.K1() + n, v);
  }
};

// db1 = sum of dh, db2 = sum of dz over the predicted rows of each group.  Block (32 columns x 8
// row slices): slice y adds rows y, y+8, ... in order, then slice 0 adds the 8 partial sums in
// order, so the result does not depend on scheduling.
constexpr int kBiasSlices = 8;
__global__ void __launch_bounds__(32 * kBiasSlices) bias_grad_kernel(Plan p, int T) {
  __shared__ float part[kBiasSlices][32];
  const int g = blockIdx.y;
  if (!group_trains(p, T, g)) return;
  const int H = p.dm.H, A = p.dm.A;
  const int c = blockIdx.x * 32 + threadIdx.x;
  const bool in = c < H + A, is1 = c < H;
  const int w = is1 ? H : A, cc = is1 ? c : c - H;
  const bf16 *src = is1 ? p.dh_b : p.dz_b;
  const int j = T - p.grp_start[g];
  float s = 0.f;
  if (in)
#pragma unroll 4
    for (int r = p.grp_lane_off[g] + threadIdx.y; r < p.grp_lane_off[g + 1]; r += kBiasSlices)
      if (j >= p.t_eff && j < p.lane_len[r]) s += __bfloat162float(src[(size_t)r * w + cc]);
  part[threadIdx.y][threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.y == 0 && in) {
    float t = 0.f;
    for (int y = 0; y < kBiasSlices; ++y) t += part[y][threadIdx.x];
    p.grad[(size_t)g * p.P + (is1 ? p.dm.off_b1() : p.dm.off_b2()) + cc] = t;
  }
}

constexpr size_t kMaxLaneMeta = 80 * 1024;

}  // namespace

bool tc_supported(const Plan &p) {
  auto ok = [](const Dims &d) { return d.E % 8 == 0 && d.H % 16 == 0 && d.A % 8 == 0; };
  // the lane-reducing GEMMs keep every lane's target and context tokens in shared memory
  return ok(p.dm) && p.P % 8 == 0 && (!p.use_static || ok(p.st)) &&
         lane_meta_bytes(p.Mmax, p.dm.t) <= kMaxLaneMeta && row_meta_bytes(p.use_static ? max(p.dm.t, p.st.t) : p.dm.t) <= kMaxLaneMeta;
}

void launch_forward_tc(const Plan &p, int T, cudaStream_t st) {
  const double R = prof_work().pred_rows;
  const int Z = p.use_static ? 2 * p.G : p.G;
  {
    double fl = 2.0 * R * p.dm.K1() * p.dm.H + (p.use_static ? 2.0 * R * p.st.K1() * p.st.H : 0.0);
    ProfScope ps("fwd_hidden_bf16", fl, 0, st);
    tc::launch(HiddenT{{p, T}}, p.Mmax, p.use_static ? max(p.dm.H, p.st.H) : p.dm.H, Z,
               row_meta_bytes(p.use_static ? max(p.dm.t, p.st.t) : p.dm.t), st);
  }
  double fl = 2.0 * R * p.dm.H * p.dm.A + (p.use_static ? 2.0 * R * p.st.H * p.st.A : 0.0);
  ProfScope ps("fwd_logits_bf16", fl, 0, st);
  tc::launch(LogitsT{{p, T}}, p.Mmax, p.dm.A, Z, row_meta_bytes(0), st);
}

void launch_backward_tc(const Plan &p, int T, cudaStream_t st) {
  const double R = prof_work().pred_rows;
  const Dims &D = p.dm;
  {
    ProfScope ps("bwd_dh_bf16", 2.0 * R * D.A * D.H, 0, st);
    tc::launch(DhT{p, T}, p.Mmax, D.H, p.G, row_meta_bytes(0), st);
  }
  {
    ProfScope ps("bwd_dw2_bf16", 2.0 * R * D.A * D.H, 0, st);
    tc::launch(DW2T{p, T}, D.H, D.A, p.G, lane_meta_bytes(p.Mmax, 0), st);
    bias_grad_kernel<<<dim3((D.H + D.A + 31) / 32, p.G), dim3(32, kBiasSlices), 0, st>>>(p, T);
  }
  {
    ProfScope ps("bwd_dx_bf16", 2.0 * R * D.K1() * D.H, 0, st);
    tc::launch(DXT{p, T}, p.Mmax, D.K1(), p.G, row_meta_bytes(D.t), st);
  }
  {
    ProfScope ps("bwd_dw1_bf16", 2.0 * R * D.K1() * D.H, 0, st);
    tc::launch(DW1T{p, T}, D.H, D.K1(), p.G, lane_meta_bytes(p.Mmax, D.t), st);
  }
}

}  // namespace pmklc
