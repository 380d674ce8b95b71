// Predictor forward, backward and optimiser update: the "plain FP32" form.
//
// Paper §2 steps (3)-(4): every dynamic model predicts the next token of each
// of its lanes from the t previous ones, then is updated by back-propagating
// the cross entropy (Eq. 2, Backward Controller §4.2.6).  The predictor is
// the MLP of the measured configurations:
//     X = [Emb[c_0] .. Emb[c_{t-1}]],  h = relu(X W1 + b1),  L = h W2 + b2.
// All groups (one dynamic model per block) advance together, so every GEMM
// here is a grouped GEMM whose z grid index is the group; the rows of a group
// are its lanes.  Each output element accumulates its K products in a fixed
// order with fmaf, independent of the tile it falls in, so the encoder and the
// decoder (which launch the same kernels on the same data) agree bit for bit.
// The embedding gradient is accumulated with 64-bit integer atomics on a
// 2^-40 fixed-point grid: integer addition is associative, so the result does
// not depend on the order of the atomics.
#include "internal.h"

namespace pmklc {

namespace {

constexpr int BM = 64, BN = 64, BK = 16;

template <class Op>
__global__ void __launch_bounds__(256) ggemm_kernel(Op op) {
  __shared__ __align__(16) float As[BK][BM + 4];
  __shared__ __align__(16) float Bs[BK][BN + 4];
  const int g = blockIdx.z;
  if (!op.active(g)) return;
  const int M = op.M(g), N = op.N(), K = op.K(g);
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  if (m0 >= M || n0 >= N) return;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  for (int k0 = 0; k0 < K; k0 += BK) {
#pragma unroll
    for (int q = 0; q < (BM * BK) / 256; ++q) {
      int e = tid + q * 256, kk = e % BK, rr = e / BK;
      As[kk][rr] = (m0 + rr < M && k0 + kk < K) ? op.a(g, m0 + rr, k0 + kk) : 0.f;
    }
#pragma unroll
    for (int q = 0; q < (BK * BN) / 256; ++q) {
      int e = tid + q * 256, cc = e % BN, kk = e / BN;
      Bs[kk][cc] = (k0 + kk < K && n0 + cc < N) ? op.b(g, k0 + kk, n0 + cc) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int r = m0 + ty * 4 + i, c = n0 + tx * 4 + j;
      if (r < M && c < N) op.epi(g, r, c, acc[i][j]);
    }
}

template <class Op>
void run_ggemm(const Op &op, int Mmax, int N, int G, cudaStream_t st) {
  if (Mmax <= 0 || N <= 0 || G <= 0) return;
  dim3 grid((Mmax + BM - 1) / BM, (N + BN - 1) / BN, G);
  ggemm_kernel<Op><<<grid, 256, 0, st>>>(op);
}

// Common row helpers: the lanes of group g are rows lane_off[g] .. lane_off[g+1)-1.
struct RowBase {
  Plan p;
  int T;
  __device__ int nrows(int g) const { return p.grp_lane_off[g + 1] - p.grp_lane_off[g]; }
  __device__ int row(int g, int r) const { return p.grp_lane_off[g] + r; }
  __device__ bool pred(int g, int row) const { return row_pred(p, T, row, g); }
  __device__ bool active(int g) const { return group_trains(p, T, g); }
  // token at context position pos (0 = oldest) of a model with context t
  __device__ int ctx_token(int g, int row, int pos, int t) const {
    int j = T - p.grp_start[g];
    return p.tokens[p.lane_tok[row] + j - t + pos];
  }
};

// h = relu(X W1 + b1) for the dynamic (stat = 0) or static (stat = 1) model
struct HiddenOp : RowBase {
  int stat;
  __device__ const float *w(int g) const { return stat ? p.static_params : p.params + (size_t)g * p.P; }
  __device__ const Dims &d() const { return stat ? p.st : p.dm; }
  __device__ int M(int g) const { return nrows(g); }
  __device__ int N() const { return d().H; }
  __device__ int K(int) const { return d().K1(); }
  __device__ float a(int g, int r, int k) const {
    int rw = row(g, r);
    if (!pred(g, rw)) return 0.f;
    const Dims &D = d();
    int pos = k / D.E, e = k - pos * D.E;
    int tok = ctx_token(g, rw, pos, D.t);
    return w(g)[D.off_emb() + (size_t)tok * D.E + e];
  }
  __device__ float b(int g, int k, int n) const { return w(g)[d().off_w1() + (size_t)k * d().H + n]; }
  __device__ void epi(int g, int r, int n, float acc) const {
    float h = fmaxf(acc + w(g)[d().off_b1() + n], 0.f);
    (stat ? p.hs : p.hd)[(size_t)row(g, r) * d().H + n] = h;
  }
};

// L = h W2 + b2
struct LogitsOp : RowBase {
  int stat;
  __device__ const float *w(int g) const { return stat ? p.static_params : p.params + (size_t)g * p.P; }
  __device__ const Dims &d() const { return stat ? p.st : p.dm; }
  __device__ int M(int g) const { return nrows(g); }
  __device__ int N() const { return d().A; }
  __device__ int K(int) const { return d().H; }
  __device__ float a(int g, int r, int k) const {
    return (stat ? p.hs : p.hd)[(size_t)row(g, r) * d().H + k];
  }
  __device__ float b(int g, int k, int n) const { return w(g)[d().off_w2() + (size_t)k * d().A + n]; }
  __device__ void epi(int g, int r, int n, float acc) const {
    (stat ? p.zu : p.zm)[(size_t)row(g, r) * d().A + n] = acc + w(g)[d().off_b2() + n];
  }
};

// dh = (dz W2^T) * [h > 0]
struct DhOp : RowBase {
  __device__ int M(int g) const { return nrows(g); }
  __device__ int N() const { return p.dm.H; }
  __device__ int K(int) const { return p.dm.A; }
  __device__ float a(int g, int r, int k) const {
    int rw = row(g, r);
    return pred(g, rw) ? p.dz[(size_t)rw * p.dm.A + k] : 0.f;
  }
  __device__ float b(int g, int k, int n) const {
    return p.params[(size_t)g * p.P + p.dm.off_w2() + (size_t)n * p.dm.A + k];
  }
  __device__ void epi(int g, int r, int n, float acc) const {
    size_t i = (size_t)row(g, r) * p.dm.H + n;
    p.dh[i] = p.hd[i] > 0.f ? acc : 0.f;
  }
};

// dW2 = h^T dz   (K = rows of the group)
struct DW2Op : RowBase {
  __device__ int M(int) const { return p.dm.H; }
  __device__ int N() const { return p.dm.A; }
  __device__ int K(int g) const { return nrows(g); }
  __device__ float a(int g, int i, int r) const {
    int rw = row(g, r);
    return pred(g, rw) ? p.hd[(size_t)rw * p.dm.H + i] : 0.f;
  }
  __device__ float b(int g, int r, int n) const {
    int rw = row(g, r);
    return pred(g, rw) ? p.dz[(size_t)rw * p.dm.A + n] : 0.f;
  }
  __device__ void epi(int g, int i, int n, float acc) const {
    p.grad[(size_t)g * p.P + p.dm.off_w2() + (size_t)i * p.dm.A + n] = acc;
  }
};

// dW1 = X^T dh   (K = rows of the group)
struct DW1Op : RowBase {
  __device__ int M(int) const { return p.dm.K1(); }
  __device__ int N() const { return p.dm.H; }
  __device__ int K(int g) const { return nrows(g); }
  __device__ float a(int g, int i, int r) const {
    int rw = row(g, r);
    if (!pred(g, rw)) return 0.f;
    int pos = i / p.dm.E, e = i - pos * p.dm.E;
    int tok = ctx_token(g, rw, pos, p.dm.t);
    return p.params[(size_t)g * p.P + p.dm.off_emb() + (size_t)tok * p.dm.E + e];
  }
  __device__ float b(int g, int r, int n) const {
    int rw = row(g, r);
    return pred(g, rw) ? p.dh[(size_t)rw * p.dm.H + n] : 0.f;
  }
  __device__ void epi(int g, int i, int n, float acc) const {
    p.grad[(size_t)g * p.P + p.dm.off_w1() + (size_t)i * p.dm.H + n] = acc;
  }
};

// dX = dh W1^T, scattered into the embedding rows of the context tokens
struct DXOp : RowBase {
  __device__ int M(int g) const { return nrows(g); }
  __device__ int N() const { return p.dm.K1(); }
  __device__ int K(int) const { return p.dm.H; }
  __device__ float a(int g, int r, int k) const { return p.dh[(size_t)row(g, r) * p.dm.H + k]; }
  __device__ float b(int g, int k, int i) const {
    return p.params[(size_t)g * p.P + p.dm.off_w1() + (size_t)i * p.dm.H + k];
  }
  __device__ void epi(int g, int r, int i, float acc) const {
    int rw = row(g, r);
    if (!pred(g, rw)) return;
    int pos = i / p.dm.E, e = i - pos * p.dm.E;
    int tok = ctx_token(g, rw, pos, p.dm.t);
    long long q = __double2ll_rn((double)acc * kEmbFix);
    atomicAdd(reinterpret_cast<unsigned long long *>(p.demb_acc + ((size_t)g * p.dm.A + tok) * p.dm.E + e),
              (unsigned long long)q);
  }
};

// db2 = sum dz, db1 = sum dh, dalpha = sum dalpha_row over the predicted rows, in row order
__global__ void bias_grad_kernel(Plan p, int T) {
  int g = blockIdx.y;
  if (!group_trains(p, T, g)) return;
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  int A = p.dm.A, H = p.dm.H;
  if (c > A + H) return;
  int r0 = p.grp_lane_off[g], r1 = p.grp_lane_off[g + 1];
  float s = 0.f;
  for (int r = r0; r < r1; ++r) {
    if (!row_pred(p, T, r, g)) continue;
    if (c < A)
      s += p.dz[(size_t)r * A + c];
    else if (c < A + H)
      s += p.dh[(size_t)r * H + (c - A)];
    else
      s += p.dalpha_row[r];
  }
  if (c < A)
    p.grad[(size_t)g * p.P + p.dm.off_b2() + c] = s;
  else if (c < A + H)
    p.grad[(size_t)g * p.P + p.dm.off_b1() + (c - A)] = s;
  else
    p.dalpha_grp[g] = s;
}

__device__ __forceinline__ void adam_one(float &th, float &m, float &v, float gr, float lr, float bc1, float bc2) {
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  m = b1 * m + (1.f - b1) * gr;
  v = b2 * v + (1.f - b2) * gr * gr;
  float mh = m / bc1, vh = v / bc2;
  th -= lr * mh / (sqrtf(vh) + eps);
}

__global__ void update_kernel(Plan p, int T) {
  int g = blockIdx.y;
  if (!group_trains(p, T, g)) return;
  int j = T - p.grp_start[g];
  int tau = p.grp_tau0[g] + (j - p.t_eff) + 1;
  float bc1 = p.bc1[tau], bc2 = p.bc2[tau];
  size_t nemb = (size_t)p.dm.A * p.dm.E;
  float *th = p.params + (size_t)g * p.P, *m = p.m + (size_t)g * p.P, *v = p.v + (size_t)g * p.P;
  const float *gr = p.grad + (size_t)g * p.P;
  long long *acc = p.demb_acc + (size_t)g * nemb;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < p.P; i += (size_t)gridDim.x * blockDim.x) {
    float gi;
    if (i < nemb) {
      gi = (float)((double)acc[i] * (1.0 / kEmbFix));
      acc[i] = 0;
    } else {
      gi = gr[i];
    }
    if (p.optimizer == PMKLC_ADAM) {
      float t = th[i], mm = m[i], vv = v[i];
      adam_one(t, mm, vv, gi, p.lr, bc1, bc2);
      th[i] = t;
      m[i] = mm;
      v[i] = vv;
    } else {
      th[i] -= p.lr * gi;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    float ga = p.dalpha_grp[g];
    if (p.optimizer == PMKLC_ADAM) {
      float t = p.alpha[g], mm = p.alpha_m[g], vv = p.alpha_v[g];
      adam_one(t, mm, vv, ga, p.lr, bc1, bc2);
      p.alpha[g] = t;
      p.alpha_m[g] = mm;
      p.alpha_v[g] = vv;
    } else {
      p.alpha[g] -= p.lr * ga;
    }
  }
}

__global__ void smp_copy_kernel(Plan p, const int *pairs, int n_pairs) {
  int q = blockIdx.y;
  if (q >= n_pairs) return;
  int child = pairs[2 * q], parent = pairs[2 * q + 1];
  size_t P = p.P;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < P; i += (size_t)gridDim.x * blockDim.x) {
    p.params[child * P + i] = p.params[parent * P + i];
    p.m[child * P + i] = p.m[parent * P + i];
    p.v[child * P + i] = p.v[parent * P + i];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    p.alpha[child] = p.alpha[parent];
    p.alpha_m[child] = p.alpha_m[parent];
    p.alpha_v[child] = p.alpha_v[parent];
  }
}

__global__ void init_groups_kernel(Plan p, const float *init, float alpha0) {
  int g = blockIdx.y;
  size_t P = p.P;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < P; i += (size_t)gridDim.x * blockDim.x) {
    p.params[g * P + i] = init[i];
    p.m[g * P + i] = 0.f;
    p.v[g * P + i] = 0.f;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    p.alpha[g] = alpha0;
    p.alpha_m[g] = 0.f;
    p.alpha_v[g] = 0.f;
  }
}

}  // namespace

void launch_forward(const Plan &p, int T, cudaStream_t st) {
  const double R = prof_work().pred_rows;
  {
    ProfScope ps("fwd_hidden_dm", 2.0 * R * p.dm.K1() * p.dm.H, 0, st);
    run_ggemm(HiddenOp{{p, T}, 0}, p.Mmax, p.dm.H, p.G, st);
  }
  {
    ProfScope ps("fwd_logits_dm", 2.0 * R * p.dm.H * p.dm.A, 0, st);
    run_ggemm(LogitsOp{{p, T}, 0}, p.Mmax, p.dm.A, p.G, st);
  }
  if (p.use_static) {
    {
      ProfScope ps("fwd_hidden_static", 2.0 * R * p.st.K1() * p.st.H, 0, st);
      run_ggemm(HiddenOp{{p, T}, 1}, p.Mmax, p.st.H, p.G, st);
    }
    ProfScope ps("fwd_logits_static", 2.0 * R * p.st.H * p.st.A, 0, st);
    run_ggemm(LogitsOp{{p, T}, 1}, p.Mmax, p.st.A, p.G, st);
  }
}

void launch_backward(const Plan &p, int T, cudaStream_t st) {
  const double R = prof_work().pred_rows;
  {
    ProfScope ps("bwd_dh", 2.0 * R * p.dm.A * p.dm.H, 0, st);
    run_ggemm(DhOp{{p, T}}, p.Mmax, p.dm.H, p.G, st);
  }
  {
    ProfScope ps("bwd_dw2", 2.0 * R * p.dm.A * p.dm.H, 0, st);
    run_ggemm(DW2Op{{p, T}}, p.dm.H, p.dm.A, p.G, st);
  }
  {
    ProfScope ps("bwd_dw1", 2.0 * R * p.dm.K1() * p.dm.H, 0, st);
    run_ggemm(DW1Op{{p, T}}, p.dm.K1(), p.dm.H, p.G, st);
  }
  {
    ProfScope ps("bwd_dx_demb", 2.0 * R * p.dm.K1() * p.dm.H, 0, st);
    run_ggemm(DXOp{{p, T}}, p.Mmax, p.dm.K1(), p.G, st);
  }
  int cols = p.dm.A + p.dm.H + 1;
  ProfScope ps("bias_grad", 0, 0, st);
  bias_grad_kernel<<<dim3((cols + 127) / 128, p.G), 128, 0, st>>>(p, T);
}

void launch_update(const Plan &p, int T, cudaStream_t st) {
  unsigned gx = (unsigned)((p.P + 1023) / 1024);
  if (gx > 64) gx = 64;
  // Adam: read w, m, v, grad (16 B) and write w, m, v (12 B) per parameter of every training group
  const double nemb = (double)p.dm.A * p.dm.E;
  ProfScope ps("update_adam", 0, prof_work().train_groups * ((double)p.P * 28.0 + nemb * 12.0), st);
  update_kernel<<<dim3(gx, p.G), 256, 0, st>>>(p, T);
}

void launch_backward_update(const Plan &p, int T, cudaStream_t st) {
  launch_backward(p, T, st);
  launch_update(p, T, st);
}

namespace {
__global__ void export_grad_kernel(Plan p, float *out) {
  int g = blockIdx.y;
  size_t nemb = (size_t)p.dm.A * p.dm.E;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < p.P; i += (size_t)gridDim.x * blockDim.x)
    out[(size_t)g * p.P + i] = i < nemb ? (float)((double)p.demb_acc[(size_t)g * nemb + i] * (1.0 / kEmbFix))
                                        : p.grad[(size_t)g * p.P + i];
}
}  // namespace

void launch_export_grad(const Plan &p, float *d_out, cudaStream_t st) {
  unsigned gx = (unsigned)((p.P + 1023) / 1024);
  if (gx > 64) gx = 64;
  export_grad_kernel<<<dim3(gx, p.G), 256, 0, st>>>(p, d_out);
}

void launch_smp_copy(const Plan &p, const int *d_pairs, int n_pairs, cudaStream_t st) {
  if (n_pairs <= 0) return;
  unsigned gx = (unsigned)((p.P + 1023) / 1024);
  if (gx > 64) gx = 64;
  smp_copy_kernel<<<dim3(gx, n_pairs), 256, 0, st>>>(p, d_pairs, n_pairs);
}

void launch_init_groups(const Plan &p, const float *d_init, float alpha0, cudaStream_t st) {
  if (p.G <= 0) return;
  unsigned gx = (unsigned)((p.P + 1023) / 1024);
  if (gx > 64) gx = 64;
  init_groups_kernel<<<dim3(gx, p.G), 256, 0, st>>>(p, d_init, alpha0);
}

}  // namespace pmklc
