// The BiGRU static predictor (paper §4.2.2 SPuM: 16-wide embedding, two BiGRU layers, a Linear
// and a Dense layer of width 128; §4.2.3 SPrM: the same with one BiGRU layer), forward in FP32.
//
// GRU cell (the form with the reset gate on the recurrent projection after its bias):
//   r = sigmoid(Wi_r x + bi_r + Wh_r h + bh_r), z = sigmoid(Wi_z x + bi_z + Wh_z h + bh_z),
//   n = tanh(Wi_n x + bi_n + r (Wh_n h + bh_n)), h' = (1 - z) n + z h, starting from h = 0.
// Layer l runs a forward GRU over the context positions 0..t-1 (oldest first) and a backward one
// over t-1..0; its output at p is [h^f_p, h^b_p].  The last layer's summary u = [h^f after t-1,
// h^b after 0] feeds the Linear layer q = relu(W3 u + b3) (128 wide), and the Dense layer forms
// the logits L = q W4 + b4.
//
// The recurrence is sequential over the t positions of a row and independent across rows, so one
// thread carries one row: its state h lives in registers, the weights of the (layer, direction)
// pass being run are staged in shared memory and read by all threads of the CTA at the same
// address (broadcast), and each new state is formed from gate values the thread parks in its own
// shared-memory column.  With two layers the first layer's outputs go to a global scratch
// [t][2 Hg][rows] (row index fastest, so a warp's accesses are coalesced); the second layer reads
// them back.  The Dense layer is the MLP's logits layer (h = q, H = 128): in the codec it runs on
// the library's logits kernels, here (pmklc_predict_bigru) on a plain row x column kernel.
#include <math.h>

#include <exception>
#include <new>

#include "internal.h"

namespace pmklc {

namespace {

constexpr int kThreads = 128;  // rows per CTA

struct GruRun {
  const float *w;
  GruOff o;
  int A, t, layers, rows;
  float *y;             // two layers: the first layer's outputs [t][2 Hg][rows]
  float *q;             // output rows (FP32), row stride ldq, or nullptr
  __nv_bfloat16 *qb;    // output rows (BF16), row stride ldq, or nullptr
  int ldq;
  int *err;             // kErrCorrupt: a context token >= A (read as token 0)
};

// context source: explicit rows of t tokens, oldest first
struct CtxRows {
  const uint16_t *ctx;
  int t;
  __device__ bool on(int) const { return true; }
  __device__ int tok(int r, int pos) const { return ctx[(size_t)r * t + pos]; }
};

// context source: the lanes predicted at global step T of a run (the static model's t tokens
// before each lane's target, oldest first)
struct CtxLanes {
  Plan p;
  int T;
  __device__ bool on(int r) const { return row_pred(p, T, r, p.lane_grp[r]); }
  __device__ int tok(int r, int pos) const {
    const long long tp = p.lane_tok[r] + (T - p.grp_start[p.lane_grp[r]]);
    return p.tokens[tp - p.st.t + pos];
  }
};

__device__ __forceinline__ float sigm(float x) { return 1.f / (1.f + expf(-x)); }

// One GRU direction over the positions of this thread's row.  sw: Wi [3 HG][IN] | Wh [3 HG][HG] |
// bi [3 HG] | bh [3 HG] in shared memory; col: this thread's shared-memory column (stride
// kThreads) of 2 HG gate values.  x_at(p, x) loads the input at position p, put(p, h) takes the
// state after it.
template <int IN, int HG, class X, class Put>
__device__ __forceinline__ void gru_dir(const float *sw, float *col, int t, bool rev, bool on, X x_at, Put put,
                                        float (&h)[HG]) {
  const float *wi = sw, *wh = sw + 3 * HG * IN, *bi = wh + 3 * HG * HG, *bh = bi + 3 * HG;
#pragma unroll
  for (int k = 0; k < HG; ++k) h[k] = 0.f;
  if (!on) return;
  for (int s = 0; s < t; ++s) {
    const int p = rev ? t - 1 - s : s;
    float x[IN];
    x_at(p, x);
#pragma unroll 1
    for (int j = 0; j < HG; ++j) {
      float ar = bi[j] + bh[j], az = bi[HG + j] + bh[HG + j], an = bi[2 * HG + j], hn = bh[2 * HG + j];
      const float *wr = wi + j * IN, *wz = wi + (HG + j) * IN, *wn = wi + (2 * HG + j) * IN;
#pragma unroll
      for (int e = 0; e < IN; ++e) {
        ar = fmaf(wr[e], x[e], ar);
        az = fmaf(wz[e], x[e], az);
        an = fmaf(wn[e], x[e], an);
      }
      const float *vr = wh + j * HG, *vz = wh + (HG + j) * HG, *vn = wh + (2 * HG + j) * HG;
#pragma unroll
      for (int k = 0; k < HG; ++k) {
        ar = fmaf(vr[k], h[k], ar);
        az = fmaf(vz[k], h[k], az);
        hn = fmaf(vn[k], h[k], hn);
      }
      const float r = sigm(ar);
      col[j * kThreads] = tanhf(fmaf(r, hn, an));  // n
      col[(HG + j) * kThreads] = sigm(az);         // z
    }
#pragma unroll
    for (int k = 0; k < HG; ++k) {
      const float n = col[k * kThreads], z = col[(HG + k) * kThreads];
      h[k] = fmaf(z, h[k], (1.f - z) * n);
    }
    put(p, h);
  }
}

// Stage n floats from global src into shared dst (all threads of the CTA).
__device__ __forceinline__ void stage(float *dst, const float *src, int n) {
  for (int i = threadIdx.x; i < n; i += kThreads) dst[i] = src[i];
}

template <int E, int HG, class Ctx>
__global__ void __launch_bounds__(kThreads) bigru_kernel(const GruRun a, const Ctx src) {
  extern __shared__ float sm[];
  const int r = blockIdx.x * kThreads + threadIdx.x;
  const bool on = r < a.rows && src.on(r);
  float *col = sm + (3 * HG * (2 * HG) + 3 * HG * HG + 6 * HG) + threadIdx.x;  // after the largest pass
  float uf[HG], ub[HG], h[HG];
  const size_t R = (size_t)a.rows;
  for (int l = 0; l < a.layers; ++l) {
    const bool last = l + 1 == a.layers;
    for (int d = 0; d < 2; ++d) {
      const int in = l == 0 ? E : 2 * HG;
      __syncthreads();  // the previous pass has read its weights
      stage(sm, a.w + a.o.wi[l][d], 3 * HG * in);
      stage(sm + 3 * HG * in, a.w + a.o.wh[l][d], 3 * HG * HG);
      stage(sm + 3 * HG * in + 3 * HG * HG, a.w + a.o.bi[l][d], 3 * HG);
      stage(sm + 3 * HG * in + 3 * HG * HG + 3 * HG, a.w + a.o.bh[l][d], 3 * HG);
      __syncthreads();
      auto put = [&](int p, const float (&hv)[HG]) {
        if (last) return;
        float *yp = a.y + ((size_t)p * 2 * HG + d * HG) * R + r;
#pragma unroll
        for (int k = 0; k < HG; ++k) yp[k * R] = hv[k];
      };
      if (l == 0) {
        auto x_at = [&](int p, float (&x)[E]) {
          int tok = src.tok(r, p);
          if (tok >= a.A) {
            atomicOr(a.err, kErrCorrupt);
            tok = 0;
          }
          const float *e = a.w + a.o.emb + (size_t)tok * E;
#pragma unroll
          for (int i = 0; i < E; ++i) x[i] = __ldg(e + i);
        };
        gru_dir<E, HG>(sm, col, a.t, d == 1, on, x_at, put, h);
      } else {
        auto x_at = [&](int p, float (&x)[2 * HG]) {
          const float *yp = a.y + (size_t)p * 2 * HG * R + r;
#pragma unroll
          for (int c = 0; c < 2 * HG; ++c) x[c] = yp[c * R];
        };
        gru_dir<2 * HG, HG>(sm, col, a.t, d == 1, on, x_at, put, h);
      }
      if (last && d == 0) {
#pragma unroll
        for (int k = 0; k < HG; ++k) uf[k] = h[k];
      } else if (last) {
#pragma unroll
        for (int k = 0; k < HG; ++k) ub[k] = h[k];
      }
    }
  }
  // Linear layer: q = relu(W3 u + b3), u = [uf, ub]
  __syncthreads();
  stage(sm, a.w + a.o.w3, kGruDense * 2 * HG);
  stage(sm + kGruDense * 2 * HG, a.w + a.o.b3, kGruDense);
  __syncthreads();
  if (!on) return;
  const float *b3 = sm + kGruDense * 2 * HG;
#pragma unroll 1
  for (int j = 0; j < kGruDense; ++j) {
    const float *w3 = sm + j * 2 * HG;
    float acc = b3[j];
#pragma unroll
    for (int c = 0; c < HG; ++c) acc = fmaf(w3[c], uf[c], acc);
#pragma unroll
    for (int c = 0; c < HG; ++c) acc = fmaf(w3[HG + c], ub[c], acc);
    acc = fmaxf(acc, 0.f);
    if (a.q)
      a.q[(size_t)r * a.ldq + j] = acc;
    else
      a.qb[(size_t)r * a.ldq + j] = __float2bfloat16_rn(acc);
  }
}

// L[r][c] = b4[c] + sum_j q[r][j] W4[j][c] (j in order): 8 rows per CTA (grid x), a thread per
// column (grid y: at most 4^8 / 128 = 512)
__global__ void __launch_bounds__(128) dense_kernel(const float *q, const float *w4, const float *b4, int rows, int A,
                                                    float *L) {
  __shared__ float sq[8][kGruDense];
  const int r0 = blockIdx.x * 8;
  for (int i = threadIdx.x; i < 8 * kGruDense; i += 128) {
    const int rr = r0 + i / kGruDense;
    sq[i / kGruDense][i % kGruDense] = rr < rows ? q[(size_t)rr * kGruDense + i % kGruDense] : 0.f;
  }
  __syncthreads();
  const int c = blockIdx.y * 128 + threadIdx.x;
  if (c >= A) return;
  float acc[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) acc[i] = b4[c];
  for (int j = 0; j < kGruDense; ++j) {
    const float w = w4[(size_t)j * A + c];
#pragma unroll
    for (int i = 0; i < 8; ++i) acc[i] = fmaf(sq[i][j], w, acc[i]);
  }
#pragma unroll
  for (int i = 0; i < 8; ++i)
    if (r0 + i < rows) L[(size_t)(r0 + i) * A + c] = acc[i];
}

template <int E, int HG, class Ctx>
cudaError_t launch_e_hg(const GruRun &a, const Ctx &src, int smem, cudaStream_t st) {
  if (!smem_optin((const void *)bigru_kernel<E, HG, Ctx>, smem)) return cudaGetLastError();
  const int grid = (a.rows + kThreads - 1) / kThreads;
  bigru_kernel<E, HG, Ctx><<<grid, kThreads, smem, st>>>(a, src);
  return cudaGetLastError();
}

template <class Ctx>
cudaError_t launch_any(const GruRun &a, int E, int Hg, const Ctx &src, cudaStream_t st) {
  if (a.rows <= 0) return cudaSuccess;
  const int smem = gru_smem_bytes(Hg);
  if (Hg == 16) {
    if (E == 8) return launch_e_hg<8, 16>(a, src, smem, st);
    if (E == 16) return launch_e_hg<16, 16>(a, src, smem, st);
    if (E == 32) return launch_e_hg<32, 16>(a, src, smem, st);
  } else if (Hg == 32) {
    if (E == 8) return launch_e_hg<8, 32>(a, src, smem, st);
    if (E == 16) return launch_e_hg<16, 32>(a, src, smem, st);
    if (E == 32) return launch_e_hg<32, 32>(a, src, smem, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

GruOff gru_offsets(int A, int E, int Hg, int layers) {
  GruOff o{};
  size_t off = 0;
  o.emb = off;
  off += (size_t)A * E;
  for (int l = 0; l < layers; ++l)
    for (int d = 0; d < 2; ++d) {
      const int in = l == 0 ? E : 2 * Hg;
      o.wi[l][d] = off;
      off += (size_t)3 * Hg * in;
      o.wh[l][d] = off;
      off += (size_t)3 * Hg * Hg;
      o.bi[l][d] = off;
      off += (size_t)3 * Hg;
      o.bh[l][d] = off;
      off += (size_t)3 * Hg;
    }
  o.w3 = off;
  off += (size_t)kGruDense * 2 * Hg;
  o.b3 = off;
  off += kGruDense;
  o.w4 = off;
  off += (size_t)kGruDense * A;
  o.b4 = off;
  off += (size_t)A;
  o.count = off;
  return o;
}

bool gru_shape_ok(int k, int E, int t, int Hg, int layers) {
  return k >= 1 && k <= 8 && (E == 8 || E == 16 || E == 32) && (Hg == 16 || Hg == 32) && (layers == 1 || layers == 2) &&
         t >= 1 && t <= 4096;
}

int gru_smem_bytes(int Hg) {
  // the largest pass (input 2 Hg) + the gate columns; the Linear layer's W3 and b3 fit in it
  const int pass = 3 * Hg * 2 * Hg + 3 * Hg * Hg + 6 * Hg, cols = 2 * Hg * kThreads;
  return (int)sizeof(float) * (pass + cols);
}

void launch_bigru_static(const Plan &p, int T, cudaStream_t st) {
  GruRun a{};
  a.w = p.st_gru;
  a.o = gru_offsets(p.st.A, p.st.E, p.gru_hg, p.gru_layers);
  a.A = p.st.A, a.t = p.st.t, a.layers = p.gru_layers, a.rows = p.NL, a.y = p.gru_y, a.err = p.err;
  if (p.hs_b)
    a.qb = p.hs_b;
  else
    a.q = p.hs;
  a.ldq = kGruDense;
  // FLOPs per predicted row: every (layer, direction) pass does t x 3 Hg x (in + Hg) FMAs, the
  // Linear layer 128 x 2 Hg
  const double Hg = p.gru_hg;
  double per = 2.0 * kGruDense * 2 * Hg;
  for (int l = 0; l < p.gru_layers; ++l) per += 2.0 * 2 * p.st.t * 3 * Hg * ((l ? 2 * Hg : p.st.E) + Hg);
  ProfScope ps("fwd_bigru_static", prof_work().pred_rows * per, 0, st);
  launch_any(a, p.st.E, p.gru_hg, CtxLanes{p, T}, st);
}

}  // namespace pmklc

using namespace pmklc;

extern "C" {

size_t pmklc_bigru_count(uint32_t k, uint32_t E, uint32_t Hg, uint32_t layers) {
  if (!gru_shape_ok((int)k, (int)E, 1, (int)Hg, (int)layers)) return 0;
  return gru_offsets(1 << (2 * k), (int)E, (int)Hg, (int)layers).count;
}

int pmklc_predict_bigru(const float *d_params, uint32_t k, uint32_t E, uint32_t t, uint32_t Hg, uint32_t layers,
                        const uint16_t *d_ctx, size_t rows, float *d_q, float *d_logits, void *stream) {
  try {
    if (!gru_shape_ok((int)k, (int)E, (int)t, (int)Hg, (int)layers)) return PMKLC_EINVAL;
    if (rows && (!d_params || !d_ctx || (!d_q && !d_logits))) return PMKLC_EINVAL;
    if (rows == 0) return PMKLC_OK;
    if (rows > (size_t)1 << 24) return PMKLC_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const int A = 1 << (2 * k);
    GruRun a{};
    a.w = d_params;
    a.o = gru_offsets(A, (int)E, (int)Hg, (int)layers);
    a.A = A, a.t = (int)t, a.layers = (int)layers, a.rows = (int)rows, a.ldq = kGruDense;
    void *y = nullptr, *q = nullptr, *err = nullptr;
    auto release = [&]() {
      if (y) cudaFreeAsync(y, st);
      if (q) cudaFreeAsync(q, st);
      if (err) cudaFreeAsync(err, st);
    };
    bool ok = cudaMallocAsync(&err, sizeof(int), st) == cudaSuccess;
    if (ok && layers == 2) ok = cudaMallocAsync(&y, sizeof(float) * (size_t)t * 2 * Hg * rows, st) == cudaSuccess;
    if (ok && !d_q) ok = cudaMallocAsync(&q, sizeof(float) * kGruDense * rows, st) == cudaSuccess;
    if (!ok) {
      release();
      cudaGetLastError();
      return PMKLC_ENOMEM;
    }
    a.y = (float *)y;
    a.q = d_q ? d_q : (float *)q;
    a.err = (int *)err;
    int rc = PMKLC_OK;
    if (cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess ||
        launch_any(a, (int)E, (int)Hg, CtxRows{d_ctx, (int)t}, st) != cudaSuccess)
      rc = PMKLC_ECUDA;
    if (!rc && d_logits) {
      dim3 grid((unsigned)((rows + 7) / 8), (A + 127) / 128);
      dense_kernel<<<grid, 128, 0, st>>>(a.q, d_params + a.o.w4, d_params + a.o.b4, (int)rows, A, d_logits);
      if (cudaGetLastError() != cudaSuccess) rc = PMKLC_ECUDA;
    }
    int h_err = 0;
    if (!rc && cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) rc = PMKLC_ECUDA;
    release();
    if (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess) return PMKLC_ECUDA;
    if (!rc && h_err) rc = PMKLC_EINVAL;
    return rc;
  } catch (const std::bad_alloc &) {
    return PMKLC_ENOMEM;
  } catch (...) {
    return PMKLC_EINVAL;
  }
}

}  // extern "C"
