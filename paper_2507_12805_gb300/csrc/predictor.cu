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
#include <algorithm>

#include "internal.h"

namespace pmklc {

namespace {

constexpr int BM = 64, BN = 64, BK = 32;
__device__ const float kOneF = 1.0f;  // the "ones" entry that turns a bias gradient into a GEMM row

__device__ __forceinline__ bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

// Register fragments of one K-chunk (each of the 256 threads holds two float4).
struct Frag {
  float4 v[2];
};

// Operand with k contiguous (A rows, or B^T rows): element e = tid + 256q covers row e/8 and
// k = 4*(e%8) .. +3 of the chunk.  ptr(rl, r, k) -> address of element (r, k), nullptr = 0.
template <class F>
__device__ __forceinline__ void fetch_kc(Frag &f, int r0, int k0, int R, int K, F ptr, bool vec_ok = true) {
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    int e = threadIdx.x + 256 * q, rl = e >> 3, r = r0 + rl, k = k0 + (e & 7) * 4;
    float t[4] = {0.f, 0.f, 0.f, 0.f};
    if (r < R && k < K) {
      const float *p = ptr(rl, r, k);
      if (p) {
        if (vec_ok && k + 3 < K && aligned16(p)) {
          float4 v = *reinterpret_cast<const float4 *>(p);
          t[0] = v.x, t[1] = v.y, t[2] = v.z, t[3] = v.w;
        } else {
          for (int i = 0; i < 4; ++i)
            if (k + i < K) {
              const float *pi = ptr(rl, r, k + i);
              t[i] = pi ? *pi : 0.f;
            }
        }
      }
    }
    f.v[q] = make_float4(t[0], t[1], t[2], t[3]);
  }
}
template <int W>
__device__ __forceinline__ void store_kc(float (*S)[W], const Frag &f) {
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    int e = threadIdx.x + 256 * q, rl = e >> 3, kk = (e & 7) * 4;
    S[kk][rl] = f.v[q].x;
    S[kk + 1][rl] = f.v[q].y;
    S[kk + 2][rl] = f.v[q].z;
    S[kk + 3][rl] = f.v[q].w;
  }
}

// Operand with its column index contiguous: element e covers k = e/16 and c = 4*(e%16) .. +3.
// Vector loads only when c + 3 < Cv (the extent that is contiguous in memory).
template <class F>
__device__ __forceinline__ void fetch_cc(Frag &f, int c0, int k0, int C, int Cv, int K, F ptr) {
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    int e = threadIdx.x + 256 * q, kl = e >> 4, k = k0 + kl, c = c0 + (e & 15) * 4;
    float t[4] = {0.f, 0.f, 0.f, 0.f};
    if (k < K && c < C) {
      const float *p = ptr(kl, k, c);
      if (c + 3 < Cv && p && aligned16(p)) {
        float4 v = *reinterpret_cast<const float4 *>(p);
        t[0] = v.x, t[1] = v.y, t[2] = v.z, t[3] = v.w;
      } else {
        for (int i = 0; i < 4; ++i)
          if (c + i < C) {
            const float *pi = ptr(kl, k, c + i);
            t[i] = pi ? *pi : 0.f;
          }
      }
    }
    f.v[q] = make_float4(t[0], t[1], t[2], t[3]);
  }
}
template <int W>
__device__ __forceinline__ void store_cc(float (*S)[W], const Frag &f) {
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    int e = threadIdx.x + 256 * q, kl = e >> 4, cc = (e & 15) * 4;
    *reinterpret_cast<float4 *>(&S[kl][cc]) = f.v[q];
  }
}

// Shared engine: C[M x N] = sum_k A[m][k] B[k][n] for group g = blockIdx.z, tiles 64 x 64,
// K-chunks of 32 staged in shared memory as As[k][m], Bs[k][n]; the next chunk is fetched into
// registers while the current one is multiplied.  Each thread owns a 4x4 block of C and
// accumulates its K products in increasing k with fmaf (the order never depends on the tile,
// so every output equals the same sequential sum whatever the launch shape).
template <class Op>
__global__ void __launch_bounds__(256) ggemm_kernel(Op op) {
  __shared__ __align__(16) float As[BK][BM + 4];
  __shared__ __align__(16) float Bs[BK][BN + 4];
  __shared__ long long mbase[BM];
  const int g = blockIdx.z;
  if (!op.active(g)) return;
  const int M = op.M(g), N = op.N(), K = op.K(g);
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  if (m0 >= M || n0 >= N) return;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  if (tid < BM) mbase[tid] = m0 + tid < M ? op.mrow_base(g, m0 + tid) : -1;
  __syncthreads();
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  Frag fa, fb;
  op.fetch_a(mbase, g, m0, 0, M, K, fa);
  op.fetch_b(g, 0, n0, K, N, fb);
  for (int k0 = 0; k0 < K; k0 += BK) {
    if (Op::kAKc)
      store_kc(As, fa);
    else
      store_cc(As, fa);
    if (Op::kBKc)
      store_kc(Bs, fb);
    else
      store_cc(Bs, fb);
    __syncthreads();
    if (k0 + BK < K) {
      op.fetch_a(mbase, g, m0, k0 + BK, M, K, fa);
      op.fetch_b(g, k0 + BK, n0, K, N, fb);
    }
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float4 a = *reinterpret_cast<const float4 *>(&As[kk][ty * 4]);
      float4 b = *reinterpret_cast<const float4 *>(&Bs[kk][tx * 4]);
      float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int r = m0 + ty * 4 + i;
    if (r >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int c = n0 + tx * 4 + j;
      if (c < N) op.epi(mbase, g, r, ty * 4 + i, c, acc[i][j]);
    }
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
  __device__ bool active(int g) const { return group_trains(p, T, g); }
  // absolute index of the row's target token (its context ends just before), or -1 if the
  // row does not predict at this step
  __device__ long long target_pos(int g, int r) const {
    int rw = row(g, r);
    if (!row_pred(p, T, rw, g)) return -1;
    return p.lane_tok[rw] + (T - p.grp_start[g]);
  }
  __device__ long long mrow_base(int g, int r) const { return target_pos(g, r); }
  // pointer to X[row][k] = Emb[token at context position k / E][k % E]
  __device__ const float *xptr(const float *w, const Dims &D, long long tpos, int k) const {
    int pos = k / D.E, e = k - pos * D.E;
    int tok = p.tokens[tpos - D.t + pos];
    return w + D.off_emb() + (size_t)tok * D.E + e;
  }
};

// h = relu(X W1 + b1) for the dynamic (stat = 0) or static (stat = 1) model
struct HiddenOp : RowBase {
  static constexpr bool kAKc = true, kBKc = true;
  int stat;
  __device__ const float *w(int g) const { return stat ? p.static_params : p.params + (size_t)g * p.P; }
  __device__ const Dims &d() const { return stat ? p.st : p.dm; }
  __device__ int M(int g) const { return nrows(g); }
  __device__ int N() const { return d().H; }
  __device__ int K(int) const { return d().K1(); }
  __device__ void fetch_a(const long long *mb, int g, int m0, int k0, int M, int K, Frag &f) const {
    const float *wg = w(g);
    const Dims &D = d();
    // four consecutive k lie in one embedding row only when E is a multiple of 4
    fetch_kc(
        f, m0, k0, M, K,
        [&](int rl, int, int k) -> const float * {
          long long b = mb[rl];
          return b < 0 ? nullptr : xptr(wg, D, b, k);
        },
        D.E % 4 == 0);
  }
  __device__ void fetch_b(int g, int k0, int n0, int K, int N, Frag &f) const {
    const float *w1t = w(g) + d().off_w1();  // B[k][n] = W1t[n][k]
    fetch_kc(f, n0, k0, N, K, [&](int, int n, int k) -> const float * { return w1t + (size_t)n * K + k; });
  }
  __device__ void epi(const long long *, int g, int r, int, int n, float acc) const {
    float h = fmaxf(acc + w(g)[d().off_b1() + n], 0.f);
    (stat ? p.hs : p.hd)[(size_t)row(g, r) * d().H + n] = h;
  }
};

// L = h W2 + b2
struct LogitsOp : RowBase {
  static constexpr bool kAKc = true, kBKc = false;
  int stat;
  __device__ const float *w(int g) const { return stat ? p.static_params : p.params + (size_t)g * p.P; }
  __device__ const Dims &d() const { return stat ? p.st : p.dm; }
  __device__ int M(int g) const { return nrows(g); }
  __device__ int N() const { return d().A; }
  __device__ int K(int) const { return d().H; }
  __device__ void fetch_a(const long long *mb, int g, int m0, int k0, int M, int K, Frag &f) const {
    const float *h = stat ? p.hs : p.hd;
    fetch_kc(f, m0, k0, M, K, [&](int rl, int m, int k) -> const float * {
      return mb[rl] < 0 ? nullptr : h + (size_t)row(g, m) * K + k;
    });
  }
  __device__ void fetch_b(int g, int k0, int n0, int K, int N, Frag &f) const {
    const float *w2 = w(g) + d().off_w2();
    fetch_cc(f, n0, k0, N, N, K, [&](int, int k, int c) -> const float * { return w2 + (size_t)k * N + c; });
  }
  __device__ void epi(const long long *mb, int g, int r, int rl, int n, float acc) const {
    if (mb[rl] < 0) return;
    (stat ? p.zu : p.zm)[(size_t)row(g, r) * d().A + n] = acc + w(g)[d().off_b2() + n];
  }
};

// dh = (dz W2^T) * [h > 0]
struct DhOp : RowBase {
  static constexpr bool kAKc = true, kBKc = true;
  __device__ int M(int g) const { return nrows(g); }
  __device__ int N() const { return p.dm.H; }
  __device__ int K(int) const { return p.dm.A; }
  __device__ void fetch_a(const long long *mb, int g, int m0, int k0, int M, int K, Frag &f) const {
    fetch_kc(f, m0, k0, M, K, [&](int rl, int m, int k) -> const float * {
      return mb[rl] < 0 ? nullptr : p.dz + (size_t)row(g, m) * K + k;
    });
  }
  __device__ void fetch_b(int g, int k0, int n0, int K, int N, Frag &f) const {
    const float *w2 = p.params + (size_t)g * p.P + p.dm.off_w2();  // B[k][n] = W2[n][k]
    fetch_kc(f, n0, k0, N, K, [&](int, int n, int k) -> const float * { return w2 + (size_t)n * K + k; });
  }
  __device__ void epi(const long long *mb, int g, int r, int rl, int n, float acc) const {
    size_t i = (size_t)row(g, r) * p.dm.H + n;
    p.dh[i] = (mb[rl] >= 0 && p.hd[i] > 0.f) ? acc : 0.f;
  }
};

// [dW2; db2] = [h 1]^T dz   (K = rows of the group; row H of the result is the bias gradient)
struct DW2Op : RowBase {
  static constexpr bool kAKc = false, kBKc = false;
  __device__ int M(int) const { return p.dm.H + 1; }
  __device__ int N() const { return p.dm.A; }
  __device__ int K(int g) const { return nrows(g); }
  __device__ void fetch_a(const long long *, int g, int m0, int k0, int M, int K, Frag &f) const {
    const int H = p.dm.H;
    fetch_cc(f, m0, k0, M, H, K, [&](int, int r, int i) -> const float * {
      if (target_pos(g, r) < 0) return nullptr;
      return i < H ? p.hd + (size_t)row(g, r) * H + i : &kOneF;
    });
  }
  __device__ void fetch_b(int g, int k0, int n0, int K, int N, Frag &f) const {
    fetch_cc(f, n0, k0, N, N, K, [&](int, int r, int c) -> const float * {
      return target_pos(g, r) < 0 ? nullptr : p.dz + (size_t)row(g, r) * N + c;
    });
  }
  __device__ void epi(const long long *, int g, int i, int, int n, float acc) const {
    float *gr = p.grad + (size_t)g * p.P;
    if (i < p.dm.H)
      gr[p.dm.off_w2() + (size_t)i * p.dm.A + n] = acc;
    else
      gr[p.dm.off_b2() + n] = acc;
  }
};

// [dW1; db1] = [X 1]^T dh   (K = rows of the group; row t*E of the result is the bias gradient)
struct DW1Op : RowBase {
  static constexpr bool kAKc = false, kBKc = false;
  __device__ int M(int) const { return p.dm.K1() + 1; }
  __device__ int N() const { return p.dm.H; }
  __device__ int K(int g) const { return nrows(g); }
  __device__ void fetch_a(const long long *, int g, int m0, int k0, int M, int K, Frag &f) const {
    // A[i][r] = X[r][i]: contiguous along i within one embedding row (E consecutive values)
    const float *wg = p.params + (size_t)g * p.P;
    const int KX = p.dm.K1(), E = p.dm.E;
    fetch_cc(f, m0, k0, M, (E % 4 == 0) ? KX : 0, K, [&](int, int r, int i) -> const float * {
      long long b = target_pos(g, r);
      if (b < 0) return nullptr;
      return i < KX ? xptr(wg, p.dm, b, i) : &kOneF;
    });
  }
  __device__ void fetch_b(int g, int k0, int n0, int K, int N, Frag &f) const {
    fetch_cc(f, n0, k0, N, N, K, [&](int, int r, int c) -> const float * {
      return target_pos(g, r) < 0 ? nullptr : p.dh + (size_t)row(g, r) * N + c;
    });
  }
  __device__ void epi(const long long *, int g, int i, int, int n, float acc) const {
    float *gr = p.grad + (size_t)g * p.P;
    if (i < p.dm.K1())
      gr[p.dm.off_w1() + (size_t)n * p.dm.K1() + i] = acc;  // W1 is stored transposed
    else
      gr[p.dm.off_b1() + n] = acc;
  }
};

// dX = dh W1^T, scattered into the embedding rows of the context tokens
struct DXOp : RowBase {
  static constexpr bool kAKc = true, kBKc = false;
  __device__ int M(int g) const { return nrows(g); }
  __device__ int N() const { return p.dm.K1(); }
  __device__ int K(int) const { return p.dm.H; }
  __device__ void fetch_a(const long long *mb, int g, int m0, int k0, int M, int K, Frag &f) const {
    fetch_kc(f, m0, k0, M, K, [&](int rl, int m, int k) -> const float * {
      return mb[rl] < 0 ? nullptr : p.dh + (size_t)row(g, m) * K + k;
    });
  }
  __device__ void fetch_b(int g, int k0, int n0, int K, int N, Frag &f) const {
    const float *w1t = p.params + (size_t)g * p.P + p.dm.off_w1();  // B[h][i] = W1[i][h] = W1t[h][i]
    fetch_cc(f, n0, k0, N, N, K, [&](int, int h, int i) -> const float * { return w1t + (size_t)h * N + i; });
  }
  __device__ void epi(const long long *mb, int g, int r, int rl, int i, float acc) const {
    long long b = mb[rl];
    if (b < 0) return;
    int pos = i / p.dm.E, e = i - pos * p.dm.E;
    int tok = p.tokens[b - p.dm.t + pos];
    long long q = fix40(acc);
    atomicAdd(reinterpret_cast<unsigned long long *>(p.demb_acc + ((size_t)g * p.dm.A + tok) * p.dm.E + e),
              (unsigned long long)q);
  }
};

// Optimiser over every parameter of every training group, streamed in float4 groups: the
// gradient comes from `grad` (W1, b1, W2, b2, and Emb when it was summed from stored dX rows),
// from the dX tiles' FP32 partials, or from the fixed-point embedding accumulators (Emb, zeroed on
// the way).  The FP32 master, Adam moments
// and, in the BF16 form, the BF16 copy are rewritten in place.  The work is cut into chunks of
// kOptChunk parameters of one group; the CTAs (one resident wave) stride over the
// (group, chunk) pairs, and a thread issues the loads of both of its float4 groups of a chunk
// before any store, so enough bytes are in flight to keep HBM busy.  Indices are 32-bit (no 64-bit
// division, whose FP64-based code is slow on GB300).  The first warp on a group's first chunk also
// updates the group's mixing weight alpha (Eq. 1) by the same rule.
constexpr int kOptThreads = 256, kOptVec = 2, kOptChunk = kOptThreads * 4 * kOptVec;

struct OptGroup {
  float *th, *mm, *vv;
  const float *gr, *part;
  long long *acc;
  __nv_bfloat16 *wb;
  int npart;
};

__device__ __forceinline__ void opt_load4(const Plan &p, const OptGroup &o, uint32_t i0, uint32_t nemb, float *t,
                                          float *m, float *v, float *gg) {
  const float4 a = *reinterpret_cast<const float4 *>(o.th + i0), b = *reinterpret_cast<const float4 *>(o.mm + i0),
               c = *reinterpret_cast<const float4 *>(o.vv + i0);
  t[0] = a.x, t[1] = a.y, t[2] = a.z, t[3] = a.w;
  m[0] = b.x, m[1] = b.y, m[2] = b.z, m[3] = b.w;
  v[0] = c.x, v[1] = c.y, v[2] = c.z, v[3] = c.w;
  if (i0 < nemb && o.part) {  // the dX tiles' FP32 partials, summed in partial order
    float4 a4 = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int k = 0; k < o.npart; ++k) {
      const float4 q = *reinterpret_cast<const float4 *>(o.part + (size_t)k * nemb + i0);
      a4.x += q.x, a4.y += q.y, a4.z += q.z, a4.w += q.w;
    }
    gg[0] = a4.x, gg[1] = a4.y, gg[2] = a4.z, gg[3] = a4.w;
  } else if (i0 < nemb && o.acc) {  // A*E is a multiple of 4: a float4 group never straddles the embedding boundary
    const longlong2 q0 = *reinterpret_cast<const longlong2 *>(o.acc + i0),
                    q1 = *reinterpret_cast<const longlong2 *>(o.acc + i0 + 2);
    gg[0] = unfix40(q0.x), gg[1] = unfix40(q0.y), gg[2] = unfix40(q1.x), gg[3] = unfix40(q1.y);
    *reinterpret_cast<longlong2 *>(o.acc + i0) = make_longlong2(0, 0);
    *reinterpret_cast<longlong2 *>(o.acc + i0 + 2) = make_longlong2(0, 0);
  } else {
    const float4 d = *reinterpret_cast<const float4 *>(o.gr + i0);
    gg[0] = d.x, gg[1] = d.y, gg[2] = d.z, gg[3] = d.w;
  }
}

__device__ __forceinline__ void opt_store4(const OptGroup &o, uint32_t i0, const float *t, const float *m,
                                           const float *v, bool adam) {
  *reinterpret_cast<float4 *>(o.th + i0) = make_float4(t[0], t[1], t[2], t[3]);
  if (adam) {
    *reinterpret_cast<float4 *>(o.mm + i0) = make_float4(m[0], m[1], m[2], m[3]);
    *reinterpret_cast<float4 *>(o.vv + i0) = make_float4(v[0], v[1], v[2], v[3]);
  }
  if (o.wb) {
    __nv_bfloat162 lo = __floats2bfloat162_rn(t[0], t[1]), hi = __floats2bfloat162_rn(t[2], t[3]);
    *reinterpret_cast<uint2 *>(o.wb + i0) =
        make_uint2(*reinterpret_cast<uint32_t *>(&lo), *reinterpret_cast<uint32_t *>(&hi));
  }
}

// The parameters the streaming optimiser updates, as a contiguous "virtual" range: all P of a
// group, or, when W1 and W2 are updated in their gradient GEMMs' epilogues (p.fused_w), the
// embedding, b1 and b2 only (their offsets and lengths are multiples of 4 there: H % 64 == 0).
__device__ __forceinline__ uint32_t opt_count(const Plan &p) {
  return p.fused_w ? (uint32_t)(p.dm.A * p.dm.E + p.dm.H + p.dm.A) : (uint32_t)p.P;
}
__device__ __forceinline__ uint32_t opt_index(const Plan &p, uint32_t i) {
  if (!p.fused_w) return i;
  const uint32_t ae = (uint32_t)(p.dm.A * p.dm.E), h = (uint32_t)p.dm.H;
  if (i < ae) return i;
  if (i < ae + h) return (uint32_t)p.dm.off_b1() + (i - ae);
  return (uint32_t)p.dm.off_b2() + (i - ae - h);
}

__global__ void __launch_bounds__(kOptThreads, 4) opt_stream_kernel(Plan p, int T, int chunks_per_group) {
  pdl_wait();
  pdl_trigger();
  const uint32_t P = opt_count(p), nemb = (uint32_t)(p.dm.A * p.dm.E);
  const bool adam = p.optimizer == PMKLC_ADAM;
  const int n_chunks = p.G * chunks_per_group;
  for (int ch = blockIdx.x; ch < n_chunks; ch += gridDim.x) {
    const int g = ch / chunks_per_group, cg = ch - g * chunks_per_group;
    if (!group_trains(p, T, g)) continue;  // the same for the whole CTA
    const size_t base = (size_t)g * p.P;
    const int tau = group_tau(p, T, g);
    const float bc1 = p.bc1[tau], bc2 = p.bc2[tau];
    OptGroup o;
    o.th = p.params + base, o.mm = p.m + base, o.vv = p.v + base, o.gr = p.grad + base;
    o.acc = p.demb_acc ? p.demb_acc + (size_t)g * nemb : nullptr;  // else the gradient buffer holds it
    // the group's partials of the embedding gradient: its row tiles x the column tiles
    o.part = p.demb_part ? p.demb_part + (size_t)g * p.dx_np * nemb : nullptr;
    o.npart = p.demb_part ? ((p.grp_lane_off[g + 1] - p.grp_lane_off[g] + 127) / 128) * p.dx_ct : 0;
    o.wb = p.wbf ? p.wbf + base : nullptr;
    if (cg == 0 && threadIdx.x < 32) {  // the mixing weight alpha of Eq. (1), same rule
      const float ga = alpha_grad(p, T, g);
      if (threadIdx.x == 0) {
        p.dalpha_grp[g] = ga;
        float t1[4] = {p.alpha[g], 0, 0, 0}, m1[4] = {p.alpha_m[g], 0, 0, 0}, v1[4] = {p.alpha_v[g], 0, 0, 0},
              g1[4] = {ga, 0, 0, 0};
        adam_n<1>(t1, m1, v1, g1, p.lr, bc1, bc2, adam);
        p.alpha[g] = t1[0];
        p.alpha_m[g] = m1[0];
        p.alpha_v[g] = v1[0];
      }
    }
    const uint32_t c0 = (uint32_t)cg * kOptChunk + 4u * threadIdx.x;
    if ((base & 3) == 0 && (uint32_t)cg * kOptChunk + kOptChunk <= P) {  // a whole, aligned chunk
      float t[kOptVec][4], m[kOptVec][4], v[kOptVec][4], gg[kOptVec][4];
#pragma unroll
      for (int q = 0; q < kOptVec; ++q)
        opt_load4(p, o, opt_index(p, c0 + q * 4 * kOptThreads), nemb, t[q], m[q], v[q], gg[q]);
#pragma unroll
      for (int q = 0; q < kOptVec; ++q) {
        adam_n<4>(t[q], m[q], v[q], gg[q], p.lr, bc1, bc2, adam);
        opt_store4(o, opt_index(p, c0 + q * 4 * kOptThreads), t[q], m[q], v[q], adam);
      }
      continue;
    }
    for (int q = 0; q < kOptVec; ++q) {  // the group's last chunk, or unaligned groups: element by element
      const uint32_t v0 = c0 + q * 4 * kOptThreads;
      for (uint32_t vi = v0; vi < v0 + 4 && vi < P; ++vi) {
        const uint32_t i = opt_index(p, vi);
        float t1[4] = {o.th[i], 0, 0, 0}, m1[4] = {o.mm[i], 0, 0, 0}, v1[4] = {o.vv[i], 0, 0, 0}, g1[4] = {0, 0, 0, 0};
        if (i < nemb && o.part) {
          for (int k = 0; k < o.npart; ++k) g1[0] += o.part[(size_t)k * nemb + i];
        } else if (i < nemb && o.acc) {
          g1[0] = unfix40(o.acc[i]);
          o.acc[i] = 0;
        } else {
          g1[0] = o.gr[i];
        }
        adam_n<1>(t1, m1, v1, g1, p.lr, bc1, bc2, adam);
        o.th[i] = t1[0];
        if (adam) o.mm[i] = m1[0], o.vv[i] = v1[0];
        if (o.wb) o.wb[i] = __float2bfloat16_rn(t1[0]);
      }
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
    if (p.wbf) p.wbf[child * P + i] = p.wbf[parent * P + i];
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
    if (p.st_gru) {  // the BiGRU static predictor's Linear layer forms the static h
      launch_bigru_static(p, T, st);
    } else {
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
    run_ggemm(DW2Op{{p, T}}, p.dm.H + 1, p.dm.A, p.G, st);
  }
  {
    ProfScope ps("bwd_dw1", 2.0 * R * p.dm.K1() * p.dm.H, 0, st);
    run_ggemm(DW1Op{{p, T}}, p.dm.K1() + 1, p.dm.H, p.G, st);
  }
  {
    ProfScope ps("bwd_dx_demb", 2.0 * R * p.dm.K1() * p.dm.H, 0, st);
    run_ggemm(DXOp{{p, T}}, p.Mmax, p.dm.K1(), p.G, st);
  }
}

void launch_update(const Plan &p, int T, cudaStream_t st) {
  // Adam: read w, m, v, grad (16 B) and write w, m, v (12 B) per parameter of every training
  // group (+2 B for the BF16 copy); the embedding part reads/clears 8-byte accumulators instead of
  // the 4-byte gradient, or reads the dX partials (dx_np of 4 bytes)
  const double nemb = (double)p.dm.A * p.dm.E;
  const double per = p.wbf ? 30.0 : 28.0;
  const double emb_extra = p.demb_part ? nemb * 4.0 * (p.dx_np - 1) : p.demb_acc ? nemb * 12.0 : 0.0;
  const size_t count = p.fused_w ? (size_t)p.dm.A * p.dm.E + p.dm.H + p.dm.A : p.P;
  {
    ProfScope ps("update_adam", 0, prof_work().train_groups * ((double)count * per + emb_extra), st);
    // one resident wave (4 blocks of 256 threads per SM, the launch bound) striding over the
    // (group, chunk) pairs
    const int per_group = (int)((count + kOptChunk - 1) / kOptChunk);
    const long long chunks = (long long)per_group * p.G;
    const unsigned grid = (unsigned)std::min<long long>(chunks, 152LL * 4);
    if (grid == 0) return;
    launch_pdl(opt_stream_kernel, dim3(grid), dim3(kOptThreads), 0, st, p, T, per_group);  // also updates alpha
  }
}

void launch_backward_update(const Plan &p, int T, cudaStream_t st) {
  launch_backward(p, T, st);
  launch_update(p, T, st);
}

namespace {
__global__ void export_grad_kernel(Plan p, float *out) {
  int g = blockIdx.y;
  size_t nemb = (size_t)p.dm.A * p.dm.E;
  const int npart = p.demb_part ? ((p.grp_lane_off[g + 1] - p.grp_lane_off[g] + 127) / 128) * p.dx_ct : 0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < p.P; i += (size_t)gridDim.x * blockDim.x) {
    float v;
    if (i >= nemb) {
      v = p.grad[(size_t)g * p.P + i];
    } else if (p.demb_part) {  // the same partial order as the optimiser
      v = 0.f;
      for (int k = 0; k < npart; ++k) v += p.demb_part[((size_t)g * p.dx_np + k) * nemb + i];
    } else if (p.demb_acc) {
      v = unfix40(p.demb_acc[(size_t)g * nemb + i]);
    } else {  // summed from the dX rows into the gradient buffer
      v = p.grad[(size_t)g * p.P + i];
    }
    out[(size_t)g * p.P + i] = v;
  }
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
