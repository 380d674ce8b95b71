// Predictor forward and backward: the "BF16 batched" form.
//
// Same mathematics as predictor.cu (paper §2 steps (3)-(4); MLP predictor
// X -> relu(X W1 + b1) -> W2, Eq. (1) mixing, Eq. (2) loss), with the
// contractions on the tensor cores: operands are BF16 (weights from per-group
// BF16 copies of the FP32 master weights, activations stored in BF16 by their
// producers) streamed into shared memory by a cp.async pipeline and multiplied
// with mma.sync m16n8k16 into FP32 accumulators.  The weight-gradient GEMMs
// store FP32 gradient tiles; the shared streaming optimiser (predictor.cu) then
// updates the FP32 master weights, moments and BF16 copies.
#include <cuda_bf16.h>

#include "internal.h"

namespace pmklc {

namespace {

using bf16 = __nv_bfloat16;
constexpr int TBM = 64, TBN = 64, TBK = 32, TTH = 128;
constexpr int SKC = TBK + 8;  // row stride (elements) of a k-contiguous tile [64][32]
constexpr int SMC = TBM + 8;  // row stride of a row/col-contiguous tile [32][64]

__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void ldm4(uint32_t (&r)[4], uint32_t a) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}
__device__ __forceinline__ void ldm4t(uint32_t (&r)[4], uint32_t a) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}
__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ bool al16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

constexpr int ASZ = TBM * SKC > TBK * SMC ? TBM * SKC : TBK * SMC;
constexpr int BSZ = TBN * SKC > TBK * SMC ? TBN * SKC : TBK * SMC;
constexpr int kMaxCtxStaged = 128;

// Gradient tile [rows m0.. x cols n0..] (staged in shared memory, leading dimension ld) to the
// gradient buffer: row r of the tile starts at parameter offset rowoff(r); four columns per store.
template <class RowOff>
__device__ __forceinline__ void store_grad_tile(const Plan &p, int g, int m0, int n0, int M, int N, const float *Cs,
                                                int ld, RowOff rowoff) {
  float *gr = p.grad + (size_t)g * p.P;
  for (int q = threadIdx.x; q < TBM * (TBN / 4); q += TTH) {
    int rl = q / (TBN / 4), cl = (q % (TBN / 4)) * 4, r = m0 + rl, c = n0 + cl;
    if (r >= M || c >= N) continue;
    size_t o = rowoff(r) + c;
    const float *src = Cs + rl * ld + cl;
    if (c + 3 < N && (((size_t)g * p.P + o) & 3) == 0)
      *reinterpret_cast<float4 *>(gr + o) = make_float4(src[0], src[1], src[2], src[3]);
    else
      for (int e = 0; e < 4 && c + e < N; ++e) gr[o + e] = src[e];
  }
}  // context tokens per row staged in shared memory (HiddenB)
__device__ const unsigned short kOneBfBits = 0x3F80;  // BF16 1.0: the "ones" entry of a bias-gradient row
__device__ const uint4 kZero16 = {0u, 0u, 0u, 0u};  // source of zero-filled async copies

__device__ __forceinline__ void cp16(bf16 *dst, const void *src, bool real) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(saddr(dst)), "l"(real ? src : &kZero16),
               "r"(real ? 16 : 0));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

// Stage 8 consecutive BF16 operand values (one 16-byte smem chunk): an asynchronous copy when the
// source holds them contiguously and aligned, a zero fill when there are none, else one by one.
template <class F>  // ptr(i) -> const bf16* of element i (0..7) or nullptr (= 0)
__device__ __forceinline__ void stage_chunk(bf16 *dst, F ptr, int valid, bool contiguous) {
  const bf16 *p0 = valid > 0 ? ptr(0) : nullptr;
  if (valid == 8 && contiguous && p0 && al16(p0)) {
    cp16(dst, p0, true);
    return;
  }
  if (valid == 0 || (contiguous && !p0)) {
    cp16(dst, nullptr, false);
    return;
  }
  unsigned short t[8];
  for (int i = 0; i < 8; ++i) {
    const bf16 *pi = i < valid ? ptr(i) : nullptr;
    t[i] = pi ? __bfloat16_as_ushort(*pi) : (unsigned short)0;
  }
  *reinterpret_cast<uint4 *>(dst) = make_uint4(t[0] | (uint32_t)t[1] << 16, t[2] | (uint32_t)t[3] << 16,
                                               t[4] | (uint32_t)t[5] << 16, t[6] | (uint32_t)t[7] << 16);
}

// Operand tile staging.  k-contiguous tile of R rows ([64][SKC]): chunk c -> row c/4, k 8*(c%4).
// Row-contiguous tile over columns ([32][SMC]): chunk c -> k c/8, column 8*(c%8).  2 chunks/thread.
template <class F>  // ptr(rl, r, k) -> element (r, k)
__device__ __forceinline__ void stage_kc(bf16 *S, int r0, int k0, int R, int K, F ptr, bool contiguous) {
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    int c = threadIdx.x + TTH * q, rl = c >> 2, r = r0 + rl, k = k0 + (c & 3) * 8;
    int valid = (r < R && k < K) ? min(8, K - k) : 0;
    stage_chunk(
        S + rl * SKC + (c & 3) * 8, [&](int i) { return ptr(rl, r, k + i); }, valid, contiguous);
  }
}
template <class F>  // ptr(kl, k, col) -> element (k, col); runs of 8 are contiguous while col + 8 <= Cv
__device__ __forceinline__ void stage_cc(bf16 *S, int c0, int k0, int C, int Cv, int K, F ptr) {
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    int c = threadIdx.x + TTH * q, kl = c >> 3, k = k0 + kl, col = c0 + (c & 7) * 8;
    int valid = (k < K && col < C) ? min(8, C - col) : 0;
    stage_chunk(
        S + kl * SMC + (c & 7) * 8, [&](int i) { return ptr(kl, k, col + i); }, valid, col + 8 <= Cv);
  }
}

// Tensor-core grouped GEMM engine (BF16 x BF16 -> FP32): C[M x N] = A[M x K] B[K x N] for
// z = blockIdx.z.  Op::kAKc: A staged [m][k] (k contiguous) else [k][m]; Op::kBKc: B staged [n][k]
// else [k][n].  K-chunks of 32 stream through a 3-stage cp.async pipeline; 4 warps each own a
// 32x32 block of the 64x64 tile (2 x 4 mma.sync m16n8k16 per 16 of K).  The accumulation order
// of an output element does not depend on its tile position.
template <class Op>
constexpr int tgemm_smem() {
  constexpr int stage = Op::kStages * (ASZ + BSZ) * 2, tile = TBM * (TBN + 4) * 4;
  return (stage > tile ? stage : tile) + TBM * Op::kTokSlots * 2;
}

template <class Op>
__global__ void __launch_bounds__(TTH) tgemm_kernel(Op op) {
  constexpr int STG = Op::kStages;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ long long mbase[TBM];
  bf16 *As = reinterpret_cast<bf16 *>(smem);
  bf16 *Bs = As + STG * ASZ;
  constexpr int stage_bytes = STG * (ASZ + BSZ) * 2, tile_bytes = TBM * (TBN + 4) * 4;
  uint16_t *toks = reinterpret_cast<uint16_t *>(smem + (stage_bytes > tile_bytes ? stage_bytes : tile_bytes));
  const int z = blockIdx.z;
  if (!op.active(z)) return;
  const int M = op.M(z), N = op.N(z), K = op.K(z);
  const int m0 = blockIdx.x * TBM, n0 = blockIdx.y * TBN;
  if (m0 >= M || n0 >= N) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int mw = (warp >> 1) * 32, nw = (warp & 1) * 32;
  if (tid < TBM) mbase[tid] = m0 + tid < M ? op.mrow_base(z, m0 + tid) : -1;
  __syncthreads();
  if constexpr (Op::kTokSlots > 0) {  // context tokens of the tile's rows, staged once
    op.stage_tokens(toks, mbase, z);
    __syncthreads();
  }
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;
  const int kb = op.kbeg(z);  // first K of this CTA (split-K ops), a multiple of TBK
  const int nk = (K - kb + TBK - 1) / TBK;
#pragma unroll
  for (int s = 0; s < STG - 1; ++s) {
    if (s < nk) {
      op.stage_a(As + s * ASZ, mbase, toks, z, m0, kb + s * TBK, M, K);
      op.stage_b(Bs + s * BSZ, z, kb + s * TBK, n0, K, N);
    }
    cp_commit();
  }
  for (int kt = 0; kt < nk; ++kt) {
    cp_wait<STG - 2>();
    __syncthreads();
    const int nxt = kt + STG - 1;
    if (nxt < nk) {
      op.stage_a(As + (nxt % STG) * ASZ, mbase, toks, z, m0, kb + nxt * TBK, M, K);
      op.stage_b(Bs + (nxt % STG) * BSZ, z, kb + nxt * TBK, n0, K, N);
    }
    cp_commit();
    const bf16 *Ak = As + (kt % STG) * ASZ, *Bk = Bs + (kt % STG) * BSZ;
#pragma unroll
    for (int kk = 0; kk < TBK; kk += 16) {
      uint32_t a[2][4], b[4][2];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        if (Op::kAKc) {
          int r = mw + 16 * i + (lane & 15), k = kk + 8 * (lane >> 4);
          ldm4(a[i], saddr(&Ak[r * SKC + k]));
        } else {
          int k = kk + (lane & 7) + 8 * (lane >> 4), m = mw + 16 * i + 8 * ((lane >> 3) & 1);
          ldm4t(a[i], saddr(&Ak[k * SMC + m]));
        }
      }
#pragma unroll
      for (int j = 0; j < 4; j += 2) {
        uint32_t r[4];
        if (Op::kBKc) {
          int n = nw + 8 * j + (lane & 7) + 8 * (lane >> 4), k = kk + 8 * ((lane >> 3) & 1);
          ldm4(r, saddr(&Bk[n * SKC + k]));
        } else {
          int k = kk + (lane & 7) + 8 * ((lane >> 3) & 1), n = nw + 8 * j + 8 * (lane >> 4);
          ldm4t(r, saddr(&Bk[k * SMC + n]));
        }
        b[j][0] = r[0], b[j][1] = r[1], b[j + 1][0] = r[2], b[j + 1][1] = r[3];
      }
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], a[i], b[j][0], b[j][1]);
    }
  }
  cp_wait<0>();
  __syncthreads();
  if constexpr (Op::kTileEpi) {
    // stage the tile in shared memory so the epilogue can walk it row-contiguously (coalesced)
    float *Cs = reinterpret_cast<float *>(smem);
    constexpr int LD = TBN + 4;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          int rl = mw + 16 * i + (lane >> 2) + 8 * h, cl = nw + 8 * j + 2 * (lane & 3);
          Cs[rl * LD + cl] = acc[i][j][2 * h];
          Cs[rl * LD + cl + 1] = acc[i][j][2 * h + 1];
        }
    __syncthreads();
    op.epi_tile(z, m0, n0, M, N, Cs, LD);
  } else {
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          int rl = mw + 16 * i + (lane >> 2) + 8 * h, r = m0 + rl;
          int c = n0 + nw + 8 * j + 2 * (lane & 3);
          if (r < M) op.epi2(mbase, z, r, rl, c, acc[i][j][2 * h], acc[i][j][2 * h + 1], N);
        }
  }
}

template <class Op>
void run_tgemm(const Op &op, int Mmax, int Nmax, int Z, cudaStream_t st) {
  if (Mmax <= 0 || Nmax <= 0 || Z <= 0) return;
  dim3 grid((Mmax + TBM - 1) / TBM, (Nmax + TBN - 1) / TBN, Z);
  constexpr int smem = tgemm_smem<Op>();
  if (!smem_optin((const void *)tgemm_kernel<Op>, smem)) return;  // error left for cudaGetLastError
  tgemm_kernel<Op><<<grid, TTH, smem, st>>>(op);
}

// ---- ops -----------------------------------------------------------------------------------
struct BBase {
  static constexpr bool kTileEpi = false;
  static constexpr int kStages = 3, kTokSlots = 0;
  Plan p;
  int T;
  __device__ void epi_tile(int, int, int, int, int, const float *, int) const {}
  __device__ int kbeg(int) const { return 0; }
  __device__ void stage_tokens(uint16_t *, const long long *, int) const {}
  __device__ int nrows(int g) const { return p.grp_lane_off[g + 1] - p.grp_lane_off[g]; }
  __device__ int row(int g, int r) const { return p.grp_lane_off[g] + r; }
  __device__ long long target_pos(int g, int r) const {
    int rw = row(g, r);
    if (!row_pred(p, T, rw, g)) return -1;
    return p.lane_tok[rw] + (T - p.grp_start[g]);
  }
  __device__ long long mrow_base(int z, int r) const { return target_pos(z % p.G, r); }
  __device__ const bf16 *xptr(const bf16 *w, const Dims &D, long long tpos, int k) const {
    int pos = k / D.E, e = k - pos * D.E;
    int tok = p.tokens[tpos - D.t + pos];
    return w + D.off_emb() + (size_t)tok * D.E + e;
  }
  __device__ const bf16 *wb(int g) const { return p.wbf + (size_t)g * p.P; }
};

// Partial sums of h = X W1 over K-slices: z = (model*G + g)*S + slice (model 0 dynamic, 1 static);
// the slices are summed in order by hidden_reduce_kernel, which adds b1, applies relu and stores
// BF16 h.  Splitting K gives enough CTAs to hide the gather and weight-stream latency.
struct HiddenB : BBase {
  static constexpr bool kAKc = true, kBKc = true;
  float *part;  // [2][S][NL][Hmax] partial sums
  int hmax;
  __device__ int zz(int z) const { return z / kHiddenSplit; }
  __device__ int slice(int z) const { return z % kHiddenSplit; }
  __device__ bool stat(int z) const { return zz(z) >= p.G; }
  __device__ int grp(int z) const { return zz(z) % p.G; }
  __device__ const Dims &d(int z) const { return stat(z) ? p.st : p.dm; }
  __device__ const bf16 *w(int z) const { return stat(z) ? p.static_bf : wb(grp(z)); }
  __device__ bool active(int z) const { return group_trains(p, T, grp(z)); }
  __device__ int M(int z) const { return nrows(grp(z)); }
  __device__ int N(int z) const { return d(z).H; }
  __device__ int kper(int z) const {
    int k = d(z).K1();
    return ((k + kHiddenSplit - 1) / kHiddenSplit + TBK - 1) / TBK * TBK;
  }
  __device__ int kbeg(int z) const { return min(d(z).K1(), slice(z) * kper(z)); }
  __device__ int K(int z) const { return min(d(z).K1(), (slice(z) + 1) * kper(z)); }
  __device__ long long mrow_base(int z, int r) const { return target_pos(grp(z), r); }
  __device__ void stage_a(bf16 *S, const long long *mb, const uint16_t *, int z, int m0, int k0, int M,
                          int K) const {
    const bf16 *wz = w(z);
    const Dims &D = d(z);
    stage_kc(
        S, m0, k0, M, K,
        [&](int rl, int, int k) -> const bf16 * {
          long long b = mb[rl];
          return b < 0 ? nullptr : xptr(wz, D, b, k);
        },
        D.E % 8 == 0);
  }
  __device__ void stage_b(bf16 *S, int z, int k0, int n0, int K, int N) const {
    const bf16 *w1t = w(z) + d(z).off_w1();  // B[k][n] = W1t[n][k]; the row stride is the full K
    const int KX = d(z).K1();
    stage_kc(
        S, n0, k0, N, K, [&](int, int n, int k) -> const bf16 * { return w1t + (size_t)n * KX + k; }, true);
  }
  __device__ void epi2(const long long *, int z, int r, int, int c, float a0, float a1, int N) const {
    float *o = part + (((size_t)(stat(z) ? 1 : 0) * kHiddenSplit + slice(z)) * p.NL + row(grp(z), r)) * hmax;
    if (c < N) o[c] = a0;
    if (c + 1 < N) o[c + 1] = a1;
  }
};

// h = relu(sum_slices + b1) -> BF16, for the predicted rows of every active group and model.
__global__ void hidden_reduce_kernel(Plan p, int T, const float *part, int hmax) {
  const int model = blockIdx.y;  // 0 dynamic, 1 static
  const Dims &D = model ? p.st : p.dm;
  const int H = D.H;
  const uint32_t total = (uint32_t)p.NL * (uint32_t)H;  // 32-bit indices: no FP64-based 64-bit division
  for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < total; w += gridDim.x * blockDim.x) {
    const int r = (int)(w / (uint32_t)H), c = (int)(w - (uint32_t)r * (uint32_t)H);
    const int g = p.lane_grp[r];
    if (!row_pred(p, T, r, g)) continue;
    float acc = 0.f;
#pragma unroll
    for (int sl = 0; sl < kHiddenSplit; ++sl)
      acc += part[(((size_t)model * kHiddenSplit + sl) * p.NL + r) * hmax + c];
    const float *b1 = (model ? p.static_params : p.params + (size_t)g * p.P) + D.off_b1();
    (model ? p.hs_b : p.hd_b)[(size_t)r * H + c] = __float2bfloat16_rn(fmaxf(acc + b1[c], 0.f));
  }
}

struct LogitsB : BBase {
  static constexpr bool kAKc = true, kBKc = false;
  __device__ bool stat(int z) const { return z >= p.G; }
  __device__ const Dims &d(int z) const { return stat(z) ? p.st : p.dm; }
  __device__ bool active(int z) const { return group_trains(p, T, z % p.G); }
  __device__ int M(int z) const { return nrows(z % p.G); }
  __device__ int N(int z) const { return d(z).A; }
  __device__ int K(int z) const { return d(z).H; }
  __device__ void stage_a(bf16 *S, const long long *mb, const uint16_t *, int z, int m0, int k0, int M,
                          int K) const {
    const bf16 *h = stat(z) ? p.hs_b : p.hd_b;
    const int g = z % p.G;
    stage_kc(
        S, m0, k0, M, K,
        [&](int rl, int m, int k) -> const bf16 * { return mb[rl] < 0 ? nullptr : h + (size_t)row(g, m) * K + k; },
        true);
  }
  __device__ void stage_b(bf16 *S, int z, int k0, int n0, int K, int N) const {
    const bf16 *w2 = (stat(z) ? p.static_bf : wb(z)) + d(z).off_w2();
    stage_cc(S, n0, k0, N, N, K, [&](int, int k, int c) -> const bf16 * { return w2 + (size_t)k * N + c; });
  }
  __device__ void epi2(const long long *mb, int z, int r, int rl, int c, float a0, float a1, int N) const {
    if (mb[rl] < 0) return;
    const float *b2 = (stat(z) ? p.static_params : p.params + (size_t)z * p.P) + d(z).off_b2();
    float *o = (stat(z) ? p.zu : p.zm) + (size_t)row(z % p.G, r) * N;
    if (c < N) o[c] = a0 + b2[c];
    if (c + 1 < N) o[c + 1] = a1 + b2[c + 1];
  }
};

// dh = (dz W2^T) * [h > 0]
struct DhB : BBase {
  static constexpr bool kAKc = true, kBKc = true;
  __device__ bool active(int z) const { return group_trains(p, T, z); }
  __device__ int M(int z) const { return nrows(z); }
  __device__ int N(int) const { return p.dm.H; }
  __device__ int K(int) const { return p.dm.A; }
  __device__ void stage_a(bf16 *S, const long long *mb, const uint16_t *, int z, int m0, int k0, int M,
                          int K) const {
    stage_kc(
        S, m0, k0, M, K,
        [&](int rl, int m, int k) -> const bf16 * {
          return mb[rl] < 0 ? nullptr : p.dz_b + (size_t)row(z, m) * K + k;
        },
        true);
  }
  __device__ void stage_b(bf16 *S, int z, int k0, int n0, int K, int N) const {
    const bf16 *w2 = wb(z) + p.dm.off_w2();  // row n of B^T = W2[n][.]
    stage_kc(
        S, n0, k0, N, K, [&](int, int n, int k) -> const bf16 * { return w2 + (size_t)n * K + k; }, true);
  }
  __device__ void epi2(const long long *mb, int z, int r, int rl, int c, float a0, float a1, int N) const {
    size_t i = (size_t)row(z, r) * N + c;
    bool ok = mb[rl] >= 0;
    if (c < N) p.dh_b[i] = __float2bfloat16_rn((ok && __bfloat162float(p.hd_b[i]) > 0.f) ? a0 : 0.f);
    if (c + 1 < N) p.dh_b[i + 1] = __float2bfloat16_rn((ok && __bfloat162float(p.hd_b[i + 1]) > 0.f) ? a1 : 0.f);
  }
};

// [dW2; db2] = [h 1]^T dz -> gradient buffer (row H of the tile is the bias gradient)
struct DW2B : BBase {
  static constexpr bool kAKc = false, kBKc = false, kTileEpi = true;
  __device__ bool active(int z) const { return group_trains(p, T, z); }
  __device__ int M(int) const { return p.dm.H + 1; }
  __device__ int N(int) const { return p.dm.A; }
  __device__ int K(int z) const { return nrows(z); }
  __device__ long long mrow_base(int, int) const { return 0; }
  __device__ void stage_a(bf16 *S, const long long *, const uint16_t *, int z, int m0, int k0, int M,
                          int K) const {
    const int H = p.dm.H;
    stage_cc(S, m0, k0, M, H, K, [&](int, int r, int i) -> const bf16 * {
      if (target_pos(z, r) < 0) return nullptr;
      return i < H ? p.hd_b + (size_t)row(z, r) * H + i : reinterpret_cast<const bf16 *>(&kOneBfBits);
    });
  }
  __device__ void stage_b(bf16 *S, int z, int k0, int n0, int K, int N) const {
    stage_cc(S, n0, k0, N, N, K, [&](int, int r, int c) -> const bf16 * {
      return target_pos(z, r) < 0 ? nullptr : p.dz_b + (size_t)row(z, r) * N + c;
    });
  }
  __device__ void epi2(const long long *, int, int, int, int, float, float, int) const {}
  __device__ void epi_tile(int z, int m0, int n0, int M, int N, const float *Cs, int ld) const {
    const int H = p.dm.H;
    store_grad_tile(p, z, m0, n0, M, N, Cs, ld,
                    [&](int i) -> size_t { return i < H ? p.dm.off_w2() + (size_t)i * N : p.dm.off_b2(); });
  }
};

// dX = dh W1^T scattered into the embedding rows (fixed-point atomics)
struct DXB : BBase {
  static constexpr bool kAKc = true, kBKc = false;
  __device__ bool active(int z) const { return group_trains(p, T, z); }
  __device__ int M(int z) const { return nrows(z); }
  __device__ int N(int) const { return p.dm.K1(); }
  __device__ int K(int) const { return p.dm.H; }
  __device__ void stage_a(bf16 *S, const long long *mb, const uint16_t *, int z, int m0, int k0, int M,
                          int K) const {
    stage_kc(
        S, m0, k0, M, K,
        [&](int rl, int m, int k) -> const bf16 * {
          return mb[rl] < 0 ? nullptr : p.dh_b + (size_t)row(z, m) * K + k;
        },
        true);
  }
  __device__ void stage_b(bf16 *S, int z, int k0, int n0, int K, int N) const {
    const bf16 *w1t = wb(z) + p.dm.off_w1();  // B[h][i] = W1[i][h] = W1t[h][i]
    stage_cc(S, n0, k0, N, N, K, [&](int, int h, int i) -> const bf16 * { return w1t + (size_t)h * N + i; });
  }
  __device__ void one(long long b, int z, int i, float acc) const {
    int pos = i / p.dm.E, e = i - pos * p.dm.E;
    int tok = p.tokens[b - p.dm.t + pos];
    long long q = fix40(acc);
    atomicAdd(reinterpret_cast<unsigned long long *>(p.demb_acc + ((size_t)z * p.dm.A + tok) * p.dm.E + e),
              (unsigned long long)q);
  }
  __device__ void epi2(const long long *mb, int z, int, int rl, int c, float a0, float a1, int N) const {
    long long b = mb[rl];
    if (b < 0) return;
    if (c < N) one(b, z, c, a0);
    if (c + 1 < N) one(b, z, c + 1, a1);
  }
};

// [dW1; db1] = [X 1]^T dh -> gradient buffer; W1 is stored transposed (W1t[h][i]), so the tile is
// written column-wise: four consecutive i of one h per store.
struct DW1B : BBase {
  static constexpr bool kAKc = false, kBKc = false, kTileEpi = true;
  __device__ bool active(int z) const { return group_trains(p, T, z); }
  __device__ int M(int) const { return p.dm.K1() + 1; }
  __device__ int N(int) const { return p.dm.H; }
  __device__ int K(int z) const { return nrows(z); }
  __device__ long long mrow_base(int, int) const { return 0; }
  __device__ void stage_a(bf16 *S, const long long *, const uint16_t *, int z, int m0, int k0, int M,
                          int K) const {
    const int KX = p.dm.K1(), E = p.dm.E;
    const bf16 *wz = wb(z);
    stage_cc(S, m0, k0, M, (E % 8 == 0) ? KX : 0, K, [&](int, int r, int i) -> const bf16 * {
      long long b = target_pos(z, r);
      if (b < 0) return nullptr;
      return i < KX ? xptr(wz, p.dm, b, i) : reinterpret_cast<const bf16 *>(&kOneBfBits);
    });
  }
  __device__ void stage_b(bf16 *S, int z, int k0, int n0, int K, int N) const {
    stage_cc(S, n0, k0, N, N, K, [&](int, int r, int c) -> const bf16 * {
      return target_pos(z, r) < 0 ? nullptr : p.dh_b + (size_t)row(z, r) * N + c;
    });
  }
  __device__ void epi2(const long long *, int, int, int, int, float, float, int) const {}
  __device__ void epi_tile(int z, int m0, int n0, int M, int N, const float *Cs, int ld) const {
    const int KX = p.dm.K1();
    float *gr = p.grad + (size_t)z * p.P;
    float *g1t = gr + p.dm.off_w1();
    for (int q = threadIdx.x; q < TBN * (TBM / 4); q += TTH) {
      int cl = q / (TBM / 4), rl = (q % (TBM / 4)) * 4, c = n0 + cl, i = m0 + rl;
      if (c >= N || i >= M) continue;
      float v[4];
      for (int e = 0; e < 4; ++e) v[e] = Cs[(rl + e) * ld + cl];
      float *dst = g1t + (size_t)c * KX + i;
      if (i + 3 < KX && ((reinterpret_cast<uintptr_t>(dst) & 15) == 0)) {
        *reinterpret_cast<float4 *>(dst) = make_float4(v[0], v[1], v[2], v[3]);
      } else {
        for (int e = 0; e < 4 && i + e < M; ++e) {
          if (i + e < KX)
            dst[e] = v[e];
          else
            gr[p.dm.off_b1() + c] = v[e];  // the bias row
        }
      }
    }
  }
};

__global__ void to_bf16_kernel(const float *src, bf16 *dst, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = __float2bfloat16_rn(src[i]);
}

}  // namespace

void launch_to_bf16(const float *src, void *dst, size_t n, cudaStream_t st) {
  if (n == 0) return;
  size_t grid = (n + 255) / 256;
  if (grid > 152 * 32) grid = 152 * 32;
  to_bf16_kernel<<<(unsigned)grid, 256, 0, st>>>(src, reinterpret_cast<bf16 *>(dst), n);
}

void launch_forward_bf16(const Plan &p, int T, cudaStream_t st, int which) {
  if (tc_supported(p)) {
    launch_forward_tc(p, T, st, which);
    return;
  }
  if (which != kFwdBoth) return;  // the mma.sync form runs both models together only
  const double R = prof_work().pred_rows;
  const int Z = p.use_static ? 2 * p.G : p.G;
  const int Hmax = p.use_static ? max(p.dm.H, p.st.H) : p.dm.H;
  // a BiGRU static predictor forms its own h: the hidden GEMM then covers the dynamic models only
  const bool s_hid = p.use_static && !p.st_gru;
  {
    double fl = 2.0 * R * p.dm.K1() * p.dm.H + (s_hid ? 2.0 * R * p.st.K1() * p.st.H : 0.0);
    ProfScope ps("fwd_hidden_bf16", fl, 0, st);
    HiddenB op{{p, T}, p.hpart, Hmax};
    run_tgemm(op, p.Mmax, Hmax, (s_hid ? Z : p.G) * kHiddenSplit, st);
    size_t n = (size_t)p.NL * Hmax, grid = (n + 255) / 256;
    if (grid > 152 * 16) grid = 152 * 16;
    hidden_reduce_kernel<<<dim3((unsigned)grid, s_hid ? 2 : 1), 256, 0, st>>>(p, T, p.hpart, Hmax);
  }
  if (p.use_static && p.st_gru) launch_bigru_static(p, T, st);
  double fl = 2.0 * R * p.dm.H * p.dm.A + (p.use_static ? 2.0 * R * p.st.H * p.st.A : 0.0);
  ProfScope ps("fwd_logits_bf16", fl, 0, st);
  run_tgemm(LogitsB{{p, T}}, p.Mmax, p.dm.A, Z, st);
}

void launch_backward_bf16(const Plan &p, int T, cudaStream_t st, const StepStreams *ss) {
  if (tc_supported(p)) {
    launch_backward_tc(p, T, st, ss);
    return;
  }
  const double R = prof_work().pred_rows;
  {
    ProfScope ps("bwd_dh_bf16", 2.0 * R * p.dm.A * p.dm.H, 0, st);
    run_tgemm(DhB{{p, T}}, p.Mmax, p.dm.H, p.G, st);
  }
  {
    ProfScope ps("bwd_dw2_bf16", 2.0 * R * p.dm.A * p.dm.H, 0, st);
    run_tgemm(DW2B{{p, T}}, p.dm.H + 1, p.dm.A, p.G, st);
  }
  {
    ProfScope ps("bwd_dx_bf16", 2.0 * R * p.dm.K1() * p.dm.H, 0, st);
    run_tgemm(DXB{{p, T}}, p.Mmax, p.dm.K1(), p.G, st);
  }
  {
    ProfScope ps("bwd_dw1_bf16", 2.0 * R * p.dm.K1() * p.dm.H, 0, st);
    run_tgemm(DW1B{{p, T}}, p.dm.K1() + 1, p.dm.H, p.G, st);
  }
}

}  // namespace pmklc
