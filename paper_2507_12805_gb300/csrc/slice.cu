// The logits layer and its input gradient restricted to the coded slice (BF16 forms, overlap-masked
// coding with s < k, paper §4.1 tokens): a row whose previous token is e codes its next token among
// the 4^s tokens that agree with e, the columns [q W, q W + W) of the alphabet with W = 4^s and
// q = e mod 4^(k-s), so only those logits are formed and only those entries of dz are non-zero:
//
//   L[r, q W + c]  = b2[q W + c] + sum_h h[r, h] W2[h, q W + c]          c < W
//   dh[r, h]       = (sum_c dz[r, q W + c] W2[h, q W + c]) [h[r, h] > 0]
//
// Both read, per row, the W columns of W2 that its slice selects (H x W BF16, 32 KB for the (3,6)
// model), so one CTA per (group, model) sorts the group's predicted rows by slice and walks the
// slices present, up to 16 rows at a time: the slice's W2 columns and the rows' operands are
// copied to shared memory in parts of 128 hidden units (cp.async into four part buffers, two CTAs
// per SM: the next three parts' copies overlap this part's products) and multiplied with mma.sync
// m16n8k16 into FP32 accumulators.  Every group's W2 is
// read about once per step, so the pass is bound by that read (about 2 FLOP per byte), not by
// the multiplies.  A row's results depend only on its own operands and the fixed K order of the
// products, not on which rows share its chunk, so encoder and decoder agree bit for bit.
#include <cuda_bf16.h>

#include "internal.h"

namespace pmklc {

namespace {

using bf16 = __nv_bfloat16;
constexpr int kSlThreads = 256;   // eight warps
constexpr int kSlRows = 16;       // rows per chunk: one m16n8k16 row tile
constexpr int kSlMaxSlices = 1024;
constexpr int kSlPad = 8;         // BF16 padding of staged rows: ldmatrix rows fall in distinct banks
constexpr int kSlMaxRows = 8192;  // rows of a group (row indices kept in 16 bits)
constexpr int kSlMaxStages = 4;   // chunk buffers: up to three chunks' copies in flight
constexpr size_t kSlSmemMax = 220 * 1024;

__device__ __forceinline__ uint32_t sl_sa(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void sl_ldm4(uint32_t (&r)[4], uint32_t a) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}
__device__ __forceinline__ void sl_ldm2(uint32_t &b0, uint32_t &b1, uint32_t a) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n" : "=r"(b0), "=r"(b1) : "r"(a));
}
__device__ __forceinline__ void sl_ldm2t(uint32_t &b0, uint32_t &b1, uint32_t a) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];\n" : "=r"(b0), "=r"(b1) : "r"(a));
}
__device__ __forceinline__ void sl_mma(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
__device__ const uint4 kSlZero16 = {0u, 0u, 0u, 0u};
// 16 bytes global -> shared, asynchronously; a zero fill when !real
__device__ __forceinline__ void sl_cp16(void *dst, const void *src, bool real) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sl_sa(dst)), "l"(real ? src : &kSlZero16),
               "r"(real ? 16 : 0));
}
__device__ __forceinline__ void sl_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void sl_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

// Shared-memory layout of one CTA (byte offsets; every region 16-byte aligned).  A chunk (up to 16
// rows of one slice) is staged in parts of hp rows of W2 (the hidden units h in [k hp, k hp + hp)):
// the logits accumulate over the parts, dh writes the part's columns, so a buffer holds hp x W of
// W2 and one part of the rows' operands, and several parts are in flight at once.
struct SliceLayout {
  int nq, mrows, hp, W, ka;  // slices, rows of the largest group, part height, slice width, A-operand K
  int dh;                    // 1: the dh pass (the rows' h of the part staged too, for the ReLU mask)
  int ns;                    // part buffers
  __host__ __device__ static size_t up16(size_t x) { return (x + 15) & ~(size_t)15; }
  __host__ __device__ size_t slab_bytes() const { return (size_t)hp * (W + kSlPad) * 2; }
  __host__ __device__ size_t arow_bytes() const { return (size_t)kSlRows * (ka + kSlPad) * 2; }
  __host__ __device__ size_t hrow_bytes() const { return dh ? (size_t)kSlRows * hp * 2 : 0; }
  __host__ __device__ size_t stage_bytes() const { return slab_bytes() + arow_bytes() + hrow_bytes(); }
  __host__ __device__ size_t red_off() const { return (size_t)ns * stage_bytes(); }  // k-split partial sums
  __host__ __device__ size_t cnt_off() const { return red_off() + (size_t)kSlThreads * 4 * 4; }
  __host__ __device__ size_t rstart_off() const { return cnt_off() + up16((size_t)nq * 4); }
  __host__ __device__ size_t cstart_off() const { return rstart_off() + up16((size_t)(nq + 1) * 4); }
  __host__ __device__ size_t rq_off() const { return cstart_off() + up16((size_t)(nq + 1) * 4); }
  __host__ __device__ size_t list_off() const { return rq_off() + up16((size_t)mrows * 2); }
  __host__ __device__ size_t chrow_off() const { return list_off() + up16((size_t)mrows * 2); }
  __host__ __device__ size_t chq_off() const { return chrow_off() + up16((size_t)mrows * 2); }
  __host__ __device__ size_t bytes() const { return chq_off() + up16((size_t)mrows * 2); }
};

// part height of a model with H hidden units (H % 64 == 0)
__host__ __device__ inline int slice_part(int H) { return H % 128 == 0 ? 128 : 64; }

// kDh false: the logits of problem z (z < G: group z's dynamic model, else the static model on group
// z - G's rows); kDh true: dh of group z.  L: the layout for the launch's largest model.
template <bool kDh>
__global__ void __launch_bounds__(kSlThreads, 2) slice_kernel(Plan p, int T, int zb, SliceLayout L) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ __align__(16) uint8_t sl_smem[];
  __shared__ int n_chunks;
  const int z = zb + blockIdx.x;
  const bool stat = !kDh && z >= p.G;
  const int g = stat ? z - p.G : z;
  if (!group_trains(p, T, g)) return;  // the same for the whole CTA
  const Dims D = stat ? p.st : p.dm;
  const int H = D.H, A = D.A, W = p.ov_w, nq = p.ov_mod;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  int *cnt = reinterpret_cast<int *>(sl_smem + L.cnt_off());
  int *rstart = reinterpret_cast<int *>(sl_smem + L.rstart_off());
  int *cstart = reinterpret_cast<int *>(sl_smem + L.cstart_off());
  short *rq = reinterpret_cast<short *>(sl_smem + L.rq_off());
  uint16_t *list = reinterpret_cast<uint16_t *>(sl_smem + L.list_off());
  uint16_t *chrow = reinterpret_cast<uint16_t *>(sl_smem + L.chrow_off());
  uint16_t *chq = reinterpret_cast<uint16_t *>(sl_smem + L.chq_off());
  const int r0 = p.grp_lane_off[g], nr = p.grp_lane_off[g + 1] - r0;
  const long long j = T - p.grp_start[g];

  // the group's predicted rows sorted by slice (counting sort; order within a slice is immaterial)
  for (int q = tid; q < nq; q += kSlThreads) cnt[q] = 0;
  __syncthreads();
  for (int r = tid; r < nr; r += kSlThreads) {
    const int rw = r0 + r;
    int q = -1;
    if (row_pred(p, T, rw, g)) q = (int)p.tokens[p.lane_tok[rw] + j - 1] % nq;  // a predicted row's index >= 1
    rq[r] = (short)q;
    if (q >= 0) atomicAdd(&cnt[q], 1);
  }
  __syncthreads();
  if (warp == 0) {  // exclusive prefix sums of the rows and of the 16-row chunks of every slice
    const int per = (nq + 31) / 32, q0 = lane * per, q1 = min(nq, q0 + per);
    int sr = 0, sc = 0;
    for (int q = q0; q < q1; ++q) sr += cnt[q], sc += (cnt[q] + kSlRows - 1) / kSlRows;
    int xr = sr, xc = sc;
    for (int o = 1; o < 32; o <<= 1) {
      const int yr = __shfl_up_sync(0xffffffffu, xr, o), yc = __shfl_up_sync(0xffffffffu, xc, o);
      if (lane >= o) xr += yr, xc += yc;
    }
    int br = xr - sr, bc = xc - sc;
    for (int q = q0; q < q1; ++q) {
      rstart[q] = br, cstart[q] = bc;
      br += cnt[q], bc += (cnt[q] + kSlRows - 1) / kSlRows;
    }
    if (lane == 31) rstart[nq] = xr, cstart[nq] = xc, n_chunks = xc;
  }
  __syncthreads();
  for (int q = tid; q < nq; q += kSlThreads) {
    for (int c = cstart[q], k = 0; c < cstart[q + 1]; ++c, ++k)
      chrow[c] = (uint16_t)(rstart[q] + k * kSlRows), chq[c] = (uint16_t)q;
    cnt[q] = rstart[q];  // placement cursor
  }
  __syncthreads();
  for (int r = tid; r < nr; r += kSlThreads) {
    const int q = rq[r];
    if (q >= 0) list[atomicAdd(&cnt[q], 1)] = (uint16_t)r;
  }
  if (kDh) {  // rows that predict nothing get dh = 0 (the lane-reducing GEMMs read the group's rows)
    const int h8 = H / 8;
    for (int idx = tid; idx < nr * h8; idx += kSlThreads) {
      const int r = idx / h8;
      if (rq[r] < 0)
        *reinterpret_cast<uint4 *>(p.dh_b + (size_t)(r0 + r) * H + 8 * (idx - r * h8)) = make_uint4(0u, 0u, 0u, 0u);
    }
  }
  __syncthreads();

  const bf16 *w2 = (stat ? p.static_bf : p.wbf + (size_t)g * p.P) + D.off_w2();
  const float *b2 = (stat ? p.static_params : p.params + (size_t)g * p.P) + D.off_b2();
  const bf16 *asrc = kDh ? p.dz_b : (stat ? p.hs_b : p.hd_b);  // rows of the A operand
  const int hp = slice_part(H), nparts = H / hp;
  const int ald = kDh ? A : H, ka = kDh ? W : hp, wc = W / 8, kc = ka / 8, hc = hp / 8;
  const int sw = W + kSlPad, sa_ = ka + kSlPad;  // staged row strides (elements)
  auto slab_of = [&](int buf) { return reinterpret_cast<bf16 *>(sl_smem + (size_t)buf * L.stage_bytes()); };
  auto arow_of = [&](int buf) {
    return reinterpret_cast<bf16 *>(sl_smem + (size_t)buf * L.stage_bytes() + L.slab_bytes());
  };
  auto hrow_of = [&](int buf) {
    return reinterpret_cast<bf16 *>(sl_smem + (size_t)buf * L.stage_bytes() + L.slab_bytes() + L.arow_bytes());
  };
  // unit u = part k of chunk c (u = c nparts + k): rows [k hp, k hp + hp) of the slice's W2 columns and
  // the chunk rows' operand part, asynchronously
  auto stage = [&](int buf, int u) {
    const int c = u / nparts, k = u - c * nparts, h0 = k * hp;
    bf16 *slab = slab_of(buf), *arow = arow_of(buf);
    const int q = chq[c], row0 = chrow[c], n = min(kSlRows, rstart[q + 1] - row0), lo = q * W;
    for (int idx = tid; idx < hp * wc; idx += kSlThreads) {
      const int h = idx / wc, cc = idx - h * wc;
      sl_cp16(slab + h * sw + 8 * cc, w2 + (size_t)(h0 + h) * A + lo + 8 * cc, true);
    }
    for (int idx = tid; idx < kSlRows * kc; idx += kSlThreads) {
      const int i = idx / kc, cc = idx - i * kc;
      const bool real = i < n;
      const bf16 *src =
          real ? asrc + (size_t)(r0 + list[row0 + i]) * ald + (kDh ? lo : h0) + 8 * cc : nullptr;
      sl_cp16(arow + i * sa_ + 8 * cc, src, real);
    }
    if (kDh) {  // the part of the rows' h (BF16, unpadded): the ReLU mask of the epilogue
      bf16 *hrow = hrow_of(buf);
      for (int idx = tid; idx < kSlRows * hc; idx += kSlThreads) {
        const int i = idx / hc, cc = idx - i * hc;
        const bool real = i < n;
        sl_cp16(hrow + i * hp + 8 * cc, real ? p.hd_b + (size_t)(r0 + list[row0 + i]) * H + h0 + 8 * cc : nullptr,
                real);
      }
    }
  };

  const int nu = n_chunks * nparts;
  const int gq = lane >> 2, tq = lane & 3;  // accumulator rows gq, gq + 8; columns 2 tq, 2 tq + 1
  float4 *red = reinterpret_cast<float4 *>(sl_smem + L.red_off());
  // L.ns buffers: units u + 1 .. u + ns - 1 in flight while unit u is multiplied; one commit group
  // per unit slot (empty past the last unit), so "all but the newest ns - 1 groups done" means unit
  // u has landed
  const int ns = L.ns;
  for (int u = 0; u < ns - 1; ++u) {
    if (u < nu) stage(u, u);
    sl_commit();
  }
  // logits: W / 8 column tiles; the eight warps split each part's K when there are fewer tiles than
  // warps, and the partial sums are added in K order after the last part
  const int ntl = W / 8, ks = 8 / ntl, ln0 = (warp % ntl) * 8, kp = warp / ntl, kst = hp / 16 / ks;
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  for (int u = 0; u < nu; ++u) {
    if (u + ns - 1 < nu) stage((u + ns - 1) % ns, u + ns - 1);
    sl_commit();
    if (ns == 2) sl_wait<1>();
    else if (ns == 3) sl_wait<2>();
    else sl_wait<3>();
    __syncthreads();
    const int buf = u % ns, c = u / nparts, k = u - c * nparts;
    const bf16 *slab = slab_of(buf), *arow = arow_of(buf);
    const int q = chq[c], row0 = chrow[c], n = min(kSlRows, rstart[q + 1] - row0), lo = q * W;
    if constexpr (!kDh) {
      if (k == 0) acc[0] = acc[1] = acc[2] = acc[3] = 0.f;
      for (int kk = kp * kst; kk < (kp + 1) * kst; ++kk) {
        const int k0 = kk * 16;
        uint32_t a[4], b0, b1;
        sl_ldm4(a, sl_sa(arow + (lane & 15) * sa_ + k0 + (lane >> 4) * 8));
        sl_ldm2t(b0, b1, sl_sa(slab + (k0 + (lane & 15)) * sw + ln0));
        sl_mma(acc, a, b0, b1);
      }
      if (k == nparts - 1) {
        if (ks > 1) {
          red[warp * 32 + lane] = make_float4(acc[0], acc[1], acc[2], acc[3]);
          __syncthreads();
          if (kp == 0)
            for (int m = 1; m < ks; ++m) {
              const float4 v = red[(warp + m * ntl) * 32 + lane];
              acc[0] += v.x, acc[1] += v.y, acc[2] += v.z, acc[3] += v.w;
            }
        }
        if (kp == 0) {
          const int col = lo + ln0 + 2 * tq;
          const float c0 = b2[col], c1 = b2[col + 1];
          float *zout = stat ? p.zu : p.zm;
#pragma unroll
          for (int hf = 0; hf < 2; ++hf) {
            const int i = gq + 8 * hf;
            if (i < n)
              *reinterpret_cast<float2 *>(zout + (size_t)(r0 + list[row0 + i]) * A + col) =
                  make_float2(acc[2 * hf] + c0, acc[2 * hf + 1] + c1);
          }
        }
      }
    } else {
      // K = W (at most four 16-deep steps, their A fragments kept); the warps take the part's hp / 8
      // column tiles in turn
      uint32_t a[4][4];
      const int nks = W / 16;
      const bf16 *hrow = hrow_of(buf);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk)
        if (kk < nks) sl_ldm4(a[kk], sl_sa(arow + (lane & 15) * sa_ + kk * 16 + (lane >> 4) * 8));
      for (int nt = warp; nt < hp / 8; nt += kSlThreads / 32) {
        const int n0 = nt * 8;
        float d[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
          if (kk < nks) {
            uint32_t b0, b1;
            sl_ldm2(b0, b1, sl_sa(slab + (n0 + (lane & 7)) * sw + kk * 16 + ((lane >> 3) & 1) * 8));
            sl_mma(d, a[kk], b0, b1);
          }
        const int hl = n0 + 2 * tq;  // column within the part
#pragma unroll
        for (int hf = 0; hf < 2; ++hf) {
          const int i = gq + 8 * hf;
          if (i < n) {
            const __nv_bfloat162 hv = *reinterpret_cast<const __nv_bfloat162 *>(hrow + i * hp + hl);
            const float x0 = __low2float(hv) > 0.f ? d[2 * hf] : 0.f;
            const float x1 = __high2float(hv) > 0.f ? d[2 * hf + 1] : 0.f;
            *reinterpret_cast<__nv_bfloat162 *>(p.dh_b + (size_t)(r0 + list[row0 + i]) * H + k * hp + hl) =
                __floats2bfloat162_rn(x0, x1);
          }
        }
      }
    }
    __syncthreads();  // the buffer is restaged ns - 1 units on
  }
}

// up to kSlMaxStages part buffers, fewer if the layout would not fit
SliceLayout slice_layout(const Plan &p, bool dh) {
  const int hp = !dh && p.use_static ? max(slice_part(p.dm.H), slice_part(p.st.H)) : slice_part(p.dm.H);
  SliceLayout L{p.ov_mod, p.Mmax, hp, p.ov_w, dh ? p.ov_w : hp, dh ? 1 : 0, kSlMaxStages};
  while (L.ns > 2 && L.bytes() > kSlSmemMax) --L.ns;
  return L;
}

}  // namespace

bool slice_rule(const Plan &p) {
  const int W = p.ov_w;
  if (W < 16 || W > 64 || W % 16 != 0 || p.ov_mod < 1 || p.ov_mod > kSlMaxSlices || p.Mmax > kSlMaxRows) return false;
  if (p.dm.H % 64 != 0 || (p.use_static && p.st.H % 64 != 0)) return false;
  return slice_layout(p, false).bytes() <= kSlSmemMax && slice_layout(p, true).bytes() <= kSlSmemMax;
}

void launch_slice_logits(const Plan &p, int T, cudaStream_t st, int zb, int Z) {
  const SliceLayout L = slice_layout(p, false);
  if (Z <= 0 || !smem_optin((const void *)slice_kernel<false>, (int)L.bytes())) return;
  launch_pdl(slice_kernel<false>, dim3(Z), dim3(kSlThreads), L.bytes(), st, p, T, zb, L);
}

void launch_slice_dh(const Plan &p, int T, cudaStream_t st) {
  const SliceLayout L = slice_layout(p, true);
  if (p.G <= 0 || !smem_optin((const void *)slice_kernel<true>, (int)L.bytes())) return;
  launch_pdl(slice_kernel<true>, dim3(p.G), dim3(kSlThreads), L.bytes(), st, p, T, 0, L);
}

}  // namespace pmklc
