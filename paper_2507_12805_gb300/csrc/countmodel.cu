// Adaptive order-m count model: the integer, exact judge and fallback coder of
// a block (not a component of the paper's method; it guards the learned path,
// which keeps a block only when it spends fewer bytes on it).
//
// It codes a block in the same lanes as the network, inside the same global
// steps: lane r's base stream is the k digits of its first token followed by
// the last s digits of each later token, so at local step j every live lane
// codes the bases its j-th token adds (k at j = 0, else s), one sub-step per
// base.  One table per block (counts c[ctx][b], ctx = previous m bases of the
// lane's stream, positions before its start read as A) is shared by all its
// lanes with a deterministic three-phase update per sub-step:
//   A  every live lane reads its context's counts and codes freq_b = 2c_b+1 out of
//      2 sum(c) + 4 (Krichevsky-Trofimov);
//   B  every live lane adds 1 to c[ctx][base] (integer atomics: order-free);
//   C  every used context whose largest count reached 1024 is halved once (by the
//      first live lane that used it).
// One thread block per data block and one thread per lane (<= 1024 lanes); table
// reads bypass L1 (ld.global.cg) so a phase sees the previous phase's atomics.
#include "internal.h"
#include "rangecoder.cuh"

namespace pmklc {

namespace {

constexpr uint32_t kCountLimit = 1024;

__global__ void __launch_bounds__(1024) count_step_kernel(Plan p, CountPlan c, int T) {
  __shared__ uint32_t sctx[1024];
  const int g = blockIdx.x;
  const int j = T - p.grp_start[g];
  if (j < 0 || j >= p.grp_steps[g]) return;
  const int cmode = c.grp_cmode[g];
  if (cmode == 0) return;
  const int r0 = p.grp_lane_off[g], M = p.grp_lane_off[g + 1] - r0;
  const int li = threadIdx.x;
  const int r = r0 + li;
  const bool live = li < M && j < p.lane_len[r];
  const int nb = j == 0 ? c.k : c.s;
  uint32_t *tab = c.table + ((size_t)g << (2 * c.m)) * 4;
  const uint32_t mask = (1u << (2 * c.m)) - 1u;
  long long tpos = live ? p.lane_tok[r] + j : 0;
  uint32_t tok = (live && cmode == 1) ? p.tokens[tpos] : 0u;
  uint32_t ctx = live ? c.ctx[r] : 0u, digits = 0;
  EncState es;
  DecState ds;
  uint8_t *buf = nullptr;
  uint32_t cap = 0;
  if (live) {
    buf = c.buf + c.buf_off[r];
    cap = c.buf_cap[r];
    if (cmode == 1)
      es = c.enc[r];
    else
      ds = c.dec[r];
  }
  for (int q = 0; q < nb; ++q) {
    uint32_t x = 0;
    if (li < 1024) sctx[li] = live ? ctx : 0xFFFFFFFFu;
    if (live) {  // phase A
      uint4 cw = __ldcg(reinterpret_cast<const uint4 *>(tab) + ctx);
      uint32_t cnt[4] = {cw.x, cw.y, cw.z, cw.w};
      uint32_t total = 2 * (cnt[0] + cnt[1] + cnt[2] + cnt[3]) + 4;
      if (cmode == 1) {
        x = (tok >> (2 * (nb - 1 - q))) & 3u;
        uint32_t cum = 0;
        for (uint32_t b = 0; b < x; ++b) cum += 2 * cnt[b] + 1;
        enc_code(es, cum, 2 * cnt[x] + 1, total, buf, cap, p.err);
      } else {
        unsigned long long rr;
        uint32_t v = dec_target(ds, total, rr);
        uint32_t cum = 0;
        x = 3;
        for (uint32_t b = 0; b < 4; ++b) {
          uint32_t f = 2 * cnt[b] + 1;
          if (v < cum + f) {
            x = b;
            break;
          }
          cum += f;
        }
        if (x == 3) cum = total - (2 * cnt[3] + 1);
        dec_consume(ds, rr, cum, 2 * cnt[x] + 1, buf, cap);
        digits = (digits << 2) | x;
      }
    }
    __syncthreads();
    if (live) atomicAdd(tab + (size_t)ctx * 4 + x, 1u);  // phase B
    __syncthreads();
    if (live) {  // phase C
      uint4 cw = __ldcg(reinterpret_cast<const uint4 *>(tab) + ctx);
      uint32_t mx = max(max(cw.x, cw.y), max(cw.z, cw.w));
      if (mx >= kCountLimit) {
        bool first = true;
        for (int o = 0; o < li && first; ++o) first = sctx[o] != ctx;
        if (first) {
          uint4 h = make_uint4(cw.x >> 1, cw.y >> 1, cw.z >> 1, cw.w >> 1);
          __stcg(reinterpret_cast<uint4 *>(tab) + ctx, h);
        }
      }
      ctx = ((ctx << 2) | x) & mask;
    }
    __syncthreads();
  }
  if (!live) return;
  c.ctx[r] = ctx;
  if (cmode == 1) {
    c.enc[r] = es;
  } else {
    c.dec[r] = ds;
    uint32_t t = digits;
    if (j > 0) {  // keep the k - s digits shared with the previous token
      uint32_t prev = p.tokens[tpos - 1];
      t = ((prev & ((1u << (2 * (c.k - c.s))) - 1u)) << (2 * c.s)) | digits;
    }
    p.tokens[tpos] = (uint16_t)t;
  }
}

__global__ void count_init_kernel(Plan p, CountPlan c, int encode) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= p.NL) return;
  c.ctx[r] = 0;
  if (encode) {
    EncState s;
    enc_init(s);
    c.enc[r] = s;
  } else {
    DecState s;
    dec_init(s, c.buf + c.buf_off[r], c.buf_cap[r]);
    c.dec[r] = s;
  }
}

__global__ void count_finish_kernel(Plan p, CountPlan c, uint32_t *lane_len) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= p.NL) return;
  EncState s = c.enc[r];
  lane_len[r] = enc_finish(s, c.buf + c.buf_off[r], c.buf_cap[r], p.err);
  c.enc[r] = s;
}

}  // namespace

void launch_count_step(const Plan &p, const CountPlan &c, int T, cudaStream_t st) {
  if (p.G <= 0 || p.Mmax <= 0) return;
  int threads = ((p.Mmax + 31) / 32) * 32;
  ProfScope ps("count_step", 0, 0, st);
  count_step_kernel<<<p.G, threads, 0, st>>>(p, c, T);
}

void launch_count_init(const Plan &p, const CountPlan &c, int encode, cudaStream_t st) {
  if (p.NL <= 0) return;
  count_init_kernel<<<(p.NL + 127) / 128, 128, 0, st>>>(p, c, encode);
}

void launch_count_finish(const Plan &p, const CountPlan &c, uint32_t *d_lane_len, cudaStream_t st) {
  if (p.NL <= 0) return;
  count_finish_kernel<<<(p.NL + 127) / 128, 128, 0, st>>>(p, c, d_lane_len);
}

}  // namespace pmklc
