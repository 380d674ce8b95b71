// Adaptive order-m count model: the integer, exact judge and fallback coder of
// a block (not a component of the paper's method; it guards the learned path,
// which codes a block only when it spends fewer bytes).
//
// One thread block per data block; the block's bases are coded one by one as a
// single range-coded stream.  Context = the previous m base codes (oldest most
// significant; positions before the block read as A).  Counts c[ctx][b] live in
// shared memory as four uint16; freq_b = 2c_b + 1, total = 2 sum c + 4
// (Krichevsky-Trofimov); after coding base x, c[ctx][x] += 1 and when it
// reaches 1024 all four counts of the context are halved.  Thread 0 codes;
// the other threads only clear the table.
#include "internal.h"
#include "rangecoder.cuh"

namespace pmklc {

namespace {

constexpr uint32_t kCountLimit = 1024;

__device__ __forceinline__ uint32_t code_of(uint32_t c) { return ((c >> 1) & 3u) ^ ((c >> 2) & 1u); }

__device__ __forceinline__ void ctx_counts(const unsigned long long *tab, uint32_t ctx, uint32_t c[4]) {
  unsigned long long w = tab[ctx];
  for (int b = 0; b < 4; ++b) c[b] = (uint32_t)(w >> (16 * b)) & 0xFFFFu;
}

__device__ __forceinline__ void ctx_update(unsigned long long *tab, uint32_t ctx, uint32_t c[4], uint32_t x) {
  c[x] += 1;
  if (c[x] >= kCountLimit)
    for (int b = 0; b < 4; ++b) c[b] >>= 1;
  tab[ctx] = (unsigned long long)c[0] | ((unsigned long long)c[1] << 16) | ((unsigned long long)c[2] << 32) |
             ((unsigned long long)c[3] << 48);
}

__global__ void count_encode_kernel(const uint8_t *__restrict__ seq, const unsigned long long *__restrict__ off, int m,
                                    uint8_t *__restrict__ out, const unsigned long long *__restrict__ out_off,
                                    const uint32_t *__restrict__ cap, uint32_t *__restrict__ len, int *err) {
  extern __shared__ unsigned long long tab[];
  const int b = blockIdx.x;
  const uint32_t nctx = 1u << (2 * m);
  for (uint32_t i = threadIdx.x; i < nctx; i += blockDim.x) tab[i] = 0ull;
  __syncthreads();
  if (threadIdx.x != 0) return;
  const uint8_t *s = seq + off[b];
  const unsigned long long n = off[b + 1] - off[b];
  uint8_t *o = out + out_off[b];
  const uint32_t cp = cap[b];
  EncState st;
  enc_init(st);
  const uint32_t mask = nctx - 1;
  uint32_t ctx = 0;
  for (unsigned long long i = 0; i < n; ++i) {
    uint32_t ch = s[i];
    if (!(ch == 'A' || ch == 'C' || ch == 'G' || ch == 'T')) {
      atomicOr(err, kErrBadBase);
      ch = 'A';
    }
    uint32_t x = code_of(ch);
    uint32_t c[4];
    ctx_counts(tab, ctx, c);
    uint32_t cum = 0;
    for (uint32_t q = 0; q < x; ++q) cum += 2 * c[q] + 1;
    uint32_t total = 2 * (c[0] + c[1] + c[2] + c[3]) + 4;
    enc_code(st, cum, 2 * c[x] + 1, total, o, cp, err);
    ctx_update(tab, ctx, c, x);
    ctx = ((ctx << 2) | x) & mask;
  }
  len[b] = enc_finish(st, o, cp, err);
}

__global__ void count_decode_kernel(const uint8_t *__restrict__ in, const unsigned long long *__restrict__ in_off,
                                    const uint32_t *__restrict__ in_len, const unsigned long long *__restrict__ off,
                                    const int *__restrict__ sel, int m, uint8_t *__restrict__ seq) {
  extern __shared__ unsigned long long tab[];
  const int b = blockIdx.x;
  if (!sel[b]) return;
  const uint32_t nctx = 1u << (2 * m);
  for (uint32_t i = threadIdx.x; i < nctx; i += blockDim.x) tab[i] = 0ull;
  __syncthreads();
  if (threadIdx.x != 0) return;
  const uint8_t *src = in + in_off[b];
  const uint32_t ln = in_len[b];
  uint8_t *dst = seq + off[b];
  const unsigned long long n = off[b + 1] - off[b];
  DecState st;
  dec_init(st, src, ln);
  const uint32_t mask = nctx - 1;
  uint32_t ctx = 0;
  for (unsigned long long i = 0; i < n; ++i) {
    uint32_t c[4];
    ctx_counts(tab, ctx, c);
    uint32_t total = 2 * (c[0] + c[1] + c[2] + c[3]) + 4;
    unsigned long long r;
    uint32_t v = dec_target(st, total, r);
    uint32_t x = 3, cum = 0;
    for (uint32_t q = 0; q < 4; ++q) {
      uint32_t f = 2 * c[q] + 1;
      if (v < cum + f) {
        x = q;
        break;
      }
      cum += f;
    }
    if (x == 3) cum = total - (2 * c[3] + 1);
    dec_consume(st, r, cum, 2 * c[x] + 1, src, ln);
    dst[i] = (uint8_t)"ACGT"[x];
    ctx_update(tab, ctx, c, x);
    ctx = ((ctx << 2) | x) & mask;
  }
}

int smem_for(int m) { return (int)(sizeof(unsigned long long) << (2 * m)); }

}  // namespace

int launch_count_encode(const uint8_t *d_seq, const unsigned long long *d_off, int n_blocks, int m, uint8_t *d_out,
                        const unsigned long long *d_out_off, const uint32_t *d_cap, uint32_t *d_len, int *d_err,
                        cudaStream_t st) {
  if (m < 0 || m > 7) return PMKLC_EINVAL;
  if (n_blocks <= 0) return PMKLC_OK;
  int smem = smem_for(m);
  PMKLC_CUDA_TRY(cudaFuncSetAttribute(count_encode_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  count_encode_kernel<<<n_blocks, 128, smem, st>>>(d_seq, d_off, m, d_out, d_out_off, d_cap, d_len, d_err);
  PMKLC_CUDA_TRY(cudaGetLastError());
  return PMKLC_OK;
}

int launch_count_decode(const uint8_t *d_in, const unsigned long long *d_in_off, const uint32_t *d_len,
                        const unsigned long long *d_off, const int *d_sel, int n_blocks, int m, uint8_t *d_seq,
                        cudaStream_t st) {
  if (m < 0 || m > 7) return PMKLC_EINVAL;
  if (n_blocks <= 0) return PMKLC_OK;
  int smem = smem_for(m);
  PMKLC_CUDA_TRY(cudaFuncSetAttribute(count_decode_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  count_decode_kernel<<<n_blocks, 128, smem, st>>>(d_in, d_in_off, d_len, d_off, d_sel, m, d_seq);
  PMKLC_CUDA_TRY(cudaGetLastError());
  return PMKLC_OK;
}

}  // namespace pmklc

using namespace pmklc;

extern "C" int pmklc_count_encode(const uint8_t *d_seq, const uint64_t *d_off, uint32_t n_blocks, uint32_t m,
                                  uint8_t *d_out, uint32_t cap, uint32_t *d_len, void *stream) {
  if (m > 7 || (n_blocks && (!d_off || !d_out || !d_len))) return PMKLC_EINVAL;
  if (n_blocks == 0) return PMKLC_OK;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned long long *d_oo = nullptr;
  uint32_t *d_cap = nullptr;
  int *d_err = nullptr;
  size_t bytes = sizeof(unsigned long long) * n_blocks + sizeof(uint32_t) * n_blocks + sizeof(int) + 16;
  char *blob = nullptr;
  PMKLC_CUDA_TRY(cudaMallocAsync((void **)&blob, bytes, st));
  d_oo = (unsigned long long *)blob;
  d_cap = (uint32_t *)(blob + sizeof(unsigned long long) * n_blocks);
  d_err = (int *)(blob + sizeof(unsigned long long) * n_blocks + sizeof(uint32_t) * n_blocks);
  unsigned long long *h_oo = new unsigned long long[n_blocks];
  uint32_t *h_cap = new uint32_t[n_blocks];
  for (uint32_t b = 0; b < n_blocks; ++b) {
    h_oo[b] = (unsigned long long)b * cap;
    h_cap[b] = cap;
  }
  cudaMemcpyAsync(d_oo, h_oo, sizeof(unsigned long long) * n_blocks, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(d_cap, h_cap, sizeof(uint32_t) * n_blocks, cudaMemcpyHostToDevice, st);
  cudaMemsetAsync(d_err, 0, sizeof(int), st);
  int rc = launch_count_encode(d_seq, (const unsigned long long *)d_off, (int)n_blocks, (int)m, d_out, d_oo, d_cap,
                               d_len, d_err, st);
  int h_err = 0;
  cudaMemcpyAsync(&h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
  cudaError_t e = cudaStreamSynchronize(st);
  cudaFreeAsync(blob, st);
  delete[] h_oo;
  delete[] h_cap;
  if (rc) return rc;
  if (e != cudaSuccess) return PMKLC_ECUDA;
  if (h_err & kErrBadBase) return PMKLC_EINVAL;
  if (h_err & kErrOverflow) return PMKLC_ENOSPC;
  return PMKLC_OK;
}

extern "C" int pmklc_count_decode(const uint8_t *d_in, const uint32_t *d_len, uint32_t cap, const uint64_t *d_off,
                                  uint32_t n_blocks, uint32_t m, uint8_t *d_seq, void *stream) {
  if (m > 7 || (n_blocks && (!d_in || !d_len || !d_off || !d_seq))) return PMKLC_EINVAL;
  if (n_blocks == 0) return PMKLC_OK;
  cudaStream_t st = (cudaStream_t)stream;
  char *blob = nullptr;
  size_t bytes = sizeof(unsigned long long) * n_blocks + sizeof(int) * n_blocks;
  PMKLC_CUDA_TRY(cudaMallocAsync((void **)&blob, bytes, st));
  unsigned long long *d_io = (unsigned long long *)blob;
  int *d_sel = (int *)(blob + sizeof(unsigned long long) * n_blocks);
  unsigned long long *h_io = new unsigned long long[n_blocks];
  int *h_sel = new int[n_blocks];
  for (uint32_t b = 0; b < n_blocks; ++b) {
    h_io[b] = (unsigned long long)b * cap;
    h_sel[b] = 1;
  }
  cudaMemcpyAsync(d_io, h_io, sizeof(unsigned long long) * n_blocks, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(d_sel, h_sel, sizeof(int) * n_blocks, cudaMemcpyHostToDevice, st);
  int rc = launch_count_decode(d_in, d_io, d_len, (const unsigned long long *)d_off, d_sel, (int)n_blocks, (int)m,
                               d_seq, st);
  cudaError_t e = cudaStreamSynchronize(st);
  cudaFreeAsync(blob, st);
  delete[] h_io;
  delete[] h_sel;
  if (rc) return rc;
  return e == cudaSuccess ? PMKLC_OK : PMKLC_ECUDA;
}
