// (s,k)-mer encoding and decoding (GskE, paper §4.1 and Fig. 3), input
// validation and a parallel CRC-32, on sm_103a.
//
// The paper's encoder maps A/C/G/T to 0..3 and reads each window of k bases,
// taken every s bases, as a base-4 number with the first base most
// significant ("CGG" -> 26).  Here a CTA reads a segment of bases with 16-byte
// loads, validates and packs them to 2 bits in shared memory, and cuts each token
// from the packed stream with a shift and a mask.
#include <stdio.h>

#include <mutex>
#include <vector>

#include "internal.h"

namespace pmklc {

__device__ __forceinline__ bool is_acgt(uint32_t c) { return c == 'A' || c == 'C' || c == 'G' || c == 'T'; }
// A=0x41 -> 0, C=0x43 -> 1, G=0x47 -> 2, T=0x54 -> 3
__device__ __forceinline__ uint32_t base_code(uint32_t c) { return ((c >> 1) & 3u) ^ ((c >> 2) & 1u); }

__device__ __forceinline__ int find_block(const long long *off, int n_blocks, long long x) {
  // largest b with off[b] <= x (off has n_blocks + 1 ascending entries)
  int lo = 0, hi = n_blocks - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= x)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// Fused validation and (s,k)-mer encoding.  Each CTA owns kTokSeg consecutive bases of one block
// (its block read from a per-CTA table, then the block's offsets in one round of loads): it reads its bases
// plus the k - 1 after them with 16-byte loads, checks the bases it owns, packs all of them to 2
// bits (16 per 32-bit word, the first base in the most significant bits) in shared memory, and
// writes the tokens j whose first base j*s lies in its range: token j is the 2k-bit field of the
// packed stream at base j*s, cut from a 64-bit window of two words.
// Four bases per 32-bit operation (byte i of x is base i): their codes, one per byte (the A/C/G/T
// map of base_code applied bytewise)...
__device__ __forceinline__ uint32_t swar_codes(uint32_t x) {
  return ((x >> 1) & 0x03030303u) ^ ((x >> 2) & 0x01010101u);
}
// ... packed to 8 bits with base 0 most significant (bytes reversed, then two shift-ors fold the
// four 2-bit codes into the low byte) ...
__device__ __forceinline__ uint32_t swar_pack(uint32_t t) {
  const uint32_t r = __byte_perm(t, 0u, 0x0123u);  // c3 | c2 << 8 | c1 << 16 | c0 << 24
  const uint32_t x = r | (r >> 6);                 // low byte c3 | c2 << 2, byte 2 c1 | c0 << 2
  return (x | (x >> 12)) & 0xFFu;
}
// ... and the bytes (under mask) that are not the letter their code stands for: the four letters
// rebuilt from the codes by a byte permutation of "ACGT" and compared with the input.
__device__ __forceinline__ uint32_t swar_bad(uint32_t x, uint32_t t, uint32_t mask) {
  // the codes as the permutation's four selector nibbles: c0 | c1 << 4 in byte 0 and c2 | c3 << 4
  // in byte 2 of t | t >> 4, moved to bytes 0 and 1 (the upper two selector bytes pick zeros)
  const uint32_t sel = __byte_perm(t | (t >> 4), 0u, 0x4420u);
  return (__byte_perm(0x54474341u, 0u, sel) ^ x) & mask;
}
// Byte mask of the window bytes [o, o + 4) that lie in the owned range [sh, sh + own).
__device__ __forceinline__ uint32_t owned_bytes(int o, int sh, int own) {
  const int lo = max(sh - o, 0), hi = min(sh + own - o, 4);
  return lo >= hi ? 0u : ((0xFFFFFFFFu >> (8 * (4 - hi))) & (0xFFFFFFFFu << (8 * lo)));
}

constexpr int kTokSeg = 8192;                     // bases owned by one CTA
constexpr int kTokWin = kTokSeg + 48;             // bytes loaded: alignment slack (< 16) + owned + k - 1 + pad
constexpr int kTokWords = kTokWin / 16 + 1;       // packed words (+1 so a window's second word exists)
constexpr int kTokThreads = 256;

__global__ void __launch_bounds__(kTokThreads) tokenize_packed_kernel(
    const uint8_t *__restrict__ seq, size_t n_all, const long long *__restrict__ base_off,
    const long long *__restrict__ tok_off, const int *__restrict__ cta_off, const int *__restrict__ cta_blk, int s,
    int k, uint16_t *__restrict__ tokens, int *err) {
  __shared__ uint32_t words[kTokWords];
  const int tid = threadIdx.x;
  const int c = blockIdx.x;
  const int b = cta_blk[c];  // the block this CTA works in
  const long long nb = base_off[b + 1] - base_off[b];
  const long long a = (long long)(c - cta_off[b]) * kTokSeg;  // first owned base (block-relative)
  const long long own = min((long long)kTokSeg, nb - a);       // owned bases
  const uint8_t *ga = seq + base_off[b] + a;
  const uint8_t *g0 = reinterpret_cast<const uint8_t *>(reinterpret_cast<uintptr_t>(ga) & ~(uintptr_t)15);
  const int sh = (int)(ga - g0);                    // window byte of owned base 0
  const uint8_t *end = seq + n_all;
  bool bad = false;
  for (int w = tid; w < kTokWords; w += kTokThreads) {
    const uint8_t *p = g0 + 16 * (size_t)w;
    uint32_t word = 0;
    if (p + 16 <= end && p >= seq) {  // whole vector inside the sequence: four bytes per operation
      const uint4 v = *reinterpret_cast<const uint4 *>(p);
      const uint32_t q[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      uint32_t t[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        t[i] = swar_codes(q[i]);
        word |= swar_pack(t[i]) << (24 - 8 * i);
      }
      if (16 * w >= sh && 16 * w + 16 <= sh + (int)own) {  // every byte owned (all but the edges)
        bad |= (swar_bad(q[0], t[0], ~0u) | swar_bad(q[1], t[1], ~0u) | swar_bad(q[2], t[2], ~0u) |
                swar_bad(q[3], t[3], ~0u)) != 0;
      } else {
#pragma unroll
        for (int i = 0; i < 4; ++i) bad |= swar_bad(q[i], t[i], owned_bytes(16 * w + 4 * i, sh, (int)own)) != 0;
      }
    } else {  // the sequence's first or last partial vector: byte loads inside it only
#pragma unroll 1
      for (int i = 0; i < 16; ++i) {
        const uint8_t *pi = p + i;
        if (pi < seq || pi >= end) continue;  // outside the sequence: code 0, never part of a token
        const uint32_t ch = *pi;
        const long long rel = 16LL * w + i - sh;
        if (rel >= 0 && rel < own) bad |= !is_acgt(ch);
        word |= base_code(ch) << (30 - 2 * i);
      }
    }
    words[w] = word;
  }
  if (__any_sync(0xffffffffu, bad) && (tid & 31) == 0) atomicOr(err, kErrBadBase);
  __syncthreads();
  // tokens j of this block with a <= j*s < a + own
  const long long l = tok_off[b + 1] - tok_off[b];
  // 64-bit integer division compiles to slow FP64-based code on GB300: blocks below 2^31 bases
  // (every practical one) divide in 32 bits
  long long j0, j1;
  if (a + own + s < (1LL << 31)) {
    j0 = (long long)((unsigned)(a + s - 1) / (unsigned)s);
    j1 = (long long)((unsigned)(a + own + s - 1) / (unsigned)s);
  } else {
    j0 = (a + s - 1) / s;
    j1 = (a + own + s - 1) / s;
  }
  j1 = min(l, j1);
  // from here on 32-bit offsets from the CTA's first token: q is the window byte of a token's first
  // base, and its 2k bits are the top of the 64-bit window (words[w], words[w + 1]) shifted left by
  // 2 (q mod 16) (one funnel shift; 2 (q mod 16) + 2k <= 46 bits stay inside the window)
  const int cnt = (int)max(0LL, j1 - j0);
  const int q0 = (int)(j0 * s - a) + sh;
  uint16_t *out = tokens + tok_off[b] + j0;
  for (int jj = tid; jj < cnt; jj += kTokThreads) {
    const int q = q0 + jj * s;
    const int w = q >> 4, o = q & 15;
    const uint32_t top = __funnelshift_l(words[w + 1], words[w], 2 * o);
    out[jj] = (uint16_t)(top >> (32 - 2 * k));
  }
}

std::vector<int> tokenize_ctas(const std::vector<long long> &base_off) {
  const size_t nb = base_off.empty() ? 0 : base_off.size() - 1;
  std::vector<int> cta(nb + 1, 0), blk;
  for (size_t b = 0; b < nb; ++b) {
    const int n = (int)((base_off[b + 1] - base_off[b] + kTokSeg - 1) / kTokSeg);
    cta[b + 1] = cta[b] + n;
    blk.insert(blk.end(), (size_t)n, (int)b);
  }
  cta.insert(cta.end(), blk.begin(), blk.end());
  return cta;
}

void launch_validate_tokenize(const uint8_t *d_seq, size_t n, const long long *d_base_off, const long long *d_tok_off,
                              const int *d_cta, int n_blocks, int n_cta, int s, int k, uint16_t *d_tokens,
                              int *d_err, cudaStream_t st) {
  if (n_cta <= 0) return;
  tokenize_packed_kernel<<<n_cta, kTokThreads, 0, st>>>(d_seq, n, d_base_off, d_tok_off, d_cta, d_cta + n_blocks + 1,
                                                        s, k, d_tokens, d_err);
}

__global__ void tails_kernel(const uint8_t *__restrict__ seq, const long long *__restrict__ base_off,
                             const long long *__restrict__ tok_off, int n_blocks, int s, int k, uint8_t *tail) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n_blocks) return;
  long long n = base_off[b + 1] - base_off[b];
  long long l = tok_off[b + 1] - tok_off[b];
  long long covered = l > 0 ? (l - 1) * s + k : 0;
  for (int i = 0; i < 8; ++i)
    tail[b * 8 + i] = (covered + i < n) ? (uint8_t)base_code(seq[base_off[b] + covered + i]) : 0;
}

void launch_tails(const uint8_t *d_seq, const long long *d_base_off, const long long *d_tok_off, int n_blocks,
                  int s, int k, uint8_t *d_tail, cudaStream_t st) {
  if (n_blocks <= 0) return;
  tails_kernel<<<(n_blocks + 127) / 128, 128, 0, st>>>(d_seq, d_base_off, d_tok_off, n_blocks, s, k, d_tail);
}

// One thread per output base of the selected blocks.  Base i of a block is digit i of
// token 0 when i < k, else digit k-s+m of token j = (i-k)/s + 1 (m = (i-k) mod s), else
// tail[i - covered].  The thread owning the first new base of token j >= 1 also checks
// that the k-s overlapping digits agree with token j-1.
__global__ void detokenize_kernel(const uint16_t *__restrict__ tokens, const uint8_t *__restrict__ tail,
                                  const long long *__restrict__ base_off, const long long *__restrict__ tok_off,
                                  const int *__restrict__ sel, int n_blocks, long long n_bases, int s, int k,
                                  uint8_t *__restrict__ seq, int *err) {
  long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (x >= n_bases) return;
  int b = find_block(base_off, n_blocks, x);
  if (!sel[b]) return;
  long long i = x - base_off[b];
  long long l = tok_off[b + 1] - tok_off[b];
  long long covered = l > 0 ? (l - 1) * s + k : 0;
  uint32_t code;
  if (i >= covered) {
    code = tail[b * 8 + (i - covered)];
  } else if (i < k) {
    uint32_t t0 = tokens[tok_off[b]];
    code = (t0 >> (2 * (k - 1 - i))) & 3u;
  } else {
    long long j = (i - k) / s + 1;
    int m = (int)((i - k) % s);
    uint32_t tj = tokens[tok_off[b] + j];
    int d = k - s + m;
    code = (tj >> (2 * (k - 1 - d))) & 3u;
    if (m == 0 && s < k) {
      uint32_t prev = tokens[tok_off[b] + j - 1];
      uint32_t lo = prev & ((1u << (2 * (k - s))) - 1u);
      if (lo != (tj >> (2 * s))) atomicOr(err, kErrCorrupt);
    }
  }
  seq[x] = "ACGT"[code];
}

void launch_detokenize(const uint16_t *d_tokens, const uint8_t *d_tail, const long long *d_base_off,
                       const long long *d_tok_off, const int *d_sel, int n_blocks, long long n_bases, int s, int k,
                       uint8_t *d_seq, int *d_err, cudaStream_t st) {
  if (n_bases <= 0) return;
  detokenize_kernel<<<(unsigned)((n_bases + 255) / 256), 256, 0, st>>>(d_tokens, d_tail, d_base_off, d_tok_off, d_sel,
                                                                        n_blocks, n_bases, s, k, d_seq, d_err);
}

// ---------------------------------------------------------------------------
// CRC-32 (reflected polynomial 0xEDB88320, zlib's).  The register update
// c <- T[(c ^ byte) & 0xFF] ^ (c >> 8) is linear over GF(2), so the register
// after a chunk D started from c equals R(D, 0) xor Z_|D| c, where Z_n is the
// 32x32 matrix of n zero bytes.  Chunks are processed in parallel from 0 and
// folded left with Z; the ragged end is finished byte by byte.

constexpr int kCrcChunk = 4096;
constexpr int kCrcFold = 256;  // threads of the folding kernel

__device__ __forceinline__ uint32_t crc_table_entry(uint32_t i) {
  uint32_t c = i;
  for (int b = 0; b < 8; ++b) c = (c & 1u) ? (0xEDB88320u ^ (c >> 1)) : (c >> 1);
  return c;
}

__device__ __forceinline__ uint32_t gf2_apply(const uint32_t *mat, uint32_t v) {
  uint32_t out = 0;
  for (int i = 0; v; ++i, v >>= 1)
    if (v & 1u) out ^= mat[i];
  return out;
}

__global__ void crc_chunks_kernel(const uint8_t *__restrict__ data, long long n_chunks, uint32_t *__restrict__ regs) {
  __shared__ uint32_t tab[256];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) tab[i] = crc_table_entry(i);
  __syncthreads();
  long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= n_chunks) return;
  const uint4 *p = reinterpret_cast<const uint4 *>(data + c * kCrcChunk);
  uint32_t r = 0;
  for (int q = 0; q < kCrcChunk / 16; ++q) {
    uint4 w = p[q];
    uint32_t words[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int t = 0; t < 4; ++t)
#pragma unroll
      for (int b = 0; b < 4; ++b) r = tab[(r ^ (words[t] >> (8 * b))) & 0xFFu] ^ (r >> 8);
  }
  regs[c] = r;
}

// mats: [0] = Z_chunk, [1] = Z_(chunk*per), [2] = Z_(chunk*last_count); 32 words each
__global__ void crc_fold_kernel(const uint8_t *__restrict__ head, int head_len, const uint32_t *__restrict__ regs,
                                long long n_chunks, long long per, const uint32_t *__restrict__ mats,
                                const uint8_t *__restrict__ rest, int rest_len, uint32_t *out) {
  __shared__ uint32_t part[kCrcFold];
  __shared__ uint32_t tab[256];
  __shared__ uint32_t m[3][32];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) tab[i] = crc_table_entry(i);
  for (int i = threadIdx.x; i < 96; i += blockDim.x) m[i / 32][i % 32] = mats[i];
  __syncthreads();
  long long lo = threadIdx.x * per, hi = lo + per < n_chunks ? lo + per : n_chunks;
  uint32_t x = 0;
  for (long long c = lo; c < hi; ++c) x = regs[c] ^ gf2_apply(m[0], x);
  part[threadIdx.x] = x;
  __syncthreads();
  if (threadIdx.x != 0) return;
  uint32_t acc = 0xFFFFFFFFu;
  for (int i = 0; i < head_len; ++i) acc = tab[(acc ^ head[i]) & 0xFFu] ^ (acc >> 8);
  for (int t = 0; t < kCrcFold; ++t) {
    long long a = t * per, e = a + per < n_chunks ? a + per : n_chunks;
    if (a >= e) break;
    acc = part[t] ^ gf2_apply(e - a == per ? m[1] : m[2], acc);
  }
  for (int i = 0; i < rest_len; ++i) acc = tab[(acc ^ rest[i]) & 0xFFu] ^ (acc >> 8);
  *out = ~acc;
}

namespace {
// column i = image of basis vector e_i
void gf2_mul(const uint32_t *a, const uint32_t *b, uint32_t *out) {  // out = a*b
  for (int i = 0; i < 32; ++i) {
    uint32_t v = b[i], r = 0;
    for (int j = 0; v; ++j, v >>= 1)
      if (v & 1u) r ^= a[j];
    out[i] = r;
  }
}
void zero_bytes_matrix(unsigned long long nbytes, uint32_t *out) {
  uint32_t one[32], acc[32], tmp[32];
  for (int i = 0; i < 32; ++i) {  // one zero byte: c -> T[c & 0xFF] ^ (c >> 8)
    uint32_t c = 1u << i, t = c & 0xFFu, e = t;
    for (int b = 0; b < 8; ++b) e = (e & 1u) ? (0xEDB88320u ^ (e >> 1)) : (e >> 1);
    one[i] = e ^ (c >> 8);
    acc[i] = 1u << i;
    (void)t;
  }
  while (nbytes) {
    if (nbytes & 1) {
      gf2_mul(one, acc, tmp);
      for (int i = 0; i < 32; ++i) acc[i] = tmp[i];
    }
    gf2_mul(one, one, tmp);
    for (int i = 0; i < 32; ++i) one[i] = tmp[i];
    nbytes >>= 1;
  }
  for (int i = 0; i < 32; ++i) out[i] = acc[i];
}
}  // namespace

int crc32_device(const uint8_t *d_all, size_t n_all, uint32_t *crc, cudaStream_t st) {
  size_t head = (16 - (reinterpret_cast<uintptr_t>(d_all) & 15)) & 15;
  if (head > n_all) head = n_all;
  const uint8_t *d_data = d_all + head;
  size_t n = n_all - head;
  long long n_chunks = (long long)(n / kCrcChunk);
  long long per = (n_chunks + kCrcFold - 1) / kCrcFold;
  if (per == 0) per = 1;
  long long last = n_chunks - (n_chunks > 0 ? ((n_chunks - 1) / per) * per : 0);
  uint32_t mats[96];
  zero_bytes_matrix(kCrcChunk, mats);
  zero_bytes_matrix((unsigned long long)kCrcChunk * per, mats + 32);
  zero_bytes_matrix((unsigned long long)kCrcChunk * (last > 0 ? last : 1), mats + 64);
  uint32_t *d_regs = nullptr, *d_mats = nullptr, *d_out = nullptr;
  size_t bytes = sizeof(uint32_t) * (size_t)(n_chunks + 96 + 1);
  PMKLC_CUDA_TRY(cudaMallocAsync((void **)&d_regs, bytes, st));
  d_mats = d_regs + n_chunks;
  d_out = d_mats + 96;
  cudaMemcpyAsync(d_mats, mats, sizeof(mats), cudaMemcpyHostToDevice, st);
  if (n_chunks > 0)
    crc_chunks_kernel<<<(unsigned)((n_chunks + 127) / 128), 128, 0, st>>>(d_data, n_chunks, d_regs);
  int rest_len = (int)(n - (size_t)n_chunks * kCrcChunk);
  crc_fold_kernel<<<1, kCrcFold, 0, st>>>(d_all, (int)head, d_regs, n_chunks, per, d_mats, d_data + (size_t)n_chunks * kCrcChunk,
                                          rest_len, d_out);
  uint32_t h = 0;
  cudaMemcpyAsync(&h, d_out, sizeof(h), cudaMemcpyDeviceToHost, st);
  cudaFreeAsync(d_regs, st);
  PMKLC_CUDA_TRY(cudaStreamSynchronize(st));
  PMKLC_CUDA_TRY(cudaGetLastError());
  *crc = h;
  return PMKLC_OK;
}

}  // namespace pmklc

namespace pmklc {

// ---------------------------------------------------------------------------
// CRC-32 without any device allocation.
//
// Its scratch (one register per 4 KiB chunk, the three zero-byte matrices and the result word)
// lives in a file-scope device array of fixed size instead of cudaMallocAsync memory, for
// callers that cannot allocate: a process whose device memory is handed out entirely by another
// framework's pool allocator, or a latency-sensitive loop that must not pay for an allocation.
// The array holds kNoAllocCrcChunks chunk registers, i.e. inputs up to 256 MiB (+ 15 head bytes
// and up to 4095 tail bytes); every device that loads the library keeps it (about 256 KiB) until
// the process exits.  All calls share it and it keeps the last call's contents; nothing in it
// needs to start at zero (each call writes every slot it reads), but calls that overlap on the
// GPU (different streams, or host threads) race on it and must be serialised by the caller.

namespace {
constexpr long long kNoAllocCrcChunks = 65536;
__device__ __align__(256) uint32_t g_crc_scratch[kNoAllocCrcChunks + 96 + 1];

constexpr int kMaxDevices = 64;
uint32_t *g_crc_scratch_addr[kMaxDevices];  // device address of g_crc_scratch, per device
std::mutex g_crc_scratch_mu;

// Set-up, once per device with that device current: the host-side name of the array is a
// stand-in, not a device address, so the kernels get the address cudaGetSymbolAddress returns.
int crc_scratch_addr(uint32_t **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PMKLC_ECUDA;
  std::lock_guard<std::mutex> lock(g_crc_scratch_mu);
  if (!g_crc_scratch_addr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_crc_scratch) != cudaSuccess || !p) return PMKLC_ECUDA;
    g_crc_scratch_addr[dev] = static_cast<uint32_t *>(p);
  }
  *out = g_crc_scratch_addr[dev];
  return PMKLC_OK;
}
}  // namespace

}  // namespace pmklc

extern "C" int pmklc_crc32_noalloc(const uint8_t *d_all, size_t n_all, uint32_t *crc, void *stream) {
  using namespace pmklc;
  if (!crc || (n_all && !d_all)) return PMKLC_EINVAL;
  size_t head = (16 - (reinterpret_cast<uintptr_t>(d_all) & 15)) & 15;
  if (head > n_all) head = n_all;
  const uint8_t *d_data = d_all + head;
  size_t n = n_all - head;
  long long n_chunks = (long long)(n / kCrcChunk);
  if (n_chunks > kNoAllocCrcChunks) return PMKLC_EINVAL;  // larger than the fixed scratch
  uint32_t *scratch = nullptr;
  int rc = crc_scratch_addr(&scratch);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  long long per = (n_chunks + kCrcFold - 1) / kCrcFold;
  if (per == 0) per = 1;
  long long last = n_chunks - (n_chunks > 0 ? ((n_chunks - 1) / per) * per : 0);
  uint32_t mats[96];
  zero_bytes_matrix(kCrcChunk, mats);
  zero_bytes_matrix((unsigned long long)kCrcChunk * per, mats + 32);
  zero_bytes_matrix((unsigned long long)kCrcChunk * (last > 0 ? last : 1), mats + 64);
  uint32_t *d_regs = scratch, *d_mats = scratch + kNoAllocCrcChunks, *d_out = d_mats + 96;
  PMKLC_CUDA_TRY(cudaMemcpyAsync(d_mats, mats, sizeof(mats), cudaMemcpyHostToDevice, st));
  if (n_chunks > 0)
    crc_chunks_kernel<<<(unsigned)((n_chunks + 127) / 128), 128, 0, st>>>(d_data, n_chunks, d_regs);
  int rest_len = (int)(n - (size_t)n_chunks * kCrcChunk);
  crc_fold_kernel<<<1, kCrcFold, 0, st>>>(d_all, (int)head, d_regs, n_chunks, per, d_mats,
                                          d_data + (size_t)n_chunks * kCrcChunk, rest_len, d_out);
  uint32_t h = 0;
  PMKLC_CUDA_TRY(cudaMemcpyAsync(&h, d_out, sizeof(h), cudaMemcpyDeviceToHost, st));
  PMKLC_CUDA_TRY(cudaStreamSynchronize(st));
  PMKLC_CUDA_TRY(cudaGetLastError());
  *crc = h;
  return PMKLC_OK;
}
