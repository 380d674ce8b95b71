// Byte-oriented range coder (the paper's unspecified entropy encoder, §2 step 3;
// the reading used: G. N. N. Martin's range encoding with a 56-bit window, carry
// propagation through a cache byte and a count of pending 0xFF bytes).
// One coder state per lane; each call is made by one thread.
#pragma once
#include "common.cuh"

namespace pmklc {

constexpr unsigned long long kTop = 1ull << 56;
constexpr unsigned long long kBot = 1ull << 48;
constexpr unsigned long long kMask = kTop - 1;

__device__ __forceinline__ void enc_init(EncState &s) {
  s.low = 0;
  s.range = kTop - 1;
  s.cache = 0;
  s.pending = 0;
  s.pos = 0;
  s.has_cache = 0;
}

__device__ __forceinline__ void enc_put(EncState &s, uint8_t *out, uint32_t cap, uint32_t byte, int *err) {
  if (s.pos < cap)
    out[s.pos] = (uint8_t)byte;
  else
    atomicOr(err, kErrOverflow);
  s.pos++;
}

__device__ __forceinline__ void enc_shift_low(EncState &s, uint8_t *out, uint32_t cap, int *err) {
  if (s.low < (0xFFull << 48) || s.low >= kTop) {
    uint32_t carry = (uint32_t)(s.low >> 56);
    if (s.has_cache) enc_put(s, out, cap, (s.cache + carry) & 0xFF, err);
    for (; s.pending; --s.pending) enc_put(s, out, cap, (0xFF + carry) & 0xFF, err);
    s.cache = (uint32_t)(s.low >> 48) & 0xFF;
    s.has_cache = 1;
  } else {
    s.pending++;
  }
  s.low = (s.low << 8) & kMask;
}

// r = range / total for total = 2^24 (network and uniform tables)
__device__ __forceinline__ void enc_code24(EncState &s, uint32_t cum, uint32_t freq, uint8_t *out, uint32_t cap,
                                           int *err) {
  unsigned long long r = s.range >> kTotalBits;
  s.low += r * cum;
  s.range = r * freq;
  while (s.range < kBot) {
    enc_shift_low(s, out, cap, err);
    s.range <<= 8;
  }
}

// general total (count model)
__device__ __forceinline__ void enc_code(EncState &s, uint32_t cum, uint32_t freq, uint32_t total, uint8_t *out,
                                         uint32_t cap, int *err) {
  unsigned long long r = s.range / total;
  s.low += r * cum;
  s.range = r * freq;
  while (s.range < kBot) {
    enc_shift_low(s, out, cap, err);
    s.range <<= 8;
  }
}

// Final value with the most trailing zero bits inside [low, low+range), two shifts,
// trailing zero bytes dropped (the decoder reads bytes past the end as zero).
__device__ __forceinline__ uint32_t enc_finish(EncState &s, uint8_t *out, uint32_t cap, int *err) {
  unsigned long long hi = s.low + s.range;
  for (int b = 56; b >= 48; --b) {
    unsigned long long g = (1ull << b) - 1;
    unsigned long long v = (s.low + g) & ~g;
    if (v < hi) {
      s.low = v;
      break;
    }
  }
  enc_shift_low(s, out, cap, err);
  enc_shift_low(s, out, cap, err);
  uint32_t n = s.pos < cap ? s.pos : cap;
  while (n > 0 && out[n - 1] == 0) --n;
  s.pos = n;
  return n;
}

__device__ __forceinline__ uint32_t dec_byte(const uint8_t *in, uint32_t len, uint32_t pos) {
  return pos < len ? in[pos] : 0u;
}

__device__ __forceinline__ void dec_init(DecState &s, const uint8_t *in, uint32_t len) {
  unsigned long long c = 0;
  for (int i = 0; i < 7; ++i) c = (c << 8) | dec_byte(in, len, i);
  s.code = c;
  s.range = kTop - 1;
  s.pos = 7;
}

// First half of a decode step: the scaled target value v in [0, total).
__device__ __forceinline__ uint32_t dec_target24(const DecState &s, unsigned long long &r) {
  r = s.range >> kTotalBits;
  unsigned long long v = s.code / r;
  return v >= kTotal ? kTotal - 1 : (uint32_t)v;
}

__device__ __forceinline__ uint32_t dec_target(const DecState &s, uint32_t total, unsigned long long &r) {
  r = s.range / total;
  unsigned long long v = s.code / r;
  return v >= total ? total - 1 : (uint32_t)v;
}

// Second half: consume the decoded symbol's (cum, freq).
__device__ __forceinline__ void dec_consume(DecState &s, unsigned long long r, uint32_t cum, uint32_t freq,
                                            const uint8_t *in, uint32_t len) {
  s.code -= r * cum;
  s.range = r * freq;
  while (s.range < kBot) {
    s.code = (s.code << 8) | dec_byte(in, len, s.pos++);
    s.range <<= 8;
  }
}

}  // namespace pmklc
