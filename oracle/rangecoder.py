"""Entropy coding: a byte-oriented range coder, plus an exact arithmetic coder.

Test infrastructure only.  The paper's entropy encoder (§2 step 3, "EE" in
Fig. 2) turns each predicted distribution and target symbol into bits but is
not specified; the reading used here is range encoding (G. N. N.
Martin, 1979) with a 56-bit window and byte output, written with Python
integers so no intermediate can overflow:

  state: low < 2^57 (bit 56 is a pending carry), range, cache byte (none at
         start), count of pending 0xFF bytes
  start: low = 0, range = 2^56 - 1
  code (cum, freq, total):  r = range // total;  low += r*cum;  range = r*freq;
         while range < 2^48: shift_low(); range <<= 8
  shift_low: if low < 0xFF<<48 or low >= 2^56:
                 emit cache+carry (unless no cache yet), then each pending 0xFF
                 byte plus carry, and make the window's top byte the new cache
             else: one more pending 0xFF
             low = (low << 8) mod 2^56
  finish: pick in [low, low+range) the value with the most trailing zero bits
          at a granularity of 2^b, b = 56..48; shift_low twice; drop trailing
          zero bytes (the decoder reads missing bytes as zero).

Decoder: code = first 7 bytes; per symbol r = range // total,
v = min(code // r, total - 1), s such that cum_s <= v < cum_{s+1},
code -= r*cum_s, range = r*freq_s, then shift in bytes while range < 2^48.

Pins (tests): round trip on random tables; exact byte equality with the CUDA
coder given the same tables; length bound 8*bytes <= sum(-log2 q) +
N*2^-24/ln2 + 8 (per symbol: the truncation of range / 2^24;
at the end: the flush), checked against the exact rational
coder below, whose output length obeys ceil(-log2 W) + 1 <= sum(-log2 q) + 2.
"""
from __future__ import annotations

from fractions import Fraction

WINDOW = 56
TOP = 1 << WINDOW
BOT = 1 << 48
MASK = TOP - 1


class Encoder:
    def __init__(self):
        self.low = 0
        self.range = TOP - 1
        self.cache = None
        self.pending = 0
        self.out = bytearray()

    def _shift_low(self):
        if self.low < (0xFF << 48) or self.low >= TOP:
            carry = self.low >> WINDOW
            if self.cache is not None:
                self.out.append((self.cache + carry) & 0xFF)
            for _ in range(self.pending):
                self.out.append((0xFF + carry) & 0xFF)
            self.pending = 0
            self.cache = (self.low >> 48) & 0xFF
        else:
            self.pending += 1
        self.low = (self.low << 8) & MASK

    def encode(self, cum: int, freq: int, total: int):
        assert 0 < freq and 0 <= cum and cum + freq <= total <= (1 << 24)
        r = self.range // total
        self.low += r * cum
        self.range = r * freq
        while self.range < BOT:
            self._shift_low()
            self.range <<= 8

    def finish(self) -> bytes:
        hi = self.low + self.range
        for b in range(WINDOW, 47, -1):
            g = (1 << b) - 1
            v = (self.low + g) & ~g
            if v < hi:
                self.low = v
                break
        self._shift_low()
        self._shift_low()
        out = bytes(self.out)
        return out.rstrip(b"\x00")


class Decoder:
    def __init__(self, data: bytes):
        self.data = data
        self.pos = 0
        self.range = TOP - 1
        self.code = 0
        for _ in range(7):
            self.code = (self.code << 8) | self._byte()

    def _byte(self) -> int:
        b = self.data[self.pos] if self.pos < len(self.data) else 0
        self.pos += 1
        return b

    def decode(self, cum, total: int) -> int:
        """cum: exclusive prefix sums with the total appended (length A+1)."""
        r = self.range // total
        v = min(self.code // r, total - 1)
        lo, hi = 0, len(cum) - 2  # largest s with cum[s] <= v
        while lo < hi:
            mid = (lo + hi + 1) >> 1
            if cum[mid] <= v:
                lo = mid
            else:
                hi = mid - 1
        s = lo
        self.code -= r * int(cum[s])
        self.range = r * int(cum[s + 1] - cum[s])
        while self.range < BOT:
            self.code = ((self.code << 8) | self._byte()) & ((1 << 64) - 1)
            self.range <<= 8
        return s


def encode_all(symbols, cums, total: int) -> bytes:
    enc = Encoder()
    for s, cum in zip(symbols, cums):
        enc.encode(int(cum[s]), int(cum[s + 1] - cum[s]), total)
    return enc.finish()


def decode_all(data: bytes, cums, total: int):
    dec = Decoder(data)
    return [dec.decode(cum, total) for cum in cums]


# ---------------------------------------------------------------------------
# Exact arithmetic coding with rationals (pin only; tiny inputs)

def exact_encode(symbols, cums, total: int) -> str:
    """Shortest binary fraction inside the final interval [L, L+W); returns its bits."""
    L, W = Fraction(0), Fraction(1)
    for s, cum in zip(symbols, cums):
        L += W * Fraction(int(cum[s]), total)
        W *= Fraction(int(cum[s + 1] - cum[s]), total)
    n = 0
    while True:
        n += 1
        scale = 1 << n
        num = -((-L.numerator * scale) // L.denominator)  # ceil(L * 2^n)
        if Fraction(num, scale) < L + W:
            return format(num, "b").zfill(n) if num else "0" * n


def exact_decode(bits: str, cums, total: int):
    x = Fraction(int(bits, 2), 1 << len(bits)) if bits else Fraction(0)
    L, W, out = Fraction(0), Fraction(1), []
    for cum in cums:
        v = (x - L) / W * total
        s = max(i for i in range(len(cum) - 1) if cum[i] <= v)
        out.append(s)
        L += W * Fraction(int(cum[s]), total)
        W *= Fraction(int(cum[s + 1] - cum[s]), total)
    return out
