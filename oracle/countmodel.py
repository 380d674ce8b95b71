"""Adaptive order-m count model: judge and fallback coder for a block.

Test infrastructure only.  Not a component of the paper's compressor: it is
the integer, exact fallback the measured configurations ask for, coding a
block with it whenever the learned path would spend more bits.  Reading
(the design doc):

  * the block's bases are coded one by one, as a single stream;
  * context = the previous m base codes as a base-4 number (oldest most
    significant); positions before the block start count as A (0);
  * counts c[ctx][b] start at 0; the Krichevsky-Trofimov estimate
    freq_b = 2*c_b + 1, total = 2*sum(c) + 4 is coded with the range coder;
  * after coding base x: c[ctx][x] += 1; when it reaches 1024 all four counts
    of that context are halved (floor).

Pins: brute-force probability of a hand-worked short string; round trip;
length within the range coder's bound of sum(-log2 q).
"""
from __future__ import annotations

import numpy as np

from .rangecoder import Decoder, Encoder

LIMIT = 1024


def _model_steps(m: int):
    counts = np.zeros((4 ** m, 4), dtype=np.int64)
    return counts, (4 ** m) - 1


def probabilities(codes, m: int):
    """(freq_b, total) used for each base of `codes` (for the length pin)."""
    counts, mask = _model_steps(m)
    ctx, out = 0, []
    for x in codes:
        c = counts[ctx]
        freq = 2 * c + 1
        out.append((int(freq[x]), int(freq.sum())))
        c[x] += 1
        if c[x] >= LIMIT:
            c //= 2
        ctx = ((ctx << 2) | int(x)) & mask if m else 0
    return out


def encode(codes, m: int) -> bytes:
    counts, mask = _model_steps(m)
    enc, ctx = Encoder(), 0
    for x in np.asarray(codes, dtype=np.int64):
        c = counts[ctx]
        freq = 2 * c + 1
        cum = int(freq[:x].sum())
        enc.encode(cum, int(freq[x]), int(freq.sum()))
        c[x] += 1
        if c[x] >= LIMIT:
            c //= 2
        ctx = ((ctx << 2) | int(x)) & mask if m else 0
    return enc.finish()


def decode(data: bytes, n: int, m: int) -> np.ndarray:
    counts, mask = _model_steps(m)
    dec, ctx = Decoder(data), 0
    out = np.zeros(n, dtype=np.uint8)
    for i in range(n):
        c = counts[ctx]
        freq = 2 * c + 1
        cum = np.concatenate([[0], np.cumsum(freq)])
        x = dec.decode(cum, int(freq.sum()))
        out[i] = x
        c[x] += 1
        if c[x] >= LIMIT:
            c //= 2
        ctx = ((ctx << 2) | x) & mask if m else 0
    return out
