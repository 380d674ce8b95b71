"""(s,k)-mer encoding (GskE), paper §4.1 and Fig. 3.  Test infrastructure only.

Bases map to numbers A:0 C:1 G:2 T:3; a window of k bases starting every s
bases is read as a base-4 number with the first base most significant (the
paper's example: "CGG" = 4^2*1 + 4^1*2 + 4^0*2 = 26).

Readings where the paper is silent:
  * only 1 <= s <= k <= 8 is lossless, so only that is accepted;
  * l = floor((n-k)/s) + 1 windows for n >= k, none for n < k;
  * the n - ((l-1)s + k) bases after the last window (fewer than s) form the
    block's raw tail (all n bases when n < k).
Pins: the worked example, brute force over all short strings, round trip.
"""
from __future__ import annotations

import numpy as np

CODE = {ord("A"): 0, ord("C"): 1, ord("G"): 2, ord("T"): 3}
LETTERS = np.frombuffer(b"ACGT", dtype=np.uint8)


class InvalidBase(ValueError):
    pass


def base_codes(seq) -> np.ndarray:
    """ASCII bases -> codes 0..3; any byte other than A, C, G, T is rejected."""
    a = np.frombuffer(bytes(seq), dtype=np.uint8) if not isinstance(seq, np.ndarray) else seq.astype(np.uint8)
    out = np.full(a.shape, 255, dtype=np.uint8)
    for ch, v in CODE.items():
        out[a == ch] = v
    if (out == 255).any():
        raise InvalidBase(f"non-ACGT byte at offset {int(np.argmax(out == 255))}")
    return out


def n_tokens(n: int, s: int, k: int) -> int:
    return 0 if n < k else (n - k) // s + 1


def tokenize(codes: np.ndarray, s: int, k: int):
    """Return (tokens int64[l], tail codes uint8[n - covered])."""
    if not (1 <= s <= k <= 8):
        raise ValueError("need 1 <= s <= k <= 8")
    codes = np.asarray(codes, dtype=np.int64)
    n = codes.size
    l = n_tokens(n, s, k)
    if l == 0:
        return np.zeros(0, dtype=np.int64), codes.astype(np.uint8)
    tok = np.zeros(l, dtype=np.int64)
    for m in range(k):  # e_j = sum_m 4^(k-1-m) * code[j*s + m]
        tok = tok * 4 + codes[m: m + (l - 1) * s + 1: s]
    covered = (l - 1) * s + k
    return tok, codes[covered:].astype(np.uint8)


def detokenize(tokens: np.ndarray, tail: np.ndarray, s: int, k: int) -> np.ndarray:
    """Inverse of tokenize; raises ValueError when overlapping windows disagree."""
    tokens = np.asarray(tokens, dtype=np.int64)
    if tokens.size == 0:
        return np.asarray(tail, dtype=np.uint8)
    if s < k:  # the last k-s digits of e_j must equal the first k-s digits of e_{j+1}
        lo = tokens[:-1] % (4 ** (k - s))
        hi = tokens[1:] // (4 ** s)
        if not np.array_equal(lo, hi):
            raise ValueError("inconsistent overlapping (s,k)-mers")
    first = [(int(tokens[0]) >> (2 * (k - 1 - m))) & 3 for m in range(k)]
    rest = np.zeros((tokens.size - 1, s), dtype=np.uint8)
    for m in range(s):  # the last s digits of each later window are its new bases
        rest[:, m] = (tokens[1:] >> (2 * (s - 1 - m))) & 3
    return np.concatenate([np.array(first, dtype=np.uint8), rest.reshape(-1), np.asarray(tail, dtype=np.uint8)])


def letters(codes: np.ndarray) -> bytes:
    return LETTERS[np.asarray(codes, dtype=np.int64)].tobytes()
