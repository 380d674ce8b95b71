"""Probabilities -> integer frequency table for the entropy coder.

Test infrastructure only.  The paper passes P to its entropy encoder (§2 step 3)
without saying how P becomes integers; the reading used here:

    T = 2^24 (total), A = alphabet size
    freq_j = 1 + floor(P_j * (T - A))      the product rounded in the working
                                           precision (float64 for the oracle's
                                           own runs, float32 to mirror a kernel)
    R = T - sum_j freq_j                   added to the first index of maximal freq
    cum_j = sum_{i<j} freq_i

Every symbol keeps freq >= 1, so any token stays codable.  The uniform table
used for the first t symbols (§2) has freq_j = T / A = 2^(24 - 2k) exactly.
Pins: sum = T, all freq >= 1, tie rule, and brute force on small alphabets.
"""
from __future__ import annotations

import numpy as np

TOTAL_BITS = 24
TOTAL = 1 << TOTAL_BITS


def quantize(P: np.ndarray, dtype=np.float64) -> np.ndarray:
    """P [..., A] -> int64 freq [..., A]; `dtype` is the precision of the product P_j*(T-A)."""
    P = np.asarray(P, dtype=dtype)
    A = P.shape[-1]
    scale = dtype(TOTAL - A)
    prod = (P * scale).astype(dtype)
    freq = 1 + np.floor(prod).astype(np.int64)
    flat = freq.reshape(-1, A)
    rem = TOTAL - flat.sum(axis=1)
    top = flat.argmax(axis=1)  # first maximal index
    flat[np.arange(flat.shape[0]), top] += rem
    return flat.reshape(freq.shape)


def cumulative(freq: np.ndarray) -> np.ndarray:
    """Exclusive prefix sums with the total appended: cum[..., A] == TOTAL."""
    freq = np.asarray(freq, dtype=np.int64)
    c = np.cumsum(freq, axis=-1)
    return np.concatenate([np.zeros(freq.shape[:-1] + (1,), dtype=np.int64), c], axis=-1)


def uniform_freq(A: int) -> np.ndarray:
    return np.full(A, TOTAL // A, dtype=np.int64)
