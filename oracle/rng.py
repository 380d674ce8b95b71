"""Counter-based splitmix64 and the dynamic model's seeded initialisation.

Test infrastructure only.  The paper initialises the dynamic model from
"randomly initialized parameters" (§4.3) without naming a generator; the
reading used here is splitmix64 (Steele, Lea & Flood,
2014) as a counter-based stream: draw i of seed S is mix(S + (i+1)*gamma).

Initial value of parameter i of a tensor with bound B:
    u = draw_i >> 40                     (24 random bits)
    w = float32((2u - 2^24) / 2^24)      (exact: an integer below 2^25 times 2^-24)
    value = float32(w * B)               (one IEEE round-to-nearest product)
with B = 1 for the embedding, float32(1/sqrt(fan_in)) for weight matrices
(fan_in = t*E for W1, H for W2) and biases exactly +0.  Pins: the published
splitmix64 test value, exact reproducibility of the float32 values.
"""
from __future__ import annotations

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
MASK = (1 << 64) - 1


def splitmix64_draws(seed: int, start: int, count: int) -> np.ndarray:
    """Draws start .. start+count-1 of the splitmix64 stream seeded with `seed` (uint64)."""
    with np.errstate(over="ignore"):
        i = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        z = np.uint64(seed & MASK) + i * np.uint64(GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def uniform_pm1(seed: int, start: int, count: int) -> np.ndarray:
    """float32 values in [-1, 1) on a 2^-23 grid, from draws start..start+count-1."""
    u = (splitmix64_draws(seed, start, count) >> np.uint64(40)).astype(np.int64)
    return ((2 * u - (1 << 24)).astype(np.float64) * 2.0 ** -24).astype(np.float32)


def fan_in_bound(fan_in: int) -> np.float32:
    return np.float32(1.0) / np.sqrt(np.float32(fan_in))
