"""Adaptive order-m count model: judge and fallback coder of a block.

Test infrastructure only.  Not a component of the paper's compressor: it is
the integer, exact fallback that guards the learned path, coding a block
whenever the network would spend more bytes on it.  Reading (the paper has no count model):

Estimator.  Counts c[ctx][b] start at 0; the Krichevsky-Trofimov estimate
freq_b = 2 c_b + 1, total = 2 sum(c) + 4 is range coded; the context is the
previous m bases (oldest most significant), positions before the start of the
stream reading as A (0).

Lanes.  The count model codes a block in the same lanes as the network: lane
r's base stream is the k digits of its first token followed by the last s
digits of each later token (exactly the bases its tokens add).  At local step
j every live lane codes the bases its j-th token adds (k at j = 0, else s),
one sub-step per base, against ONE table per block:
  A  every live lane reads the counts of its context and codes its base;
  B  every live lane adds 1 to c[ctx][base] (increments commute);
  C  every context that some live lane used and whose largest count is now
     >= 1024 has all four counts halved (floor), once.
With one lane and (s, k) = (1, 1) this is the plain sequential adaptive model
(`sequential_probabilities`), which the tests use as the pin.
"""
from __future__ import annotations

import numpy as np

LIMIT = 1024


class Table:
    """The count table of one block and the per-lane contexts."""

    def __init__(self, m: int, n_lanes: int):
        self.m = m
        self.mask = (1 << (2 * m)) - 1
        self.c = np.zeros((1 << (2 * m), 4), dtype=np.int64)
        self.ctx = [0] * n_lanes

    def freqs(self, r: int):
        """(freq[4], total) for lane r's current context."""
        f = 2 * self.c[self.ctx[r]] + 1
        return f, int(f.sum())

    def finish_substep(self, lanes, bases):
        """Phases B and C for the lanes that coded `bases` in this sub-step, then advance contexts."""
        used = []
        for r, x in zip(lanes, bases):
            self.c[self.ctx[r], x] += 1
            used.append(self.ctx[r])
        for ctx in dict.fromkeys(used):  # each used context once, in lane order
            if self.c[ctx].max() >= LIMIT:
                self.c[ctx] //= 2
        for r, x in zip(lanes, bases):
            self.ctx[r] = ((self.ctx[r] << 2) | int(x)) & self.mask


def new_digits(token: int, j: int, s: int, k: int):
    """Bases that token j of a lane adds to the lane's stream (digits, first base first)."""
    n = k if j == 0 else s
    return [(int(token) >> (2 * (n - 1 - q))) & 3 for q in range(n)]


def sequential_probabilities(codes, m: int):
    """(freq, total) of every base of one stream coded alone: the one-lane, (1,1) special case."""
    t = Table(m, 1)
    out = []
    for x in codes:
        f, tot = t.freqs(0)
        out.append((int(f[x]), tot))
        t.finish_substep([0], [int(x)])
    return out
