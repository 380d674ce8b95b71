"""MLP knowledge predictor, its backward pass and the optimiser, in FP64.

Test infrastructure only.  Paper §2 steps (3)-(4): a model maps the t
historical symbols to a distribution over the next symbol and is updated by
back-propagating the cross-entropy loss.  The predictor architecture used here
is the one the measured configurations fix (embedding E, context t, one ReLU
hidden layer H, 4^k output logits), in place of the paper's BiGRU/Transformer.

Flat parameter layout (float32 storage, one model):
    Emb [A][E] | W1^T [H][t*E] | b1 [H] | W2 [H][A] | b2 [A]
(W1 is stored transposed: row j holds the t*E weights into hidden unit j.)
For a row with context tokens c_0..c_{t-1} (oldest first):
    X   = [Emb[c_0], ..., Emb[c_{t-1}]]            (t*E)
    a   = X W1 + b1,   h = relu(a)                 (H)
    L   = h W2 + b2                                (A logits)
Backward from dL (rows x A): dW2 = h^T dL, db2 = sum dL, dh = dL W2^T,
da = dh * [a > 0], dW1 = X^T da, db1 = sum da, dX = da W1^T, and dEmb[c] adds
the slice of dX of every context position holding token c.

Optimiser (paper silent; the reading used): Adam with beta1 0.9,
beta2 0.999, eps 1e-8 and bias correction by the update count tau, or plain
SGD.  Pins: central finite differences of the loss (tests), closed-form Adam
first step (|update| = lr for every parameter with nonzero gradient).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .rng import fan_in_bound, uniform_pm1

BETA1, BETA2, ADAM_EPS = 0.9, 0.999, 1e-8


@dataclass(frozen=True)
class Shape:
    A: int  # alphabet 4^k
    E: int  # embedding width
    t: int  # context tokens
    H: int  # hidden width

    @property
    def sizes(self):
        A, E, t, H = self.A, self.E, self.t, self.H
        return {"emb": A * E, "w1": t * E * H, "b1": H, "w2": H * A, "b2": A}

    @property
    def count(self) -> int:
        return sum(self.sizes.values())

    def offsets(self):
        off, out = 0, {}
        for name, n in self.sizes.items():
            out[name] = (off, off + n)
            off += n
        return out


def init_params(shape: Shape, seed: int) -> np.ndarray:
    """Seeded initial parameters (float32), see oracle.rng for the draw-to-value rule."""
    out = np.zeros(shape.count, dtype=np.float32)
    off = shape.offsets()
    bounds = {"emb": np.float32(1.0), "w1": fan_in_bound(shape.t * shape.E), "w2": fan_in_bound(shape.H)}
    for name, bound in bounds.items():
        lo, hi = off[name]
        out[lo:hi] = uniform_pm1(seed, lo, hi - lo) * bound
    return out  # biases stay exactly +0


def views(flat: np.ndarray, shape: Shape):
    off = shape.offsets()
    A, E, t, H = shape.A, shape.E, shape.t, shape.H
    get = lambda n: flat[off[n][0]:off[n][1]]
    return (get("emb").reshape(A, E), get("w1").reshape(H, t * E).T, get("b1"),
            get("w2").reshape(H, A), get("b2"))


def forward(flat: np.ndarray, shape: Shape, ctx: np.ndarray):
    """ctx: int [R, t] tokens.  Returns (X, a, h, logits), all float64."""
    emb, w1, b1, w2, b2 = (np.asarray(v, dtype=np.float64) for v in views(flat, shape))
    ctx = np.asarray(ctx, dtype=np.int64).reshape(-1, shape.t)
    X = emb[ctx].reshape(ctx.shape[0], shape.t * shape.E)
    a = X @ w1 + b1
    h = np.maximum(a, 0.0)
    return X, a, h, h @ w2 + b2


def backward(flat: np.ndarray, shape: Shape, ctx: np.ndarray, X, a, h, dlogits) -> np.ndarray:
    """Gradient (float64, flat layout) of sum_rows <dlogits, logits> w.r.t. the parameters."""
    emb, w1, b1, w2, b2 = (np.asarray(v, dtype=np.float64) for v in views(flat, shape))
    ctx = np.asarray(ctx, dtype=np.int64).reshape(-1, shape.t)
    dL = np.asarray(dlogits, dtype=np.float64)
    g = np.zeros(shape.count, dtype=np.float64)
    gemb, gw1, gb1, gw2, gb2 = views(g, shape)
    gw2[...] = h.T @ dL
    gb2[...] = dL.sum(axis=0)
    da = (dL @ w2.T) * (a > 0)
    gw1[...] = X.T @ da
    gb1[...] = da.sum(axis=0)
    dX = (da @ w1.T).reshape(ctx.shape[0], shape.t, shape.E)
    np.add.at(gemb, ctx.reshape(-1), dX.reshape(-1, shape.E))
    return g


def bias_corrections(tau: int):
    return 1.0 - BETA1 ** tau, 1.0 - BETA2 ** tau


def adam_step(theta: np.ndarray, m: np.ndarray, v: np.ndarray, g: np.ndarray, tau: int, lr: float):
    """One Adam update (in place, FP64 arrays); tau is the 1-based update count."""
    m *= BETA1
    m += (1.0 - BETA1) * g
    v *= BETA2
    v += (1.0 - BETA2) * g * g
    c1, c2 = bias_corrections(tau)
    theta -= lr * (m / c1) / (np.sqrt(v / c2) + ADAM_EPS)


def sgd_step(theta: np.ndarray, g: np.ndarray, lr: float):
    theta -= lr * g
