"""BiGRU static predictor (the paper's SPuM / SPrM architecture), forward in FP64.

Test infrastructure only.  Paper §4.2.2: the static public model reads the t
historical symbols through a 16-wide embedding, two bidirectional GRU layers and
a Linear and a Dense layer of width 128, and outputs the logits L^u over the 4^k
tokens; §4.2.3: the static private model has the same structure and parameters
with one BiGRU layer.  Both are frozen while coding, so only the forward pass is
needed here.

Readings (the paper names the layers, not their equations):
  * GRU cell, in the form with the reset gate applied to the recurrent
    projection after its bias (as in cuDNN and torch.nn.GRU):
        r  = sigmoid(Wi_r x + bi_r + Wh_r h + bh_r)
        z  = sigmoid(Wi_z x + bi_z + Wh_z h + bh_z)
        n  = tanh(Wi_n x + bi_n + r * (Wh_n h + bh_n))
        h' = (1 - z) * n + z * h,          state before the first position: 0
  * a BiGRU layer runs one GRU forward over the context positions 0..t-1
    (oldest first) and another backward over t-1..0; its output at position p
    is [h^f_p, h^b_p] (2 Hg wide), the next layer's input at p;
  * the summary of the last layer is u = [h^f after position t-1, h^b after
    position 0]: each direction's state once it has read the whole context;
  * "a Linear and Dense layer with a dimension of 128": q = relu(W3 u + b3) with
    D = 128 units, then L = q W4 + b4 (4^k logits);
  * Hg, the GRU width per direction, is not stated: a parameter;
  * SPrM's parameters are SPuM's without the second BiGRU layer (the paper: the
    two share structure and parameters), see drop_second_layer.

Flat parameter layout (float32 storage, one model; A = 4^k):
    Emb [A][E]
    for layer l = 0 .. layers-1, direction d = forward, backward:
        Wi [3 Hg][in_l] | Wh [3 Hg][Hg] | bi [3 Hg] | bh [3 Hg]
        (gate rows in the order r, z, n; in_0 = E, in_l = 2 Hg for l >= 1)
    W3 [D][2 Hg] | b3 [D] | W4 [D][A] | b4 [A]
The size does not depend on t.  Seeded initialisation as the MLP's (oracle.rng):
weights uniform in +-1/sqrt(fan_in) with fan_in = in_l for Wi, Hg for Wh, 2 Hg for
W3 and D for W4; the embedding in +-1; biases exactly +0.

Pins (tests/test_oracle_bigru.py): torch.nn.GRU in float64 (bidirectional, one
and two layers) on the same weights; the closed form of the recurrence with the
recurrent and input weights at zero (h_p = c (1 - 2^-(p+1)) for z = 1/2); the
reset gate's placement with saturated gates; the direction-swap symmetry;
drop_second_layer against a one-layer model.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .rng import fan_in_bound, uniform_pm1

DENSE = 128  # width of the Linear layer (§4.2.2)


@dataclass(frozen=True)
class GruShape:
    A: int       # alphabet 4^k
    E: int       # embedding width (paper: 16)
    t: int       # context tokens
    Hg: int      # GRU width per direction
    layers: int  # BiGRU layers: 2 for SPuM, 1 for SPrM
    D: int = DENSE

    def in_width(self, layer: int) -> int:
        return self.E if layer == 0 else 2 * self.Hg

    @property
    def sizes(self):
        A, E, Hg, D = self.A, self.E, self.Hg, self.D
        out = {"emb": A * E}
        for l in range(self.layers):
            for d in ("f", "b"):
                out[f"wi{l}{d}"] = 3 * Hg * self.in_width(l)
                out[f"wh{l}{d}"] = 3 * Hg * Hg
                out[f"bi{l}{d}"] = 3 * Hg
                out[f"bh{l}{d}"] = 3 * Hg
        out.update({"w3": D * 2 * Hg, "b3": D, "w4": D * A, "b4": A})
        return out

    @property
    def count(self) -> int:
        return sum(self.sizes.values())

    def offsets(self):
        off, out = 0, {}
        for name, n in self.sizes.items():
            out[name] = (off, off + n)
            off += n
        return out


def init_bigru(shape: GruShape, seed: int) -> np.ndarray:
    """Seeded initial parameters (float32); draw i of the stream sets flat parameter i."""
    out = np.zeros(shape.count, dtype=np.float32)
    off = shape.offsets()
    bounds = {"emb": np.float32(1.0), "w3": fan_in_bound(2 * shape.Hg), "w4": fan_in_bound(shape.D)}
    for l in range(shape.layers):
        for d in ("f", "b"):
            bounds[f"wi{l}{d}"] = fan_in_bound(shape.in_width(l))
            bounds[f"wh{l}{d}"] = fan_in_bound(shape.Hg)
    for name, bound in bounds.items():
        lo, hi = off[name]
        out[lo:hi] = uniform_pm1(seed, lo, hi - lo) * bound
    return out


def params(flat: np.ndarray, shape: GruShape) -> dict:
    """Named float64 views of the flat parameters (matrices in their row-major shapes)."""
    off = shape.offsets()
    f = np.asarray(flat, dtype=np.float64)
    Hg = shape.Hg
    out = {}
    for name, (lo, hi) in off.items():
        v = f[lo:hi]
        if name == "emb":
            v = v.reshape(shape.A, shape.E)
        elif name.startswith("wi"):
            v = v.reshape(3 * Hg, shape.in_width(int(name[2])))
        elif name.startswith("wh"):
            v = v.reshape(3 * Hg, Hg)
        elif name == "w3":
            v = v.reshape(shape.D, 2 * Hg)
        elif name == "w4":
            v = v.reshape(shape.D, shape.A)
        out[name] = v
    return out


def _sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def gru_pass(x: np.ndarray, wi, wh, bi, bh, reverse: bool) -> np.ndarray:
    """One GRU direction over x [R, t, in]: the state after every position [R, t, Hg] (for the
    backward direction, the state at p has read positions t-1 .. p)."""
    R, t, _ = x.shape
    Hg = wh.shape[1]
    h = np.zeros((R, Hg))
    seq = np.zeros((R, t, Hg))
    for p in (range(t - 1, -1, -1) if reverse else range(t)):
        gi = x[:, p, :] @ wi.T + bi
        gh = h @ wh.T + bh
        r = _sigmoid(gi[:, :Hg] + gh[:, :Hg])
        z = _sigmoid(gi[:, Hg:2 * Hg] + gh[:, Hg:2 * Hg])
        n = np.tanh(gi[:, 2 * Hg:] + r * gh[:, 2 * Hg:])
        h = (1.0 - z) * n + z * h
        seq[:, p, :] = h
    return seq


def states(flat: np.ndarray, shape: GruShape, ctx: np.ndarray):
    """ctx: int [R, t] tokens (oldest first).  Returns (the output of every BiGRU layer, each
    [R, t, 2 Hg], and the summary u [R, 2 Hg])."""
    w = params(flat, shape)
    ctx = np.asarray(ctx, dtype=np.int64).reshape(-1, shape.t)
    x = w["emb"][ctx]
    outs = []
    for l in range(shape.layers):
        fwd = gru_pass(x, w[f"wi{l}f"], w[f"wh{l}f"], w[f"bi{l}f"], w[f"bh{l}f"], reverse=False)
        bwd = gru_pass(x, w[f"wi{l}b"], w[f"wh{l}b"], w[f"bi{l}b"], w[f"bh{l}b"], reverse=True)
        x = np.concatenate([fwd, bwd], axis=2)
        outs.append(x)
    Hg = shape.Hg
    u = np.concatenate([x[:, -1, :Hg], x[:, 0, Hg:]], axis=1)
    return outs, u


def forward(flat: np.ndarray, shape: GruShape, ctx: np.ndarray):
    """Returns (q, logits): the Linear layer's output q = relu(W3 u + b3) [R, D] and the Dense
    layer's logits L = q W4 + b4 [R, A], float64."""
    w = params(flat, shape)
    _, u = states(flat, shape, ctx)
    q = np.maximum(u @ w["w3"].T + w["b3"], 0.0)
    return q, q @ w["w4"] + w["b4"]


def drop_second_layer(flat: np.ndarray, shape: GruShape):
    """The one-layer model (SPrM's structure) that shares SPuM's embedding, first BiGRU layer and
    head: SPuM's flat parameters without layer 1.  Returns (flat, shape)."""
    assert shape.layers == 2
    one = GruShape(shape.A, shape.E, shape.t, shape.Hg, 1, shape.D)
    off = shape.offsets()
    keep = ["emb"] + [f"{p}0{d}" for d in ("f", "b") for p in ("wi", "wh", "bi", "bh")] + ["w3", "b3", "w4", "b4"]
    # one.offsets() orders the kept tensors as the two-layer layout does
    parts = [np.asarray(flat)[off[n][0]:off[n][1]] for n in one.offsets()]
    assert list(one.offsets()) == [n for n in shape.offsets() if n in keep]
    return np.concatenate(parts), one
