"""FP8 E4M3 codes and the frozen static predictor's FP8 form, in FP64.

Test infrastructure only.  The measured configuration with a large pre-trained
static predictor freezes it in FP8 (the paper's static public model, §4.2.2, is
frozen and never updated; its precision is not stated).  Reading used here:

E4M3 (the OCP 8-bit floating-point format): 1 sign bit, 4 exponent bits with
bias 7, 3 mantissa bits.  Exponent field 0 holds the subnormals m * 2^-9; the
code S.1111.111 is NaN; there are no infinities; the largest finite magnitude is
1.75 * 2^8 = 448.  encode() rounds to the nearest code, ties to the even
mantissa (even code), and saturates magnitudes above 448 to 448.

Quantisation of a frozen model (flat layout of model.py):
    scale  = float32(amax / 448)      amax = largest |w| of the channel, float32
                                      division; an all-zero channel has scale 1
    code   = encode(float32(w / scale))   float32 division
    value  = decode(code) * scale        (exact in float64)
with one scale for the whole embedding table, one per hidden unit for W1 (a row
of W1^T) and one per output logit for W2 (a column of W2).  Biases stay FP32.

FP8 forward of the static predictor (the kernels' quantisation points):
    a  = (X_q . W1_q^T) * (s_emb * s_1[h]) + b1      X_q: codes of the context rows
    h  = relu(a)
    s_r = max_h h / 448  (1 if the row is all zero),  h_q = encode(h / s_r)
    L  = (h_q . W2_q) * (s_r * s_2[a]) + b2
FP8-hidden form (precision 3): the embedding and W1 as above, h unrounded, the logits layer
with the stored (FP32) W2 and b2:
    a  = (X_q . W1_q^T) * (s_emb * s_1[h]) + b1,   h = relu(a),   L = h . W2 + b2
Pins (tests): every finite code decodes and re-encodes to itself; the format's
landmarks (1.0, 448, the smallest normal and subnormal, NaN); ties to even;
saturation; brute-force nearest-code search; each channel's largest magnitude
maps to the code of 448; dequantised weights within half a code step.
"""
from __future__ import annotations

import numpy as np

from .model import Shape, views

MAX = 448.0
NAN_CODE = 0x7F


def decode(code) -> np.ndarray:
    """Value(s) of E4M3 code(s) (float64; NaN for the NaN codes)."""
    c = np.asarray(code, dtype=np.int64) & 0xFF
    sign = np.where(c & 0x80, -1.0, 1.0)
    e = (c >> 3) & 0xF
    m = c & 0x7
    mag = np.where(e == 0, m * 2.0 ** -9, (1.0 + m / 8.0) * np.exp2(e.astype(np.float64) - 7.0))
    mag = np.where((e == 15) & (m == 7), np.nan, mag)
    return sign * mag


# the 127 non-negative finite codes 0x00 .. 0x7E and their values, ascending
_POS_CODES = np.arange(0x7F, dtype=np.int64)
_POS_VALUES = decode(_POS_CODES)
assert np.all(np.diff(_POS_VALUES) > 0)


def encode(x) -> np.ndarray:
    """E4M3 codes (uint8) of x: nearest code, ties to the even code, saturated at 448."""
    x = np.asarray(x, dtype=np.float64)
    mag = np.minimum(np.abs(x), MAX)
    i = np.searchsorted(_POS_VALUES, mag)          # first value >= mag
    i = np.clip(i, 1, len(_POS_VALUES) - 1)
    lo, hi = _POS_VALUES[i - 1], _POS_VALUES[i]
    pick_hi = (mag - lo > hi - mag) | ((mag - lo == hi - mag) & (_POS_CODES[i] % 2 == 0))
    code = np.where(pick_hi, _POS_CODES[i], _POS_CODES[i - 1])
    code = np.where(mag == 0.0, 0, code)
    code = code | np.where(np.signbit(x), 0x80, 0)
    return code.astype(np.uint8)


def channel_scales(amax) -> np.ndarray:
    """float32 scales amax / 448 (1 where amax is 0)."""
    amax = np.asarray(amax, dtype=np.float32)
    s = (amax / np.float32(MAX)).astype(np.float32)
    return np.where(amax == 0, np.float32(1.0), s).astype(np.float32)


def quantize_rows(w) -> tuple[np.ndarray, np.ndarray]:
    """Codes and per-row float32 scales of a 2-D float32 array (one channel per row)."""
    w = np.asarray(w, dtype=np.float32)
    s = channel_scales(np.abs(w).max(axis=1))
    q = encode((w / s[:, None]).astype(np.float32))
    return q, s


def quantize_model(flat: np.ndarray, shape: Shape) -> dict:
    """FP8 form of a frozen model: codes and scales of Emb, W1 (by hidden unit), W2 (by logit)."""
    emb, w1, b1, w2, b2 = views(np.asarray(flat, dtype=np.float32), shape)
    w1t = np.ascontiguousarray(w1.T)               # [H][t*E]
    s_emb = channel_scales(np.abs(emb).max())
    q_emb = encode((emb / s_emb).astype(np.float32))
    q_w1t, s_w1 = quantize_rows(w1t)
    q_w2t, s_w2 = quantize_rows(np.ascontiguousarray(w2.T))   # [A][H]: one channel per logit
    return {"emb": q_emb, "s_emb": np.float32(s_emb), "w1t": q_w1t, "s_w1": s_w1,
            "w2t": q_w2t, "s_w2": s_w2, "b1": np.asarray(b1, np.float32).copy(),
            "b2": np.asarray(b2, np.float32).copy(), "shape": shape}


def dequantize_model(fq: dict) -> np.ndarray:
    """The frozen model the FP8 codes represent, in the flat layout (float64)."""
    shape = fq["shape"]
    out = np.zeros(shape.count, dtype=np.float64)
    emb, w1, b1, w2, b2 = views(out, shape)
    emb[...] = decode(fq["emb"]) * np.float64(fq["s_emb"])
    w1[...] = (decode(fq["w1t"]) * fq["s_w1"].astype(np.float64)[:, None]).T
    b1[...] = fq["b1"]
    w2[...] = (decode(fq["w2t"]) * fq["s_w2"].astype(np.float64)[:, None]).T
    b2[...] = fq["b2"]
    return out


def forward(fq: dict, ctx: np.ndarray) -> np.ndarray:
    """Static logits [R, A] of the FP8 form for context tokens ctx [R, t] (float64)."""
    shape = fq["shape"]
    ctx = np.asarray(ctx, dtype=np.int64).reshape(-1, shape.t)
    xq = decode(fq["emb"])[ctx].reshape(ctx.shape[0], shape.t * shape.E)
    a = (xq @ decode(fq["w1t"]).T) * (np.float64(fq["s_emb"]) * fq["s_w1"].astype(np.float64)) + fq["b1"]
    h = np.maximum(a, 0.0)
    amax = h.max(axis=1)
    s_r = np.where(amax > 0, amax / MAX, 1.0)
    hq = decode(encode(h / s_r[:, None]))
    return (hq @ decode(fq["w2t"]).T) * (s_r[:, None] * fq["s_w2"].astype(np.float64)[None, :]) + fq["b2"]


def forward_hidden(fq: dict, flat: np.ndarray, ctx: np.ndarray) -> np.ndarray:
    """Static logits [R, A] of the FP8-hidden form: E4M3 embedding and W1, stored W2 (float64)."""
    shape = fq["shape"]
    ctx = np.asarray(ctx, dtype=np.int64).reshape(-1, shape.t)
    xq = decode(fq["emb"])[ctx].reshape(ctx.shape[0], shape.t * shape.E)
    a = (xq @ decode(fq["w1t"]).T) * (np.float64(fq["s_emb"]) * fq["s_w1"].astype(np.float64)) + fq["b1"]
    h = np.maximum(a, 0.0)
    _, _, _, w2, b2 = views(np.asarray(flat, dtype=np.float32).astype(np.float64), shape)
    return h @ w2 + b2
