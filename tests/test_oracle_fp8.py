"""Pins of oracle.fp8: the E4M3 format's definition and the frozen model's FP8 form."""
import itertools

import numpy as np
import pytest

from oracle import fp8
from oracle.model import Shape, forward, init_params


def test_landmark_values():
    """Values fixed by the format: bias 7, 3 mantissa bits, no infinities, S.1111.111 NaN."""
    assert fp8.decode(0x38) == 1.0
    assert fp8.decode(0x7E) == 448.0            # largest finite: 1.75 * 2^8
    assert fp8.decode(0x08) == 2.0 ** -6        # smallest normal
    assert fp8.decode(0x01) == 2.0 ** -9        # smallest subnormal
    assert fp8.decode(0x07) == 7 * 2.0 ** -9    # largest subnormal
    assert fp8.decode(0x77) == 1.875 * 2.0 ** 7  # 0.1110.111
    assert np.isnan(fp8.decode(0x7F)) and np.isnan(fp8.decode(0xFF))
    assert fp8.decode(0xB8) == -1.0 and fp8.decode(0x80) == 0.0
    assert not np.isnan(fp8.decode(0x78)) and fp8.decode(0x78) == 256.0  # exponent 15 is finite


def test_every_finite_code_round_trips():
    codes = np.array([c for c in range(256) if c not in (0x7F, 0xFF)])
    back = fp8.encode(fp8.decode(codes))
    assert np.array_equal(back, codes.astype(np.uint8))


def test_brute_force_nearest_with_ties_to_even():
    """encode(x) is the nearest finite code by exhaustive search; exact midpoints take the even code."""
    vals = fp8.decode(np.arange(0x7F))
    rng = np.random.default_rng(3)
    xs = np.concatenate([rng.uniform(0, 460, 4000), rng.uniform(0, 0.05, 2000),
                         (vals[1:] + vals[:-1]) / 2])  # every midpoint
    for x in xs:
        d = np.abs(vals - min(x, 448.0))
        best = np.flatnonzero(d == d.min())
        want = best[0] if len(best) == 1 else [b for b in best if b % 2 == 0][0]
        assert fp8.encode(x) == want, x


def test_ties_and_saturation_examples():
    assert fp8.encode(1.0625) == 0x38   # between 1.0 (0x38) and 1.125 (0x39): even code
    assert fp8.encode(1.1875) == 0x3A   # between 1.125 (0x39) and 1.25 (0x3A)
    assert fp8.encode(464.0) == 0x7E and fp8.encode(1e30) == 0x7E
    assert fp8.encode(-1e30) == 0xFE
    assert fp8.encode(2.0 ** -10) == 0x00     # midpoint of 0 and the smallest subnormal: even (0)
    assert fp8.encode(3 * 2.0 ** -11) == 0x01
    assert fp8.encode(-0.0) == 0x80


def test_channel_maximum_maps_to_448_and_error_bound():
    shape = Shape(64, 8, 4, 32)
    flat = init_params(shape, 11)
    fq = fp8.quantize_model(flat, shape)
    assert np.all(np.abs(fp8.decode(fq["w1t"])).max(axis=1) == 448.0)
    assert np.all(np.abs(fp8.decode(fq["w2t"])).max(axis=1) == 448.0)
    assert np.abs(fp8.decode(fq["emb"])).max() == 448.0
    deq = fp8.dequantize_model(fq)
    w = flat.astype(np.float64)
    # half a code step: relative 2^-4 for normals, absolute 2^-10 * scale below the normal range
    err = np.abs(deq - w)
    off = shape.offsets()
    for name, scale in (("emb", np.full(shape.A * shape.E, fq["s_emb"])),):
        lo, hi = off[name]
        tol = np.maximum(np.abs(w[lo:hi]) * 2.0 ** -4, scale * 2.0 ** -10) * (1 + 1e-6)
        assert np.all(err[lo:hi] <= tol)
    lo, hi = off["b1"]
    assert np.array_equal(deq[lo:hi], w[lo:hi])


def test_fp8_forward_within_activation_rounding_bound():
    """The FP8 forward is the plain forward of the dequantised model except that h is rounded to
    its row's E4M3 grid: each |h_q - h| is at most half a code step (2^-4 relative, or 2^-10 s_r
    below the normal range), so |L8 - L| <= sum_h that step * |W2[h][a]|, element by element."""
    shape = Shape(16, 8, 3, 16)
    flat = init_params(shape, 5)
    fq = fp8.quantize_model(flat, shape)
    deq = fp8.dequantize_model(fq)
    ctx = np.array(list(itertools.product(range(16), repeat=3))[:200])
    L8 = fp8.forward(fq, ctx)
    _, _, h, L = forward(deq, shape, ctx)
    w2 = np.abs(deq[shape.offsets()["w2"][0]:shape.offsets()["w2"][1]].reshape(shape.H, shape.A))
    amax = h.max(axis=1)
    s_r = np.where(amax > 0, amax / 448.0, 1.0)
    step = np.maximum(h * 2.0 ** -4, s_r[:, None] * 2.0 ** -10)
    bound = step @ w2
    assert np.all(np.abs(L8 - L) <= bound * (1 + 1e-9) + 1e-12)
    assert np.max(np.abs(L8 - L)) > 0  # the activation rounding is really applied


@pytest.mark.parametrize("bad", [np.float32(np.inf), np.float32(-np.inf)])
def test_infinities_saturate(bad):
    assert fp8.decode(fp8.encode(bad)) == np.sign(bad) * 448.0


def test_fp8_hidden_forward_is_the_plain_forward_with_e4m3_embedding_and_w1():
    """The FP8-hidden form equals the plain forward of the model whose embedding and W1 are the
    dequantised E4M3 values and whose b1, W2 and b2 are the stored ones, element by element."""
    shape = Shape(16, 8, 3, 16)
    rng = np.random.default_rng(9)
    flat = (init_params(shape, 6) + rng.normal(0, 0.05, shape.count)).astype(np.float32)
    fq = fp8.quantize_model(flat, shape)
    deq = fp8.dequantize_model(fq)
    mixed = flat.astype(np.float64).copy()
    off = shape.offsets()
    for name in ("emb", "w1"):
        lo, hi = off[name]
        mixed[lo:hi] = deq[lo:hi]
    ctx = np.array(list(itertools.product(range(16), repeat=3))[:300])
    got = fp8.forward_hidden(fq, flat, ctx)
    want = forward(mixed, shape, ctx)[3]
    assert np.allclose(got, want, rtol=1e-12, atol=1e-12)
    # the logits layer really is the stored one: the FP8 form (E4M3 W2 and h) differs
    assert np.max(np.abs(fp8.forward(fq, ctx) - got)) > 1e-6


def test_encoder_matches_torch_float8_e4m3fn_within_range():
    """torch's float8_e4m3fn cast (round to nearest even; the same OCP E4M3 format) on values within
    +-448: random magnitudes over every exponent, the subnormals, and every midpoint between two
    consecutive codes (the ties), both signs.  Beyond 448 the two differ by design: the oracle
    saturates at 448, the cast gives NaN."""
    torch = pytest.importorskip("torch")
    if not hasattr(torch, "float8_e4m3fn"):
        pytest.skip("this torch has no float8_e4m3fn")
    from oracle.fp8 import decode, encode
    rng = np.random.default_rng(21)
    pos = decode(np.arange(0x7F))
    mids = (pos[:-1] + pos[1:]) / 2
    vals = np.concatenate([np.exp2(rng.uniform(-12, np.log2(448.0), 20000)), mids, pos,
                           rng.uniform(0, 2.0 ** -6, 2000)])
    vals = np.concatenate([vals, -vals]).astype(np.float32)  # float32 inputs: mids are exact in float32
    assert np.abs(vals).max() <= 448.0
    want = torch.from_numpy(vals).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    assert np.array_equal(encode(vals), want)
