"""The frozen static predictor in FP8 (E4M3): the quantiser's codes and scales equal the oracle's
bit for bit; the FP8 forward (kind::f8f6f4 GEMMs) matches the oracle's FP8 forward; compress /
decompress round trips with the FP8 static model and stays within 0.5 % of the oracle's size.
The same for the FP8-hidden form (E4M3 embedding and hidden layer, BF16 logits layer)."""
import numpy as np
import pytest

import synth
from oracle import codec as ocodec
from oracle import fp8
from oracle.mixer import softmax
from oracle.model import Shape, init_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2507_12805_gb300 as P
    return P


@pytest.fixture(scope="module")
def torch():
    import torch
    return torch


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _model(sh, seed, spread=0.05, zero_rows=True):
    rng = np.random.default_rng(seed)
    w = (init_params(sh, seed).astype(np.float64) + rng.normal(0, spread, sh.count)).astype(np.float32)
    off = sh.offsets()
    lo, hi = off["w1"]
    w1t = w[lo:hi].reshape(sh.H, sh.t * sh.E)
    if zero_rows:
        w1t[1] = 0.0                      # an all-zero channel: scale 1, codes 0
        w1t[2, :5] = [1e-12, -3e-9, 5e-8, 1e3, -2e-6]  # subnormal codes and a dominant entry
    w[lo:hi] = w1t.reshape(-1)
    return w


@pytest.mark.parametrize("k,E,t,H", [(3, 16, 4, 64), (4, 32, 8, 128), (6, 32, 4, 256)])
def test_quantizer_codes_and_scales_equal_oracle(P, torch, k, E, t, H):
    sh = Shape(4 ** k, E, t, H)
    w = _model(sh, k * 7 + H)
    ref = fp8.quantize_model(w, sh)
    n_codes = sh.A * E + H * t * E + sh.A * H
    d_codes = torch.zeros(n_codes, dtype=torch.uint8, device="cuda")
    d_scales = torch.zeros(1 + H + sh.A, dtype=torch.float32, device="cuda")
    P.pmklc_quantize_static_fp8(dev(torch, w), k, E, t, H, d_codes, d_scales)
    codes, scales = d_codes.cpu().numpy(), d_scales.cpu().numpy()
    want_codes = np.concatenate([ref["emb"].reshape(-1), ref["w1t"].reshape(-1), ref["w2t"].reshape(-1)])
    want_scales = np.concatenate([[ref["s_emb"]], ref["s_w1"], ref["s_w2"]]).astype(np.float32)
    assert np.array_equal(codes, want_codes)
    assert np.array_equal(scales.view(np.uint32), want_scales.view(np.uint32))


# every dimension on the FP8 engine: two column tiles (H 256, 4^6 logits), K of several stages
@pytest.mark.parametrize("k,E,t,H,rows", [(4, 32, 8, 128, 130), (6, 32, 8, 256, 70), (3, 16, 16, 64, 260)])
def test_fp8_static_forward_matches_oracle(P, torch, k, E, t, H, rows):
    """pmklc_predict in the FP8 form against the oracle's FP8 forward: the same codes, FP32
    accumulation against FP64; an activation whose FP32 and FP64 values straddle an E4M3 rounding
    boundary takes the neighbouring code, so the bar is on the probabilities (2e-2, as for BF16)
    and on the logits relative to their spread."""
    rng = np.random.default_rng(k * 31 + rows)
    sh = Shape(4 ** k, E, t, H)
    w = _model(sh, 5 + k, zero_rows=False)
    ctx = rng.integers(0, sh.A, (rows, t))
    want = fp8.forward(fp8.quantize_model(w, sh), ctx)
    d_out = torch.zeros((rows, sh.A), dtype=torch.float32, device="cuda")
    P.pmklc_predict(dev(torch, w), k, E, t, H, dev(torch, ctx.astype(np.uint16).view(np.int16)), d_out,
                    precision=P.PMKLC_BF16_FP8STATIC)
    got = d_out.cpu().numpy().astype(np.float64)
    assert np.abs(softmax(got) - softmax(want)).max() < 2e-2
    assert np.median(np.abs(got - want)) < 1e-3 * np.abs(want).max()
    assert np.abs(got - want).max() < 0.05 * np.abs(want).max()


def test_fp8_round_trip_and_size_against_oracle(P):
    """The FP8 static form end to end: exact round trip, identical header, coded size within 0.5 %
    of the oracle's FP8 form (network only, so the static model is really used)."""
    seq = synth.markov(12000, 5, 0.40, 1002).tobytes()
    kw = dict(s=2, k=4, use_static=True, emb_s=32, ctx_s=8, hid_s=128, emb_d=16, ctx_d=8, hid_d=64,
              lanes_per_block=8, count_order=5, smp_mode=2, fallback=0)
    sw = _model(Shape(256, 32, 8, 128), 2001, zero_rows=False)
    lens = [4096, 4096, 3808]
    cfg = P.ModelConfig(**kw, static_weights=sw, precision=P.PMKLC_BF16_FP8STATIC)
    out = P.pmklc_compress(seq, lens, cfg)
    back, bl = P.pmklc_decompress(out, sw)
    assert back == seq and list(bl) == lens
    ref = ocodec.compress(seq, lens, ocodec.Config(**kw, precision=2), sw)
    assert out[:80] == ref[:80]
    assert abs(len(out) - len(ref)) <= 0.005 * len(ref), (len(out), len(ref))
    # the FP8 form is recorded in the container: decoding needs no precision argument
    assert ocodec.parse_header(out)[0].precision == 2


def test_fp8_rejects_unsupported_static_shape(P):
    """E4M3 gathers move 16 embedding codes at a time: a static embedding width that is not a
    multiple of 16 is refused up front (no fallback engine for the FP8 form)."""
    seq = synth.markov(3000, 5, 0.40, 7).tobytes()
    kw = dict(s=2, k=4, use_static=True, emb_s=8, ctx_s=8, hid_s=64, emb_d=16, ctx_d=8, hid_d=64,
              lanes_per_block=4, count_order=5, smp_mode=0, fallback=0)
    sw = init_params(Shape(256, 8, 8, 64), 3)
    with pytest.raises(P.PmklcError) as e:
        P.pmklc_compress(seq, [3000], P.ModelConfig(**kw, static_weights=sw, precision=P.PMKLC_BF16_FP8STATIC))
    assert e.value.rc == P.PMKLC_EINVAL


@pytest.mark.parametrize("k,E,t,H,rows", [(4, 32, 8, 128, 130), (6, 32, 8, 256, 70)])
def test_fp8_hidden_forward_matches_oracle(P, torch, k, E, t, H, rows):
    """pmklc_predict in the FP8-hidden form against the oracle's: the same E4M3 embedding and W1
    codes, h rounded to BF16 and W2 in BF16 on the GPU (FP64 and the stored W2 in the oracle), so
    the bars are the BF16 form's (probabilities within 2e-2)."""
    rng = np.random.default_rng(k * 37 + rows)
    sh = Shape(4 ** k, E, t, H)
    w = _model(sh, 7 + k, zero_rows=False)
    ctx = rng.integers(0, sh.A, (rows, t))
    want = fp8.forward_hidden(fp8.quantize_model(w, sh), w, ctx)
    d_out = torch.zeros((rows, sh.A), dtype=torch.float32, device="cuda")
    P.pmklc_predict(dev(torch, w), k, E, t, H, dev(torch, ctx.astype(np.uint16).view(np.int16)), d_out,
                    precision=P.PMKLC_BF16_FP8HIDDEN)
    got = d_out.cpu().numpy().astype(np.float64)
    assert np.abs(softmax(got) - softmax(want)).max() < 2e-2
    assert np.median(np.abs(got - want)) < 1e-2 * np.abs(want).max()


def test_fp8_hidden_round_trip_and_size_against_oracle(P):
    seq = synth.markov(12000, 5, 0.40, 1002).tobytes()
    kw = dict(s=2, k=4, use_static=True, emb_s=32, ctx_s=8, hid_s=128, emb_d=16, ctx_d=8, hid_d=64,
              lanes_per_block=8, count_order=5, smp_mode=2, fallback=0)
    sw = _model(Shape(256, 32, 8, 128), 2001, zero_rows=False)
    lens = [4096, 4096, 3808]
    cfg = P.ModelConfig(**kw, static_weights=sw, precision=P.PMKLC_BF16_FP8HIDDEN)
    out = P.pmklc_compress(seq, lens, cfg)
    back, bl = P.pmklc_decompress(out, sw)
    assert back == seq and list(bl) == lens
    ref = ocodec.compress(seq, lens, ocodec.Config(**kw, precision=3), sw)
    assert out[:80] == ref[:80]
    assert abs(len(out) - len(ref)) <= 0.005 * len(ref), (len(out), len(ref))
    assert ocodec.parse_header(out)[0].precision == 3
