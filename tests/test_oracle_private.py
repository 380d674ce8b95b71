"""Pins of the oracle's static private model (SPrM, §4.2.3) and Model Selector (§4.2.1): the
selector's 500 MB threshold, BF16 storage, pre-training that starts from the public model,
round trips, the knowledge the private model brings, and container errors."""
import numpy as np
import pytest

import synth
from oracle import codec
from oracle.codec import Config, CorruptStream
from oracle.model import Shape, init_params


def _cfg(**kw):
    base = dict(s=1, k=3, emb_s=8, ctx_s=6, hid_s=16, emb_d=4, ctx_d=4, hid_d=8, lanes_per_block=4,
                count_order=3, fallback=0, private_model=1, private_epochs=2, lr=3e-3)
    base.update(kw)
    return Config(**base)


def _repeats(n_unit=300, copies=12, seed=3):
    unit = synth.markov(n_unit, 1, 0.5, seed)
    return np.tile(unit, copies).tobytes()


def test_selector_threshold():
    for mode, n, want in [(0, 10 ** 9, False), (1, 10, True), (2, 500_000_000, False), (2, 500_000_001, True)]:
        assert codec.select_private(Config(private_model=mode), n) == want


def test_bf16_rounding_ties_to_even():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 1.0 + 2 ** -9, -2.5, 0.0], np.float32)
    got = codec.bf16_round(x)
    # 1 + 2^-8 is halfway between 1 and 1 + 2^-7: ties to the even mantissa (1.0); 1 + 3 2^-8 to 1 + 2^-6
    assert np.array_equal(got, np.array([1.0, 1.0, 1.0 + 2 ** -6, 1.0, -2.5, 0.0], np.float32))
    y = np.random.default_rng(0).normal(0, 1, 1000).astype(np.float32)
    r = codec.bf16_round(y)
    assert np.all(r.view(np.uint32) & 0xFFFF == 0)
    assert np.all(np.abs(r - y) <= np.abs(y) * 2.0 ** -8)


def test_round_trip_without_any_given_model():
    seq = _repeats()
    cfg = _cfg()
    out = codec.compress(seq, [len(seq)], cfg)
    hdr, meta = codec.parse_header(out)
    assert meta["private"] and hdr.use_static
    assert codec.decompress(out) == seq
    assert codec.decompress(out, init_params(Shape(64, 8, 6, 16), 1)) == seq  # a given model is ignored


def test_stored_model_is_the_bf16_pretrained_one():
    seq = _repeats()
    cfg = _cfg()
    codes = np.frombuffer(seq, np.uint8)
    want = codec.bf16_round(codec.pretrain(codec.base_codes(codes), cfg, init_params(cfg.static_shape, cfg.seed),
                                           cfg.private_epochs))
    out = codec.compress(seq, [len(seq)], cfg)
    assert want.size == cfg.static_shape.count
    assert (want.view(np.uint32) >> 16).astype("<u2").tobytes() in out
    assert codec.compress(seq, [len(seq)], cfg, private_w=want) == out


def test_pretraining_starts_from_the_public_model():
    """With no token past the context (nothing to train on) the private model is the public one,
    rounded to BF16."""
    sw = init_params(Shape(64, 8, 6, 16), 11)
    cfg = _cfg(use_static=True)
    codes = codec.base_codes(b"ACGTA")
    got = codec.pretrain(codes, cfg, sw, 1)
    assert np.array_equal(got, sw)


def test_private_knowledge_shrinks_the_payload():
    """On a highly repetitive input the pre-trained private model predicts the repeats: the coded
    payload (the container minus the stored model) is smaller than with no static model."""
    seq = _repeats(400, 15, 5)
    with_p = codec.compress(seq, [len(seq)], _cfg(private_epochs=3))
    without = codec.compress(seq, [len(seq)], _cfg(private_model=0))
    model_bytes = 2 * Shape(64, 8, 6, 16).count
    assert len(with_p) - model_bytes < 0.9 * len(without)


def test_damaged_private_section_is_corrupt():
    seq = _repeats(200, 6)
    out = codec.compress(seq, [len(seq)], _cfg())
    with pytest.raises(CorruptStream):
        codec.decompress(out[:-1] if len(out) > 0 else out)
    bad = bytearray(out)
    bad[7] &= ~1  # clear the static-slot flag while the private flag stays
    with pytest.raises(CorruptStream):
        codec.decompress(bytes(bad))
    # one bit of the stored model: its hash no longer matches
    cfg = _cfg()
    w = codec.bf16_round(codec.pretrain(codec.base_codes(seq), cfg, init_params(cfg.static_shape, cfg.seed),
                                        cfg.private_epochs))
    pos = out.find((w.view(np.uint32) >> 16).astype("<u2").tobytes(), 80)
    assert pos > 80
    flip = bytearray(out)
    flip[pos + 101] ^= 0x01
    with pytest.raises(CorruptStream):
        codec.decompress(bytes(flip))
