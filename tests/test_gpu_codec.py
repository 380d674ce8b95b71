"""Whole-method tests of the CUDA path: exact round trips, determinism, errors,
and compressed size against the oracle (within 0.5 %)."""
import numpy as np
import pytest

import synth
from oracle import codec as ocodec
from oracle.model import init_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2507_12805_gb300 as P
    return P


def _cfg(P, **kw):
    base = dict(s=2, k=3, use_static=True, emb_s=4, ctx_s=3, hid_s=8, emb_d=4, ctx_d=4, hid_d=8,
                lanes_per_block=3, count_order=3, smp_mode=P.PMKLC_SMP_TREE, smp_fraction=0.2)
    base.update(kw)
    return base


CASES = [
    dict(),
    dict(s=1, k=1, ctx_s=2, ctx_d=2),
    dict(s=3, k=3),
    dict(use_static=False, smp_mode=1),
    dict(smp_mode=0, fallback=0),
    dict(fallback=2, smp_mode=1),
    dict(optimizer=1, lr=0.05),
    dict(s=4, k=5, lanes_per_block=1),
    dict(lanes_per_block=50),
    dict(s=3, k=6, emb_d=8, ctx_d=6, hid_d=24, lanes_per_block=7, fallback=0),
    dict(lanes_per_block=40, lane_tokens=30),
]


def _static(kw):
    from oracle.model import Shape
    return init_params(Shape(4 ** kw["k"], kw["emb_s"], kw["ctx_s"], kw["hid_s"]), 5) if kw["use_static"] else None


@pytest.mark.parametrize("kw", CASES)
def test_round_trip_and_size_vs_oracle(P, kw):
    kw = _cfg(P, **kw)
    sw = _static(kw)
    seq = synth.markov(1500, 2, 0.4, 21).tobytes()
    lens = [700, 500, 2, 0, 298]
    cfg = P.ModelConfig(**kw, static_weights=sw)
    out = P.pmklc_compress(seq, lens, cfg)
    back, bl = P.pmklc_decompress(out, sw)
    assert back == seq and list(bl) == lens
    ref = ocodec.compress(seq, lens, ocodec.Config(**kw), sw)
    assert out[:80] == ref[:80]  # identical header fields, CRC included
    # tiny inputs: sizes agree to a few bytes (learning trajectories differ only by rounding)
    assert abs(len(out) - len(ref)) <= max(8, 0.05 * len(ref))


def test_empty_and_tiny_inputs(P):
    kw = _cfg(P)
    sw = _static(kw)
    cfg = P.ModelConfig(**kw, static_weights=sw)
    for seq, lens in [(b"", []), (b"", [0]), (b"G", [1]), (b"ACGTTGCA", [8]), (b"ACG" * 7, [7, 7, 7])]:
        out = P.pmklc_compress(seq, lens, cfg)
        back, bl = P.pmklc_decompress(out, sw)
        assert back == seq and list(bl) == lens
        assert out == ocodec.compress(seq, lens, ocodec.Config(**kw), sw)


def test_uniform_prefix_bytes_equal_oracle(P):
    # every token inside the uniform prefix: no floating point decides anything,
    # so the whole container must equal the oracle's byte for byte
    kw = _cfg(P, use_static=False, ctx_d=50, lanes_per_block=4, fallback=0)
    seq = synth.markov(800, 2, 0.4, 4).tobytes()  # (s,k)=(2,3): 200 + 198 tokens, 4 lanes of <= 50
    out = P.pmklc_compress(seq, [402, 398], P.ModelConfig(**kw))
    assert out == ocodec.compress(seq, [402, 398], ocodec.Config(**kw))


def test_count_model_fallback_bytes_equal_oracle(P):
    kw = _cfg(P, use_static=False, count_order=6, fallback=1)
    seq = (b"ACGTTGCAAC" * 200) + synth.markov(300, 2, 0.4, 2).tobytes()
    out = P.pmklc_compress(seq, [2000, 300], P.ModelConfig(**kw))
    ref = ocodec.compress(seq, [2000, 300], ocodec.Config(**kw))
    assert P.pmklc_last_stats()["count_blocks"] >= 1
    assert P.pmklc_decompress(out)[0] == seq
    assert abs(len(out) - len(ref)) <= 8


def test_determinism_and_device_path(P):
    import torch
    kw = _cfg(P, k=4, s=2, emb_d=8, ctx_d=8, hid_d=32, lanes_per_block=16)
    sw = _static(kw)
    cfg = P.ModelConfig(**kw, static_weights=sw)
    w = synth.workload("plain", scale=1 / 64)
    a = P.pmklc_compress(w.seq, w.block_lens, cfg)
    b = P.pmklc_compress(w.seq, w.block_lens, cfg)
    assert a == b
    d_seq = torch.from_numpy(w.seq).cuda()
    cap = P.pmklc_compress_bound(w.seq.size, w.block_lens, cfg)
    d_out = torch.zeros(cap, dtype=torch.uint8, device="cuda")
    n = P.pmklc_compress_dev(d_seq, w.block_lens, cfg, d_out)
    assert d_out[:n].cpu().numpy().tobytes() == a
    d_back = torch.zeros(w.seq.size, dtype=torch.uint8, device="cuda")
    m = P.pmklc_decompress_dev(d_out, n, d_back, sw)
    assert m == w.seq.size and torch.equal(d_back, d_seq)


def test_corruption_and_model_errors(P):
    kw = _cfg(P)
    sw = _static(kw)
    cfg = P.ModelConfig(**kw, static_weights=sw)
    seq = synth.markov(3000, 2, 0.4, 12).tobytes()
    out = P.pmklc_compress(seq, [1500, 1500], cfg)
    codes = {}
    for name, bad, w in [("magic", b"XMKL" + out[4:], sw), ("truncated", out[:-5], sw),
                         ("extra", out + b"\0", sw), ("header", out[:60], sw),
                         ("model", out, sw + np.float32(1e-3)), ("nomodel", out, None)]:
        with pytest.raises(P.PmklcError) as e:
            P.pmklc_decompress(bad, w)
        codes[name] = e.value.rc
    assert codes["model"] == codes["nomodel"] == P.PMKLC_EMODEL
    assert codes["magic"] == codes["truncated"] == codes["extra"] == codes["header"] == P.PMKLC_ECORRUPT
    # flipped payload bits: never a crash; either ECORRUPT or a decode that passed the CRC-32 of the
    # input, which then is the input (a flip past the bytes the decoder needs changes nothing)
    rng = np.random.default_rng(0)
    for _ in range(5):
        b = bytearray(out)
        i = int(rng.integers(len(out) - 200, len(out)))
        b[i] ^= 0x10
        try:
            back, _ = P.pmklc_decompress(bytes(b), sw)
        except P.PmklcError as e:
            assert e.rc == P.PMKLC_ECORRUPT
        else:
            assert back == seq
    with pytest.raises(P.PmklcError) as e:
        P.pmklc_compress(seq[:-1] + b"N", [1500, 1500], cfg)
    assert e.value.rc == P.PMKLC_EINVAL


@pytest.mark.slow
def test_tiny_workload_size_within_half_percent_of_oracle(P):
    """The 100,000-base tiny workload, one lane, dynamic model only: the full oracle run."""
    w = synth.workload("tiny")
    kw = dict(s=1, k=3, use_static=False, emb_d=16, ctx_d=16, hid_d=32, lanes_per_block=1, smp_mode=0,
              count_order=6, fallback=1)
    out = P.pmklc_compress(w.seq, w.block_lens, P.ModelConfig(**kw))
    assert P.pmklc_decompress(out)[0] == w.seq.tobytes()
    ref = ocodec.compress(w.seq.tobytes(), w.block_lens, ocodec.Config(**kw))
    assert abs(len(out) - len(ref)) <= 0.005 * len(ref), (len(out), len(ref))
