"""Pins of the overlap-masked coding (s < k): only the 4^s tokens that agree with the previous
token on their k - s shared digits are coded over."""
import numpy as np
import pytest

import synth
from oracle import codec
from oracle.codec import SMP_CHAIN, SMP_TREE, Config
from oracle.mixer import loss_grads, softmax
from oracle.model import init_params


def _cfg(**kw):
    base = dict(s=2, k=3, use_static=True, emb_s=4, ctx_s=3, hid_s=8, emb_d=4, ctx_d=4, hid_d=8,
                lanes_per_block=3, count_order=3, smp_mode=SMP_TREE, smp_fraction=0.2, overlap_mask=1)
    base.update(kw)
    return Config(**base)


@pytest.mark.parametrize("kw", [dict(), dict(s=1, k=3), dict(s=3, k=5, lanes_per_block=1),
                                dict(s=1, k=4, smp_mode=SMP_CHAIN, fallback=0), dict(fallback=2),
                                dict(lanes_per_block=40, lane_tokens=30)])
def test_round_trip(kw):
    cfg = _cfg(**kw)
    sw = init_params(cfg.static_shape, 5) if cfg.use_static else None
    seq = synth.markov(1500, 2, 0.4, 31).tobytes()
    lens = [700, 500, 2, 0, 298]
    out = codec.compress(seq, lens, cfg, sw)
    assert codec.parse_header(out)[0].overlap_mask == 1
    assert codec.decompress(out, sw) == seq


def test_no_overlap_no_change():
    """With s = k no token shares digits with the previous one: the payload equals the unmasked one."""
    cfg = _cfg(s=3, k=3)
    sw = init_params(cfg.static_shape, 5)
    seq = synth.markov(1200, 2, 0.4, 32).tobytes()
    a = codec.compress(seq, [1200], cfg, sw)
    b = codec.compress(seq, [1200], _cfg(s=3, k=3, overlap_mask=0), sw)
    assert a[:72] == b[:72] and a[76:] == b[76:] and a != b  # only the variant field differs


def test_uniform_prefix_costs_2s_bits_per_later_token():
    """Every token in the uniform prefix: token 0 of a lane costs 2k bits, each later one 2s."""
    cfg = _cfg(use_static=False, ctx_d=50, lanes_per_block=4, fallback=0)
    seq = synth.markov(402, 2, 0.4, 4).tobytes()  # (s,k)=(2,3): 200 tokens, 4 lanes of 50
    out = codec.compress(seq, [402], cfg)
    payload = len(out) - (80 + 2 + 1 + 1 + 4)
    ideal = 4 * (2 * 3 + 49 * 2 * 2)
    assert abs(8 * payload - ideal) <= 4 * 8
    assert codec.decompress(out) == seq


def test_coded_distribution_is_the_consistent_slice():
    cfg = _cfg(s=1, k=3, use_static=False, ctx_d=2, lanes_per_block=2, fallback=0)
    seq = synth.markov(300, 2, 0.4, 33).tobytes()
    toks = codec.tokenize(codec.base_codes(seq), 1, 3)[0]
    starts, lens = codec.lanes(toks.size, 2)
    seen = []

    def probs(g, j, P):
        seen.append((j, P.copy()))

    codec.compress(seq, [300], cfg, on_probs=probs)
    assert seen
    for j, P in seen:
        for i, st in enumerate(starts):  # both lanes predict at every j >= t
            prev = int(toks[st + j - 1])
            base = (prev % 16) * 4
            assert np.isclose(P[i, base:base + 4].sum(), 1.0, atol=1e-12)
            assert np.all(P[i, :base] == 0) and np.all(P[i, base + 4:] == 0)


def test_slice_loss_gradient_matches_central_differences():
    """dL/dz of the slice's cross entropy: softmax(slice) - onehot inside it, zero outside."""
    rng = np.random.default_rng(4)
    z = rng.normal(0, 1.5, (3, 64))
    bases, tgt = [8, 40, 0], np.array([10, 43, 2])

    def loss(zz):
        return np.mean([-np.log(softmax(zz[i, b:b + 4])[tgt[i] - b]) for i, b in enumerate(bases)])

    P = np.zeros_like(z)
    for i, b in enumerate(bases):
        P[i, b:b + 4] = softmax(z[i, b:b + 4])
    # alpha = 0, no static model: dL/dLm = dL/dz
    dLm, _ = loss_grads(P, tgt, None, z, 0.0, S=(0, 0, 1))
    num = np.zeros_like(z)
    for idx in np.ndindex(*z.shape):
        zp, zm = z.copy(), z.copy()
        zp[idx] += 1e-6
        zm[idx] -= 1e-6
        num[idx] = (loss(zp) - loss(zm)) / 2e-6
    assert np.allclose(dLm, num, atol=1e-8)


def test_masking_saves_bits_on_a_markov_source():
    cfg = _cfg(s=1, k=3, use_static=False, fallback=0, ctx_d=4)
    seq = synth.markov(3000, 3, 0.4, 34).tobytes()
    masked = codec.compress(seq, [1500, 1500], cfg)
    plain = codec.compress(seq, [1500, 1500], _cfg(s=1, k=3, use_static=False, fallback=0, ctx_d=4,
                                                    overlap_mask=0))
    assert len(masked) < 0.8 * len(plain)
