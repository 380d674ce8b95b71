"""Overlap-masked coding (s < k) on the GPU: round trips, the container's variant bit, coded size
within 0.5 % of the oracle's masked form, and the saving against the unmasked coding."""
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


CASES = [
    (dict(s=2, k=4, emb_d=16, ctx_d=8, hid_d=64), 0),      # slice of 16 (generic rows)
    (dict(s=2, k=4, emb_d=16, ctx_d=8, hid_d=64), 1),
    (dict(s=3, k=6, emb_d=16, ctx_d=8, hid_d=64), 1),      # slice of 64 (register rows)
    (dict(s=1, k=3, emb_d=8, ctx_d=8, hid_d=32), 0),       # slice of 4
]


@pytest.mark.parametrize("shape,precision", CASES)
def test_round_trip_and_size_vs_oracle(P, shape, precision):
    seq = synth.markov(9000, 4, 0.42, 61).tobytes()
    lens = [4000, 3000, 2000]
    kw = dict(**shape, use_static=True, emb_s=16, ctx_s=8, hid_s=64, lanes_per_block=8, count_order=4,
              smp_mode=2, fallback=0, overlap_mask=1)
    sw = init_params(ocodec.Config(**kw).static_shape, 2001)
    out = P.pmklc_compress(seq, lens, P.ModelConfig(**kw, static_weights=sw, precision=precision))
    back, bl = P.pmklc_decompress(out, sw)
    assert back == seq and list(bl) == lens
    assert ocodec.parse_header(out)[0].overlap_mask == 1
    ref = ocodec.compress(seq, lens, ocodec.Config(**kw, precision=precision), sw)
    assert out[:80] == ref[:80]
    assert abs(len(out) - len(ref)) <= 0.005 * len(ref), (len(out), len(ref))


def test_masking_saves_bits(P):
    seq = synth.markov(40000, 5, 0.40, 62).tobytes()
    kw = dict(s=2, k=4, emb_d=16, ctx_d=16, hid_d=64, lanes_per_block=16, fallback=0,
              precision=P.PMKLC_BF16_BATCHED)
    masked = P.pmklc_compress(seq, [20000, 20000], P.ModelConfig(**kw, overlap_mask=1))
    plain = P.pmklc_compress(seq, [20000, 20000], P.ModelConfig(**kw))
    print(f"bits/base: masked {8 * len(masked) / len(seq):.4f}, unmasked {8 * len(plain) / len(seq):.4f}")
    assert len(masked) < len(plain)
    assert P.pmklc_decompress(masked)[0] == seq
