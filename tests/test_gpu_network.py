"""Whole-run parity of the learned path itself: network-only coding (fallback 0, so no block is left
to the count model) on inputs of 2^16 bases, on shapes that take the tcgen05 engine in the BF16
form ((2,4) with E 32, t 32, H 128 and (3,6) with E 32, t 64, H 256), with and without overlap
masking, chain and tree step-wise model passing: exact round trips, the oracle's header, and a
compressed size within 0.5 % of the oracle's."""
import pytest

import synth
from oracle import codec as ocodec
from oracle.model import init_params

pytestmark = pytest.mark.gpu

K4 = dict(s=2, k=4, use_static=True, emb_s=32, ctx_s=32, hid_s=128, emb_d=32, ctx_d=32, hid_d=128)
K6 = dict(s=3, k=6, use_static=True, emb_s=32, ctx_s=64, hid_s=256, emb_d=32, ctx_d=64, hid_d=256)
CASES = [
    (K4, dict(overlap_mask=1, smp_mode=2), 1),
    (K4, dict(overlap_mask=1, smp_mode=2), 0),
    (K4, dict(overlap_mask=0, smp_mode=1), 1),
    (K6, dict(overlap_mask=1, smp_mode=2), 1),
    (K6, dict(overlap_mask=1, smp_mode=1), 0),
]


@pytest.fixture(scope="module")
def P():
    import paper_2507_12805_gb300 as P
    return P


@pytest.mark.parametrize("shape,opts,precision", CASES)
def test_network_only_size_within_half_percent_of_oracle(P, shape, opts, precision):
    n_blocks, block = 4, 1 << 14
    if shape["k"] == 6:
        seq = synth.human_like(n_blocks * block, 1003).tobytes()
    else:
        seq = synth.markov(n_blocks * block, 5, 0.40, 1002).tobytes()
    lens = [block] * n_blocks
    kw = dict(**shape, **opts, lanes_per_block=32, smp_fraction=0.05, fallback=0, alpha_init=0.5)
    sw = init_params(ocodec.Config(**kw).static_shape, 2001)
    out = P.pmklc_compress(seq, lens, P.ModelConfig(**kw, static_weights=sw, precision=precision))
    assert P.pmklc_last_stats()["net_blocks"] == n_blocks
    back, bl = P.pmklc_decompress(out, sw)
    assert back == seq and list(bl) == lens
    ref = ocodec.compress(seq, lens, ocodec.Config(**kw, precision=precision), sw)
    assert out[:80] == ref[:80]
    print(f"{shape['s']},{shape['k']} {opts} precision {precision}: GPU {8 * len(out) / len(seq):.4f} "
          f"oracle {8 * len(ref) / len(seq):.4f} bits/base ({(len(out) - len(ref)) / len(ref):+.3%})")
    assert abs(len(out) - len(ref)) <= 0.005 * len(ref), (len(out), len(ref))
