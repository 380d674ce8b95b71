"""GPU parity of the BiGRU static predictor (§4.2.2 SPuM, §4.2.3 SPrM) against the FP64 oracle.

Through the C ABI: pmklc_predict_bigru's Linear-layer output q and logits, on rows that span
several CTAs of 128 rows and a ragged tail, held to the benchmark spec's tolerance for FP32 predictors
(probabilities within 1e-4 absolute of the oracle's).
"""
import numpy as np
import pytest

from oracle.bigru import GruShape, forward, init_bigru
from oracle.mixer import softmax

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


def _model(sh, seed, noise=0.15):
    p = init_bigru(sh, seed).astype(np.float64)
    p += np.random.default_rng(seed).normal(0, noise, p.size)
    return p.astype(np.float32)


@pytest.mark.parametrize("k,E,t,Hg,layers,rows", [
    (3, 16, 16, 32, 2, 300),    # SPuM's structure (two layers, E 16), three CTAs and a tail of 44
    (3, 16, 16, 32, 1, 129),    # SPrM's structure (one layer)
    (6, 16, 64, 32, 2, 257),    # the (3,6) alphabet, a 64-token context
    (4, 8, 5, 16, 2, 1),        # one row
    (2, 32, 1, 16, 1, 70),      # t = 1
])
def test_predict_bigru_matches_oracle(P, torch, k, E, t, Hg, layers, rows):
    sh = GruShape(4 ** k, E, t, Hg, layers)
    assert P.pmklc_bigru_count(k, E, Hg, layers) == sh.count
    params = _model(sh, 11 + k)
    rng = np.random.default_rng(k * 1000 + rows)
    ctx = rng.integers(0, sh.A, (rows, t))
    ctx[0, :] = ctx[0, 0]  # a context of one repeated token
    q_want, L_want = forward(params, sh, ctx)
    d_q = torch.zeros((rows, 128), dtype=torch.float32, device="cuda")
    d_L = torch.zeros((rows, sh.A), dtype=torch.float32, device="cuda")
    P.pmklc_predict_bigru(dev(torch, params), k, E, t, Hg, layers, dev(torch, ctx.astype(np.uint16).view(np.int16)),
                          d_q=d_q, d_logits=d_L)
    q, L = d_q.cpu().numpy(), d_L.cpu().numpy()
    assert np.abs(q - q_want).max() < 1e-5 * max(1.0, np.abs(q_want).max())
    assert np.abs(L - L_want).max() < 1e-4 * max(1.0, np.abs(L_want).max())
    assert np.abs(softmax(L.astype(np.float64)) - softmax(L_want)).max() < 1e-4
    # q alone (no logits) gives the same values
    d_q2 = torch.zeros_like(d_q)
    P.pmklc_predict_bigru(dev(torch, params), k, E, t, Hg, layers, dev(torch, ctx.astype(np.uint16).view(np.int16)),
                          d_q=d_q2)
    assert torch.equal(d_q, d_q2)


def test_predict_bigru_rejects_tokens_outside_the_alphabet(P, torch):
    k, E, t, Hg = 2, 16, 4, 16
    sh = GruShape(16, E, t, Hg, 1)
    ctx = np.zeros((3, t), np.uint16)
    ctx[1, 2] = 16  # = A
    d_L = torch.zeros((3, 16), dtype=torch.float32, device="cuda")
    with pytest.raises(P.PmklcError) as e:
        P.pmklc_predict_bigru(dev(torch, _model(sh, 1)), k, E, t, Hg, 1, dev(torch, ctx.view(np.int16)), d_logits=d_L)
    assert e.value.rc == P.PMKLC_EINVAL
    # the context is still usable afterwards
    P.pmklc_predict_bigru(dev(torch, _model(sh, 1)), k, E, t, Hg, 1, dev(torch, np.zeros((3, t), np.int16)),
                          d_logits=d_L)
    torch.cuda.synchronize()


# ---------------------------------------------------------------- the BiGRU in the codec's static slot

import synth  # noqa: E402
from oracle import codec as ocodec  # noqa: E402

# (s,k), dynamic model, BiGRU static predictor (E 16 as in §4.2.2, t, GRU width, layers), options, form
CODEC_CASES = [
    (dict(s=2, k=4, emb_d=32, ctx_d=32, hid_d=128), dict(emb_s=16, ctx_s=16, hid_s=32, static_arch=2),
     dict(overlap_mask=1, smp_mode=2), 1),
    (dict(s=2, k=4, emb_d=32, ctx_d=32, hid_d=128), dict(emb_s=16, ctx_s=16, hid_s=32, static_arch=2),
     dict(overlap_mask=0, smp_mode=1), 0),
    (dict(s=3, k=6, emb_d=16, ctx_d=16, hid_d=64), dict(emb_s=16, ctx_s=16, hid_s=32, static_arch=1),
     dict(overlap_mask=1, smp_mode=1), 1),
    (dict(s=3, k=6, emb_d=16, ctx_d=16, hid_d=64), dict(emb_s=16, ctx_s=12, hid_s=16, static_arch=2),
     dict(overlap_mask=1, smp_mode=2), 0),
    # a dynamic model the tcgen05 engine does not take (H 48): the BF16 form on mma.sync
    (dict(s=2, k=4, emb_d=16, ctx_d=16, hid_d=48), dict(emb_s=8, ctx_s=8, hid_s=16, static_arch=1),
     dict(overlap_mask=1, smp_mode=2), 1),
]


@pytest.mark.parametrize("dm,st,opts,precision", CODEC_CASES)
def test_codec_with_bigru_static_model_matches_oracle(P, dm, st, opts, precision):
    """Network-only coding (fallback 0) with the BiGRU static predictor in the static slot of
    Eq. (1): exact round trip, the oracle's header and a size within 0.5 % of the oracle's, in the
    FP32 plain and BF16 batched forms (the BiGRU runs in FP32 on the CUDA cores in both; its h is
    rounded to BF16 for the BF16 logits GEMM)."""
    n_blocks, block = 2, 1 << 14
    if dm["k"] == 6:
        seq = synth.human_like(n_blocks * block, 1003).tobytes()
    else:
        seq = synth.markov(n_blocks * block, 5, 0.40, 1002).tobytes()
    lens = [block] * n_blocks
    kw = dict(**dm, **st, **opts, use_static=True, lanes_per_block=32, smp_fraction=0.05, fallback=0, alpha_init=0.5)
    sh = GruShape(4 ** dm["k"], st["emb_s"], st["ctx_s"], st["hid_s"], st["static_arch"])
    sw = _model(sh, 2001, noise=0.1)
    out = P.pmklc_compress(seq, lens, P.ModelConfig(**kw, static_weights=sw, precision=precision))
    assert P.pmklc_last_stats()["net_blocks"] == n_blocks
    back, bl = P.pmklc_decompress(out, sw)
    assert back == seq and list(bl) == lens
    with pytest.raises(P.PmklcError) as e:
        P.pmklc_decompress(out, (sw * 1.01).astype(np.float32))
    assert e.value.rc == P.PMKLC_EMODEL
    ref = ocodec.compress(seq, lens, ocodec.Config(**kw, precision=precision), sw)
    assert out[:80] == ref[:80]
    print(f"BiGRU static ({st['static_arch']} layers) {dm['s']},{dm['k']} {opts} precision {precision}: GPU "
          f"{8 * len(out) / len(seq):.4f} oracle {8 * len(ref) / len(seq):.4f} bits/base "
          f"({(len(out) - len(ref)) / len(ref):+.3%})")
    assert abs(len(out) - len(ref)) <= 0.005 * len(ref), (len(out), len(ref))
