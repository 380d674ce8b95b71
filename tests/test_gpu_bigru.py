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
