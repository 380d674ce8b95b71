"""Per-step parity of the CUDA path against the oracle (element by element, same seeded inputs).

Bars: bit-exact for tokens, frequency tables, coder bytes and count-model bytes;
FP32 probabilities within 1e-4 absolute of the FP64 oracle; gradients and
updated parameters within the tolerances stated per test.
"""
import zlib

import numpy as np
import pytest

import synth
from oracle.mixer import loss_grads, mix, softmax
from oracle.model import Shape, adam_step, backward, forward, init_params
from oracle.quantize import TOTAL, cumulative, quantize
from oracle.rangecoder import decode_all, encode_all
from oracle.tokenizer import base_codes, tokenize

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


# ---------------------------------------------------------------- tokenizer

@pytest.mark.parametrize("s,k", [(1, 1), (1, 3), (2, 4), (3, 3), (3, 6), (5, 8), (8, 8)])
def test_tokenize_bit_exact(P, torch, s, k):
    for n, seed in [(0, 1), (1, 2), (k - 1, 3), (k, 4), (1000, 5), (100_003, 6)]:
        seq = synth.markov(n, 3, 0.42, seed) if n else np.zeros(0, np.uint8)
        want, tail = tokenize(base_codes(seq.tobytes()), s, k)
        d_seq = dev(torch, seq) if n else torch.zeros(1, dtype=torch.uint8, device="cuda")[:0]
        d_tok = torch.zeros(max(len(want), 1), dtype=torch.int16, device="cuda")
        d_tail = torch.zeros(8, dtype=torch.uint8, device="cuda")
        l = P.pmklc_tokenize(d_seq, s, k, d_tok, d_tail)
        assert l == len(want)
        got = d_tok[:l].cpu().numpy().view(np.uint16).astype(np.int64)
        assert np.array_equal(got, want)
        assert np.array_equal(d_tail[:len(tail)].cpu().numpy(), tail)


def test_tokenize_unaligned_and_invalid(P, torch):
    seq = synth.markov(20000, 2, 0.5, 9)
    buf = dev(torch, np.concatenate([np.frombuffer(b"xyz", np.uint8), seq]))
    d = buf[3:]  # 3-byte offset: not 16-byte aligned
    d_tok = torch.zeros(20000, dtype=torch.int16, device="cuda")
    d_tail = torch.zeros(8, dtype=torch.uint8, device="cuda")
    l = P.pmklc_tokenize(d, 1, 4, d_tok, d_tail)
    want, _ = tokenize(base_codes(seq.tobytes()), 1, 4)
    assert np.array_equal(d_tok[:l].cpu().numpy().view(np.uint16), want)
    # every position class: the first bytes, inside a 16-byte vector, the edges of a CTA's 8,192-base
    # segment, the last byte
    for i, pos in enumerate((0, 1, 17, 4095, 8191, 8192, 8193, 8207, 16383, 19999)):
        bad = seq.copy()
        bad[pos] = ord("Na\nt"[i % 4])  # N, lower case, a line break
        with pytest.raises(P.PmklcError) as e:
            P.pmklc_tokenize(dev(torch, bad), 1, 4, d_tok, d_tail)
        assert e.value.rc == P.PMKLC_EINVAL


# ---------------------------------------------------------------- quantiser / mixer

def _probs(rng, rows, A, temp):
    z = rng.normal(0, temp, (rows, A))
    return softmax(z).astype(np.float32)


@pytest.mark.parametrize("A", [4, 16, 64, 256, 4096])
def test_quantize_bit_exact(P, torch, A):
    rng = np.random.default_rng(A)
    Pm = np.concatenate([_probs(rng, 37, A, t) for t in (0.1, 1.0, 4.0, 30.0)])
    Pm[0] = np.float32(1.0 / A)  # uniform
    Pm[1] = 0
    Pm[1, A // 2] = 1  # one-hot
    Pm[2] = 0
    Pm[2, :2] = 0.5  # a tie
    want = quantize(Pm, np.float32)
    d_f = torch.zeros(Pm.shape, dtype=torch.int32, device="cuda")
    P.pmklc_quantize(dev(torch, Pm), d_f)
    got = d_f.cpu().numpy().view(np.uint32).astype(np.int64)
    assert np.array_equal(got, want)
    assert np.all(got.sum(axis=1) == TOTAL) and got.min() >= 1


@pytest.mark.parametrize("A,use_static", [(4, 1), (64, 0), (256, 1), (4096, 1)])
def test_mix_softmax_within_tolerance(P, torch, A, use_static):
    rng = np.random.default_rng(7 + A)
    Lu = rng.normal(0, 3, (50, A)).astype(np.float32)
    Lm = rng.normal(0, 3, (50, A)).astype(np.float32)
    alpha = np.float32(0.3125)
    want = softmax(mix(Lu, Lm, float(alpha), S=(use_static, 0, 1)))
    d_P = torch.zeros((50, A), dtype=torch.float32, device="cuda")
    d_f = torch.zeros((50, A), dtype=torch.int32, device="cuda")
    P.pmklc_mix_quantize(dev(torch, Lu), dev(torch, Lm), float(alpha), bool(use_static), d_P, d_f)
    got = d_P.cpu().numpy()
    assert np.abs(got - want).max() < 1e-4
    f = d_f.cpu().numpy().view(np.uint32).astype(np.int64)
    assert np.all(f.sum(axis=1) == TOTAL) and f.min() >= 1
    # the kernel's table is the quantiser applied to the kernel's own probabilities
    assert np.array_equal(f, quantize(got, np.float32))


# ---------------------------------------------------------------- range coder

@pytest.mark.parametrize("A,L", [(4, 2000), (64, 700), (4096, 300)])
def test_range_coder_bytes_match_oracle(P, torch, A, L):
    rng = np.random.default_rng(A * 3 + L)
    S = 9
    freq = quantize(_probs(rng, S * L, A, 3.0).astype(np.float64)).reshape(S, L, A)
    sym = np.array([[rng.choice(A, p=freq[i, j] / TOTAL) for j in range(L)] for i in range(S)])
    sym[:, ::97] = freq[:, ::97].argmin(axis=-1)  # some improbable symbols
    cap = 3 * L + 8
    d_out = torch.zeros(S * cap, dtype=torch.uint8, device="cuda")
    d_len = torch.zeros(S, dtype=torch.int32, device="cuda")
    d_freq = dev(torch, freq.astype(np.uint32).view(np.int32))
    d_sym = dev(torch, sym.astype(np.uint16).view(np.int16))
    P.pmklc_range_encode(d_freq, d_sym, S, L, A, d_out, cap, d_len)
    out = d_out.cpu().numpy().reshape(S, cap)
    lens = d_len.cpu().numpy()
    for i in range(S):
        want = encode_all(list(sym[i]), cumulative(freq[i]), TOTAL)
        assert out[i, :lens[i]].tobytes() == want
    # GPU decoder on oracle-written bytes
    buf = np.zeros((S, cap), np.uint8)
    for i in range(S):
        b = encode_all(list(sym[i]), cumulative(freq[i]), TOTAL)
        buf[i, :len(b)] = np.frombuffer(b, np.uint8)
    d_sym2 = torch.zeros_like(d_sym)
    P.pmklc_range_decode(d_freq, dev(torch, buf.reshape(-1)), d_len, S, L, A, cap, d_sym2)
    assert np.array_equal(d_sym2.cpu().numpy().view(np.uint16), sym.astype(np.uint16))


# ---------------------------------------------------------------- predictor, train step

def _model(rng, sh, seed, noise=0.2):
    p = init_params(sh, seed).astype(np.float64)
    p += rng.normal(0, noise, p.size)
    return p.astype(np.float32)


@pytest.mark.parametrize("k,E,t,H,rows", [(3, 16, 16, 32, 70), (4, 32, 32, 128, 130), (6, 32, 8, 256, 65)])
def test_predict_within_tolerance(P, torch, k, E, t, H, rows):
    rng = np.random.default_rng(k * 100 + rows)
    sh = Shape(4 ** k, E, t, H)
    params = _model(rng, sh, 3, 0.05)
    ctx = rng.integers(0, sh.A, (rows, t))
    want = forward(params, sh, ctx)[3]
    d_out = torch.zeros((rows, sh.A), dtype=torch.float32, device="cuda")
    P.pmklc_predict(dev(torch, params), k, E, t, H, dev(torch, ctx.astype(np.uint16).view(np.int16)), d_out)
    got = d_out.cpu().numpy()
    assert np.abs(got - want).max() < 1e-4 * max(1.0, np.abs(want).max())


def _oracle_step(cfg, params, m, v, alpha, am, av, static, ctx, tgt, tau, G, M):
    """FP64 oracle of one update per group; returns P, grads, dalpha, new state."""
    dsh, ssh = cfg.dm_shape, cfg.static_shape
    S = (1 if cfg.use_static else 0, 0, 1)
    outs = []
    for g in range(G):
        rows = slice(g * M, (g + 1) * M)
        th = params[g].astype(np.float64)
        cd = ctx[rows, ctx.shape[1] - cfg.ctx_d:]
        X, a, h, Lm = forward(th, dsh, cd)
        Lu = forward(static.astype(np.float64), ssh, ctx[rows, ctx.shape[1] - cfg.ctx_s:])[3] if cfg.use_static else None
        Pr = softmax(mix(Lu, Lm, float(alpha[g]), S))
        dLm, dal = loss_grads(Pr, tgt[rows], Lu, Lm, float(alpha[g]), S)
        gr = backward(th, dsh, cd, X, a, h, dLm)
        mm, vv = m[g].astype(np.float64), v[g].astype(np.float64)
        adam_step(th, mm, vv, gr, tau, float(np.float32(cfg.lr)))
        al, alm, alv = np.array([alpha[g]], np.float64), np.array([am[g]], np.float64), np.array([av[g]], np.float64)
        adam_step(al, alm, alv, np.array([dal]), tau, float(np.float32(cfg.lr)))
        outs.append((Pr, gr, dal, th, mm, vv, al[0]))
    return outs


@pytest.mark.parametrize("use_static", [0, 1])
def test_train_step_within_tolerance(P, torch, use_static):
    from oracle.codec import Config
    rng = np.random.default_rng(11 + use_static)
    cfg_o = Config(s=2, k=4, use_static=bool(use_static), emb_s=16, ctx_s=12, hid_s=48, emb_d=32, ctx_d=8,
                   hid_d=64, lr=1e-3)
    G, M = 3, 37
    dsh = cfg_o.dm_shape
    params = np.stack([_model(rng, dsh, 5 + g, 0.05) for g in range(G)])
    m = (rng.normal(0, 1e-3, params.shape)).astype(np.float32)
    v = (rng.random(params.shape) * 1e-5).astype(np.float32)
    alpha = np.array([0.5, 0.25, 0.8], np.float32)
    am = np.array([1e-3, 0, -1e-3], np.float32)
    av = np.array([1e-6, 0, 2e-6], np.float32)
    static = _model(rng, cfg_o.static_shape, 77, 0.05) if use_static else None
    te = cfg_o.t_eff
    ctx = rng.integers(0, dsh.A, (G * M, te))
    tgt = rng.integers(0, dsh.A, G * M)
    tau = 5
    want = _oracle_step(cfg_o, params, m, v, alpha, am, av, static, ctx, tgt, tau, G, M)
    cfg = P.ModelConfig(s=2, k=4, use_static=bool(use_static), emb_s=16, ctx_s=12, hid_s=48, emb_d=32, ctx_d=8,
                        hid_d=64, lr=1e-3, static_weights=static)
    d = {k: dev(torch, x) for k, x in dict(params=params, m=m, v=v, alpha=alpha, am=am, av=av).items()}
    d_P = torch.zeros((G * M, dsh.A), dtype=torch.float32, device="cuda")
    d_grad = torch.zeros(params.shape, dtype=torch.float32, device="cuda")
    d_da = torch.zeros(G, dtype=torch.float32, device="cuda")
    P.pmklc_train_step(cfg, G, M, d["params"], d["m"], d["v"], d["alpha"], d["am"], d["av"],
                       dev(torch, static) if use_static else None,
                       dev(torch, ctx.astype(np.uint16).view(np.int16)), dev(torch, tgt.astype(np.uint16).view(np.int16)),
                       tau, d_P, d_grad, d_da)
    gP, gg, gda = d_P.cpu().numpy(), d_grad.cpu().numpy(), d_da.cpu().numpy()
    gth, gm, gv, gal = d["params"].cpu().numpy(), d["m"].cpu().numpy(), d["v"].cpu().numpy(), d["alpha"].cpu().numpy()
    for g in range(G):
        Pr, gr, dal, th, mm, vv, al = want[g]
        assert np.abs(gP[g * M:(g + 1) * M] - Pr).max() < 1e-4
        scale = np.abs(gr).max()
        assert np.abs(gg[g] - gr).max() <= 1e-4 * scale, (g, np.abs(gg[g] - gr).max(), scale)
        assert abs(gda[g] - dal) <= 1e-4 * max(1.0, abs(dal))
        assert np.abs(gm[g] - mm).max() <= 1e-5 * max(np.abs(mm).max(), 1e-6) + 1e-9
        # Adam's step is lr * m_hat / (sqrt(v_hat) + eps): bounded by ~lr, compare to lr
        assert np.abs(gth[g] - th).max() <= 2e-2 * cfg.lr
        assert abs(gal[g] - al) <= 2e-2 * cfg.lr


# ---------------------------------------------------------------- count model, CRC

@pytest.mark.parametrize("s,k,M,m", [(1, 1, 1, 0), (1, 1, 1, 6), (2, 4, 16, 6), (3, 6, 64, 7), (1, 3, 200, 2)])
def test_count_model_bytes_equal_oracle(P, s, k, M, m):
    """Count model only (fallback 2): integer arithmetic end to end, so the whole container
    must equal the oracle's byte for byte, including lanes that share a context."""
    from oracle import codec as ocodec
    seq = np.concatenate([synth.markov(n, 3, 0.4, 40 + n) for n in (1, 700, 20_000, 3)]).tobytes()
    lens = [1, 700, 20_000, 3]
    kw = dict(s=s, k=k, emb_d=2, ctx_d=2, hid_d=2, lanes_per_block=M, count_order=m, fallback=2)
    out = P.pmklc_compress(seq, lens, P.ModelConfig(**kw))
    assert out == ocodec.compress(seq, lens, ocodec.Config(**kw))
    back, bl = P.pmklc_decompress(out)
    assert back == seq and list(bl) == lens


def test_crc32_matches_zlib(P, torch):
    rng = np.random.default_rng(1)
    data = rng.integers(0, 256, 3 * 4096 * 300 + 123, dtype=np.uint8)
    d = dev(torch, data)
    for n in (0, 1, 15, 4096, 4097, 4096 * 257 + 3, data.size):
        for off in (0, 1, 7):
            if off + n <= data.size:
                assert P.pmklc_crc32(d[off:], n) == zlib.crc32(data[off:off + n].tobytes())
