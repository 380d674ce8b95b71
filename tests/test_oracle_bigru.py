"""Pins of the oracle's BiGRU static predictor (§4.2.2 SPuM, §4.2.3 SPrM)."""
import math

import numpy as np
import pytest

from oracle.bigru import DENSE, GruShape, drop_second_layer, forward, init_bigru, params, states


def _generic(sh: GruShape, seed=5):
    """Seeded weights moved to a generic point (nonzero biases, gates away from 1/2)."""
    p = init_bigru(sh, seed).astype(np.float64)
    p += np.random.default_rng(seed).normal(0, 0.4, p.size)
    return p


def _set(flat, sh, name, value):
    lo, hi = sh.offsets()[name]
    flat[lo:hi] = np.asarray(value, dtype=np.float64).reshape(-1)


@pytest.mark.parametrize("layers", [1, 2])
def test_matches_torch_gru(layers):
    """torch.nn.GRU (float64, bidirectional) on the same weights gives the same layer outputs and
    final states: an independent implementation of the recurrence pins gate order, reset-gate
    placement, direction and the layer stacking."""
    torch = pytest.importorskip("torch")
    sh = GruShape(A=64, E=5, t=7, Hg=4, layers=layers)
    flat = _generic(sh)
    rng = np.random.default_rng(1)
    ctx = rng.integers(0, sh.A, (9, sh.t))
    ctx[2, :] = ctx[2, 0]  # one context of a single repeated token
    outs, u = states(flat, sh, ctx)
    w = params(flat, sh)
    gru = torch.nn.GRU(sh.E, sh.Hg, num_layers=layers, bidirectional=True, batch_first=True, dtype=torch.float64)
    with torch.no_grad():
        for l in range(layers):
            for d, suf in (("f", ""), ("b", "_reverse")):
                getattr(gru, f"weight_ih_l{l}{suf}").copy_(torch.from_numpy(w[f"wi{l}{d}"]))
                getattr(gru, f"weight_hh_l{l}{suf}").copy_(torch.from_numpy(w[f"wh{l}{d}"]))
                getattr(gru, f"bias_ih_l{l}{suf}").copy_(torch.from_numpy(w[f"bi{l}{d}"]))
                getattr(gru, f"bias_hh_l{l}{suf}").copy_(torch.from_numpy(w[f"bh{l}{d}"]))
        x = torch.from_numpy(w["emb"][ctx])
        out, hn = gru(x)
    np.testing.assert_allclose(outs[-1], out.numpy(), rtol=0, atol=1e-13)
    # u = [forward state after t-1, backward state after 0] = torch's final states of the last layer
    np.testing.assert_allclose(u, np.concatenate([hn[-2].numpy(), hn[-1].numpy()], axis=1), rtol=0, atol=1e-13)
    if layers == 2:  # the first layer's output: a one-layer torch GRU on its weights
        g1 = torch.nn.GRU(sh.E, sh.Hg, num_layers=1, bidirectional=True, batch_first=True, dtype=torch.float64)
        with torch.no_grad():
            for d, suf in (("f", ""), ("b", "_reverse")):
                for a, b in (("weight_ih", "wi"), ("weight_hh", "wh"), ("bias_ih", "bi"), ("bias_hh", "bh")):
                    getattr(g1, f"{a}_l0{suf}").copy_(torch.from_numpy(w[f"{b}0{d}"]))
            o1, _ = g1(x)
        np.testing.assert_allclose(outs[0], o1.numpy(), rtol=0, atol=1e-13)


def test_recurrence_closed_form():
    """Input and recurrent weights 0, gate biases 0 (z = r = 1/2) and tanh of the candidate bias c:
    h_p = c/2 + h_{p-1}/2, so the forward state after position p is c (1 - 2^-(p+1)), the backward
    one after position p is c' (1 - 2^-(t-p)).  With W3 the identity on u, b3 = 0, W4 = I and b4 = 0
    the logits are relu(u) padded with zeros."""
    sh = GruShape(A=16, E=3, t=5, Hg=1, layers=1, D=2)
    flat = np.zeros(sh.count)
    _set(flat, sh, "emb", np.random.default_rng(0).normal(0, 1, sh.A * sh.E))  # unread: Wi = 0
    _set(flat, sh, "bi0f", [0.0, 0.0, math.log(2.0)])    # tanh(ln 2) = 0.6
    _set(flat, sh, "bi0b", [0.0, 0.0, 0.5 * math.log(3.0)])  # tanh(ln 3 / 2) = 0.5
    _set(flat, sh, "w3", np.eye(2))
    w4 = np.zeros((2, sh.A))
    w4[0, 0] = w4[1, 1] = 1.0
    _set(flat, sh, "w4", w4)
    ctx = np.random.default_rng(1).integers(0, sh.A, (3, sh.t))
    outs, u = states(flat, sh, ctx)
    p = np.arange(sh.t)
    np.testing.assert_allclose(outs[0][:, :, 0], np.broadcast_to(0.6 * (1 - 2.0 ** -(p + 1)), (3, sh.t)), atol=1e-15)
    np.testing.assert_allclose(outs[0][:, :, 1], np.broadcast_to(0.5 * (1 - 2.0 ** -(sh.t - p)), (3, sh.t)),
                               atol=1e-15)
    q, L = forward(flat, sh, ctx)
    want = np.zeros((3, sh.A))
    want[:, 0] = 0.6 * (1 - 2.0 ** -sh.t)
    want[:, 1] = 0.5 * (1 - 2.0 ** -sh.t)
    np.testing.assert_allclose(L, want, atol=1e-15)
    np.testing.assert_allclose(q, want[:, :2], atol=1e-15)


def test_reset_gate_applies_to_the_recurrent_projection_after_its_bias():
    """Hg = 1, t = 2, z = 1/2, candidate weight w and recurrent bias c on the n row.  With the reset
    gate saturated at 0 the candidate ignores h and c: h_2 = 3/4 tanh(b).  Saturated at 1:
    h_1 = tanh(b + c)/2 and h_2 = tanh(b + w h_1 + c)/2 + h_1/2."""
    sh = GruShape(A=4, E=1, t=2, Hg=1, layers=1, D=2)
    b, c, w = 0.3, 0.7, -1.1
    for r_bias, want in ((-60.0, None), (60.0, None)):
        flat = np.zeros(sh.count)
        _set(flat, sh, "bi0f", [r_bias, 0.0, b])
        _set(flat, sh, "bh0f", [0.0, 0.0, c])
        _set(flat, sh, "wh0f", [[0.0], [0.0], [w]])
        outs, _ = states(flat, sh, np.zeros((1, sh.t), dtype=int))
        h2 = outs[0][0, 1, 0]
        if r_bias < 0:
            assert abs(h2 - 0.75 * math.tanh(b)) < 1e-15
        else:
            h1 = math.tanh(b + c) / 2
            assert abs(outs[0][0, 0, 0] - h1) < 1e-15
            assert abs(h2 - (math.tanh(b + w * h1 + c) / 2 + h1 / 2)) < 1e-15


def test_saturated_update_gate_keeps_the_zero_state():
    """z = 1 everywhere (large update-gate bias): the state never leaves 0, so u = 0 and the logits
    are relu(b3) W4 + b4 whatever the context."""
    sh = GruShape(A=16, E=4, t=6, Hg=3, layers=2)
    flat = _generic(sh)
    for l in range(2):
        for d in ("f", "b"):
            lo, _ = sh.offsets()[f"bi{l}{d}"]
            flat[lo + sh.Hg:lo + 2 * sh.Hg] = 80.0
    w = params(flat, sh)
    ctx = np.random.default_rng(2).integers(0, sh.A, (4, sh.t))
    _, u = states(flat, sh, ctx)
    assert np.abs(u).max() < 1e-30
    _, L = forward(flat, sh, ctx)
    np.testing.assert_allclose(L, np.broadcast_to(np.maximum(w["b3"], 0) @ w["w4"] + w["b4"], L.shape), atol=1e-12)


def test_direction_swap_symmetry():
    """Swapping each layer's forward and backward GRU, reversing every context, and swapping the
    halves of the inputs that read [forward, backward] (W3's columns, layer 1's Wi columns) gives
    the same logits: catches a direction or position index taken from the wrong side."""
    sh = GruShape(A=64, E=4, t=6, Hg=3, layers=2)
    flat = _generic(sh, seed=9)
    sw = flat.copy()
    off = sh.offsets()
    Hg = sh.Hg

    def swap_cols(m):
        return np.concatenate([m[:, Hg:], m[:, :Hg]], axis=1)

    w = params(flat, sh)
    for l in range(2):
        for a, b in (("f", "b"), ("b", "f")):
            for p in ("wi", "wh", "bi", "bh"):
                v = w[f"{p}{l}{b}"]
                if p == "wi" and l == 1:
                    v = swap_cols(v)
                _set(sw, sh, f"{p}{l}{a}", v)
    _set(sw, sh, "w3", swap_cols(w["w3"]))
    ctx = np.random.default_rng(3).integers(0, sh.A, (5, sh.t))
    _, L = forward(flat, sh, ctx)
    _, Ls = forward(sw, sh, ctx[:, ::-1])
    np.testing.assert_allclose(Ls, L, rtol=0, atol=1e-12)
    # and the logits do depend on the order of the context (so the check above is not vacuous)
    _, Lr = forward(flat, sh, ctx[:, ::-1])
    assert np.abs(Lr - L).max() > 1e-3
    assert off["b4"][1] == sh.count


def test_layout_init_and_private_view():
    sh = GruShape(A=256, E=16, t=32, Hg=32, layers=2)
    # sizes: embedding, 2 layers x 2 directions of (3Hg x in + 3Hg x Hg + 6 Hg), head
    want = 256 * 16 + 2 * (96 * 16 + 96 * 32 + 192) + 2 * (96 * 64 + 96 * 32 + 192) + 128 * 64 + 128 + 128 * 256 + 256
    assert sh.count == want and DENSE == 128
    assert GruShape(256, 16, 8, 32, 2).count == sh.count  # independent of t
    p = init_bigru(sh, 2001)
    w = params(p, sh)
    assert p.dtype == np.float32
    assert np.all(w["b3"] == 0) and np.all(w["bi1b"] == 0) and not np.signbit(w["b4"]).any()
    assert np.abs(w["emb"]).max() <= 1 and np.abs(w["wi0f"]).max() <= 0.25 and np.abs(w["wi1f"]).max() <= 0.125
    assert np.abs(w["w4"]).max() <= 1 / math.sqrt(128) + 1e-7 and np.abs(w["wh0b"]).max() <= 1 / math.sqrt(32) + 1e-7
    # SPrM's structure: the same embedding, first layer and head; a model of one layer
    one_flat, one = drop_second_layer(p, sh)
    assert one.layers == 1 and one_flat.size == one.count
    w1 = params(one_flat, one)
    for n in ("emb", "wi0f", "wh0b", "bh0f", "w3", "b4"):
        assert np.array_equal(w1[n], w[n])
    ctx = np.random.default_rng(4).integers(0, sh.A, (3, sh.t))
    sh1 = GruShape(256, 16, 32, 32, 1)
    q1, L1 = forward(one_flat, sh1, ctx)
    # the one-layer model's summary is the first layer's [forward last, backward first] of SPuM
    outs, _ = states(p, sh, ctx)
    u0 = np.concatenate([outs[0][:, -1, :32], outs[0][:, 0, 32:]], axis=1)
    np.testing.assert_allclose(q1, np.maximum(u0 @ w["w3"].T + w["b3"], 0), atol=1e-12)


# ---------------------------------------------------------------- the BiGRU in the codec's static slot

def _codec_case(arch, k=2):
    import synth
    from oracle import codec
    seq = synth.markov(2400, 3, 0.45, 77).tobytes()
    cfg = codec.Config(s=1, k=k, use_static=True, emb_s=8, ctx_s=4, hid_s=16, emb_d=8, ctx_d=6, hid_d=16,
                       lanes_per_block=4, fallback=0, static_arch=arch, smp_mode=codec.SMP_CHAIN)
    sh = GruShape(4 ** k, 8, 4, 16, arch)
    return codec, seq, cfg, sh


@pytest.mark.parametrize("arch", [1, 2])
def test_codec_round_trip_and_header(arch):
    codec, seq, cfg, sh = _codec_case(arch)
    sw = _generic(sh, seed=3).astype(np.float32)
    blob = codec.compress(seq, [1200, 1200], cfg, sw)
    assert blob[7] >> 4 == arch and blob[7] & 1
    pc, meta = codec.parse_header(blob)
    assert pc.static_arch == arch and (pc.emb_s, pc.ctx_s, pc.hid_s) == (8, 4, 16)
    assert codec.decompress(blob, sw) == seq
    with pytest.raises(codec.ModelMismatch):
        codec.decompress(blob, (sw * 1.5).astype(np.float32))
    bad = bytearray(blob)
    bad[7] |= 0x30  # static_arch 3
    with pytest.raises(codec.CorruptStream):
        codec.decompress(bytes(bad), sw)
    bad[7] = blob[7] | 0x40
    with pytest.raises(codec.CorruptStream):
        codec.decompress(bytes(bad), sw)


def test_codec_bigru_slot_enters_eq1_as_the_static_logits():
    """A BiGRU whose Dense layer is zero gives L^u = 0, and Eq. (1) with L^u = 0 equals Eq. (1) with
    S0 = 0: the payload is byte for byte that of the run without a static model (same t_eff).  Any
    nonzero Dense layer changes it."""
    codec, seq, cfg, sh = _codec_case(2)
    sw = _generic(sh, seed=4)
    lo, hi = sh.offsets()["w4"][0], sh.count
    sw[lo:hi] = 0.0
    sw = sw.astype(np.float32)
    blob = codec.compress(seq, [2400], cfg, sw)
    from dataclasses import replace
    plain = codec.compress(seq, [2400], replace(cfg, use_static=False, static_arch=0, emb_s=0, ctx_s=0, hid_s=0))
    hl = codec.HEADER.size
    assert blob[hl:] == plain[hl:]
    sw2 = sw.copy()
    sw2[lo:hi] = _generic(sh, seed=5)[lo:hi]
    assert codec.compress(seq, [2400], cfg, sw2)[hl:] != plain[hl:]


def test_codec_bigru_config_errors():
    from dataclasses import replace
    codec, seq, cfg, sh = _codec_case(1)
    sw = init_bigru(sh, 1)
    with pytest.raises(ValueError):
        codec.compress(seq, [2400], replace(cfg, private_model=1), sw)
    with pytest.raises(ValueError):
        codec.compress(seq, [2400], replace(cfg, precision=2), sw)
    with pytest.raises(ValueError):
        codec.compress(seq, [2400], cfg, sw[:-1])


def test_planted_recurrence_mistakes_fail_the_torch_pin():
    """Plausible mistakes in the recurrence, planted in a copy of the oracle's pass, each move the
    layer output away from torch.nn.GRU's by far more than the pin's 1e-13: the reset gate applied
    to h before the recurrent product (the other published GRU form), the update gate's two terms
    swapped, the backward pass run oldest first, and the summary taken from the wrong end."""
    torch = pytest.importorskip("torch")
    from oracle import bigru as B
    sh = GruShape(A=64, E=5, t=7, Hg=4, layers=1)
    flat = _generic(sh, seed=13)
    w = params(flat, sh)
    ctx = np.random.default_rng(6).integers(0, sh.A, (9, sh.t))
    x = w["emb"][ctx]
    gru = torch.nn.GRU(sh.E, sh.Hg, num_layers=1, bidirectional=True, batch_first=True, dtype=torch.float64)
    with torch.no_grad():
        for d, suf in (("f", ""), ("b", "_reverse")):
            for a, b in (("weight_ih", "wi"), ("weight_hh", "wh"), ("bias_ih", "bi"), ("bias_hh", "bh")):
                getattr(gru, f"{a}_l0{suf}").copy_(torch.from_numpy(w[f"{b}0{d}"]))
        want, hn = gru(torch.from_numpy(x))
    want, hn = want.numpy(), hn.numpy()

    def planted(wi, wh, bi, bh, reverse, mistake):
        R, t, _ = x.shape
        Hg = wh.shape[1]
        h = np.zeros((R, Hg))
        seq = np.zeros((R, t, Hg))
        order = range(t - 1, -1, -1) if reverse and mistake != "backward_oldest_first" else range(t)
        for p in order:
            gi = x[:, p, :] @ wi.T + bi
            gh = h @ wh.T + bh
            r = B._sigmoid(gi[:, :Hg] + gh[:, :Hg])
            z = B._sigmoid(gi[:, Hg:2 * Hg] + gh[:, Hg:2 * Hg])
            if mistake == "reset_before_product":
                n = np.tanh(gi[:, 2 * Hg:] + (r * h) @ wh[2 * Hg:].T + bh[2 * Hg:])
            else:
                n = np.tanh(gi[:, 2 * Hg:] + r * gh[:, 2 * Hg:])
            h = z * n + (1.0 - z) * h if mistake == "update_swapped" else (1.0 - z) * n + z * h
            seq[:, p, :] = h
        return seq

    def layer(mistake):
        f = planted(w["wi0f"], w["wh0f"], w["bi0f"], w["bh0f"], False, mistake)
        b = planted(w["wi0b"], w["wh0b"], w["bi0b"], w["bh0b"], True, mistake)
        return np.concatenate([f, b], axis=2)

    assert np.abs(layer(None) - want).max() < 1e-13  # the planted copy without a mistake is the oracle
    for mistake in ("reset_before_product", "update_swapped", "backward_oldest_first"):
        assert np.abs(layer(mistake) - want).max() > 1e-3, mistake
    # the summary from the wrong ends (forward state after position 0, backward after t-1)
    out = layer(None)
    wrong_u = np.concatenate([out[:, 0, :sh.Hg], out[:, -1, sh.Hg:]], axis=1)
    assert np.abs(wrong_u - np.concatenate([hn[-2], hn[-1]], axis=1)).max() > 1e-3
