"""Pins of the oracle's range coder, exact arithmetic coder and count model."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import countmodel
from oracle.quantize import TOTAL, cumulative, quantize
from oracle.rangecoder import Decoder, Encoder, decode_all, encode_all, exact_decode, exact_encode
from oracle.mixer import softmax
from oracle.tokenizer import base_codes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _random_tables(rng, n, A, temp):
    P = softmax(rng.normal(0, temp, (n, A)))
    f = quantize(P)
    return f, cumulative(f)


def _ideal_bits(sym, freq, total):
    return sum(-math.log2(freq[i][s] / total) for i, s in enumerate(sym))


@pytest.mark.parametrize("A,temp", [(4, 1.0), (64, 3.0), (256, 8.0), (4096, 0.5)])
def test_round_trip_and_length_bound(A, temp):
    rng = np.random.default_rng(A)
    n = 600
    freq, cum = _random_tables(rng, n, A, temp)
    # draw symbols from the coded distributions, plus some very unlikely ones
    sym = [int(rng.choice(A, p=freq[i] / TOTAL)) for i in range(n)]
    for i in range(0, n, 50):
        sym[i] = int(freq[i].argmin())
    data = encode_all(sym, cum, TOTAL)
    assert decode_all(data, cum, TOTAL) == sym
    ideal = _ideal_bits(sym, freq, TOTAL)
    assert 8 * len(data) <= ideal + n * 2.0 ** -24 / math.log(2) * 1.0001 + 8
    assert 8 * len(data) >= ideal - 56  # cannot beat the information content by more than the window


def test_carry_propagation_exercised():
    class Counting(Encoder):
        carries = 0

        def _shift_low(self):
            if self.low >= 1 << 56:
                Counting.carries += 1
            super()._shift_low()

    rng = np.random.default_rng(11)
    A = 16
    freq, cum = _random_tables(rng, 20000, A, 6.0)
    sym = [int(rng.choice(A, p=freq[i] / TOTAL)) for i in range(20000)]
    enc = Counting()
    for i, s in enumerate(sym):
        enc.encode(int(cum[i][s]), int(freq[i][s]), TOTAL)
    data = enc.finish()
    assert Counting.carries > 0
    assert decode_all(data, cum, TOTAL) == sym


@pytest.mark.parametrize("k", [1, 3, 6, 8])
def test_uniform_tokens_cost_2k_bits(k):
    A = 4 ** k
    u = TOTAL // A
    cum = [np.arange(A + 1, dtype=np.int64) * u] * 300
    rng = np.random.default_rng(k)
    sym = [int(x) for x in rng.integers(0, A, 300)]
    data = encode_all(sym, cum, TOTAL)
    assert decode_all(data, cum, TOTAL) == sym
    assert 300 * 2 * k - 8 <= 8 * len(data) <= 300 * 2 * k + 8


def test_exact_coder_bound_and_round_trip():
    rng = np.random.default_rng(3)
    for trial in range(20):
        n, A = int(rng.integers(1, 12)), int(rng.integers(2, 9))
        freq, cum = _random_tables(rng, n, A, 2.0)
        sym = [int(rng.integers(0, A)) for _ in range(n)]
        bits = exact_encode(sym, cum, TOTAL)
        W = Fraction(1)
        for i, s in enumerate(sym):
            W *= Fraction(int(freq[i][s]), TOTAL)
        assert len(bits) <= math.ceil(-math.log2(W)) + 1 <= _ideal_bits(sym, freq, TOTAL) + 2
        assert exact_decode(bits, cum, TOTAL) == sym
        data = encode_all(sym, cum, TOTAL)
        assert 8 * len(data) <= len(bits) + 8 + 1  # range coder within a byte of the ideal coder


def test_empty_and_single_symbol_streams():
    assert Encoder().finish() == b""
    cum = [np.array([0, 1, TOTAL])]
    for s in (0, 1):
        data = encode_all([s], cum, TOTAL)
        assert decode_all(data, cum, TOTAL) == [s]
    dec = Decoder(b"")
    assert dec.decode(np.array([0, TOTAL // 2, TOTAL]), TOTAL) == 0


def test_count_model_hand_worked():
    for line in open(os.path.join(GOLDEN, "countmodel_acac.txt")):
        if line.startswith("#") or not line.strip():
            continue
        s, m, *qs = line.split()
        probs = countmodel.sequential_probabilities(base_codes(s.encode()), int(m))
        want = [Fraction(q) for q in qs]
        assert [Fraction(f, t) for f, t in probs] == want


@pytest.mark.parametrize("m", [0, 1, 3, 6])
def test_count_model_one_lane_is_the_sequential_model(m):
    """With one lane and (s,k) = (1,1) the lane coder codes every base in order with the
    plain sequential adaptive model: its length obeys that model's bound, and it round-trips."""
    import synth
    from oracle import codec
    seq = synth.markov(4000, 2, 0.45, 17 + m).tobytes()
    cfg = codec.Config(s=1, k=1, emb_d=2, ctx_d=2, hid_d=2, lanes_per_block=1, fallback=2, count_order=m)
    out = codec.compress(seq, [len(seq)], cfg)
    assert codec.decompress(out) == seq
    ideal = sum(-math.log2(f / t) for f, t in countmodel.sequential_probabilities(base_codes(seq), m))
    payload = len(out) - 80 - len(codec.varint(len(seq))) - 1 - len(codec.varint(len(out) - 80 - 5))
    assert 8 * payload <= ideal + 8 + 1e-3
    assert 8 * payload >= ideal - 56


def test_count_model_lanes_share_one_table():
    import synth
    from oracle import codec
    seq = synth.markov(6000, 2, 0.45, 5).tobytes()
    for s_, k_, M in [(1, 1, 7), (2, 4, 16), (3, 6, 5)]:
        cfg = codec.Config(s=s_, k=k_, emb_d=2, ctx_d=2, hid_d=2, lanes_per_block=M, fallback=2, count_order=4)
        out = codec.compress(seq, [3000, 3000], cfg)
        assert codec.decompress(out) == seq


def test_count_model_halving():
    codes = np.zeros(5000, dtype=np.uint8)  # one context, counts hit the limit repeatedly
    probs = countmodel.sequential_probabilities(codes, 2)
    assert max(t for _, t in probs) <= 2 * 4 * countmodel.LIMIT + 4
    t = countmodel.Table(2, 3)  # three lanes in one context: increments land together, halving once
    for _ in range(400):
        t.finish_substep([0, 1, 2], [0, 0, 0])
        t.ctx = [0, 0, 0]
    assert t.c[0].max() < countmodel.LIMIT and t.c[0, 0] > 0


def test_count_model_totals_stay_below_2_13_with_1024_lanes():
    """With up to 1024 lanes adding to one context in a sub-step, every count read is below the
    halving limit (1024), so a total is at most 2 * 4 * 1023 + 4 = 8188 < 2^13 and no base costs
    more than 13 bits: the 2-bytes-per-base capacity of a count-model stream."""
    rng = np.random.default_rng(3)
    M = 1024
    t = countmodel.Table(1, M)
    lanes = list(range(M))
    worst = 0
    for step in range(300):
        # all lanes in one of two contexts; skewed bases so one count races ahead of the others
        t.ctx = [int(step % 2)] * M
        bases = np.where(rng.random(M) < 0.9, step % 4, rng.integers(0, 4, M))
        for r in lanes:
            f, tot = t.freqs(r)
            assert t.c[t.ctx[r]].max() < countmodel.LIMIT
            worst = max(worst, tot)
            assert -math.log2(f.min() / tot) < 13
        t.finish_substep(lanes, bases.tolist())
    assert 2 * 4 * (countmodel.LIMIT - 1) + 4 >= worst > 4 * countmodel.LIMIT  # reached the high range


def _two_lane_golden():
    """The two hand-worked multi-lane examples of tests/golden/countmodel_two_lanes.txt."""
    sections, cur = {}, None
    for line in open(os.path.join(GOLDEN, "countmodel_two_lanes.txt")):
        if line.startswith("#") or not line.strip():
            continue
        w = line.split()
        if w[0] in ("lanes", "halving"):
            cur = sections[w[0]] = {"args": w[1:], "rows": []}
        else:
            cur["rows"].append(w)
    return sections


def test_count_model_lanes_share_one_table_hand_worked():
    """Lane streams (k digits of a lane's first token, then s per later token), one table per block
    read by every lane before any lane adds, and cross-lane sharing of counts, against a two-lane
    example worked by hand (the oracle's lane coder, recording what it codes)."""
    from oracle import codec
    g = _two_lane_golden()["lanes"]
    block, s_, k_, m, M = g["args"][0], *map(int, g["args"][1:])
    cfg = codec.Config(s=s_, k=k_, emb_d=2, ctx_d=2, hid_d=2, lanes_per_block=M, fallback=2, count_order=m)
    (b,), _ = codec._prepare(cfg, [base_codes(block.encode())])
    seen = []

    class Recorder:
        def __init__(self, r):
            self.r = r

        def encode(self, cum, freq, total):
            seen.append((self.r, Fraction(freq, total), cum))

    b.count_encode, b.cenc, b.table = True, [Recorder(r) for r in range(len(b.lens))], countmodel.Table(m, len(b.lens))
    got = []
    for j in range(max(b.lens)):
        before = len(seen)
        codec._count_step(cfg, b, j)
        live = sorted({r for r, _, _ in seen[before:]})
        per_lane = {r: 0 for r in live}
        for r, q, cum in seen[before:]:
            got.append((j, per_lane[r], r, q, cum))
            per_lane[r] += 1
    want = [(int(st), int(sub), int(lane), Fraction(q)) for st, sub, lane, base, q in g["rows"]]
    assert [(j, sub, r, q) for j, sub, r, q, _ in got] == want
    # the coded base is the one worked by hand: A alone starts at cumulative frequency 0
    for (j, sub, r, q, cum), row in zip(got, g["rows"]):
        assert (row[3] == "A") == (cum == 0)


def test_count_model_halving_once_per_context_hand_worked():
    """Two lanes in one context at the halving limit: both read the old counts, the context is halved
    once after both have added (hand-worked)."""
    g = _two_lane_golden()["halving"]
    m = int(g["args"][0])
    t = countmodel.Table(m, 2)
    ctx0, counts0 = g["args"][1].split(":")
    t.c["ACGT".index(ctx0)] = [int(x) for x in counts0.split(",")]
    rows = g["rows"]
    i = 0
    while i < len(rows):
        sub = [r for r in rows[i:] if r[0] != "after"]
        sub = sub[:2]
        lanes, bases = [], []
        for sub_i, lane, ctx, base, q in sub:
            t.ctx[int(lane)] = "ACGT".index(ctx)
        for sub_i, lane, ctx, base, q in sub:
            f, tot = t.freqs(int(lane))
            assert Fraction(int(f["ACGT".index(base)]), tot) == Fraction(q), (sub_i, lane)
            lanes.append(int(lane))
            bases.append("ACGT".index(base))
        t.finish_substep(lanes, bases)
        i += len(sub)
        assert rows[i][0] == "after"
        ctx, counts = rows[i][1].split(":")
        assert t.c["ACGT".index(ctx)].tolist() == [int(x) for x in counts.split(",")]
        i += 1
