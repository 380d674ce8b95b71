"""Pins of the oracle's whole method: round trip, SMP, uniform prefix, container, judge."""
import math

import numpy as np
import pytest

import synth
from oracle import codec
from oracle.codec import SMP_CHAIN, SMP_NONE, SMP_TREE, Config, CorruptStream, ModelMismatch
from oracle.model import init_params
from oracle.tokenizer import InvalidBase


def _small(**kw):
    base = dict(s=2, k=3, use_static=True, emb_s=4, ctx_s=3, hid_s=8, emb_d=4, ctx_d=4, hid_d=8,
                lanes_per_block=3, count_order=3, smp_mode=SMP_TREE, smp_fraction=0.2)
    base.update(kw)
    return Config(**base)


CASES = [
    dict(),
    dict(s=1, k=1, ctx_s=2, ctx_d=2),
    dict(s=3, k=3),
    dict(use_static=False, smp_mode=SMP_CHAIN),
    dict(smp_mode=SMP_NONE, fallback=0),
    dict(fallback=2),
    dict(optimizer=1, lr=0.05),
    dict(s=4, k=5, lanes_per_block=1),
    dict(lanes_per_block=50),
    dict(lanes_per_block=40, lane_tokens=30),
    dict(precision=2, fallback=0),
    dict(precision=3, fallback=0),
]


@pytest.mark.parametrize("kw", CASES)
def test_round_trip(kw):
    cfg = _small(**kw)
    sw = init_params(cfg.static_shape, 5) if cfg.use_static else None
    seq = synth.markov(1500, 2, 0.4, 21).tobytes()
    lens = [700, 500, 2, 0, 298]  # includes n < k and an empty block
    out = codec.compress(seq, lens, cfg, sw)
    assert codec.decompress(out, sw) == seq


def test_empty_and_tiny_inputs():
    cfg = _small()
    sw = init_params(cfg.static_shape, 5)
    for seq, lens in [(b"", []), (b"", [0]), (b"G", [1]), (b"ACGTTGCA", [8])]:
        out = codec.compress(seq, lens, cfg, sw)
        assert codec.decompress(out, sw) == seq


def test_schedule_closed_forms():
    assert codec.schedule([10] * 4, SMP_NONE, 0.05) == ([0] * 4, [-1] * 4)
    assert codec.schedule([100] * 4, SMP_CHAIN, 0.05) == ([0, 5, 10, 15], [-1, 0, 1, 2])
    start, parent = codec.schedule([100] * 8, SMP_TREE, 0.05)
    assert parent == [-1, 0, 0, 1, 0, 1, 2, 3] and start == [0, 5, 10, 10, 15, 15, 15, 15]
    # every group starts after its parent, and the tree has depth ceil(log2 G)
    start, parent = codec.schedule([40] * 64, SMP_TREE, 0.05)
    assert all(start[g] > start[parent[g]] for g in range(1, 64)) and max(start) == 6 * 2


def test_lanes_partition():
    for l in [0, 1, 5, 99, 100, 101]:
        for M in [1, 3, 100]:
            starts, lens = codec.lanes(l, M)
            assert sum(lens) == l and len(lens) == min(M, l)
            assert all(starts[i] + lens[i] == (starts[i + 1] if i + 1 < len(lens) else l) for i in range(len(lens)))
            assert (max(lens) - min(lens) <= 1) if lens else True
            for L in [1, 7, 1000]:
                starts, lens = codec.lanes(l, M, L)
                assert sum(lens) == l and len(lens) == (0 if l == 0 else min(M, l, max(1, -(-l // L))))


def test_smp_child_starts_from_parent_state():
    cfg = _small(smp_mode=SMP_CHAIN, smp_fraction=0.25, fallback=0)
    sw = init_params(cfg.static_shape, 5)
    seq = synth.markov(2000, 2, 0.4, 3).tobytes()
    snaps = {}

    def hook(kind, g, T, st):
        snaps[(kind, g, T)] = st.theta.copy()

    blocks = codec._prepare(cfg, [np.frombuffer(seq[:1000], np.uint8) % 4,
                                  np.frombuffer(seq[1000:], np.uint8) % 4])[0]
    for b in blocks:
        b.replay = True  # known tokens, no coding: only the training trajectory matters here
    codec._run(cfg, blocks, sw.astype(np.float64), on_state=hook)
    start, _ = codec.schedule([math.ceil(499 / 3), math.ceil(499 / 3)], SMP_CHAIN, float(np.float32(0.25)))
    child_start = snaps[("start", 1, start[1])]
    assert np.array_equal(child_start, snaps[("step", 0, start[1] - 1)])


def test_f_zero_smp_equals_no_smp():
    sw = init_params(_small().static_shape, 5)
    seq = synth.markov(1200, 2, 0.4, 8).tobytes()
    outs = {mode: codec.compress(seq, [400, 400, 400], _small(smp_mode=mode, smp_fraction=0.0, fallback=0), sw)
            for mode in (SMP_NONE, SMP_CHAIN, SMP_TREE)}
    strip = lambda b: b[:10] + b[11:]  # the smp-mode byte differs
    assert strip(outs[SMP_NONE]) == strip(outs[SMP_CHAIN]) == strip(outs[SMP_TREE])


def test_uniform_prefix_costs_2k_bits_per_token():
    # context longer than every lane: every token is coded with the uniform table
    cfg = _small(use_static=False, ctx_d=50, lanes_per_block=4, fallback=0)
    seq = synth.markov(402, 2, 0.4, 4).tobytes()  # (s,k)=(2,3): 200 tokens, 4 lanes of 50
    out = codec.compress(seq, [402], cfg)
    hdr = 80 + 2 + 1 + 1 + 4  # varint(402) + mode + tail byte + 4 one-byte lane lengths
    payload = len(out) - hdr
    assert abs(8 * payload - 200 * 2 * 3) <= 4 * 8
    assert codec.decompress(out) == seq


def test_header_and_errors():
    cfg = _small()
    sw = init_params(cfg.static_shape, 5)
    seq = synth.markov(600, 2, 0.4, 2).tobytes()
    out = codec.compress(seq, [600], cfg, sw)
    c2, meta = codec.parse_header(out)
    assert (c2.s, c2.k, c2.lanes_per_block, meta["n"], meta["n_blocks"]) == (2, 3, 3, 600, 1)
    assert meta["static_hash"] == codec.static_hash(sw)
    with pytest.raises(ModelMismatch):
        codec.decompress(out, init_params(cfg.static_shape, 6))
    with pytest.raises(CorruptStream):
        codec.decompress(b"XMKL" + out[4:], sw)
    with pytest.raises(CorruptStream):
        codec.decompress(out[:-3], sw)
    with pytest.raises(CorruptStream):
        codec.decompress(out[:40], sw)
    with pytest.raises(InvalidBase):
        codec.compress(b"ACGN", [4], cfg, sw)
    with pytest.raises(ValueError):
        codec.compress(seq, [599], cfg, sw)


def test_judge_picks_the_smaller_coding():
    # a periodic block is cheap for the order-6 count model and a fresh network
    # cannot match it; a short random block is not
    cfg = _small(use_static=False, count_order=6, fallback=1)
    seq = (b"ACGTTGCAAC" * 200) + synth.markov(300, 2, 0.4, 2).tobytes()
    out = codec.compress(seq, [2000, 300], cfg)
    blocks = _modes(out)
    assert blocks[0] == 1
    assert codec.decompress(out) == seq
    off = codec.compress(seq, [2000, 300], _small(use_static=False, fallback=0))
    only = codec.compress(seq, [2000, 300], _small(use_static=False, fallback=2))
    assert len(out) <= min(len(off), len(only)) + 2  # never worse than either coder alone (flag bytes aside)


def _modes(data):
    cfg, meta = codec.parse_header(data)
    pos, modes = 80, []
    for _ in range(meta["n_blocks"]):
        n, pos = codec.read_varint(data, pos)
        modes.append(data[pos])
        pos += 1 + (codec.tail_len(n, cfg.s, cfg.k) * 2 + 7) // 8
        for _ in codec.lanes(codec.n_tokens(n, cfg.s, cfg.k), cfg.lanes_per_block, cfg.lane_tokens)[0]:
            _, pos = codec.read_varint(data, pos)
    return modes


def test_online_learning_beats_uniform():
    # an order-1 source with strong structure: the dynamic model must learn it
    table = np.array([[0.85, 0.05, 0.05, 0.05], [0.05, 0.85, 0.05, 0.05],
                      [0.05, 0.05, 0.85, 0.05], [0.05, 0.05, 0.05, 0.85]])
    seq = synth.sample(6000, table, 9).tobytes()
    cfg = Config(s=1, k=1, emb_d=4, ctx_d=4, hid_d=16, lanes_per_block=1, fallback=0, lr=1e-2)
    out = codec.compress(seq, [6000], cfg)
    entropy = -(0.85 * math.log2(0.85) + 3 * 0.05 * math.log2(0.05))
    bpb = 8 * len(out) / 6000
    assert bpb < 0.5 * (2 + entropy)  # far below 2 bits/base
    assert codec.decompress(out) == seq


@pytest.mark.parametrize("smp_mode", [0, 1, 2])
def test_block_streams_equal_the_full_runs_payloads(smp_mode):
    """block_streams(g) runs only g's ancestors, each until its child starts: its lane streams equal
    block g's payloads in the whole network-only run, for every block of a 5-block input."""
    import synth
    seq = synth.markov(2600, 2, 0.45, 13).tobytes()
    lens = [700, 500, 600, 400, 400]
    kw = dict(s=2, k=3, use_static=True, emb_s=4, ctx_s=3, hid_s=8, emb_d=4, ctx_d=4, hid_d=8,
              lanes_per_block=3, smp_mode=smp_mode, smp_fraction=0.2, fallback=0, overlap_mask=1)
    sw = init_params(codec.Config(**kw).static_shape, 5)
    full = codec.compress(seq, lens, codec.Config(**kw), sw)
    cfg, meta = codec.parse_header(full)
    pos, sizes = 80, []
    for n in lens:
        n_b, pos = codec.read_varint(full, pos)
        pos += 1 + (codec.tail_len(n_b, 2, 3) * 2 + 7) // 8
        lane_sizes = []
        for _ in codec.lanes(codec.n_tokens(n_b, 2, 3), 3)[0]:
            x, pos = codec.read_varint(full, pos)
            lane_sizes.append(x)
        sizes.append(lane_sizes)
    payload = full[pos:]
    off = 0
    for g, lane_sizes in enumerate(sizes):
        want = []
        for x in lane_sizes:
            want.append(payload[off:off + x])
            off += x
        assert codec.block_streams(seq, lens, codec.Config(**kw), sw, g) == want, g
