"""The measured configurations' shapes on the CUDA path: exact round trips, sizes against the
oracle on scaled-down inputs, and sampled outputs of the full-size 2^24-base workload that the
oracle can compute on its own (per-block count-model payloads, tails, header fields)."""
import zlib

import numpy as np
import pytest

import synth
from oracle import codec as ocodec
from oracle.model import Shape, init_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2507_12805_gb300 as P
    return P


def _sizes_close(P, seq, lens, kw, sw, tol):
    out = P.pmklc_compress(seq, lens, P.ModelConfig(**kw, static_weights=sw))
    back, bl = P.pmklc_decompress(out, sw)
    assert back == seq and list(bl) == list(lens)
    ref = ocodec.compress(seq, lens, ocodec.Config(**{k: v for k, v in kw.items() if k != "precision"}), sw)
    assert out[:80] == ref[:80] or kw.get("precision")  # the precision byte differs in the BF16 form
    assert abs(len(out) - len(ref)) <= tol * len(ref), (len(out), len(ref))
    return out


@pytest.mark.parametrize("precision", [0, 1])
def test_human_like_k6_shape(P, precision):
    """(s,k) = (3,6): 4096-symbol alphabet, E 32, t 64, H 256 static + dynamic; two 8 KiB blocks."""
    seq = synth.human_like(1 << 14, 1003).tobytes()
    kw = dict(s=3, k=6, use_static=True, emb_s=32, ctx_s=64, hid_s=256, emb_d=32, ctx_d=64, hid_d=256,
              lanes_per_block=8, count_order=6, smp_mode=2, fallback=1, precision=precision)
    sw = init_params(Shape(4096, 32, 64, 256), 2001)
    _sizes_close(P, seq, [1 << 13, 1 << 13], kw, sw, 0.005)


def test_uneven_sequences_lane_target(P):
    """Uneven blocks with lanes proportional to length (batching workload shape, scaled)."""
    w = synth.workload("batch", scale=1 / 8192)  # a few sequences of uneven length
    kw = dict(s=3, k=6, emb_d=8, ctx_d=8, hid_d=32, lanes_per_block=16, lane_tokens=40, count_order=5,
              smp_mode=2, fallback=1)
    _sizes_close(P, w.seq.tobytes(), [int(x) for x in w.block_lens], kw, None, 0.01)


def test_large_static_model_shape(P):
    """Static predictor of the held-out workload's shape (E 32, t 128, H 512) with a smaller dynamic one."""
    seq = synth.markov(6000, 3, 0.45, 5).tobytes()
    kw = dict(s=3, k=6, use_static=True, emb_s=32, ctx_s=128, hid_s=512, emb_d=16, ctx_d=16, hid_d=64,
              lanes_per_block=4, count_order=5, smp_mode=1, fallback=1)
    sw = init_params(Shape(4096, 32, 128, 512), 7)
    for prec in (0, 1):
        cfg = P.ModelConfig(**kw, static_weights=sw, precision=prec)
        out = P.pmklc_compress(seq, [3000, 3000], cfg)
        assert P.pmklc_decompress(out, sw)[0] == seq


def test_full_size_plain_workload_sampled(P):
    """The 2^24-base workload in the bench's launch configuration (both forms): exact round trip,
    and for a sampled block everything the oracle can compute alone: its tail, and its count-model
    payload (integer arithmetic, independent of the network) byte for byte."""
    import bench
    w, kw = bench.load_workload("plain")
    sw = bench.static_weights(P, kw)
    b = 37  # sampled block: recompute its count-model lanes with the oracle alone
    off = int(np.sum(w.block_lens[:b]))
    blk = w.seq[off: off + int(w.block_lens[b])].tobytes()
    ref = ocodec.compress(blk, [len(blk)], ocodec.Config(**{**kw, "fallback": 2, "smp_mode": 0}), sw)
    ref_rec, ref_pay = _records(ref)[0]
    for prec in (1, 0):
        cfg = P.ModelConfig(**kw, static_weights=sw, precision=prec)
        out = P.pmklc_compress(w.seq, w.block_lens, cfg)
        back, bl = P.pmklc_decompress(out, sw)
        assert back == w.seq.tobytes() and list(bl) == list(w.block_lens)
        c, meta = ocodec.parse_header(out)
        assert meta["n"] == w.seq.size and meta["crc"] == zlib.crc32(w.seq.tobytes())
        rec, pay = _records(out)[b]
        if rec[1] == 1:  # count-coded in the full run: identical record and payload
            assert (rec, pay) == (ref_rec, ref_pay)
        else:
            assert rec[2] == ref_rec[2]  # the raw tail is coder-independent


def _records(data):
    """Per block: ((n, mode, tail bytes, lane lengths), payload bytes) of a container."""
    cfg, meta = ocodec.parse_header(data)
    pos, recs = 80, []
    for _ in range(meta["n_blocks"]):
        n, pos = ocodec.read_varint(data, pos)
        mode = data[pos]
        pos += 1
        nb = (ocodec.tail_len(n, cfg.s, cfg.k) * 2 + 7) // 8
        tail = data[pos:pos + nb]
        pos += nb
        sizes = []
        for _ in ocodec.lanes(ocodec.n_tokens(n, cfg.s, cfg.k), cfg.lanes_per_block, cfg.lane_tokens)[0]:
            x, pos = ocodec.read_varint(data, pos)
            sizes.append(x)
        recs.append([n, mode, tail, sizes])
    out = []
    for n, mode, tail, sizes in recs:
        out.append(((n, mode, tail, tuple(sizes)), data[pos:pos + sum(sizes)]))
        pos += sum(sizes)
    assert pos == len(data)
    return out
