"""Host-side checks of the C ABI that run before any CUDA call (no GPU): malformed container
headers are rejected with PMKLC_ECORRUPT, invalid configurations with PMKLC_EINVAL, and the
container size bound (pmklc_compress_bound, the capacity every compression allocates) covers the
costliest inputs.  The containers are written by the oracle (the same format), then damaged field
by field."""
import struct

import numpy as np
import pytest

from oracle import codec as ocodec


@pytest.fixture(scope="module")
def P():
    import paper_2507_12805_gb300 as P
    return P


@pytest.fixture(scope="module")
def container():
    seq = b"ACGTTGCAAC" * 30
    cfg = ocodec.Config(s=2, k=4, emb_d=8, ctx_d=4, hid_d=16, lanes_per_block=2, count_order=3, fallback=1)
    return ocodec.compress(seq, [len(seq)], cfg)


def _rc(P, fn):
    with pytest.raises(P.PmklcError) as e:
        fn()
    return e.value.rc


def _patched(data: bytes, offset: int, fmt: str, value) -> bytes:
    b = bytearray(data)
    struct.pack_into(fmt, b, offset, value)
    return bytes(b)


@pytest.mark.parametrize("offset,fmt,value", [
    (0, "<4s", b"PMKX"),   # magic
    (4, "<B", 2),          # version
    (5, "<B", 0),          # s = 0
    (5, "<B", 5),          # s > k
    (6, "<B", 9),          # k > 8 (and s <= k)
    (8, "<B", 4),          # precision
    (9, "<B", 2),          # optimiser
    (10, "<B", 3),         # SMP mode
    (11, "<B", 8),         # count order
    (12, "<H", 0),         # dynamic embedding width
    (24, "<I", 0),         # lanes per block
    (36, "<f", 1.5),       # SMP fraction above 1
    (28, "<f", float("inf")),  # learning rate
    (28, "<f", -1e-3),     # learning rate not positive
    (32, "<f", float("nan")),  # alpha_0
    (12, "<H", 4097),      # embedding width above the configuration limit
    (14, "<H", 65535),     # context width: t x E would overflow 32 bits
    (24, "<I", (1 << 20) + 1),  # lanes per block above the limit
    (56, "<Q", 1 << 57),   # n beyond any real input
    (56, "<Q", 299),       # n differs from the block lengths' sum
    (64, "<I", 0xFFFFFFFF),  # block count the input cannot hold
    (64, "<I", 2),         # block count: the records run out
    (64, "<I", 32768),     # more blocks (model groups) than one launch grid dimension holds
    (80, "<H", 0x7FFF),    # first block length 16383 (varint FF 7F), above n
    (72, "<I", 1 << 4),    # a variant bit no kernel choice uses
    (72, "<I", 3 << 8),    # GEMM tile variant 3 (0-2 exist)
    (72, "<I", 3 << 10),   # update path 3 (0-2 exist)
])
def test_damaged_header_fields_are_corrupt(P, container, offset, fmt, value):
    bad = _patched(container, offset, fmt, value)
    if offset == 6:
        bad = _patched(bad, 5, "<B", 1)
    assert _rc(P, lambda: P.pmklc_decompress(bad)) == P.PMKLC_ECORRUPT


def test_damaged_containers_never_crash_the_host_parser(P, container):
    """Random damage to the header and block records: the host parser answers ECORRUPT or lets
    the container through to the device stage (ECUDA without a GPU), and never aborts."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("host-parser fuzzing only: with a GPU, damaged payloads would be decoded")
    rng = np.random.default_rng(5)
    seen = set()
    for it in range(3000):
        c = bytearray(container)
        for _ in range(int(rng.integers(1, 4))):
            c[int(rng.integers(0, min(100, len(c))))] ^= int(rng.integers(1, 256))
        if it % 3 == 0:
            c = c[: int(rng.integers(0, len(c) + 1))]
        try:
            P.pmklc_decompress(bytes(c))
            rc = 0
        except P.PmklcError as e:
            rc = e.rc
        seen.add(rc)
    assert seen <= {P.PMKLC_ECORRUPT, P.PMKLC_ECUDA} and P.PMKLC_ECORRUPT in seen


@pytest.mark.parametrize("cut", [0, 1, 40, 79])
def test_short_inputs_are_corrupt(P, container, cut):
    assert _rc(P, lambda: P.pmklc_decompress(container[:cut])) == P.PMKLC_ECORRUPT


@pytest.mark.parametrize("change", [dict(s=5, k=4), dict(s=1, k=9), dict(precision=4), dict(optimizer=2),
                                    dict(smp_mode=3), dict(count_order=8), dict(fallback=3),
                                    dict(emb_d=0), dict(smp_fraction=1.5), dict(lanes_per_block=(1 << 20) + 1),
                                    dict(gemm_tiles=3), dict(update_path=3)])
def test_invalid_configurations_are_rejected(P, change):
    kw = dict(s=2, k=4, emb_d=8, ctx_d=4, hid_d=16, lanes_per_block=2)
    kw.update(change)
    cfg = P.ModelConfig(**kw)
    seq = b"ACGT" * 64
    assert _rc(P, lambda: P.pmklc_compress(seq, [len(seq)], cfg)) == P.PMKLC_EINVAL



def _de_bruijn(n: int) -> np.ndarray:
    """A de Bruijn sequence of order n over the four bases (the Fredricksen-Kessler-Maiorana
    construction: the Lyndon words whose length divides n, in lexicographic order)."""
    a = [0] * (n + 1)
    out = []

    def gen(t, p):
        if t > n:
            if n % p == 0:
                out.extend(a[1:p + 1])
        else:
            a[t] = a[t - p]
            gen(t + 1, p)
            for j in range(a[t - p] + 1, 4):
                a[t] = j
                gen(t + 1, t)

    gen(1, 1)
    return np.array(out, np.uint8)


def test_de_bruijn_helper_visits_every_window_once():
    for n in (1, 2, 3, 5):
        d = _de_bruijn(n)
        assert d.size == 4 ** n
        wins = {tuple(np.roll(d, -i)[:n]) for i in range(d.size)}
        assert len(wins) == 4 ** n


@pytest.mark.parametrize("s,k,M,m,fallback", [
    (8, 8, 4, 5, 2), (4, 4, 64, 4, 2), (2, 2, 32, 3, 2), (1, 1, 64, 2, 2),
    (4, 4, 8, 4, 1), (4, 4, 8, 4, 0),
])
def test_compress_bound_holds_for_adversarial_lanes(P, s, k, M, m, fallback):
    """M identical lanes, each an order-(m+1) de Bruijn sequence, against the order-m count
    model: every context is met four times, each time with a base it has not seen, while all
    lanes read one table -- the count model's costliest input.  The container the oracle writes
    (integer coding, the same bytes as the library's) fits the library's size bound."""
    lane = _de_bruijn(m + 1)
    seq = bytes(b"ACGT"[x] for x in lane) * M
    kw = dict(s=s, k=k, emb_d=8, ctx_d=4, hid_d=16, lanes_per_block=M, count_order=m, fallback=fallback)
    out = ocodec.compress(seq, [len(seq)], ocodec.Config(**kw))
    assert len(out) <= P.pmklc_compress_bound(len(seq), [len(seq)], P.ModelConfig(**kw))


@pytest.mark.parametrize("fallback", [0, 1, 2])
def test_compress_bound_holds_for_random_ragged_blocks(P, fallback):
    rng = np.random.default_rng(11 + fallback)
    lens = [0, 3, 5, 1000, 2047]
    seq = bytes(b"ACGT"[x] for x in rng.integers(0, 4, sum(lens)))
    kw = dict(s=2, k=4, emb_d=8, ctx_d=4, hid_d=16, lanes_per_block=3, count_order=4, fallback=fallback)
    out = ocodec.compress(seq, lens, ocodec.Config(**kw))
    assert len(out) <= P.pmklc_compress_bound(len(seq), lens, P.ModelConfig(**kw))


def test_block_count_limit(P):
    """Each block is a model group and both models' groups share one grid dimension of the GEMM
    launches (at most 65,535): more than 32,767 blocks are refused before any device work."""
    cfg = P.ModelConfig(s=2, k=4, emb_d=8, ctx_d=4, hid_d=16, lanes_per_block=2)
    assert P.pmklc_compress_bound(0, [0] * 32768, cfg) == 0
    assert P.pmklc_compress_bound(0, [0] * 32767, cfg) > 0
    assert _rc(P, lambda: P.pmklc_compress(b"", [0] * 32768, cfg)) == P.PMKLC_EINVAL


def test_layout_limits(P):
    """A call's layout is checked on the host before any allocation: at most 2^24 lanes, lanes x
    hidden width below 2^31, at most 2^27 tokens per lane and 2^30 schedule steps.  The size bound
    answers 0 (the library's refusal) past any of them; the benchmarked layout fits."""
    def bound(lens, **kw):
        base = dict(s=1, k=1, emb_d=8, ctx_d=4, hid_d=16, lanes_per_block=1)
        base.update(kw)
        return P.pmklc_compress_bound(sum(lens), lens, P.ModelConfig(**base))

    assert bound([1 << 27]) > 0                           # one lane of 2^27 tokens ((s,k) = (1,1))
    assert bound([(1 << 27) + 1]) == 0                    # one token more
    assert bound([4096] * 16384, lanes_per_block=1024) > 0          # 2^24 lanes
    assert bound([4096] * 16385, lanes_per_block=1024) == 0
    assert bound([4096] * 32, lanes_per_block=1024, hid_d=65535) > 0  # 32768 lanes x 65535 < 2^31
    assert bound([4096] * 33, lanes_per_block=1024, hid_d=65535) == 0
    # chained model passing at f = 1 runs the blocks one after another: 2^30 steps at most
    assert bound([1 << 16] * 16384, smp_mode=P.PMKLC_SMP_CHAIN, smp_fraction=1.0) > 0
    assert bound([1 << 16] * 16385, smp_mode=P.PMKLC_SMP_CHAIN, smp_fraction=1.0) == 0
    assert bound([1 << 16] * 16385, smp_mode=P.PMKLC_SMP_TREE, smp_fraction=1.0) > 0
    assert bound([1 << 18] * 64, s=2, k=4, emb_d=32, ctx_d=32, hid_d=128, lanes_per_block=64) > 0


def test_model_widths_are_bounded(P):
    assert P.model_count(4, 32, 32, 128) == 172416
    for bad in [(0, 8, 8, 8), (9, 8, 8, 8), (4, 4097, 8, 8), (4, 8, 4097, 8), (4, 8, 8, 65536), (4, 0, 8, 8),
                (4, 1 << 31, 8, 8)]:
        assert P.model_count(*bad) == 0
    with pytest.raises(P.PmklcError) as e:
        P.pmklc_init_model(4, 4097, 8, 8, 1)
    assert e.value.rc == P.PMKLC_EINVAL


def test_lane_partition_matches_oracle_through_the_size_bound(P):
    """The size bound is a closed form of each block's token count l and lane count M_b (section
    "Size bound" of the container format), so equality with the formula evaluated on the
    oracle's tokenizer and lane partition pins the library's token and lane counts, including the
    lane-length target, on random ragged layouts."""
    from oracle.tokenizer import n_tokens
    rng = np.random.default_rng(17)
    for it in range(300):
        k = int(rng.integers(1, 9))
        s = int(rng.integers(1, k + 1))
        M = int(rng.integers(1, 400))
        L = int(rng.choice([0, int(rng.integers(1, 3000))]))
        fallback = int(rng.integers(0, 3))
        lens = [int(x) for x in rng.choice([0, 1, k - 1, k, k + 1, int(rng.integers(0, 1 << 20))],
                                            int(rng.integers(1, 12)))]
        kw = dict(s=s, k=k, emb_d=8, ctx_d=4, hid_d=16, lanes_per_block=M, lane_tokens=L, fallback=fallback)
        want = 80
        for n in lens:
            l = n_tokens(n, s, k)
            Mb = len(ocodec.lanes(l, M, L)[1])
            stream = 3 * l + 8 * Mb if fallback != 2 else 2 * (k * Mb + s * (l - Mb)) + 8 * Mb
            want += 13 + 10 * Mb + stream
        assert P.pmklc_compress_bound(sum(lens), lens, P.ModelConfig(**kw)) == want, (kw, lens)


def _private_container():
    from oracle.codec import Config
    seq = (b"ACGTTGCAAC" * 40)
    cfg = Config(s=1, k=3, emb_s=8, ctx_s=4, hid_s=16, emb_d=4, ctx_d=4, hid_d=8, lanes_per_block=2,
                 count_order=3, fallback=0, private_model=1)
    return ocodec.compress(seq, [len(seq)], cfg), cfg


def test_private_model_container_parses_on_the_host(P):
    """An oracle-written container with a stored private model passes the host parser (the call
    then reaches the device stage: ECUDA without a GPU); a private flag without the static slot,
    a cut model and a flipped model bit are corrupt."""
    out, cfg = _private_container()
    assert ocodec.parse_header(out)[1]["private"]
    assert _rc(P, lambda: P.pmklc_decompress(out)) == P.PMKLC_ECUDA
    bad = bytearray(out)
    bad[7] &= ~1
    assert _rc(P, lambda: P.pmklc_decompress(bytes(bad))) == P.PMKLC_ECORRUPT
    # one block record (varint n, mode, no tail bytes, one length per lane), then the model
    p = 80 + len(ocodec.varint(400)) + 1
    for _ in ocodec.lanes(ocodec.n_tokens(400, 1, 3), 2)[1]:
        _, p = ocodec.read_varint(out, p)
    n_model = 2 * P.model_count(3, 8, 4, 16)
    flip = bytearray(out)
    flip[p + 11] ^= 0x02
    assert _rc(P, lambda: P.pmklc_decompress(bytes(flip))) == P.PMKLC_ECORRUPT
    assert _rc(P, lambda: P.pmklc_decompress(out[:p + n_model - 1])) == P.PMKLC_ECORRUPT


def test_private_model_bound_and_configuration(P):
    kw = dict(s=1, k=3, emb_d=4, ctx_d=4, hid_d=8, lanes_per_block=2, fallback=0)
    plain = P.pmklc_compress_bound(400, [400], P.ModelConfig(**kw))
    with_p = P.pmklc_compress_bound(400, [400], P.ModelConfig(**kw, private_model=1, emb_s=8, ctx_s=4, hid_s=16))
    assert with_p - plain == 2 * P.model_count(3, 8, 4, 16)
    # automatic selection: only inputs above 500 MB get the private model
    auto = P.pmklc_compress_bound(400, [400], P.ModelConfig(**kw, private_model=2, emb_s=8, ctx_s=4, hid_s=16))
    assert auto == plain
    for bad in [dict(private_model=3, emb_s=8, ctx_s=4, hid_s=16), dict(private_model=1)]:
        assert P.pmklc_compress_bound(400, [400], P.ModelConfig(**kw, **bad)) == 0


def test_bigru_static_configurations(P):
    """A BiGRU static predictor (static_arch 1 or 2) is accepted with use_static, FP32 or BF16, no
    private model and a built shape (pmklc_compress_bound, host only); anything else is refused."""
    from oracle.bigru import GruShape, init_bigru
    sw = init_bigru(GruShape(256, 16, 8, 32, 2), 1)
    ok = dict(s=2, k=4, emb_d=32, ctx_d=8, hid_d=64, lanes_per_block=4, use_static=True, emb_s=16, ctx_s=8,
              hid_s=32, static_arch=2, static_weights=sw)
    lens = [4096, 4096]
    assert P.pmklc_compress_bound(8192, lens, P.ModelConfig(**ok)) > 0
    assert P.pmklc_compress_bound(8192, lens, P.ModelConfig(**dict(ok, precision=P.PMKLC_BF16_BATCHED))) > 0
    for change in [dict(static_arch=3), dict(use_static=False), dict(private_model=1),
                   dict(precision=P.PMKLC_BF16_FP8STATIC), dict(precision=P.PMKLC_BF16_FP8HIDDEN),
                   dict(emb_s=12), dict(hid_s=24), dict(ctx_s=0)]:
        cfg = P.ModelConfig(**dict(ok, **change))
        if not cfg.use_static:
            cfg.static_weights = None
        assert P.pmklc_compress_bound(8192, lens, cfg) == 0, change


def test_bigru_container_flags_checked_by_the_host_parser(P):
    """Flag bits 4-5 carry the BiGRU's layer count: 3, bits 6-7, or a BiGRU without the static slot,
    with a private model or in an FP8 form are corrupt; an intact oracle-written container passes
    the host parser (and then needs its static weights or the device)."""
    from oracle.bigru import GruShape, init_bigru
    seq = b"ACGTTGCAAC" * 30
    cfg = ocodec.Config(s=2, k=4, emb_d=8, ctx_d=4, hid_d=16, lanes_per_block=2, count_order=3, fallback=1,
                        use_static=True, emb_s=8, ctx_s=4, hid_s=16, static_arch=1)
    good = ocodec.compress(seq, [len(seq)], cfg, init_bigru(GruShape(256, 8, 4, 16, 1), 2))
    assert good[7] == 0x13  # static, judge, one BiGRU layer
    for flags in (0x33, 0x53, 0x93, 0x12, 0x1B):
        assert _rc(P, lambda: P.pmklc_decompress(_patched(good, 7, "<B", flags))) == P.PMKLC_ECORRUPT, hex(flags)
    assert _rc(P, lambda: P.pmklc_decompress(_patched(good, 8, "<B", 2))) == P.PMKLC_ECORRUPT  # FP8 form
    assert _rc(P, lambda: P.pmklc_decompress(_patched(good, 22, "<H", 24))) == P.PMKLC_ECORRUPT  # GRU width
    assert _rc(P, lambda: P.pmklc_decompress(good)) in (P.PMKLC_ECUDA, P.PMKLC_EMODEL)
