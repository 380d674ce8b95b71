"""Host-side checks of the C ABI that run before any CUDA call (no GPU): malformed container
headers are rejected with PMKLC_ECORRUPT, invalid configurations with PMKLC_EINVAL.  The
containers are written by the oracle (the same format), then damaged field by field."""
import struct

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
    (8, "<B", 3),          # precision
    (9, "<B", 2),          # optimiser
    (10, "<B", 3),         # SMP mode
    (11, "<B", 8),         # count order
    (12, "<H", 0),         # dynamic embedding width
    (24, "<I", 0),         # lanes per block
    (36, "<f", 1.5),       # SMP fraction above 1
    (28, "<f", float("inf")),  # learning rate
])
def test_damaged_header_fields_are_corrupt(P, container, offset, fmt, value):
    bad = _patched(container, offset, fmt, value)
    if offset == 6:
        bad = _patched(bad, 5, "<B", 1)
    assert _rc(P, lambda: P.pmklc_decompress(bad)) == P.PMKLC_ECORRUPT


@pytest.mark.parametrize("cut", [0, 1, 40, 79])
def test_short_inputs_are_corrupt(P, container, cut):
    assert _rc(P, lambda: P.pmklc_decompress(container[:cut])) == P.PMKLC_ECORRUPT


@pytest.mark.parametrize("change", [dict(s=5, k=4), dict(s=1, k=9), dict(precision=3), dict(optimizer=2),
                                    dict(smp_mode=3), dict(count_order=8), dict(fallback=3),
                                    dict(emb_d=0), dict(smp_fraction=1.5), dict(lanes_per_block=(1 << 20) + 1)])
def test_invalid_configurations_are_rejected(P, change):
    kw = dict(s=2, k=4, emb_d=8, ctx_d=4, hid_d=16, lanes_per_block=2)
    kw.update(change)
    cfg = P.ModelConfig(**kw)
    seq = b"ACGT" * 64
    assert _rc(P, lambda: P.pmklc_compress(seq, [len(seq)], cfg)) == P.PMKLC_EINVAL

