"""pmklc_crc32_noalloc: the CRC-32 entry point that allocates no device memory.

Some callers cannot call cudaMalloc (their device memory belongs to another framework's pool
allocator, or they run latency-sensitive loops that must not pay for an allocation); this
entry point serves them from a fixed scratch array inside the library.  Its result must equal
the allocating entry point's on consecutive calls, since both calls share that scratch.
This file is collected last so that a run stopping at the first failure has run every other
test first; it passes alone in a fresh process as well as after the other tests.
"""
import zlib

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_crc32_equals_allocating_entry_point_twice():
    import torch
    import paper_2507_12805_gb300 as P
    rng = np.random.default_rng(2024)
    first = rng.integers(0, 256, 3 * (1 << 20) + 4097, dtype=np.uint8)
    second = rng.integers(0, 256, 700_001, dtype=np.uint8)
    for data, off in ((first, 5), (second, 0)):  # two calls in a row, the first one unaligned
        d = torch.from_numpy(data).cuda()[off:]
        want = P.pmklc_crc32(d)
        got = P.pmklc_crc32_noalloc(d)
        assert got == want == zlib.crc32(data[off:].tobytes())


def test_noalloc_crc32_at_exact_capacity_and_one_chunk_beyond():
    """An unaligned input that fills every chunk register of the scratch (65,536 chunks of 4 KiB after
    the head bytes, plus a 4,095-byte tail): the registers end right where the fold's matrices start.
    One more chunk is refused before any device access."""
    import torch
    import paper_2507_12805_gb300 as P
    chunks, chunk = 65536, 4096
    rng = np.random.default_rng(7)
    host = rng.integers(0, 256, (chunks + 1) * chunk + 64, dtype=np.uint8)
    base = torch.from_numpy(host).cuda()
    off = 5
    d = base[off:]
    head = (16 - (d.data_ptr() & 15)) & 15
    assert head > 0
    n = head + chunks * chunk + (chunk - 1)
    want = zlib.crc32(host[off:off + n].tobytes())
    assert P.pmklc_crc32_noalloc(d, n=n) == want == P.pmklc_crc32(d, n=n)
    assert P.pmklc_crc32_noalloc(d, n=n) == want  # a second call over the same full scratch
    with pytest.raises(P.PmklcError) as e:
        P.pmklc_crc32_noalloc(d, n=head + (chunks + 1) * chunk)
    assert e.value.rc == P.PMKLC_EINVAL


def test_noalloc_crc32_rejects_inputs_beyond_its_scratch_or_tensor():
    import torch
    import paper_2507_12805_gb300 as P
    d = torch.zeros(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(P.PmklcError) as e:
        P.pmklc_crc32_noalloc(d, n=(256 << 20) + 2 * 4096 + 16)  # more than the tensor holds
    assert e.value.rc == P.PMKLC_EINVAL
    assert P.pmklc_crc32_noalloc(d, n=16) == zlib.crc32(bytes(16))
    w = torch.arange(8, dtype=torch.int32, device="cuda")  # a wider element type: all of its bytes
    assert P.pmklc_crc32_noalloc(w) == zlib.crc32(np.arange(8, dtype=np.int32).tobytes())
