"""Pins of the oracle's container helpers against published values and hand-worked bytes: the
FNV-1a 64 hash that identifies the static model (the published test vectors of the FNV
reference), LEB128 varints (the protocol-buffers encoding example 300 -> AC 02), and the 2-bit
little-endian packing of the raw tail bases."""
import numpy as np
import pytest

from oracle import codec


@pytest.mark.parametrize("data,want", [
    (b"", 0xCBF29CE484222325),          # the offset basis
    (b"a", 0xAF63DC4C8601EC8C),
    (b"foobar", 0x85944171F73967E8),
])
def test_fnv1a64_published_vectors(data, want):
    assert codec.fnv1a64(data) == want


def test_static_hash_hashes_little_endian_float32_bytes():
    w = np.array([1.0, -2.5, 3e-8], dtype=np.float64)      # converted to float32 first
    assert codec.static_hash(w) == codec.fnv1a64(w.astype("<f4").tobytes())
    assert codec.static_hash(None) == 0
    # 1.0f is 00 00 80 3F: one changed byte changes the hash
    assert codec.static_hash(np.array([1.0], np.float32)) == codec.fnv1a64(b"\x00\x00\x80\x3f")
    assert codec.static_hash(np.array([1.0], np.float32)) != codec.static_hash(np.array([-1.0], np.float32))


@pytest.mark.parametrize("x,enc", [
    (0, b"\x00"), (1, b"\x01"), (127, b"\x7f"), (128, b"\x80\x01"), (300, b"\xac\x02"),
    (16383, b"\xff\x7f"), (16384, b"\x80\x80\x01"), ((1 << 64) - 1, b"\xff" * 9 + b"\x01"),
])
def test_varint_encoding(x, enc):
    assert codec.varint(x) == enc
    assert codec.read_varint(b"\x55" + enc + b"\x00", 1) == (x, 1 + len(enc))


@pytest.mark.parametrize("bad", [b"", b"\x80", b"\xff\xff", b"\x80" * 10 + b"\x01"])
def test_truncated_or_overlong_varint_is_corrupt(bad):
    with pytest.raises(codec.CorruptStream):
        codec.read_varint(bad, 0)


def test_tail_packing_hand_worked():
    # bases 1, 2, 3 (C, G, T) in bit pairs from the low end: 0b11_10_01 = 0x39
    assert codec.pack_tail([1, 2, 3]) == b"\x39"
    # five bases take two bytes; the fifth sits in the low bits of the second
    assert codec.pack_tail([3, 0, 0, 0, 2]) == b"\x03\x02"
    assert codec.pack_tail([]) == b""
    for n in range(0, 9):
        t = np.arange(n, dtype=np.uint8) % 4
        assert np.array_equal(codec.unpack_tail(codec.pack_tail(t), n), t)


@pytest.mark.parametrize("n,s,k,want", [(0, 2, 4, 0), (3, 2, 4, 3), (4, 2, 4, 0), (5, 2, 4, 1), (6, 2, 4, 0),
                                        (10, 3, 3, 1), (2 ** 18, 3, 6, 1)])
def test_tail_length(n, s, k, want):
    """The bases after the last token's window: n - ((l-1) s + k), all n when no token fits;
    a 2^18-base block at (s,k) = (3,6) has 87,380 tokens and one tail base."""
    assert codec.tail_len(n, s, k) == want
