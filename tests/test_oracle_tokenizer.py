"""Pins of the oracle's (s,k)-mer encoder (paper §4.1, Fig. 3)."""
import itertools
import os

import numpy as np
import pytest

from oracle.tokenizer import InvalidBase, base_codes, detokenize, n_tokens, tokenize

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _brute(seq: str, s: int, k: int):
    # independent construction: Python's base-4 integer parser over each window
    digits = seq.translate(str.maketrans("ACGT", "0123"))
    toks = [int(digits[i:i + k], 4) for i in range(0, len(seq) - k + 1, s)]
    covered = (len(toks) - 1) * s + k if toks else 0
    return toks, digits[covered:]


def test_paper_worked_example():
    for line in open(os.path.join(GOLDEN, "gske_cgg.txt")):
        if line.startswith("#") or not line.strip():
            continue
        bases, s, k, *toks = line.split()
        got, tail = tokenize(base_codes(bases.encode()), int(s), int(k))
        assert list(got) == [int(x) for x in toks] and tail.size == 0


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_brute_force_all_short_strings(k):
    for n in range(0, 8):
        for tup in itertools.product("ACGT", repeat=n):
            seq = "".join(tup)
            codes = base_codes(seq.encode())
            for s in range(1, k + 1):
                toks, tail = tokenize(codes, s, k)
                bt, btail = _brute(seq, s, k)
                assert list(toks) == bt, (seq, s, k)
                assert "".join(map(str, tail)) == btail
                assert n_tokens(n, s, k) == len(bt)
                assert np.array_equal(detokenize(toks, tail, s, k), codes)


def test_long_round_trip_k8():
    rng = np.random.default_rng(5)
    codes = rng.integers(0, 4, 10_001).astype(np.uint8)
    for s, k in [(1, 8), (3, 8), (8, 8), (5, 7)]:
        toks, tail = tokenize(codes, s, k)
        assert toks.max() < 4 ** k
        assert np.array_equal(detokenize(toks, tail, s, k), codes)


def test_inconsistent_overlap_rejected():
    toks, tail = tokenize(base_codes(b"ACGTACGT"), 1, 3)
    bad = toks.copy()
    bad[2] ^= 1
    with pytest.raises(ValueError):
        detokenize(bad, tail, 1, 3)


def test_invalid_bytes_and_params():
    with pytest.raises(InvalidBase):
        base_codes(b"ACGN")
    with pytest.raises(InvalidBase):
        base_codes(b"acgt")
    with pytest.raises(ValueError):
        tokenize(base_codes(b"ACGT"), 3, 2)
    with pytest.raises(ValueError):
        tokenize(base_codes(b"ACGT"), 1, 9)
