"""Pins of the probability mixer (Eq. 1), the loss (Eq. 2) and the quantiser."""
import numpy as np
import pytest

from oracle.mixer import cross_entropy, mix, softmax
from oracle.quantize import TOTAL, cumulative, quantize, uniform_freq


def test_softmax_closed_form():
    P = softmax(np.log([[1.0, 2.0, 3.0]]))
    assert np.allclose(P, [[1 / 6, 2 / 6, 3 / 6]], atol=1e-15)
    assert np.allclose(softmax([[1000.0, 1000.0]]), [[0.5, 0.5]])


def test_mixer_special_cases():
    rng = np.random.default_rng(0)
    Lu, Lm = rng.normal(size=(3, 8)), rng.normal(size=(3, 8))
    assert np.allclose(mix(Lu, Lm, 0.0), Lm)                   # alpha = 0: dynamic model only
    assert np.allclose(mix(Lu, Lm, 1.0), Lu)                   # alpha = 1: static model only
    assert np.allclose(mix(Lu, Lm, 0.3, S=(0, 0, 1)), 0.7 * Lm)  # S0 = 0 reduces Eq. 1
    assert np.allclose(mix(Lu, Lm, 0.3, S=(1, 0, 0)), 0.3 * Lu)


def test_cross_entropy_uniform():
    A = 64
    P = np.full((5, A), 1.0 / A)
    assert np.isclose(cross_entropy(P, [0, 1, 2, 3, 63]), 5 * np.log(A))


@pytest.mark.parametrize("A", [4, 16, 64, 256, 4096])
def test_uniform_and_invariants(A):
    assert np.all(quantize(np.full((1, A), 1.0 / A)) == TOTAL // A)  # closed form
    assert np.all(uniform_freq(A) * A == TOTAL)
    rng = np.random.default_rng(A)
    for temp in [0.1, 1.0, 10.0]:
        P = softmax(rng.normal(0, temp, (20, A)))
        for dt in (np.float64, np.float32):
            f = quantize(P, dt)
            assert np.all(f.sum(axis=1) == TOTAL) and f.min() >= 1
            err = np.abs(f / TOTAL - P).max()
            assert err <= (A + 1) / TOTAL + A * 2.0 ** -24 + 1e-9
            c = cumulative(f)
            assert np.all(c[:, -1] == TOTAL) and np.all(np.diff(c, axis=1) == f)


def test_tie_rule_first_maximum():
    P = np.array([[0.25, 0.25, 0.25, 0.25 - 1e-12]])
    f = quantize(P)
    base = 1 + np.floor(P * (TOTAL - 4)).astype(np.int64)
    rem = TOTAL - base.sum()
    assert f[0, 0] == base[0, 0] + rem and np.all(f[0, 1:] == base[0, 1:])


def test_brute_force_small_alphabet():
    # all distributions on a 1/8 grid over A = 4: exact rational products, exact floors
    from fractions import Fraction
    from itertools import product
    for parts in product(range(9), repeat=3):
        if sum(parts) > 8:
            continue
        p = [Fraction(x, 8) for x in parts] + [Fraction(8 - sum(parts), 8)]
        want = [1 + (q * (TOTAL - 4)).__floor__() for q in p]
        top = max(range(4), key=lambda i: (want[i], -i))
        want[top] += TOTAL - sum(want)
        got = quantize(np.array([[float(q) for q in p]]))[0]
        assert list(got) == want
