"""The seeded input generator follows the recipe the workloads state (no method arithmetic here):
ACGT bytes only, determinism per seed, target GC content, the CpG depletion rule, the repeat
coverages, the uneven length draw and the 20 % table perturbation."""
import numpy as np

import synth

C, G = ord("C"), ord("G")


def _gc(s):
    return float(np.isin(np.asarray(s), [C, G]).mean())


def test_bases_and_determinism():
    a = synth.markov(50_000, 5, 0.40, 1002)
    assert a.dtype == np.uint8 and set(np.unique(a).tolist()) <= set(b"ACGT")
    assert np.array_equal(a, synth.markov(50_000, 5, 0.40, 1002))
    assert not np.array_equal(a, synth.markov(50_000, 5, 0.40, 1003))
    h = synth.human_like(1 << 16, 1003)
    assert set(np.unique(h).tolist()) <= set(b"ACGT") and np.array_equal(h, synth.human_like(1 << 16, 1003))
    # another sample of the same species: same length, other bases
    assert not np.array_equal(h, synth.human_like(1 << 16, 1003, sample_seed=7))


def test_markov_tables_and_gc_content():
    """The GC target sets the base weights pi of p(b | ctx) ~ pi_b exp(0.5 z); the sampled GC content
    follows it within 0.015 for the order-5 and order-6 tables (4^5 and more random rows average
    out) and within 0.05 for order 3 (64 rows)."""
    for order, gc in ((3, 0.42), (5, 0.40), (6, 0.30), (6, 0.65)):
        t = synth.markov_table(order, gc, 11)
        assert t.shape == (4 ** order, 4) and np.abs(t.sum(axis=1) - 1).max() < 1e-12 and t.min() > 0
        assert abs(_gc(synth.sample(1 << 19, t, 12)) - gc) < (0.05 if order < 5 else 0.015), (order, gc)
    # the five species profiles of the batching and held-out workloads: GC 0.30 .. 0.65
    for gc, t in zip(synth.SPECIES_GC, synth.species_tables()):
        assert abs(_gc(synth.sample(1 << 18, t, 3)) - gc) < 0.015


def test_cpg_depletion_rule():
    """p(G | context ending in C) divided by 4, then the row renormalised: every other entry of
    such a row keeps its ratio to the others, and G's ratio to them drops 4x; other rows are
    unchanged."""
    t1 = synth.markov_table(6, 0.41, 1003, cpg_factor=1.0)
    t4 = synth.markov_table(6, 0.41, 1003, cpg_factor=4.0)
    ends_c = (np.arange(4 ** 6) % 4) == 1  # the newest base of the context is the low digit (C = 1)
    ratio1 = t1[ends_c, 2] / t1[ends_c, 0]
    ratio4 = t4[ends_c, 2] / t4[ends_c, 0]
    assert np.allclose(ratio4, ratio1 / 4, rtol=1e-12)
    assert np.allclose(t4[ends_c][:, [0, 1, 3]] / t4[ends_c][:, [0]], t1[ends_c][:, [0, 1, 3]] / t1[ends_c][:, [0]])
    assert np.allclose(t4[~ends_c], t1[~ends_c], rtol=1e-12)
    # and in the sampled genome CG dinucleotides are under-represented against C and G's frequencies
    s = synth.human_like(1 << 20, 1003)
    oe = ((s[:-1] == C) & (s[1:] == G)).mean() / ((s == C).mean() * (s == G).mean())
    assert oe < 0.6 and abs(_gc(s) - 0.41) < 0.02


def test_repeat_coverage():
    """Alu-like families cover about 10 % of the bases and tandem repeats about 5 %: planted into a
    run of A, 3/4 of a planted random base differs from A.  Planted repeats carry their mutation
    rate."""
    buf = np.full(1 << 20, ord("A"), np.uint8)
    synth.plant_families(buf, 30, 300, 0.10, 0.12, 5)
    assert 0.085 < (buf != ord("A")).mean() / 0.75 < 0.11
    buf = np.full(1 << 20, ord("A"), np.uint8)
    synth.plant_tandem(buf, 0.05, 2, 6, 40.0, 5)
    assert 0.04 < (buf != ord("A")).mean() / 0.75 < 0.06
    # the tiny workload's 20 copies of 200-base segments at 10 % point mutation: copied from a run of
    # A, only the mutated bases differ (a mutation picks another base): about 20 x 200 x 0.1 = 400
    buf = np.full(100_000, ord("A"), np.uint8)
    synth.plant_repeats(buf, 20, 200, 0.10, 1008)
    assert 320 < int((buf != ord("A")).sum()) < 480


def test_uneven_lengths_and_perturbation():
    # the batching workload's draw: 1 KB to 8 MB, exactly 2^30 bases (the cap holds after scaling)
    lens = synth.lognormal_lengths(2000, 12.0, 1.5, 1 << 10, 1 << 23, 1 << 30, 1004)
    assert lens.size == 2000 and int(lens.sum()) == 1 << 30
    assert lens.min() >= 1 << 10 and lens.max() <= 1 << 23 and (lens == 1 << 23).sum() >= 1
    assert np.median(lens) < np.mean(lens)  # log-normal: right-skewed
    t = synth.markov_table(6, 0.40, 3)
    p = synth.perturb_table(t, 0.2, 4)
    assert np.abs(p.sum(axis=1) - 1).max() < 1e-12
    r = p / t  # (1 + 0.2 u) / row normaliser, u in [-1, 1]
    spread = r.max(axis=1) / r.min(axis=1)
    assert spread.max() <= 1.2 / 0.8 + 1e-12 and spread.max() > 1.3


def test_even_blocks():
    assert list(synth.even_blocks(10, 4)) == [4, 4, 2]
    assert list(synth.even_blocks(8, 4)) == [4, 4]
    assert int(synth.even_blocks(1 << 28, 1 << 18).size) == 1024
