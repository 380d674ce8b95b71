"""Pins of the oracle's static-model pre-training (oracle.codec.train_model): the returned
predictor carries the mixer's (1 - alpha) in its logits layer; a deterministic source is learned to
near zero entropy; epochs continue from each other."""
import numpy as np

from oracle import codec
from oracle.model import forward, init_params
from oracle.tokenizer import base_codes, tokenize


def _ce_bits_per_token(theta, shape, seq, s, k):
    """Cross entropy of the predictor alone (softmax of its logits) on every token with a full context."""
    tok, _ = tokenize(base_codes(seq), s, k)
    t = shape.t
    ctx = np.stack([tok[i - t:i] for i in range(t, tok.size)])
    L = forward(np.asarray(theta, dtype=np.float64), shape, ctx)[3]
    L = L - L.max(1, keepdims=True)
    lp = L - np.log(np.exp(L).sum(1, keepdims=True))
    return float(-lp[np.arange(ctx.shape[0]), tok[t:]].mean() / np.log(2))


def test_returned_logits_are_the_mixers():
    """forward(returned) = (1 - alpha) forward(final weights) for every context: the factor goes into
    W2 and b2 (the logits layer is linear in both) and nowhere else."""
    import synth
    seq = synth.markov(1200, 2, 0.45, 3).tobytes()
    cfg = codec.Config(s=1, k=2, emb_d=4, ctx_d=3, hid_d=8, lanes_per_block=4, lr=1e-2, seed=7)
    got = codec.train_model(seq, cfg, epochs=1)
    c = codec.replace(cfg, use_static=False, smp_mode=codec.SMP_CHAIN, smp_fraction=1.0, fallback=0)
    blocks, _ = codec._prepare(c, [base_codes(seq)])
    blocks[0].replay = True
    st = codec._run(c, blocks, None)[-1]
    assert abs(st.alpha - 0.5) > 1e-4  # alpha moved, so the check below is not vacuous
    rng = np.random.default_rng(0)
    ctx = rng.integers(0, 16, (50, 3))
    want = (1.0 - st.alpha) * forward(st.theta, c.dm_shape, ctx)[3]
    assert np.allclose(forward(got, c.dm_shape, ctx)[3], want, rtol=1e-12, atol=1e-12)
    lo = c.dm_shape.offsets()["w2"][0]
    assert np.array_equal(got[:lo], st.theta[:lo])


def test_deterministic_source_is_learned():
    """A period-4 sequence has entropy 0: the trained predictor alone predicts it almost surely,
    from about 2 bits per token (the uniform distribution over 4^k = 4 tokens) at its initialisation."""
    seq = b"ACGT" * 600
    cfg = codec.Config(s=1, k=1, emb_d=4, ctx_d=2, hid_d=8, lanes_per_block=4, lr=2e-2, seed=11)
    shape = cfg.dm_shape
    before = _ce_bits_per_token(init_params(shape, 11), shape, seq, 1, 1)
    after = _ce_bits_per_token(codec.train_model(seq, cfg, epochs=2), shape, seq, 1, 1)
    assert before > 1.5 and after < 0.05, (before, after)


def test_epochs_continue_from_each_other():
    import synth
    seq = synth.markov(3000, 1, 0.45, 9).tobytes()
    cfg = codec.Config(s=1, k=1, emb_d=4, ctx_d=2, hid_d=8, lanes_per_block=8, lr=1e-2, seed=5)
    one = codec.train_model(seq, cfg, epochs=1)
    two = codec.train_model(seq, cfg, epochs=2)
    assert not np.array_equal(one, two)
    shape = cfg.dm_shape
    assert _ce_bits_per_token(two, shape, seq, 1, 1) <= _ce_bits_per_token(one, shape, seq, 1, 1) + 1e-3
