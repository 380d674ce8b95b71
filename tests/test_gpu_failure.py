"""Failure detection without a GPU fault: every device wait of the library is bounded, and an
expired wait comes back as PMKLC_ETIMEOUT with the CUDA context still usable.  The self-test
entry point waits on an mbarrier that nothing ever arrives on (a flag nobody sets)."""
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2507_12805_gb300 as P
    return P


@pytest.mark.parametrize("polls", [1, 1000, 100000])
def test_expired_wait_reports_timeout(P, polls):
    assert P.pmklc_wait_selftest(polls) == P.PMKLC_ETIMEOUT


def test_context_survives_an_expired_wait(P):
    assert P.pmklc_wait_selftest(1000) == P.PMKLC_ETIMEOUT
    seq = synth.markov(4000, 3, 0.40, 9).tobytes()
    cfg = P.ModelConfig(s=2, k=4, emb_d=8, ctx_d=8, hid_d=64, lanes_per_block=4, precision=P.PMKLC_BF16_BATCHED)
    out = P.pmklc_compress(seq, [2000, 2000], cfg)
    back, lens = P.pmklc_decompress(out)
    assert back == seq and list(lens) == [2000, 2000]
