"""The C-ABI library loads on the CPU and exports every entry point of include/pmklc.h.

No call here touches a GPU: only host-side entry points and argument checks that
return before any CUDA call.
"""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def P():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2507_12805_gb300 as P
    return P


def _declared():
    src = open(os.path.join(ROOT, "include", "pmklc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pmklc_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(P):
    names = _declared()
    assert len(names) >= 20
    for name in names:
        assert hasattr(P.lib, name), name
    assert set(names) == set(P.EXPORTED)


def test_host_entry_points(P):
    assert P.pmklc_abi_version() == 4
    assert P.lib.pmklc_strerror(P.PMKLC_ECORRUPT) == b"corrupt compressed stream"
    # parameter count: A*E + t*E*H + H + H*A + A
    assert P.model_count(4, 32, 32, 128) == 256 * 32 + 1024 * 128 + 128 + 128 * 256 + 256 == 172416
    assert P.model_count(6, 32, 64, 256) == 1708288
    c = P.CModelCfg()
    P.lib.pmklc_default_cfg(ctypes.byref(c), 2, 4, 32, 32, 128)
    assert c.struct_size == ctypes.sizeof(P.CModelCfg) and (c.s, c.k, c.hid_d) == (2, 4, 128)


def test_init_model_matches_oracle_bit_for_bit(P):
    from oracle.model import Shape, init_params
    for (k, E, t, H, seed) in [(3, 16, 16, 32, 42), (4, 32, 32, 128, 7), (1, 3, 5, 7, 0)]:
        a = P.pmklc_init_model(k, E, t, H, seed)
        b = init_params(Shape(4 ** k, E, t, H), seed)
        assert np.array_equal(a.view(np.uint32), b.view(np.uint32))


def test_bad_config_rejected_before_any_device_work(P):
    cfg = P.ModelConfig(s=4, k=3)
    with pytest.raises(P.PmklcError) as e:
        P.pmklc_compress(b"ACGTACGT", [8], cfg)
    assert e.value.rc == P.PMKLC_EINVAL
    cfg = P.ModelConfig(s=1, k=9)
    assert P.pmklc_compress_bound(8, [8], cfg) == 0
    with pytest.raises(P.PmklcError) as e:
        P.pmklc_decompress(b"XMKL" + bytes(100))
    assert e.value.rc == P.PMKLC_ECORRUPT


def test_wait_selftest_rejects_bad_poll_counts():
    """Argument checks come before any CUDA call (no GPU needed)."""
    import paper_2507_12805_gb300 as P
    assert P.pmklc_wait_selftest(0) == P.PMKLC_EINVAL
    assert P.pmklc_wait_selftest((1 << 30) + 1) == P.PMKLC_EINVAL


def test_step_entry_points_check_sizes_before_any_cuda_call():
    """Row and stream counts past what the per-row and per-stream kernels index are refused
    before any device work (no GPU needed; the pointers are never dereferenced)."""
    import ctypes
    import paper_2507_12805_gb300 as P
    lib, fake = P.lib, ctypes.c_void_p(16)
    assert lib.pmklc_quantize(fake, (1 << 26) + 1, 4, fake, None) == P.PMKLC_EINVAL
    assert lib.pmklc_quantize(fake, 8, 5, fake, None) == P.PMKLC_EINVAL          # A not a power of 4
    assert lib.pmklc_mix_quantize(fake, fake, (1 << 26) + 1, 4, ctypes.c_float(0.5), 1, fake, fake,
                                  None) == P.PMKLC_EINVAL
    assert lib.pmklc_range_encode(fake, fake, 1 << 31, 1, 4, fake, 8, fake, None) == P.PMKLC_EINVAL
    assert lib.pmklc_range_encode(fake, fake, 1, 1 << 31, 4, fake, 8, fake, None) == P.PMKLC_EINVAL
    assert lib.pmklc_range_decode(fake, fake, fake, 1 << 31, 1, 4, 8, fake, None) == P.PMKLC_EINVAL
    assert lib.pmklc_range_decode(fake, fake, fake, 1, 1 << 31, 4, 8, fake, None) == P.PMKLC_EINVAL


def test_tokenize_and_predict_check_sizes_before_any_cuda_call():
    import ctypes
    import paper_2507_12805_gb300 as P
    lib, fake = P.lib, ctypes.c_void_p(16)
    n_tok = ctypes.c_size_t(0)
    assert lib.pmklc_tokenize(fake, (1 << 56) + 1, 2, 4, fake, fake, ctypes.byref(n_tok), None) == P.PMKLC_EINVAL
    assert lib.pmklc_tokenize(fake, 100, 5, 4, fake, fake, ctypes.byref(n_tok), None) == P.PMKLC_EINVAL  # s > k
    assert lib.pmklc_predict(fake, 4, 32, 32, 128, fake, (1 << 24) + 1, 0, fake, None) == P.PMKLC_EINVAL
    assert lib.pmklc_predict(fake, 4, 32, 32, 65535, fake, (1 << 15) + 1, 0, fake, None) == P.PMKLC_EINVAL
    assert lib.pmklc_predict(fake, 9, 32, 32, 128, fake, 8, 0, fake, None) == P.PMKLC_EINVAL


def test_header_constants_equal_the_binding_and_the_library():
    """Every value #define of include/pmklc.h has the same value in the Python binding; the ABI
    version is also what the library reports, and every error code has its own message."""
    import os
    import re
    import paper_2507_12805_gb300 as P
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    with open(os.path.join(root, "include", "pmklc.h")) as f:
        defs = dict(re.findall(r"^#define (PMKLC_[A-Z0-9_]+) \(?(-?\d+)\)?", f.read(), re.M))
    assert len(defs) >= 17
    for name, value in defs.items():
        if name == "PMKLC_ABI_VERSION":
            assert P.lib.pmklc_abi_version() == int(value)
            continue
        assert getattr(P, name) == int(value), name
    codes = [int(v) for n, v in defs.items() if n.startswith("PMKLC_E") or n == "PMKLC_OK"]
    msgs = {P.lib.pmklc_strerror(c) for c in codes}
    assert len(msgs) == len(codes)


def test_bigru_count_and_argument_checks(P):
    """The BiGRU static predictor's parameter count equals the oracle layout's; shapes outside
    those built and bad arguments are refused before any device work."""
    from oracle.bigru import GruShape
    for (k, E, Hg, layers) in [(6, 16, 32, 2), (3, 16, 32, 1), (2, 8, 16, 2), (8, 32, 16, 1)]:
        assert P.pmklc_bigru_count(k, E, Hg, layers) == GruShape(4 ** k, E, 7, Hg, layers).count
    for bad in [(6, 12, 32, 2), (6, 16, 24, 2), (6, 16, 32, 3), (0, 16, 32, 1), (9, 16, 32, 1)]:
        assert P.pmklc_bigru_count(*bad) == 0
    f = P.lib.pmklc_predict_bigru
    one = ctypes.c_void_p(16)  # never dereferenced: every call below returns before device work
    assert f(None, 3, 16, 8, 32, 2, None, 0, None, None, None) == P.PMKLC_OK  # no rows
    assert f(one, 3, 16, 0, 32, 2, one, 4, one, None, None) == P.PMKLC_EINVAL  # t = 0
    assert f(one, 3, 16, 8, 32, 2, one, 4, None, None, None) == P.PMKLC_EINVAL  # no output
    assert f(one, 3, 12, 8, 32, 2, one, 4, one, None, None) == P.PMKLC_EINVAL  # E not built
    assert f(one, 3, 16, 8, 32, 2, one, (1 << 24) + 1, one, None, None) == P.PMKLC_EINVAL  # rows
