"""Python binding of libpmklc.so: PMKLC's per-block learned-compression loop on GB300.

The binding only marshals arguments (ctypes): every step of compression runs in
the library's CUDA kernels.  Device buffers are torch CUDA tensors (torch is
used for device memory and streams only).  The functions carry the names of the
C ABI in ``include/pmklc.h``; importing this package fails loudly when the
library has not been built (``python -m paper_2507_12805_gb300.build``).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field

import numpy as np

from .build import LIB as _LIB_PATH

if not os.path.exists(_LIB_PATH):
    raise ImportError(f"libpmklc.so is not built ({_LIB_PATH}); run paper_2507_12805_gb300/build.py")

lib = ctypes.CDLL(_LIB_PATH)

PMKLC_OK, PMKLC_EINVAL, PMKLC_ENOMEM, PMKLC_ECUDA = 0, -1, -2, -3
PMKLC_ECORRUPT, PMKLC_EMODEL, PMKLC_ETIMEOUT, PMKLC_ENOSPC = -4, -5, -6, -7
PMKLC_FP32_PLAIN, PMKLC_BF16_BATCHED, PMKLC_BF16_FP8STATIC, PMKLC_BF16_FP8HIDDEN = 0, 1, 2, 3
PMKLC_UPDATE_AUTO, PMKLC_UPDATE_STREAM, PMKLC_UPDATE_FUSED = 0, 1, 2
PMKLC_ADAM, PMKLC_SGD = 0, 1
PMKLC_SMP_NONE, PMKLC_SMP_CHAIN, PMKLC_SMP_TREE = 0, 1, 2


class PmklcError(RuntimeError):
    def __init__(self, rc: int, where: str):
        self.rc = rc
        super().__init__(f"{where}: {lib.pmklc_strerror(rc).decode()} ({rc})")


class CModelCfg(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("s", ctypes.c_uint32), ("k", ctypes.c_uint32),
                ("use_static", ctypes.c_uint32), ("emb_s", ctypes.c_uint32), ("ctx_s", ctypes.c_uint32),
                ("hid_s", ctypes.c_uint32), ("emb_d", ctypes.c_uint32), ("ctx_d", ctypes.c_uint32),
                ("hid_d", ctypes.c_uint32), ("lanes_per_block", ctypes.c_uint32), ("precision", ctypes.c_uint32),
                ("optimizer", ctypes.c_uint32), ("lr", ctypes.c_float), ("alpha_init", ctypes.c_float),
                ("smp_mode", ctypes.c_uint32), ("smp_fraction", ctypes.c_float), ("count_order", ctypes.c_uint32),
                ("fallback", ctypes.c_uint32), ("seed", ctypes.c_uint64),
                ("static_weights", ctypes.POINTER(ctypes.c_float)), ("lane_tokens", ctypes.c_uint32),
                ("overlap_mask", ctypes.c_uint32), ("update_path", ctypes.c_uint32),
                ("private_model", ctypes.c_uint32), ("private_epochs", ctypes.c_uint32),
                ("private_bases", ctypes.c_uint64), ("private_threshold", ctypes.c_uint64),
                ("gemm_tiles", ctypes.c_uint32), ("static_arch", ctypes.c_uint32)]


class CKernelProf(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_uint64), ("ms", ctypes.c_double),
                ("flops", ctypes.c_double), ("bytes", ctypes.c_double)]


class CStats(ctypes.Structure):
    _fields_ = [("net_blocks", ctypes.c_uint64), ("count_blocks", ctypes.c_uint64),
                ("global_steps", ctypes.c_uint64), ("kernel_launches", ctypes.c_uint64),
                ("ms_total", ctypes.c_double), ("net_bytes", ctypes.c_uint64), ("count_bytes", ctypes.c_uint64)]


_vp, _sz, _u32, _u64, _i = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
_cfgp = ctypes.POINTER(CModelCfg)
_sigs = {
    "pmklc_abi_version": ([], _i),
    "pmklc_strerror": ([_i], ctypes.c_char_p),
    "pmklc_free": ([_vp], None),
    "pmklc_model_count": ([_u32, _u32, _u32, _u32], _sz),
    "pmklc_default_cfg": ([_cfgp, _u32, _u32, _u32, _u32, _u32], None),
    "pmklc_compress": ([_vp, _sz, _vp, _sz, _cfgp, _vp, ctypes.POINTER(_vp), ctypes.POINTER(_sz)], _i),
    "pmklc_decompress": ([_vp, _sz, _vp, _sz, _vp, ctypes.POINTER(_vp), ctypes.POINTER(_sz),
                          ctypes.POINTER(_vp), ctypes.POINTER(_sz)], _i),
    "pmklc_compress_bound": ([_sz, _vp, _sz, _cfgp], _sz),
    "pmklc_compress_dev": ([_vp, _sz, _vp, _sz, _cfgp, _vp, _vp, _sz, ctypes.POINTER(_sz)], _i),
    "pmklc_decompress_dev": ([_vp, _sz, _vp, _sz, _vp, _vp, _sz, ctypes.POINTER(_sz)], _i),
    "pmklc_tokenize": ([_vp, _sz, _u32, _u32, _vp, _vp, ctypes.POINTER(_sz), _vp], _i),
    "pmklc_quantize": ([_vp, _sz, _u32, _vp, _vp], _i),
    "pmklc_mix_quantize": ([_vp, _vp, _sz, _u32, ctypes.c_float, _u32, _vp, _vp, _vp], _i),
    "pmklc_range_encode": ([_vp, _vp, _u32, _u32, _u32, _vp, _u32, _vp, _vp], _i),
    "pmklc_range_decode": ([_vp, _vp, _vp, _u32, _u32, _u32, _u32, _vp, _vp], _i),
    "pmklc_predict": ([_vp, _u32, _u32, _u32, _u32, _vp, _sz, _u32, _vp, _vp], _i),
    "pmklc_bigru_count": ([_u32, _u32, _u32, _u32], _sz),
    "pmklc_predict_bigru": ([_vp, _u32, _u32, _u32, _u32, _u32, _vp, _sz, _vp, _vp, _vp], _i),
    "pmklc_train_step": ([_cfgp, _u32, _u32, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _u32, _vp, _vp, _vp,
                          _vp], _i),
    "pmklc_quantize_static_fp8": ([_vp, _u32, _u32, _u32, _u32, _vp, _vp, _vp], _i),
    "pmklc_wait_selftest": ([_u64, _vp], _i),
    "pmklc_crc32": ([_vp, _sz, ctypes.POINTER(_u32), _vp], _i),
    "pmklc_crc32_noalloc": ([_vp, _sz, ctypes.POINTER(_u32), _vp], _i),
    "pmklc_last_stats": ([ctypes.POINTER(CStats)], _i),
    "pmklc_init_model": ([_u32, _u32, _u32, _u32, _u64, _vp], _i),
    "pmklc_train_model": ([_vp, _sz, _cfgp, _u32, _vp, _vp], _i),
    "pmklc_autotune_lanes": ([_vp, _sz, _vp, _sz, _sz, _cfgp, _vp, _sz, ctypes.c_float, _vp, _vp, _vp], _i),
    "pmklc_autotune_variant": ([_vp, _sz, _vp, _sz, _u64, _cfgp, _vp, _sz, _vp, _vp], _i),
    "pmklc_profile_enable": ([_i], _i),
    "pmklc_profile_read": ([ctypes.POINTER(CKernelProf), _i, ctypes.POINTER(_i)], _i),
}
for _name, (_args, _res) in _sigs.items():
    _f = getattr(lib, _name)
    _f.argtypes = _args
    _f.restype = _res
EXPORTED = tuple(_sigs)


def _check(rc: int, where: str):
    if rc != PMKLC_OK:
        raise PmklcError(rc, where)


@dataclass
class ModelConfig:
    """Mirror of ``pmklc_model_cfg`` (paper §4.2 predictors, §4.3 DC + SMP, §5.1.4 parameters)."""
    s: int = 3
    k: int = 3
    emb_d: int = 16
    ctx_d: int = 16
    hid_d: int = 32
    use_static: bool = False
    emb_s: int = 0
    ctx_s: int = 0
    hid_s: int = 0
    lanes_per_block: int = 64
    precision: int = PMKLC_FP32_PLAIN
    optimizer: int = PMKLC_ADAM
    lr: float = 1e-3
    alpha_init: float = 0.5
    smp_mode: int = PMKLC_SMP_TREE
    smp_fraction: float = 0.05
    count_order: int = 6
    fallback: int = 1
    seed: int = 42
    static_weights: np.ndarray | None = field(default=None, repr=False)
    lane_tokens: int = 0
    overlap_mask: int = 0    # 1: code token j >= 1 over the 4^s tokens consistent with token j - 1
    update_path: int = 0     # PMKLC_UPDATE_AUTO / _STREAM / _FUSED (same bytes either way)
    private_model: int = 0   # Model Selector: 0 static model as given, 1 SPrM, 2 SPrM above 500 MB
    private_epochs: int = 1
    private_bases: int = 0
    private_threshold: int = 0  # private_model 2: SPrM above this many bases (0 = 5e8)
    gemm_tiles: int = 0      # row GEMMs' column tiles: 0 default, 1 at most 128, 2 at most 64 (same bytes)
    static_arch: int = 0     # static predictor: 0 MLP, 1 / 2 BiGRU layers (SPrM / SPuM structure; hid_s = GRU width)

    def to_c(self) -> CModelCfg:
        c = CModelCfg()
        c.struct_size = ctypes.sizeof(CModelCfg)
        for name, _ in CModelCfg._fields_:
            if name in ("struct_size", "static_weights"):
                continue
            setattr(c, name, int(getattr(self, name)) if not isinstance(getattr(self, name), float)
                    else getattr(self, name))
        if self.use_static:
            w = np.ascontiguousarray(self.static_weights, dtype=np.float32)
            self._keep = w  # keep alive for the call
            c.static_weights = w.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
        return c


def model_count(k: int, emb: int, ctx: int, hid: int) -> int:
    return int(lib.pmklc_model_count(k, emb, ctx, hid))


def _stream(stream=None):
    if stream is not None:
        return ctypes.c_void_p(int(stream))
    try:
        import torch
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except Exception:
        pass
    return ctypes.c_void_p(0)


def _ptr(t):
    return ctypes.c_void_p(0 if t is None else int(t.data_ptr()))


def _host(a) -> np.ndarray:
    if isinstance(a, (bytes, bytearray, memoryview)):
        return np.frombuffer(bytes(a), dtype=np.uint8)
    return np.ascontiguousarray(a, dtype=np.uint8)


def pmklc_compress(seq, block_lens, cfg: ModelConfig, stream=None) -> bytes:
    """Host buffers in, container bytes out (the C-ABI call a user makes)."""
    a = _host(seq)
    bl = np.ascontiguousarray(block_lens, dtype=np.uint64)
    c = cfg.to_c()
    out, out_len = ctypes.c_void_p(), ctypes.c_size_t()
    rc = lib.pmklc_compress(a.ctypes.data_as(_vp), a.size, bl.ctypes.data_as(_vp), bl.size, ctypes.byref(c),
                            _stream(stream), ctypes.byref(out), ctypes.byref(out_len))
    _check(rc, "pmklc_compress")
    try:
        return ctypes.string_at(out, out_len.value)
    finally:
        lib.pmklc_free(out)


def pmklc_decompress(data: bytes, static_weights=None, stream=None):
    """Container bytes in, (bases, block_lens) out."""
    d = _host(data)
    w = None if static_weights is None else np.ascontiguousarray(static_weights, dtype=np.float32)
    seq, n, bl, nb = ctypes.c_void_p(), ctypes.c_size_t(), ctypes.c_void_p(), ctypes.c_size_t()
    rc = lib.pmklc_decompress(d.ctypes.data_as(_vp), d.size, None if w is None else w.ctypes.data_as(_vp),
                              0 if w is None else w.size, _stream(stream), ctypes.byref(seq), ctypes.byref(n),
                              ctypes.byref(bl), ctypes.byref(nb))
    _check(rc, "pmklc_decompress")
    try:
        out = ctypes.string_at(seq, n.value)
        lens = np.frombuffer(ctypes.string_at(bl, 8 * nb.value), dtype=np.uint64).copy()
        return out, lens
    finally:
        lib.pmklc_free(seq)
        lib.pmklc_free(bl)


def pmklc_compress_bound(n: int, block_lens, cfg: ModelConfig) -> int:
    bl = np.ascontiguousarray(block_lens, dtype=np.uint64)
    c = cfg.to_c()
    return int(lib.pmklc_compress_bound(n, bl.ctypes.data_as(_vp), bl.size, ctypes.byref(c)))


def pmklc_compress_dev(d_seq, block_lens, cfg: ModelConfig, d_out, stream=None) -> int:
    """Device tensors in/out; returns the container length written to d_out."""
    bl = np.ascontiguousarray(block_lens, dtype=np.uint64)
    c = cfg.to_c()
    out_len = ctypes.c_size_t()
    rc = lib.pmklc_compress_dev(_ptr(d_seq), d_seq.numel(), bl.ctypes.data_as(_vp), bl.size, ctypes.byref(c),
                                _stream(stream), _ptr(d_out), d_out.numel(), ctypes.byref(out_len))
    _check(rc, "pmklc_compress_dev")
    return out_len.value


def pmklc_decompress_dev(d_in, in_len: int, d_seq, static_weights=None, stream=None) -> int:
    w = None if static_weights is None else np.ascontiguousarray(static_weights, dtype=np.float32)
    n = ctypes.c_size_t()
    rc = lib.pmklc_decompress_dev(_ptr(d_in), in_len, None if w is None else w.ctypes.data_as(_vp),
                                  0 if w is None else w.size, _stream(stream), _ptr(d_seq), d_seq.numel(),
                                  ctypes.byref(n))
    _check(rc, "pmklc_decompress_dev")
    return n.value


def pmklc_tokenize(d_seq, s: int, k: int, d_tokens, d_tail, stream=None) -> int:
    n = ctypes.c_size_t()
    rc = lib.pmklc_tokenize(_ptr(d_seq), d_seq.numel(), s, k, _ptr(d_tokens), _ptr(d_tail), ctypes.byref(n),
                            _stream(stream))
    _check(rc, "pmklc_tokenize")
    return n.value


def pmklc_quantize(d_P, d_freq, stream=None):
    rows, A = d_P.shape
    _check(lib.pmklc_quantize(_ptr(d_P), rows, A, _ptr(d_freq), _stream(stream)), "pmklc_quantize")


def pmklc_mix_quantize(d_Lu, d_Lm, alpha: float, use_static: bool, d_P, d_freq, stream=None):
    rows, A = d_Lm.shape
    _check(lib.pmklc_mix_quantize(_ptr(d_Lu), _ptr(d_Lm), rows, A, alpha, int(use_static), _ptr(d_P), _ptr(d_freq),
                                  _stream(stream)), "pmklc_mix_quantize")


def pmklc_range_encode(d_freq, d_sym, n_streams: int, L: int, A: int, d_out, cap: int, d_len, stream=None):
    _check(lib.pmklc_range_encode(_ptr(d_freq), _ptr(d_sym), n_streams, L, A, _ptr(d_out), cap, _ptr(d_len),
                                  _stream(stream)), "pmklc_range_encode")


def pmklc_range_decode(d_freq, d_in, d_len, n_streams: int, L: int, A: int, cap: int, d_sym, stream=None):
    _check(lib.pmklc_range_decode(_ptr(d_freq), _ptr(d_in), _ptr(d_len), n_streams, L, A, cap, _ptr(d_sym),
                                  _stream(stream)), "pmklc_range_decode")


def pmklc_predict(d_params, k: int, E: int, t: int, H: int, d_ctx, d_logits, precision=PMKLC_FP32_PLAIN, stream=None):
    rows = d_ctx.shape[0]
    _check(lib.pmklc_predict(_ptr(d_params), k, E, t, H, _ptr(d_ctx), rows, precision, _ptr(d_logits),
                             _stream(stream)), "pmklc_predict")


def pmklc_bigru_count(k: int, E: int, Hg: int, layers: int) -> int:
    """Parameters of a BiGRU static predictor (0 for shapes the library does not build)."""
    return int(lib.pmklc_bigru_count(k, E, Hg, layers))


def pmklc_predict_bigru(d_params, k: int, E: int, t: int, Hg: int, layers: int, d_ctx, d_q=None, d_logits=None,
                        stream=None):
    """BiGRU static predictor forward: q (rows x 128) and/or logits (rows x 4^k) of the rows of d_ctx."""
    rows = d_ctx.shape[0]
    _check(lib.pmklc_predict_bigru(_ptr(d_params), k, E, t, Hg, layers, _ptr(d_ctx), rows, _ptr(d_q),
                                   _ptr(d_logits), _stream(stream)), "pmklc_predict_bigru")


def pmklc_train_step(cfg: ModelConfig, G: int, M: int, d_params, d_m, d_v, d_alpha, d_alpha_m, d_alpha_v, d_static,
                     d_ctx, d_target, tau: int, d_P=None, d_grad=None, d_dalpha=None, stream=None):
    c = cfg.to_c()
    _check(lib.pmklc_train_step(ctypes.byref(c), G, M, _ptr(d_params), _ptr(d_m), _ptr(d_v), _ptr(d_alpha),
                                _ptr(d_alpha_m), _ptr(d_alpha_v), _ptr(d_static), _ptr(d_ctx), _ptr(d_target), tau,
                                _ptr(d_P), _ptr(d_grad), _ptr(d_dalpha), _stream(stream)), "pmklc_train_step")


def pmklc_quantize_static_fp8(d_params, k: int, E: int, t: int, H: int, d_codes, d_scales, stream=None):
    """FP8 (E4M3) codes [Emb | W1t | W2 transposed] and scales [s_emb | s_w1 | s_w2] of a frozen model."""
    _check(lib.pmklc_quantize_static_fp8(_ptr(d_params), k, E, t, H, _ptr(d_codes), _ptr(d_scales),
                                         _stream(stream)), "pmklc_quantize_static_fp8")


def pmklc_wait_selftest(polls: int, stream=None) -> int:
    """Return code of the bounded-wait self-test (PMKLC_ETIMEOUT when the wait gave up)."""
    return lib.pmklc_wait_selftest(polls, _stream(stream))


def _byte_count(d_data, n, where: str) -> int:
    """The bytes to read from a contiguous device tensor: all of them, or the first n (n larger than
    the tensor is refused here, before the library could read past it)."""
    if not d_data.is_contiguous():
        raise PmklcError(PMKLC_EINVAL, where)
    nbytes = d_data.numel() * d_data.element_size()
    if n is None:
        return nbytes
    if n < 0 or n > nbytes:
        raise PmklcError(PMKLC_EINVAL, where)
    return int(n)


def pmklc_crc32(d_data, n: int | None = None, stream=None) -> int:
    crc = ctypes.c_uint32()
    _check(lib.pmklc_crc32(_ptr(d_data), _byte_count(d_data, n, "pmklc_crc32"), ctypes.byref(crc), _stream(stream)),
           "pmklc_crc32")
    return crc.value


def pmklc_crc32_noalloc(d_data, n: int | None = None, stream=None) -> int:
    """CRC-32 of device bytes without any device allocation (fixed library scratch, inputs up to 256 MiB)."""
    crc = ctypes.c_uint32()
    _check(lib.pmklc_crc32_noalloc(_ptr(d_data), _byte_count(d_data, n, "pmklc_crc32_noalloc"), ctypes.byref(crc),
                                   _stream(stream)), "pmklc_crc32_noalloc")
    return crc.value


def pmklc_last_stats() -> dict:
    st = CStats()
    _check(lib.pmklc_last_stats(ctypes.byref(st)), "pmklc_last_stats")
    return {name: getattr(st, name) for name, _ in CStats._fields_}


def pmklc_profile_enable(every: int) -> None:
    _check(lib.pmklc_profile_enable(every), "pmklc_profile_enable")


def pmklc_profile_read() -> dict:
    """Per-kernel totals over the sampled launches: {name: dict(launches, ms, flops, bytes)}."""
    buf = (CKernelProf * 64)()
    n = ctypes.c_int()
    _check(lib.pmklc_profile_read(buf, 64, ctypes.byref(n)), "pmklc_profile_read")
    return {buf[i].name.decode(): {"launches": buf[i].launches, "ms": buf[i].ms, "flops": buf[i].flops,
                                   "bytes": buf[i].bytes} for i in range(min(n.value, 64))}


def pmklc_abi_version() -> int:
    return int(lib.pmklc_abi_version())


def pmklc_autotune_lanes(d_seq, block_lens, cfg: ModelConfig, candidates, sample_blocks: int = 8,
                         max_rel_size: float = 0.005, stream=None):
    """Pick lanes per block (batch size) for `cfg` on a sample of the device input; returns
    (chosen, sizes, ms) and sets cfg.lanes_per_block."""
    bl = np.ascontiguousarray(block_lens, dtype=np.uint64)
    cand = np.ascontiguousarray(candidates, dtype=np.uint32)
    c = cfg.to_c()
    sizes = np.zeros(cand.size, dtype=np.uint64)
    ms = np.zeros(cand.size, dtype=np.float32)
    _check(lib.pmklc_autotune_lanes(_ptr(d_seq), d_seq.numel(), bl.ctypes.data_as(_vp), bl.size, sample_blocks,
                                    ctypes.byref(c), cand.ctypes.data_as(_vp), cand.size, max_rel_size,
                                    _stream(stream), sizes.ctypes.data_as(_vp), ms.ctypes.data_as(_vp)),
           "pmklc_autotune_lanes")
    cfg.lanes_per_block = int(c.lanes_per_block)
    return cfg.lanes_per_block, sizes, ms


def pmklc_train_model(seq, cfg: ModelConfig, epochs: int = 1, stream=None) -> np.ndarray:
    """Pre-train a static predictor of shape (emb_d, ctx_d, hid_d) on host bases with the library's kernels."""
    a = _host(seq)
    out = np.zeros(model_count(cfg.k, cfg.emb_d, cfg.ctx_d, cfg.hid_d), dtype=np.float32)
    c = cfg.to_c()
    _check(lib.pmklc_train_model(a.ctypes.data_as(_vp), a.size, ctypes.byref(c), epochs, _stream(stream),
                                 out.ctypes.data_as(_vp)), "pmklc_train_model")
    return out


def pmklc_init_model(k: int, E: int, t: int, H: int, seed: int) -> np.ndarray:
    """Seeded initial parameters of an MLP predictor in the library's layout (counter-based splitmix64 draws)."""
    n = model_count(k, E, t, H)
    out = np.zeros(n, dtype=np.float32)
    _check(lib.pmklc_init_model(k, E, t, H, seed, out.ctypes.data_as(_vp)), "pmklc_init_model")
    return out


def pmklc_autotune_variant(d_seq, block_lens, cfg: ModelConfig, variants, head_bases: int, stream=None):
    """Pick the fastest kernel variant (gemm_tiles | update_path << 2) for `cfg` on the heads of all
    blocks; returns (chosen code, ms) and sets cfg.gemm_tiles and cfg.update_path."""
    bl = np.ascontiguousarray(block_lens, dtype=np.uint64)
    codes = np.ascontiguousarray(variants, dtype=np.uint32)
    c = cfg.to_c()
    ms = np.zeros(codes.size, dtype=np.float32)
    _check(lib.pmklc_autotune_variant(_ptr(d_seq), d_seq.numel(), bl.ctypes.data_as(_vp), bl.size, head_bases,
                                      ctypes.byref(c), codes.ctypes.data_as(_vp), codes.size, _stream(stream),
                                      ms.ctypes.data_as(_vp)), "pmklc_autotune_variant")
    cfg.gemm_tiles, cfg.update_path = int(c.gemm_tiles), int(c.update_path)
    return cfg.gemm_tiles | (cfg.update_path << 2), ms
