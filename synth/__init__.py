"""Seeded synthetic genomes shaped like the paper's workloads.

The paper evaluates on real genomic datasets (Table 2) that are not available;
these seeded generators stand in for them.  The module holds no compressor
arithmetic: it only produces ASCII ``ACGT`` byte arrays and block partitions,
which both the CUDA path (tests, benchmark) and the CPU oracle consume.

The sampling core is plain C (``synth.c``), compiled on first use with gcc.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "_synth.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C sampler into ``synth/_synth.so`` (idempotent)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u64, i32, dbl = ctypes.c_uint64, ctypes.c_int, ctypes.c_double
            vp = ctypes.c_void_p
            lib.synth_markov_table.argtypes = [vp, i32, dbl, dbl, dbl, u64]
            lib.synth_perturb_table.argtypes = [vp, i32, dbl, u64]
            lib.synth_markov_sample.argtypes = [vp, u64, i32, vp, u64]
            lib.synth_markov_sample.restype = i32
            lib.synth_plant_repeats.argtypes = [vp, u64, i32, u64, dbl, u64]
            lib.synth_plant_families.argtypes = [vp, u64, i32, u64, dbl, dbl, u64, u64]
            lib.synth_plant_families.restype = i32
            lib.synth_plant_tandem.argtypes = [vp, u64, dbl, i32, i32, dbl, u64]
            lib.synth_lognormal_lengths.argtypes = [vp, i32, dbl, dbl, u64, u64, u64, u64]
            lib.synth_lognormal_lengths.restype = i32
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def markov_table(order: int, gc: float, seed: int, cpg_factor: float = 1.0, z_scale: float = 0.5) -> np.ndarray:
    """p(b | previous `order` bases) as a [4**order, 4] float64 table."""
    t = np.zeros((4 ** order, 4), dtype=np.float64)
    _load().synth_markov_table(_ptr(t), order, gc, cpg_factor, z_scale, seed)
    return t


def perturb_table(table: np.ndarray, amount: float, seed: int) -> np.ndarray:
    order = int(round(np.log(table.shape[0]) / np.log(4)))
    t = np.ascontiguousarray(table, dtype=np.float64).copy()
    _load().synth_perturb_table(_ptr(t), order, amount, seed)
    return t


def sample(n: int, table: np.ndarray, seed: int) -> np.ndarray:
    order = int(round(np.log(table.shape[0]) / np.log(4)))
    out = np.empty(n, dtype=np.uint8)
    t = np.ascontiguousarray(table, dtype=np.float64)
    if n and _load().synth_markov_sample(_ptr(out), n, order, _ptr(t), seed) != 0:
        raise MemoryError("synth_markov_sample")
    return out


def markov(n: int, order: int, gc: float, seed: int, cpg_factor: float = 1.0) -> np.ndarray:
    return sample(n, markov_table(order, gc, seed, cpg_factor), seed + 0x5151)


def plant_repeats(buf: np.ndarray, count: int, length: int, mu: float, seed: int) -> np.ndarray:
    _load().synth_plant_repeats(_ptr(buf), buf.size, count, length, mu, seed)
    return buf


def plant_families(buf: np.ndarray, n_fam: int, fam_len: int, coverage: float, mu: float, seed: int,
                   place_seed: int | None = None):
    """Copies of n_fam consensus sequences (drawn from `seed`) at `mu` point mutation until `coverage`
    of buf is covered; their places and mutations come from `place_seed` (default: the same stream)."""
    ps = seed if place_seed is None else place_seed
    if _load().synth_plant_families(_ptr(buf), buf.size, n_fam, fam_len, coverage, mu, seed, ps) != 0:
        raise MemoryError("synth_plant_families")
    return buf


def plant_tandem(buf: np.ndarray, coverage: float, pmin: int, pmax: int, mean_run: float, seed: int):
    _load().synth_plant_tandem(_ptr(buf), buf.size, coverage, pmin, pmax, mean_run, seed)
    return buf


def lognormal_lengths(count: int, mu: float, sigma: float, lo: int, hi: int, total: int, seed: int):
    lens = np.zeros(count, dtype=np.uint64)
    if _load().synth_lognormal_lengths(_ptr(lens), count, mu, sigma, lo, hi, total, seed) != 0:
        raise MemoryError("synth_lognormal_lengths")
    return lens


def even_blocks(n: int, block: int) -> np.ndarray:
    """Data Chunker: an even partition of n bases into blocks of `block` bases (last one shorter)."""
    nb = max(1, -(-n // block))
    lens = np.full(nb, block, dtype=np.uint64)
    lens[-1] = n - block * (nb - 1)
    return lens


@dataclass
class Workload:
    name: str
    seq: np.ndarray          # uint8 ASCII ACGT
    block_lens: np.ndarray   # uint64, sums to seq.size
    s: int
    k: int
    recipe: str


def human_like(n: int, seed: int, sample_seed: int | None = None) -> np.ndarray:
    """GC 0.41, CpG depleted 4x, order-6 background; 10% of bases from 30 Alu-like 300-bp
    families at 12% mutation; 5% tandem repeats with periods 2-6 (mean run 40 bp).

    `seed` fixes the "species" (the order-6 table and the family consensus sequences) and, by
    default, the sample; another `sample_seed` draws another genome of the same species (its own
    background sample, family copies and tandem repeats), e.g. the public data a static model is
    pre-trained on."""
    ss = seed if sample_seed is None else sample_seed
    seq = sample(n, markov_table(6, 0.41, seed, cpg_factor=4.0), ss + 1)
    plant_families(seq, 30, 300, 0.10, 0.12, seed + 2, ss + 2)
    plant_tandem(seq, 0.05, 2, 6, 40.0, ss + 3)
    return seq


SPECIES_GC = (0.30, 0.3875, 0.475, 0.5625, 0.65)


def species_tables(seed: int = 2001):
    return [markov_table(6, gc, seed + 17 * i) for i, gc in enumerate(SPECIES_GC)]


def pretrain_corpus(name: str, n: int, seed: int = 2001) -> np.ndarray:
    """n bases of other genomes from the same source as a workload (its "species"), drawn with their
    own sample seed: the public data a static model is pre-trained on.  plain: the order-5 table of
    seed 1002; human: the human-like species of seed 1003 (its table and repeat families); batch /
    heldout: the five species profiles in turn (unperturbed)."""
    if name == "plain":
        return sample(n, markov_table(5, 0.40, 1002), seed)
    if name == "human":
        return human_like(n, 1003, sample_seed=seed)
    if name in ("batch", "heldout"):
        tabs = species_tables()
        part = -(-n // 5)
        return np.concatenate([sample(min(part, n - i * part), tabs[i], seed + i) for i in range(5)])
    if name == "tiny":
        return sample(n, markov_table(3, 0.42, 1001), seed)
    raise KeyError(name)


def workload(name: str, scale: float = 1.0) -> Workload:
    """The measured configurations.  `scale` < 1 shrinks the input (same recipe) for tests.

    tiny   : 100,000 bases, order-3 Markov (GC 0.42) + 20 planted 200-bp repeats at 10%
             mutation; one block; (s,k) = (1,3).                         seed 1001
    plain  : 2**24 bases, order-5 Markov (GC 0.40); 64 blocks of 2**18; (s,k) = (2,4).  seed 1002
    human  : 2**28 bases human-like (see human_like); 1024 blocks of 2**18; (3,6).     seed 1003
    batch  : 2,000 sequences, ln L ~ N(12, 1.5) clipped to [2**10, 2**23], 2**30 total,
             5 species profiles (order 6, GC 0.30-0.65), one block per sequence; (3,6).  seed 1004
    heldout: 2**30 bases from the species profiles with tables perturbed 20%,
             4096 blocks of 2**18; (3,6).                                    seed 1005
    """
    if name == "tiny":
        n = max(64, int(100_000 * scale))
        seq = markov(n, 3, 0.42, 1001)
        plant_repeats(seq, 20, min(200, n // 4), 0.10, 1001 + 7)
        return Workload(name, seq, np.array([n], dtype=np.uint64), 1, 3,
                        "order-3 Markov GC 0.42 + 20x200bp repeats mu=0.10")
    if name == "plain":
        n = max(1 << 10, int((1 << 24) * scale))
        seq = markov(n, 5, 0.40, 1002)
        return Workload(name, seq, even_blocks(n, 1 << 18 if scale >= 1 else max(1 << 10, int((1 << 18) * scale))),
                        2, 4, "order-5 Markov GC 0.40, 256 KB blocks")
    if name == "human":
        n = max(1 << 12, int((1 << 28) * scale))
        return Workload(name, human_like(n, 1003), even_blocks(n, 1 << 18), 3, 6,
                        "human-like GC 0.41 CpG/4, 10% Alu-like, 5% tandem, 256 KB blocks")
    if name == "batch":
        total = max(1 << 16, int((1 << 30) * scale))
        count = 2000 if scale >= 1 else max(4, int(2000 * scale))
        lens = lognormal_lengths(count, 12.0, 1.5, 1 << 10, 1 << 23, total, 1004)
        tabs = species_tables()
        parts = [sample(int(L), tabs[i % 5], 1004_000 + i) for i, L in enumerate(lens)]
        return Workload(name, np.concatenate(parts), lens, 3, 6, "5 species, log-normal lengths")
    if name == "heldout":
        n = max(1 << 16, int((1 << 30) * scale))
        tabs = [perturb_table(t, 0.2, 1005 + i) for i, t in enumerate(species_tables())]
        blocks = even_blocks(n, 1 << 18)
        parts = [sample(int(L), tabs[i % 5], 1005_000 + i) for i, L in enumerate(blocks)]
        return Workload(name, np.concatenate(parts), blocks, 3, 6, "perturbed species profiles")
    raise KeyError(name)
