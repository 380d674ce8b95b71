"""CPU oracle of the PMKLC per-block learned-compression loop.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code with the CUDA path (``paper_2507_12805_gb300``) and imports nothing
from it; the only module both sides use is the seeded input generator
``synth``, which holds none of the method's arithmetic.

It is a plain, slow, FP64 restatement of the method, written from the paper:

  tokenizer   (s,k)-mer encoding GskE                     paper §4.1, Fig. 3
  rng         counter-based splitmix64 initialisation      (published generator)
  model       MLP predictor forward/backward, Adam         §2 steps (3)-(4), §4.2
  bigru       BiGRU static predictor (SPuM/SPrM) forward   §4.2.2, §4.2.3
  mixer       probability mixer, softmax, cross entropy    Eq. (1), Eq. (2)
  quantize    probabilities -> integer frequency table     (paper silent; see module)
  rangecoder  byte-oriented range coder + exact rational   §2 step (3) "entropy encoder"
              arithmetic coder used only as a pin
  countmodel  adaptive order-m count model (judge/fallback)
  codec       lanes, step-wise model passing, container,   §2, §4.3, Fig. 5
              compress / decompress

Parity status of each function is stated in its module header; every function
is pinned by tests in ``tests/test_oracle_*.py`` against closed forms, the
paper's worked example, brute force or invariants.  The full-run probability
trajectory of one block's online training is pinned against an independent
float64 restatement in torch; only the CUDA path's trajectory against this one
is compared by compressed size (FP32/BF16 and FP64 diverge over a long run).
"""
