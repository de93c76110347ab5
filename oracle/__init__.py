"""Exact CPU oracle for the RNS-CKKS statistics path.

TEST INFRASTRUCTURE ONLY: this package is what the GPU library is checked
against. Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg
may import it; the product library never does, and the two share no code.

* ckks_oracle.c -- exact per-limb primitives (__int128 modular arithmetic,
  negacyclic transform, base conversion, ChaCha20 samplers);
* ckks.py       -- parameters, keys, encryption, evaluator ops;
* stats.py      -- Chebyshev / Newton inverse square root and the five
  statistics, on the exact evaluator or a noise-free FP64 simulation.
"""
from ._clib import build  # noqa: F401
