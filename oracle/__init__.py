"""CPU oracle of the robust LOBPCG hot path -- TEST INFRASTRUCTURE ONLY.

Plain FP64 numpy code written from the paper (Duersch, Shao, Yang, Gu, 2018).
Only tests/, the smoke check in __graft_entry__ and bench.py's CPU-baseline
leg may import it.  The CUDA library (paper_1704_07458_gb300) never imports or
links it; the two share no code.  Inputs come from the seeded generators in
synth/, which hold none of the method's arithmetic.
"""
from . import dense, lobpcg, kernels  # noqa: F401
