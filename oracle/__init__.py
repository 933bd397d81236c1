"""FP64 CPU oracle of the damped-gradient Skyrme-DFT iteration.

TEST INFRASTRUCTURE: only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it.  It shares no code with the CUDA
path.  Parity of every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, invariants, brute force and library special cases.
"""
from .sky_oracle import *  # noqa: F401,F403
