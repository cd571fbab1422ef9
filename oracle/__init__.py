"""CPU oracle of Bootstrap AMG for Markov chains (FP64, numpy/scipy).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
CPU-baseline leg of bench.py, never by the product path.  It shares no code with the
CUDA library; only the input generators in `workloads` serve both.
"""
from . import bamg, exact  # noqa: F401
