"""FP64 CPU oracle of the ICM time step (arXiv:1212.6427).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
CPU legs of bench.py, never by the CUDA library, with which it shares no code.
Every function is pinned by the `-m "not gpu"` tests in tests/test_oracle_*.py.
"""
from . import icm, philox  # noqa: F401
