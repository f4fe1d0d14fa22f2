"""Plain FP64 CPU oracle of the filtered time-domain Krylov eigensolver.

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
CPU-baseline / reference arm of bench.py. The CUDA library does not use it.
"""
from .kes_oracle import *  # noqa: F401,F403
from . import spectra  # noqa: F401
