"""CPU oracle for the interpolated pseudodifferential Helmholtz solver.

TEST INFRASTRUCTURE ONLY: imported by tests/, by __graft_entry__.smoke() and
by the CPU-baseline leg of bench.py, never by the library.  It shares no code
with the CUDA path.
"""
from .hz_oracle import *  # noqa: F401,F403
