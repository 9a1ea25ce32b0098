"""GB300-native interpolated pseudodifferential Helmholtz solver.

The compute path lives in the CUDA library built from ``csrc/`` and is
reached through the thin ctypes binding in ``hz.py``.  ``synth.py`` holds the
seeded input generators.  Importing the package does not load the CUDA
library; ``paper_2409_16172_gb300.hz`` does, and raises if it is missing.
"""
__all__ = ["synth"]
