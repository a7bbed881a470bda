"""GB300-native low-rank Poisson solver (Muravleva & Oseledets, arXiv:1306.2150).

The solve of Section 4.2: the factors of a low-rank right-hand side are taken to
frequency space by DST-I, the frequency-space solution is built by a cross
approximation, recompressed by QR + a small SVD (Section 3, rounding) and
transformed back.

Sub-modules:
  lr      -- ctypes binding of the C-ABI library ``liblrpoisson.so`` (CUDA, sm_103a)
  inputs  -- seeded synthetic right-hand sides (holds none of the solver's arithmetic)
  build   -- compiles the CUDA library in-tree with nvcc

Nothing is imported eagerly, so ``inputs`` can be used on machines without the
compiled library.
"""
__all__ = ["lr", "inputs", "build"]
