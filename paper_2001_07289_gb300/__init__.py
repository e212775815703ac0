"""GB300-native BDDC-SO hot path (Badia, Martin, Nguyen, arXiv 2001.07289).

The CUDA library (csrc/, built into _lib/libbddc_so.so) holds every step of
the preconditioner setup, its application inside PCG, the matrix-free Q1
operator and the adjoint gradient.  `bddc` is the thin ctypes binding over
its C ABI (include/bddc_so.h); `inputs` draws the seeded synthetic problems.
Importing the package loads nothing; `paper_2001_07289_gb300.bddc` loads the
library and fails loudly when it is missing.
"""
__all__ = ["inputs", "bddc"]
