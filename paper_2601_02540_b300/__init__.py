"""B300-native split-form SBP solver for the 2D hyperbolized Serre-Green-Naghdi
equations (arXiv 2601.02540): hand-written sm_103a CUDA kernels behind a C ABI
(``libsgn.so``), with a thin ctypes binding in :mod:`.sgn`.

Importing the package loads nothing; the CUDA library is loaded on first use
and a missing library raises immediately (there is no CPU fallback).
"""

__all__ = ["inputs", "sgn"]
