"""GB300-native SISPH hot path (arXiv 1908.01762): C-ABI library + thin binding.

The compute lives in ``libsisph.so`` (hand-written CUDA for sm_103a, declared
in ``include/sisph.h``).  ``paper_1908_01762_gb300.sisph`` is the ctypes
binding with the same function names; importing this package does not load
the library, the first call does, and it raises if the library is missing.
"""
from .buildlib import build  # noqa: F401

__all__ = ["build", "sisph"]
