"""GB300-native FP64 finite-difference + RK4 hot path of the Chemora method
(arXiv 1410.1764).

The compute path is the CUDA library libchemora.so (C ABI declared in
include/chemora.h); this package is a thin ctypes binding over it.  Importing
the package does not load the library; the first call that needs it does, and
raises if it is missing.
"""
__all__ = ["api", "synth"]
