"""GB300-native structured divide-and-conquer tridiagonal eigensolver.

The compute path is the C-ABI library ``libtdc.so`` (hand-written sm_103a CUDA,
declared in ``include/tdc.h``); :mod:`.tdc` is a thin ctypes binding with the
same entry-point names.  Importing this package does not load the library;
the first call into :mod:`.tdc` does, and it raises if the library is missing.
"""

__all__ = ["tdc", "inputs"]
