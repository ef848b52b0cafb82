"""B300-native CVD memory operations (software hybrid address space).

``paper_1304_3771_b300.cvd`` is the ctypes binding of ``libcvd.so`` (the
C-ABI declared in ``include/cvd.h``); ``paper_1304_3771_b300.workload`` holds
the seeded input generators.  Nothing is imported eagerly so that the input
generators can be used without loading the CUDA library.
"""
__all__ = ["cvd", "workload"]
