"""MAGNUS SpGEMM for GB300 (sm_103a): C = A * B in CSR with FP64 values.

The compute path is the CUDA library ``libmagnus.so`` built from ``csrc/``
and reached through its C ABI (``include/magnus.h``).  ``magnus`` holds the
thin ctypes binding; importing this package does not load the library, so
the seeded input generators (``inputs``) work on machines without a GPU.  Any
call into the binding raises if the library is missing: there is no CPU
fallback.
"""
__all__ = ["inputs"]
