"""GB300-native RNS-CKKS encrypted CSR matrix factorisation.

The compute path lives in the CUDA library built from ``csrc/``; ``capi`` is a
thin ctypes binding over its C ABI (declared in ``include/ckks_mf.h``).
Importing this package does not load the library; ``capi.lib()`` does, and it
raises if the library has not been built.
"""
