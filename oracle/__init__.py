"""CPU oracle for the encrypted CSR matrix-factorisation path — TEST INFRASTRUCTURE.

Plain, slow, obviously-correct reference code: exact u128 ring arithmetic in C
(ring.c), the RNS-CKKS scheme in coefficient form (ckks.py) and the plaintext
and encrypted MF epochs (mf.py). Only tests/, ``__graft_entry__.smoke()`` and the
benchmark's ``cpu_baseline`` / ``--impl reference`` legs may import, link or run
anything in this package. It shares no code with the CUDA library.
"""
from . import ring  # noqa: F401
