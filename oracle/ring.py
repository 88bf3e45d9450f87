"""ctypes wrapper over the oracle's plain-C ring arithmetic (oracle/ring.c).

TEST INFRASTRUCTURE ONLY: tests/, the smoke check and the benchmark's
CPU-baseline leg may use this; the product path never does.

The shared object is compiled from ring.c with gcc on first use (or by
``build()``), into ``oracle/_oracle_ring.so``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ring.c")
_SO = os.path.join(_HERE, "_oracle_ring.so")
_lock = threading.Lock()
_lib = None

_u64p = ctypes.POINTER(ctypes.c_uint64)


def build(force: bool = False) -> str:
    """Compile ring.c into a shared object (plain -O2; no vector intrinsics)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_SO)
            u64 = ctypes.c_uint64
            for name in ("or_addmod", "or_submod", "or_mulmod", "or_powmod"):
                f = getattr(L, name)
                f.argtypes = [u64, u64, u64]
                f.restype = u64
            L.or_invmod.argtypes = [u64, u64]
            L.or_invmod.restype = u64
            L.or_is_prime.argtypes = [u64]
            L.or_is_prime.restype = ctypes.c_int
            L.or_find_psi.argtypes = [ctypes.c_int, u64]
            L.or_find_psi.restype = u64
            L.or_negacyclic_schoolbook.argtypes = [_u64p, _u64p, _u64p, ctypes.c_int, u64]
            L.or_negacyclic_dot.argtypes = [_u64p, _u64p, ctypes.c_int, _u64p, ctypes.c_int, u64]
            L.or_negacyclic_dot.restype = ctypes.c_int
            L.or_negacyclic_dot_rows.argtypes = [_u64p, _u64p, ctypes.c_int, ctypes.c_int, _u64p,
                                                 ctypes.c_int, _u64p]
            L.or_negacyclic_dot_rows.restype = ctypes.c_int
            L.or_scalar_mul.argtypes = [_u64p, u64, _u64p, ctypes.c_int, u64]
            L.or_automorphism.argtypes = [_u64p, _u64p, ctypes.c_int, u64, u64]
            L.or_fast_base_conv.argtypes = [_u64p, _u64p, ctypes.c_int, _u64p, _u64p, ctypes.c_int,
                                            ctypes.c_int]
            L.or_rescale.argtypes = [_u64p, _u64p, ctypes.c_int, _u64p, ctypes.c_int]
            _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.uint64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_u64p)


def _c(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.uint64)


def is_prime(n: int) -> bool:
    return bool(lib().or_is_prime(n))


def mulmod(a: int, b: int, q: int) -> int:
    return int(lib().or_mulmod(a, b, q))


def powmod(a: int, e: int, q: int) -> int:
    return int(lib().or_powmod(a, e, q))


def find_psi(n: int, q: int) -> int:
    return int(lib().or_find_psi(n, q))


def schoolbook(a, b, q: int) -> np.ndarray:
    a, b = _c(a), _c(b)
    out = np.zeros_like(a)
    lib().or_negacyclic_schoolbook(_p(a), _p(b), _p(out), a.shape[-1], q)
    return out


def polymul(a, b, q: int) -> np.ndarray:
    """Product in Z_q[X]/(X^N+1) of two coefficient vectors."""
    return polydot(np.asarray(a)[None], np.asarray(b)[None], q)


def polydot(A, B, q: int) -> np.ndarray:
    """sum_t A[t] * B[t] in Z_q[X]/(X^N+1); A, B: [count, N]."""
    A, B = _c(A), _c(B)
    assert A.shape == B.shape and A.ndim == 2
    out = np.zeros(A.shape[1], dtype=np.uint64)
    rc = lib().or_negacyclic_dot(_p(A), _p(B), A.shape[0], _p(out), A.shape[1], q)
    if rc:
        raise RuntimeError(f"or_negacyclic_dot failed ({rc})")
    return out


def polydot_rows(A, B, primes) -> np.ndarray:
    """Row r: sum_t A[r, t] * B[r, t] mod primes[r]; A, B: [rows, count, N]."""
    A, B = _c(A), _c(B)
    pr = _c(primes)
    rows, count, n = A.shape
    out = np.zeros((rows, n), dtype=np.uint64)
    rc = lib().or_negacyclic_dot_rows(_p(A), _p(B), rows, count, _p(out), n, _p(pr))
    if rc:
        raise RuntimeError(f"or_negacyclic_dot_rows failed ({rc})")
    return out


def scalar_mul(a, s: int, q: int) -> np.ndarray:
    a = _c(a)
    out = np.zeros_like(a)
    lib().or_scalar_mul(_p(a), s % q, _p(out), a.shape[-1], q)
    return out


def automorphism(a, g: int, q: int) -> np.ndarray:
    a = _c(a)
    out = np.zeros_like(a)
    lib().or_automorphism(_p(a), _p(out), a.shape[-1], g, q)
    return out


def fast_base_conv(x, src, dst) -> np.ndarray:
    """x: [len(src), N] residues -> [len(dst), N] residues of x + u*prod(src)."""
    x = _c(x)
    s, d = _c(src), _c(dst)
    out = np.zeros((len(dst), x.shape[1]), dtype=np.uint64)
    lib().or_fast_base_conv(_p(x), _p(s), len(src), _p(out), _p(d), len(dst), x.shape[1])
    return out


def rescale(x, primes) -> np.ndarray:
    """x: [l+1, N] residues modulo primes[0..l] -> [l, N], exact round(x / q_l)."""
    x = _c(x)
    pr = _c(primes)
    l = len(primes) - 1
    out = np.zeros((l, x.shape[1]), dtype=np.uint64)
    lib().or_rescale(_p(x), _p(pr), l, _p(out), x.shape[1])
    return out
