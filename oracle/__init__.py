"""CPU oracle for batched multi-precision and Montgomery arithmetic (ctypes wrapper).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers. The CUDA product path never
imports this package and shares no code with it.

All arrays are instance-major ``[batch, n]`` little-endian uint32 (numpy).
Functions and the passages they follow:

* ``mul(a, b)`` / ``sqr(a)``      C = A*B, C = A^2 (Alg. 1 / Alg. 2 "Ensure")
* ``ctx(N)``                      N' = (-N)^{-1} mod R, R mod N, R^2 mod N with R = 2^(32n) (Sec. 4)
* ``mont_def(a, b, N)``           a*b*R^{-1} mod N, canonical (Alg. 3/5 "Ensure", canonical reading)
* ``modexp(a, e, ebits, N)``      a^e mod N by left-to-right square-and-multiply (Alg. 7 "Ensure")
* ``mont_model(a, b, N, red)``    the paper's reductions: red=0 truncated (Alg. 6), 1 classical (Alg. 5),
                                  3 truncated with the Karatsuba high half (Sec. 5.1; n even)
* ``montred_alg6(T, N, Np)``      one truncated reduction with its intermediates (Thm. 1, Thm. 2)
* ``montred_tkara(T, N, Np)``     the same in the truncated Karatsuba form (Sec. 5.1)
* ``modexp_alg7(a, e, ebits, N, w, red)``  fixed-window exponentiation (Alg. 7)
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_lib = None
_u32p = ctypes.POINTER(ctypes.c_uint32)


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        P, I, L = _u32p, ctypes.c_int, ctypes.c_long
        sig = {
            "or_batch_mul": [P, P, P, L, I, I],
            "or_batch_sqr": [P, P, L, I, I],
            "or_batch_ctx": [P, P, P, P, L, I, I],
            "or_batch_mont_def": [P, P, P, P, L, I, I],
            "or_batch_mont_model": [P, P, P, P, L, I, I, I],
            "or_batch_modexp": [P, P, P, I, P, L, I, I],
            "or_batch_modexp_alg7": [P, P, P, I, P, L, I, I, I, I],
            "or_montred_alg6": [P, P, P, P, P, I, P, ctypes.POINTER(ctypes.c_long)],
            "or_montred_alg5": [P, P, P, P, P, I],
            "or_montred_tkara": [P, P, P, P, P, I, P, ctypes.POINTER(ctypes.c_long)],
            "or_threads_used": [I],
            "or_mod": [P, P, I, P, I],
        }
        for name, args in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = ctypes.c_int if name not in ("or_batch_mul", "or_batch_sqr",
                                                     "or_montred_alg6", "or_montred_alg5") else None
        _lib = lib
    return _lib


def _c(x: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(x, dtype=np.uint32)


def _p(x: np.ndarray):
    return x.ctypes.data_as(_u32p)


def threads_used(nthreads: int = 0) -> int:
    return int(_load().or_threads_used(nthreads))


def mul(a, b, nthreads: int = 0) -> np.ndarray:
    a, b = _c(a), _c(b)
    B, n = a.shape
    c = np.zeros((B, 2 * n), np.uint32)
    _load().or_batch_mul(_p(c), _p(a), _p(b), B, n, nthreads)
    return c


def sqr(a, nthreads: int = 0) -> np.ndarray:
    a = _c(a)
    B, n = a.shape
    c = np.zeros((B, 2 * n), np.uint32)
    _load().or_batch_sqr(_p(c), _p(a), B, n, nthreads)
    return c


def ctx(N, nthreads: int = 0):
    """(N', R mod N, R^2 mod N) for R = 2^(32n), n = N.shape[1]."""
    N = _c(N)
    B, n = N.shape
    Np, r1, r2 = (np.zeros((B, n), np.uint32) for _ in range(3))
    if _load().or_batch_ctx(_p(Np), _p(r1), _p(r2), _p(N), B, n, nthreads):
        raise ValueError("even modulus")
    return Np, r1, r2


def mont_def(a, b, N, nthreads: int = 0) -> np.ndarray:
    a, b, N = _c(a), _c(b), _c(N)
    B, n = N.shape
    c = np.zeros((B, n), np.uint32)
    if _load().or_batch_mont_def(_p(c), _p(a), _p(b), _p(N), B, n, nthreads):
        raise ValueError("even modulus")
    return c


def mont_model(a, b, N, red: int = 0, nthreads: int = 0) -> np.ndarray:
    a, b, N = _c(a), _c(b), _c(N)
    B, n = N.shape
    c = np.zeros((B, n), np.uint32)
    if _load().or_batch_mont_model(_p(c), _p(a), _p(b), _p(N), B, n, red, nthreads):
        raise ValueError("even modulus")
    return c


def _exp_words(e, ebits):
    e = _c(e)
    ne = max(1, (ebits + 31) // 32)
    if e.shape[1] < ne:
        e = np.concatenate([e, np.zeros((e.shape[0], ne - e.shape[1]), np.uint32)], axis=1)
    return _c(e[:, :ne])


def modexp(a, e, ebits: int, N, nthreads: int = 0) -> np.ndarray:
    a, N = _c(a), _c(N)
    e = _exp_words(e, ebits)
    B, n = N.shape
    y = np.zeros((B, n), np.uint32)
    if _load().or_batch_modexp(_p(y), _p(a), _p(e), ebits, _p(N), B, n, nthreads):
        raise ValueError("zero modulus")
    return y


def modexp_alg7(a, e, ebits: int, N, w: int = 5, red: int = 0, nthreads: int = 0) -> np.ndarray:
    a, N = _c(a), _c(N)
    e = _exp_words(e, ebits)
    B, n = N.shape
    y = np.zeros((B, n), np.uint32)
    if _load().or_batch_modexp_alg7(_p(y), _p(a), _p(e), ebits, _p(N), B, n, w, red, nthreads):
        raise ValueError("even modulus or bad window")
    return y


def montred_alg6(T, N, Np):
    """One truncated reduction of a single T (2n words). Returns a dict with
    C (canonical), Cpre (n+1 words), c_add, S (64-bit), kappa, H (n+1 words), pp."""
    T, N, Np = _c(T).ravel(), _c(N).ravel(), _c(Np).ravel()
    n = N.size
    C = np.zeros(n, np.uint32)
    Cpre = np.zeros(n + 1, np.uint32)
    dbg = np.zeros(n + 5, np.uint32)
    pp = ctypes.c_long(0)
    _load().or_montred_alg6(_p(C), _p(Cpre), _p(T), _p(N), _p(Np), n, _p(dbg), ctypes.byref(pp))
    return {"C": C, "Cpre": Cpre, "c_add": int(dbg[0]),
            "S": int(dbg[1]) | (int(dbg[2]) << 32), "kappa": int(dbg[3]),
            "H": dbg[4:4 + n + 1].copy(), "pp": int(pp.value)}


def montred_tkara(T, N, Np):
    """One truncated reduction in the Karatsuba form (Sec. 5.1) of a single T (2n words,
    n even). Returns a dict with C (canonical), Cpre (n+1 words), c_add, e (the signed
    error of the column-(n-1) estimate), H (n+1 words) and pp."""
    T, N, Np = _c(T).ravel(), _c(N).ravel(), _c(Np).ravel()
    n = N.size
    C = np.zeros(n, np.uint32)
    Cpre = np.zeros(n + 1, np.uint32)
    dbg = np.zeros(n + 3, np.uint32)
    pp = ctypes.c_long(0)
    rc = _load().or_montred_tkara(_p(C), _p(Cpre), _p(T), _p(N), _p(Np), n, _p(dbg), ctypes.byref(pp))
    if rc:
        raise ValueError("odd n" if rc == -1 else "estimate outside the recoverable range")
    e = int(dbg[1])
    return {"C": C, "Cpre": Cpre, "c_add": int(dbg[0]), "e": e - (1 << 32) if e >= 1 << 31 else e,
            "H": dbg[2:2 + n + 1].copy(), "pp": int(pp.value)}


def montred_alg5(T, N, Np):
    T, N, Np = _c(T).ravel(), _c(N).ravel(), _c(Np).ravel()
    n = N.size
    C = np.zeros(n, np.uint32)
    Cpre = np.zeros(n + 1, np.uint32)
    _load().or_montred_alg5(_p(C), _p(Cpre), _p(T), _p(N), _p(Np), n)
    return {"C": C, "Cpre": Cpre}


def mod(u, v) -> np.ndarray:
    """u mod v for single values given as 1-D word arrays (Algorithm D)."""
    u, v = _c(u).ravel(), _c(v).ravel()
    r = np.zeros(v.size, np.uint32)
    if _load().or_mod(_p(r), _p(u), u.size, _p(v), v.size):
        raise ZeroDivisionError
    return r
