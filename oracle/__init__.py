"""FP64 CPU oracle for the FDAS overlap-save power plane (ctypes over plain C).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py``.  The library's product path never imports
it.  It shares no code with the CUDA path; inputs come from the seeded
generators in ``synth``.

Functions (each restates the paper, see ``fdas_oracle.c``):
  direct_conv   Eq. (1), complex output          direct_power   Eq. (1) + |y|^2
  direct_points Eq. (1) + |y|^2 at chosen points fft            unnormalised radix-2 DFT
  ols_power     Algorithm 2 (overlap-save) + |y|^2
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fdas_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP) into ``oracle/_build/liboracle.so``."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i64 = ctypes.c_int64
            ci = ctypes.c_int
            lib.oracle_set_threads.argtypes = [ci]
            lib.oracle_threads.restype = ci
            lib.oracle_direct_conv.argtypes = [P, i64, P, ci, ci, P]
            lib.oracle_power.argtypes = [P, i64, P]
            lib.oracle_direct_power.argtypes = [P, i64, P, ci, ci, P]
            lib.oracle_direct_points.argtypes = [P, i64, P, ci, ci, P, P, i64, P]
            lib.oracle_fft.argtypes = [P, ci, ci]
            lib.oracle_fft.restype = ci
            lib.oracle_ols_power.argtypes = [P, i64, P, ci, ci, ci, ci, P]
            lib.oracle_ols_power.restype = ci
            _lib = lib
    return _lib


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a), dtype=np.complex128)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def set_threads(n: int) -> None:
    _load().oracle_set_threads(int(n))


def threads() -> int:
    return int(_load().oracle_threads())


def direct_conv(x, h) -> np.ndarray:
    """Eq. (1) for every template row of ``h`` ([m, K]): complex128 [m, n]."""
    x, h = _c128(x), _c128(np.atleast_2d(h))
    m, k = h.shape
    y = np.empty((m, x.size), dtype=np.complex128)
    _load().oracle_direct_conv(_ptr(x), x.size, _ptr(h), m, k, _ptr(y))
    return y


def power(y) -> np.ndarray:
    """|y|^2 of complex values, float64, same shape."""
    y = _c128(y)
    p = np.empty(y.shape, dtype=np.float64)
    _load().oracle_power(_ptr(y), y.size, _ptr(p))
    return p


def direct_power(x, h) -> np.ndarray:
    """Eq. (1) followed by |y|^2: float64 [m, n]."""
    x, h = _c128(x), _c128(np.atleast_2d(h))
    m, k = h.shape
    p = np.empty((m, x.size), dtype=np.float64)
    _load().oracle_direct_power(_ptr(x), x.size, _ptr(h), m, k, _ptr(p))
    return p


def direct_points(x, h, zi, ii) -> np.ndarray:
    """|y_z[i]|^2 of Eq. (1) at the points (zi[j], ii[j]): float64 [len(zi)]."""
    x, h = _c128(x), _c128(np.atleast_2d(h))
    m, k = h.shape
    zi = np.ascontiguousarray(zi, dtype=np.int32)
    ii = np.ascontiguousarray(ii, dtype=np.int64)
    if zi.shape != ii.shape:
        raise ValueError("zi and ii must have the same shape")
    if zi.size and (zi.min() < 0 or zi.max() >= m or ii.min() < 0 or ii.max() >= x.size):
        raise ValueError("point out of range")
    p = np.empty(zi.shape, dtype=np.float64)
    _load().oracle_direct_points(_ptr(x), x.size, _ptr(h), m, k, _ptr(zi), _ptr(ii), zi.size, _ptr(p))
    return p


def fft(v, sign: int = -1) -> np.ndarray:
    """Unnormalised radix-2 DFT: X[k] = sum_j v[j] exp(sign 2 pi i jk / L)."""
    v = _c128(v).copy()
    if _load().oracle_fft(_ptr(v), v.size, int(sign)) != 0:
        raise ValueError("length must be a power of two")
    return v


def ols_power(x, h, L: int = 2048, S: int | None = None) -> np.ndarray:
    """Algorithm 2 (overlap-save, FFT length L, step S = L-K+1 by default) + |y|^2."""
    x, h = _c128(x), _c128(np.atleast_2d(h))
    m, k = h.shape
    if S is None:
        S = L - k + 1
    p = np.empty((m, x.size), dtype=np.float64)
    if _load().oracle_ols_power(_ptr(x), x.size, _ptr(h), m, k, int(L), int(S), _ptr(p)) != 0:
        raise ValueError(f"invalid overlap-save arguments (n={x.size}, K={k}, L={L}, S={S})")
    return p
