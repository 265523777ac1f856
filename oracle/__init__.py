"""FP64 CPU oracle for the FDAS overlap-save power plane (ctypes over plain C).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py``.  The library's product path never imports
it.  It shares no code with the CUDA path; inputs come from the seeded
generators in ``synth``.

Functions (each restates the paper, see ``fdas_oracle.c``):
  direct_conv   Eq. (1), complex output          direct_power   Eq. (1) + |y|^2
  direct_points Eq. (1) + |y|^2 at chosen points fft            unnormalised radix-2 DFT
  ols_power     Algorithm 2 (overlap-save) + |y|^2
  harmonic_sums / harmonic_candidates
                the harmonic-summing stage on the power plane (Sec. 3 names it;
                read as the incoherent sum of the powers at bin k r, drift k z)
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
            lib.oracle_harmonic_sums.argtypes = [P, ci, i64, i64, ci, P]
            lib.oracle_harmonic_sums.restype = ci
            lib.oracle_harmonic_candidates.argtypes = [P, ci, i64, i64, ci, P, P, P, P, P, i64]
            lib.oracle_harmonic_candidates.restype = i64
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


def _plane32(P) -> np.ndarray:
    P = np.ascontiguousarray(P, dtype=np.float32)
    if P.ndim != 2:
        raise ValueError("the plane must be 2-D [m, n]")
    return P


def harmonic_levels(max_harm: int) -> list[int]:
    """The harmonic counts h = 1, 2, 4, .., max_harm summed."""
    return [1 << j for j in range(int(max_harm).bit_length())]


def harmonic_sums(P, bin0: int, max_harm: int) -> np.ndarray:
    """S_h(r, z) = sum_{k<=h} P[c + k z][bin0 + k r] for h = 1, 2, .., max_harm, float64
    [nlev, m, n] at (level, c + z, bin0 + r); NaN where undefined (r < 1, |h z| > c or
    bin0 + h r > n - 1).  P: float32 [m, n], m odd, c = (m - 1) / 2."""
    P = _plane32(P)
    m, n = P.shape
    S = np.empty((len(harmonic_levels(max_harm)), m, n), dtype=np.float64)
    if _load().oracle_harmonic_sums(_ptr(P), m, n, int(bin0), int(max_harm), _ptr(S)) != 0:
        raise ValueError(f"invalid harmonic-sum arguments (m={m}, n={n}, bin0={bin0}, max_harm={max_harm})")
    return S


def harmonic_candidates(P, bin0: int, max_harm: int, thresholds) -> dict:
    """Crossings S_h > thresholds[j] (h = 2^j) in (level, row, bin) order: a dict of arrays
    ``level`` (j), ``row`` (c + z), ``bin`` (bin0 + r) and ``value`` (S_h, float64)."""
    P = _plane32(P)
    m, n = P.shape
    nlev = len(harmonic_levels(max_harm))
    thr = np.ascontiguousarray(thresholds, dtype=np.float64)
    if thr.shape != (nlev,):
        raise ValueError(f"need {nlev} thresholds")
    lib = _load()
    empty = [np.empty(0, dtype=t) for t in (np.int32, np.int32, np.int64, np.float64)]
    total = lib.oracle_harmonic_candidates(_ptr(P), m, n, int(bin0), int(max_harm), _ptr(thr),
                                           *[_ptr(a) for a in empty], 0)
    if total < 0:
        raise ValueError(f"invalid harmonic-sum arguments (m={m}, n={n}, bin0={bin0}, max_harm={max_harm})")
    out = [np.empty(total, dtype=t) for t in (np.int32, np.int32, np.int64, np.float64)]
    got = lib.oracle_harmonic_candidates(_ptr(P), m, n, int(bin0), int(max_harm), _ptr(thr),
                                         *[_ptr(a) for a in out], total)
    assert got == total
    return dict(zip(("level", "row", "bin", "value"), out))
