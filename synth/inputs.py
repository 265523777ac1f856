"""Seeded synthetic Fourier-domain input arrays shaped like the paper's workload.

The FT-convolution module receives 2^22 complex single-precision Fourier bins per
dedispersion trial (Sec. 3).  No telescope data ship with the paper, so arrays are
synthesised:

  1. real series  s[n] = g[n] + sum_c a_c cos(2 pi (r_c u + z_c u^2 / 2)),
     n = 0 .. 2N-1, u = n / (2N), g ~ N(0, 1)  (r_c: start bin, z_c: drift in bins);
  2. X = rFFT(s) in FP64, keep bins 0 .. N-1 (the Nyquist bin is dropped),
     x = X / sqrt(2N) so that the noise has E|x|^2 = 1;
  3. cast to complex64.

A chirp of amplitude a, start bin r and drift z then appears around bin r + z/2 as
a sqrt(N/2) R_z(k - r - z/2) (see ``synth.templates.response``).  Nothing here is
part of the convolution; the oracle and the CUDA path both consume these arrays.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass(frozen=True)
class Chirp:
    r: float        # start frequency, bins
    z: float        # drift over the observation, bins
    a: float = 0.05  # amplitude relative to unit-variance noise


@dataclass(frozen=True)
class ArraySpec:
    n: int
    seed: int
    chirps: tuple = field(default_factory=tuple)
    noise: bool = True


def make_series(spec: ArraySpec) -> np.ndarray:
    """Step 1: the 2N-sample real time series (FP64)."""
    n2 = 2 * spec.n
    rng = np.random.default_rng(spec.seed)
    s = rng.standard_normal(n2) if spec.noise else np.zeros(n2)
    u = np.arange(n2, dtype=np.float64) / n2
    for c in spec.chirps:
        cycles = c.r * u + c.z * u * u / 2.0
        cycles -= np.floor(cycles)          # keep the phase argument small before 2 pi
        s += c.a * np.cos(2.0 * np.pi * cycles)
    return s


def make_input(spec: ArraySpec, dtype=np.complex64) -> np.ndarray:
    """Steps 2-3: Fourier bins 0..N-1 of the series, unit noise power, as ``dtype``."""
    s = make_series(spec)
    X = np.fft.rfft(s)[: spec.n] / np.sqrt(2.0 * spec.n)
    return X.astype(dtype)


# ---------------------------------------------------------------------------
# The workloads: a small single array, the SKA-sized single array, a batch of
# dedispersion trials of uneven lengths and a Poisson request stream.
# ---------------------------------------------------------------------------

def single_small(n: int = 1 << 14, seed: int = 0) -> ArraySpec:
    """N = 2^14, one chirp at 0.3 of Nyquist (bin 0.3 N) drifting z = +20 bins."""
    return ArraySpec(n=n, seed=seed, chirps=(Chirp(r=0.3 * n, z=20.0, a=0.05),))


def single_ska(n: int = 1 << 22, seed: int = 1, n_chirps: int = 8) -> ArraySpec:
    """N = 2^22, 8 chirps at seeded start bins U[0.05N, 0.95N] and drifts U{-40..40}."""
    rng = np.random.default_rng(seed + 10_000)
    chirps = tuple(
        Chirp(r=float(rng.uniform(0.05 * n, 0.95 * n)), z=float(rng.integers(-40, 41)), a=0.05)
        for _ in range(n_chirps)
    )
    return ArraySpec(n=n, seed=seed, chirps=chirps)


def log_uniform_lengths(count: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """Lengths drawn log-uniformly in [lo, hi] and rounded to the nearest integer."""
    rng = np.random.default_rng(seed)
    return np.rint(np.exp(rng.uniform(np.log(lo), np.log(hi), size=count))).astype(np.int64)


def batch_trials(count: int = 64, lo: int = 1 << 18, hi: int = 1 << 22,
                 length_seed: int = 999, first_seed: int = 1000) -> list[ArraySpec]:
    """Dedispersion trials of uneven length, one chirp each as in ``single_small``."""
    ns = log_uniform_lengths(count, lo, hi, length_seed)
    return [single_small(int(n), first_seed + i) for i, n in enumerate(ns)]


def poisson_requests(count: int, rate_hz: float = 200.0, lo: int = 1 << 16, hi: int = 1 << 22,
                     arrival_seed: int = 2000, first_seed: int = 2001):
    """Arrival times (s) of a Poisson stream and the arrays it carries."""
    rng = np.random.default_rng(arrival_seed)
    t = np.cumsum(rng.exponential(1.0 / rate_hz, size=count))
    ns = log_uniform_lengths(count, lo, hi, arrival_seed + 1)
    return t, [single_small(int(n), first_seed + i) for i, n in enumerate(ns)]
