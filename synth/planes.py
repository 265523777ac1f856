"""Seeded power planes for the harmonic-summing stage, and a pulsar-like input array.

The harmonic-summing module receives the power plane (Sec. 3).  Its own parity
tests feed it planes made here directly, so that its inputs do not depend on the
convolution: noise powers drawn from the unit exponential (the distribution of
|x|^2 for unit-power complex Gaussian noise) plus trains of raised cells.  Nothing
here sums harmonics; the oracle and the CUDA path both consume these planes.
"""
from __future__ import annotations

import numpy as np

from .inputs import ArraySpec, Chirp


def noise_plane(m: int, n: int, seed: int) -> np.ndarray:
    """float32 [m, n] of unit-exponential powers."""
    rng = np.random.default_rng(seed)
    return rng.standard_exponential(size=(m, n), dtype=np.float32)


def add_train(P: np.ndarray, bin0: int, r: int, z: int, amps) -> np.ndarray:
    """Raise the cells of a harmonic train in place: amps[k-1] is added at row
    (m-1)/2 + k z, column bin0 + k r, for every k whose cell lies in the plane."""
    m, n = P.shape
    c = (m - 1) // 2
    for k, a in enumerate(amps, start=1):
        y, i = c + k * z, bin0 + k * r
        if 0 <= y < m and 0 <= i < n:
            P[y, i] += np.float32(a)
    return P


def pulsar(n: int, seed: int, r: float, z: float, amps) -> ArraySpec:
    """An array whose signal has harmonics: harmonic k (amplitude amps[k-1]) starts at
    bin k r and drifts k z bins, as the k-th harmonic of a constant-fdot signal does."""
    return ArraySpec(n=n, seed=seed,
                     chirps=tuple(Chirp(r=k * r, z=k * z, a=float(a)) for k, a in enumerate(amps, start=1)))
