"""Constant-acceleration (constant fdot) template bank for the FDAS convolution.

The paper applies 85 templates per dedispersion trial, the longest with 421 taps,
and treats them as complex FIR filters (Sec. 3).  It cites the Fourier-domain
correlation technique for them but prints no formula, so the bank is built here
from the Fourier response of a signal whose frequency drifts linearly by ``z``
bins over the observation:

    R_z(q) = int_0^1 exp(2 pi i (-(q + z/2) t + z t^2 / 2)) dt        (q: bin offset
                                                                        from mid-sweep)

For z > 0 completing the square gives a Fresnel-integral closed form,
R_{-z}(q) = conj(R_z(-q)), and R_0(q) is the rectangular-window kernel
(1 at q = 0, 0 at the other integers).

Template z has K_z = 10|z| + 1 taps (q = -5|z| .. 5|z|, 421 taps at |z| = 42)
and is the unit-energy matched filter, centred in a 421-tap frame:

    h_z[k] = conj(R_z(210 - k)) / sqrt(sum_{|q| <= 5|z|} |R_z(q)|^2),  |210 - k| <= 5|z|

so every row of the power plane has the same 210-bin delay.  This module is an
input generator: it holds none of the convolution arithmetic and serves the
oracle and the CUDA path alike.
"""
from __future__ import annotations

import numpy as np
from scipy.special import fresnel

ZMAX = 42               # z = -42 .. +42 -> 85 templates (Sec. 3: 84 filters + the input)
FRAME = 421             # longest template (Sec. 3)
TAPS_PER_Z = 10         # K_z = 10 |z| + 1
CENTRE = (FRAME - 1) // 2


def _fresnel_e(s: np.ndarray) -> np.ndarray:
    """E(s) = C(s) + i S(s), the Fresnel integrals with argument pi s^2 / 2."""
    S, C = fresnel(s)
    return C + 1j * S


def response(z: float, q) -> np.ndarray:
    """R_z(q) for a scalar drift z (bins) at bin offsets q (array), complex128."""
    q = np.asarray(q, dtype=np.float64)
    if z == 0:
        out = np.empty(q.shape, dtype=np.complex128)
        zero = q == 0
        qq = np.where(zero, 1.0, q)
        out[...] = (np.exp(-2j * np.pi * qq) - 1.0) / (-2j * np.pi * qq)
        out[zero] = 1.0
        return out
    if z < 0:
        return np.conj(response(-z, -q))
    c = np.sqrt(2.0 / z)
    s1 = -(q + z / 2.0) * c
    s2 = (z / 2.0 - q) * c
    phase = np.exp(-1j * np.pi * (q + z / 2.0) ** 2 / z)
    return phase / np.sqrt(2.0 * z) * (_fresnel_e(s2) - _fresnel_e(s1))


def response_quadrature(z: float, q, nodes: int = 8192, panels: int = 64) -> np.ndarray:
    """R_z(q) by composite Gauss-Legendre quadrature of its defining integral.

    Independent of the closed form; used to pin it.
    """
    q = np.atleast_1d(np.asarray(q, dtype=np.float64))
    per = nodes // panels
    xg, wg = np.polynomial.legendre.leggauss(per)
    edges = np.linspace(0.0, 1.0, panels + 1)
    t = (0.5 * (edges[1:] - edges[:-1])[:, None] * (xg[None, :] + 1.0) + edges[:-1, None]).ravel()
    w = (0.5 * (edges[1:] - edges[:-1])[:, None] * wg[None, :]).ravel()
    ph = 2.0 * np.pi * (-(q[:, None] + z / 2.0) * t[None, :] + z * t[None, :] ** 2 / 2.0)
    return (np.exp(1j * ph) * w[None, :]).sum(axis=1)


def template_taps(z: int) -> int:
    return TAPS_PER_Z * abs(int(z)) + 1


def template_bank(zmax: int = ZMAX, frame: int = FRAME, dtype=np.complex64):
    """Return (h, zs): h[m, k] for z = zs[m] = -zmax .. zmax, each in a ``frame``-tap frame.

    The bank is computed in FP64 and cast to ``dtype`` (complex64 by default: the
    templates the method consumes are complex single precision, Sec. 3).
    """
    zs = np.arange(-zmax, zmax + 1)
    centre = (frame - 1) // 2
    h = np.zeros((zs.size, frame), dtype=np.complex128)
    for m, z in enumerate(zs):
        half = (template_taps(z) - 1) // 2
        if half > centre:
            raise ValueError(f"template z={z} ({template_taps(z)} taps) does not fit a {frame}-tap frame")
        q = np.arange(-half, half + 1)
        r = response(float(z), q)
        r = r / np.sqrt(np.sum(np.abs(r) ** 2))
        # h[k] = conj(R(centre - k))  ->  k = centre - q
        h[m, centre - q] = np.conj(r)
    return h.astype(dtype), zs
