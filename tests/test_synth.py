"""Pins for the seeded input generators (templates and Fourier-domain arrays)."""
import numpy as np
import pytest

import synth
from synth import templates as T


@pytest.mark.parametrize("z", [1, 2, 5, 13, 20, 31, 42, -7, -42])
def test_closed_form_matches_quadrature(z):
    # The Fresnel closed form against Gauss-Legendre quadrature of the defining integral.
    half = 5 * abs(z)
    q = np.arange(-half - 20, half + 21)
    closed = T.response(float(z), q)
    quad = T.response_quadrature(float(z), q)
    assert np.max(np.abs(closed - quad)) <= 1e-12


def test_response_symmetry_and_zero_drift():
    q = np.arange(-60, 61)
    for z in (3, 17, 42):
        np.testing.assert_allclose(T.response(float(-z), q), np.conj(T.response(float(z), -q)), atol=1e-15)
    r0 = T.response(0.0, q)
    assert r0[q == 0][0] == 1.0
    assert np.max(np.abs(r0[q != 0])) < 1e-14           # integer offsets of the rectangular kernel
    # non-integer offsets follow (e^{-2 pi i q} - 1) / (-2 pi i q)
    qf = np.array([0.25, 0.5, -1.5])
    np.testing.assert_allclose(T.response(0.0, qf), T.response_quadrature(0.0, qf), atol=1e-13)


def test_response_energy_parseval():
    # sum over all integer q of |R_z(q)|^2 = int_0^1 |e^{i phi}|^2 dt = 1 (Parseval for the
    # unit-length window); the 5|z| truncation keeps most of it.
    for z in (4, 20, 42):
        q = np.arange(-4000, 4001)
        tot = np.sum(np.abs(T.response(float(z), q)) ** 2)
        assert abs(tot - 1.0) < 2e-4
        half = 5 * z
        kept = np.sum(np.abs(T.response(float(z), np.arange(-half, half + 1))) ** 2)
        assert 0.98 <= kept <= 1.0


def test_template_bank_layout():
    h, zs = T.template_bank(dtype=np.complex128)
    assert h.shape == (85, 421) and list(zs) == list(range(-42, 43))
    for m, z in enumerate(zs):
        nz = np.nonzero(np.abs(h[m]) > 0)[0]
        half = 5 * abs(z)
        assert nz.min() == 210 - half and nz.max() == 210 + half          # centred, 10|z|+1 taps
        np.testing.assert_allclose(np.sum(np.abs(h[m]) ** 2), 1.0, rtol=1e-13)  # unit energy
    # z = 0 is the single-tap delta at the frame centre
    assert h[42, 210] == 1.0 and np.count_nonzero(h[42]) == 1
    # h_{-z}[k] = conj(h_z[420 - k]) (time reversal + conjugation)
    np.testing.assert_allclose(h[0], np.conj(h[84][::-1]), atol=1e-15)
    hc, _ = T.template_bank()
    assert hc.dtype == np.complex64


def test_input_noise_power_and_seed():
    spec = synth.ArraySpec(n=1 << 15, seed=3)
    x = synth.make_input(spec)
    assert x.dtype == np.complex64 and x.shape == (1 << 15,)
    assert abs(np.mean(np.abs(x[1:]) ** 2) - 1.0) < 0.03       # E|x|^2 = 1 after normalisation
    np.testing.assert_array_equal(x, synth.make_input(spec))      # deterministic
    assert not np.array_equal(x, synth.make_input(synth.ArraySpec(n=1 << 15, seed=4)))


def test_chirp_spectrum_matches_response():
    # noise-free chirp: x[k] ~ a sqrt(N/2) R_z(k - r - z/2) near the sweep
    n, r, z, a = 1 << 14, 4000.0, 20.0, 0.05
    x = synth.make_input(synth.ArraySpec(n=n, seed=0, chirps=(synth.Chirp(r, z, a),), noise=False),
                         dtype=np.complex128)
    k = np.arange(int(r) - 30, int(r) + 51)
    pred = a * np.sqrt(n / 2.0) * T.response(z, k - r - z / 2.0)
    err = np.max(np.abs(x[k] - pred)) / np.max(np.abs(pred))
    assert err < 2e-2


def test_workload_specs():
    s0 = synth.single_small()
    assert s0.n == 1 << 14 and s0.chirps[0].r == pytest.approx(0.3 * (1 << 14)) and s0.chirps[0].z == 20
    s1 = synth.single_ska()
    assert s1.n == 1 << 22 and len(s1.chirps) == 8
    assert all(-40 <= c.z <= 40 and 0.05 * s1.n <= c.r <= 0.95 * s1.n for c in s1.chirps)
    b = synth.batch_trials()
    ns = np.array([s.n for s in b])
    assert len(b) == 64 and ns.min() >= 1 << 18 and ns.max() <= 1 << 22
    assert len({s.seed for s in b}) == 64
    t, reqs = synth.poisson_requests(100)
    assert np.all(np.diff(t) > 0) and len(reqs) == 100


def test_pulsar_harmonics_and_planes():
    s = synth.pulsar(1 << 14, 5, 1000.5, 2.0, [0.05, 0.04, 0.03])
    assert [(c.r, c.z, c.a) for c in s.chirps] == [(1000.5, 2.0, 0.05), (2001.0, 4.0, 0.04), (3001.5, 6.0, 0.03)]
    P = synth.noise_plane(5, 20000, 9)
    assert P.dtype == np.float32 and P.shape == (5, 20000) and P.min() >= 0
    assert abs(P.mean() - 1.0) < 0.02 and abs(P.var() - 1.0) < 0.05        # unit exponential
    np.testing.assert_array_equal(P, synth.noise_plane(5, 20000, 9))
    Z = synth.add_train(np.zeros((5, 100), np.float32), 10, 7, 1, [3.0, 2.0, 1.0])
    assert Z[3, 17] == 3.0 and Z[4, 24] == 2.0 and Z.sum() == 5.0            # k = 3 falls outside the rows
