"""Pins for the FP64 oracle against facts that do not come from the oracle itself.

Each pin is chosen so that a plausible slip in the oracle fails it:
  * brute force vs numpy.convolve and a hand-written double loop: a dropped term,
    a wrong index or sign, a transposed operand (correlation instead of convolution);
  * the delta template: the identity and the 210-bin delay of the centred frame;
  * linearity; |y|^2 is the power;
  * the radix-2 FFT against numpy.fft and Parseval;
  * Algorithm 2 (overlap-save) against Eq. (1) for every segment length;
  * the noise-free chirp: the matched template's peak value and position follow
    from the template closed form.
"""
import numpy as np
import pytest

import synth
from synth import templates as T


def _rand_c(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


@pytest.mark.parametrize("n,k", [(1, 1), (5, 3), (16, 5), (7, 7), (3, 5), (16, 1)])
def test_direct_bruteforce(oracle_mod, n, k):
    rng = np.random.default_rng(100 + 10 * n + k)
    x = _rand_c(rng, n)
    h = _rand_c(rng, 3, k)
    y = oracle_mod.direct_conv(x, h)
    for m in range(3):
        # library special case: full linear convolution, first n outputs (Eq. 1 is causal)
        np.testing.assert_allclose(y[m], np.convolve(x, h[m])[:n], rtol=1e-14, atol=1e-14)
        # the sum written out
        ref = np.zeros(n, dtype=complex)
        for i in range(n):
            for kk in range(k):
                if i - kk >= 0:
                    ref[i] += x[i - kk] * h[m, kk]
        np.testing.assert_allclose(y[m], ref, rtol=1e-14, atol=1e-14)
    np.testing.assert_allclose(oracle_mod.direct_power(x, h), np.abs(y) ** 2, rtol=1e-14, atol=1e-14)


def test_bruteforce_rejects_correlation(oracle_mod):
    # the pin above must distinguish convolution from correlation (a reversed operand)
    rng = np.random.default_rng(7)
    x, h = _rand_c(rng, 16), _rand_c(rng, 1, 5)
    wrong = oracle_mod.direct_conv(x, h[:, ::-1])
    assert not np.allclose(wrong[0], np.convolve(x, h[0])[:16], rtol=1e-6)


def test_delta_template(oracle_mod):
    rng = np.random.default_rng(1)
    x = _rand_c(rng, 1000).astype(np.complex64)
    p = oracle_mod.direct_power(x, np.ones((1, 1)))
    xd = x.astype(np.complex128)
    np.testing.assert_array_equal(p[0], xd.real ** 2 + xd.imag ** 2)
    h, _ = T.template_bank(dtype=np.complex128)
    p0 = oracle_mod.direct_power(x, h[42:43])           # z = 0: centred delta
    assert np.all(p0[0, :210] == 0.0)
    np.testing.assert_array_equal(p0[0, 210:], (xd.real ** 2 + xd.imag ** 2)[:-210])


def test_linearity(oracle_mod):
    rng = np.random.default_rng(2)
    x1, x2 = _rand_c(rng, 3000), _rand_c(rng, 3000)
    h = _rand_c(rng, 4, 421)
    al, be = 0.7 - 1.3j, -2.1 + 0.4j
    lhs = oracle_mod.direct_conv(al * x1 + be * x2, h)
    rhs = al * oracle_mod.direct_conv(x1, h) + be * oracle_mod.direct_conv(x2, h)
    assert np.max(np.abs(lhs - rhs)) <= 1e-13 * np.max(np.abs(lhs))


def test_power_is_abs_squared(oracle_mod):
    rng = np.random.default_rng(3)
    y = _rand_c(rng, 257)
    np.testing.assert_allclose(oracle_mod.power(y), np.abs(y) ** 2, rtol=1e-15)


@pytest.mark.parametrize("L", [1, 2, 8, 1024, 2048, 4096])
def test_fft_against_numpy_and_parseval(oracle_mod, L):
    rng = np.random.default_rng(L)
    v = _rand_c(rng, L)
    f = oracle_mod.fft(v, -1)
    np.testing.assert_allclose(f, np.fft.fft(v), rtol=0, atol=1e-12 * np.sqrt(L) * 4)
    np.testing.assert_allclose(oracle_mod.fft(v, +1), np.fft.ifft(v) * L, rtol=0, atol=1e-12 * np.sqrt(L) * 4)
    assert abs(np.sum(np.abs(f) ** 2) - L * np.sum(np.abs(v) ** 2)) <= 1e-12 * L * np.sum(np.abs(v) ** 2)
    np.testing.assert_allclose(oracle_mod.fft(f, +1) / L, v, atol=1e-13)


def test_fft_rejects_non_power_of_two(oracle_mod):
    with pytest.raises(ValueError):
        oracle_mod.fft(np.ones(12), -1)


@pytest.mark.parametrize("L", [1024, 2048, 4096])
@pytest.mark.parametrize("n", [1, 7, 419, 1000, 1627, 1628, 1629, 2048, 5000, 9001])
def test_ols_equals_direct(oracle_mod, L, n):
    rng = np.random.default_rng(L + n)
    x = _rand_c(rng, n).astype(np.complex64)
    h, _ = T.template_bank(dtype=np.complex128)
    hs = h[::12]                                      # 8 templates incl. short and long ones
    pd = oracle_mod.direct_power(x, hs)
    po = oracle_mod.ols_power(x, hs, L=L)
    assert np.max(np.abs(po - pd)) <= 1e-12 * max(np.max(pd), 1e-300)


@pytest.mark.parametrize("k,L,S", [(1, 1024, 1024), (5, 8, 4), (421, 2048, 1600), (421, 2048, 1),
                                   (64, 128, 65), (1024, 1024, 1)])
def test_ols_any_step(oracle_mod, k, L, S):
    rng = np.random.default_rng(k + S)
    x = _rand_c(rng, 3001)
    h = _rand_c(rng, 2, k)
    pd = oracle_mod.direct_power(x, h)
    po = oracle_mod.ols_power(x, h, L=L, S=S)
    assert np.max(np.abs(po - pd)) <= 1e-12 * np.max(pd)


def test_ols_rejects_bad_step(oracle_mod):
    with pytest.raises(ValueError):
        oracle_mod.ols_power(np.ones(10), np.ones((1, 421)), L=2048, S=1629)


@pytest.mark.parametrize("z,r", [(20, 4000.0), (-30, 9000.0), (7, 2500.5)])
def test_chirp_peak(oracle_mod, z, r):
    # Noise-free chirp centred at integer bin c = r + z/2: the matched template's power
    # peaks at output index c + 210 with value (a^2 N / 2) sum_{|q|<=5|z|} |R_z(q)|^2.
    n, a = 1 << 14, 0.05
    x = synth.make_input(synth.ArraySpec(n=n, seed=0, noise=False,
                                         chirps=(synth.Chirp(float(r), float(z), a),)))
    h, zs = T.template_bank(dtype=np.complex128)
    p = oracle_mod.direct_power(x, h)
    m = int(np.nonzero(zs == z)[0][0])
    c = r + z / 2
    assert c == int(c)          # the sweep centre falls on a bin: no scalloping loss
    c = int(c)
    half = 5 * abs(z)
    energy = np.sum(np.abs(T.response(float(z), np.arange(-half, half + 1))) ** 2)
    expect = a * a * n / 2.0 * energy
    i_peak = int(np.argmax(p[m]))
    assert abs(i_peak - (c + 210)) <= 1
    assert p[m, i_peak] == pytest.approx(expect, rel=0.05)
    # the matched row beats rows whose drift is off by several bins
    assert p[m, i_peak] > 1.2 * max(p[m - 4].max(), p[min(m + 4, 84)].max())


def test_direct_points_match_plane(oracle_mod):
    rng = np.random.default_rng(5)
    x = _rand_c(rng, 2000)
    h = _rand_c(rng, 5, 33)
    p = oracle_mod.direct_power(x, h)
    zi = rng.integers(0, 5, 50)
    ii = rng.integers(0, 2000, 50)
    np.testing.assert_array_equal(oracle_mod.direct_points(x, h, zi, ii), p[zi, ii])


def test_threads_do_not_change_results(oracle_mod):
    rng = np.random.default_rng(6)
    x = _rand_c(rng, 5000)
    h, _ = T.template_bank(dtype=np.complex128)
    n0 = oracle_mod.threads()
    try:
        oracle_mod.set_threads(1)
        a = oracle_mod.ols_power(x, h[::20])
        oracle_mod.set_threads(max(2, n0))
        b = oracle_mod.ols_power(x, h[::20])
    finally:
        oracle_mod.set_threads(n0)
    np.testing.assert_array_equal(a, b)
