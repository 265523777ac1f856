"""Pins of the oracle's harmonic-summing stage (Sec. 3 names the harmonic-summing module
that receives the power plane; the reading is the incoherent sum of the powers at bin k r,
drift k z, k = 1..h).  Each expectation below comes from a closed form or from the cells'
side (which fundamentals a raised cell feeds), not from the sum re-typed."""
import numpy as np
import pytest

import oracle
import synth

M, C = 9, 4   # rows z = -4 .. 4


def _domain(m, n, bin0, max_harm):
    """bool [nlev, m, n]: where S_h is defined (r >= 1, |h z| <= c, bin0 + h r <= n - 1)."""
    c = (m - 1) // 2
    lev = np.array(oracle.harmonic_levels(max_harm))[:, None, None]
    z = (np.arange(m) - c)[None, :, None]
    r = (np.arange(n) - bin0)[None, None, :]
    return (r >= 1) & (lev * np.abs(z) <= c) & (bin0 + lev * r <= n - 1)


@pytest.mark.parametrize("max_harm", [1, 2, 4, 8])
def test_linear_plane_closed_form(max_harm):
    """P[y][i] = a (y - c) + b i + g sums to a z T + b (h bin0 + r T) + g h, T = h (h+1)/2:
    a wrong row, column, sign or bin offset changes it."""
    n, bin0, a, b, g = 300, 7, 3.0, 1.0, 1000.0
    y, i = np.meshgrid(np.arange(M), np.arange(n), indexing="ij")
    P = (a * (y - C) + b * i + g).astype(np.float32)
    S = oracle.harmonic_sums(P, bin0, max_harm)
    dom = _domain(M, n, bin0, max_harm)
    assert np.array_equal(~np.isnan(S), dom)
    for j, h in enumerate(oracle.harmonic_levels(max_harm)):
        T = h * (h + 1) / 2
        z = (np.arange(M) - C)[:, None]
        r = (np.arange(n) - bin0)[None, :]
        want = a * z * T + b * (h * bin0 + r * T) + g * h
        assert np.array_equal(S[j][dom[j]], np.broadcast_to(want, (M, n))[dom[j]])


def test_constant_plane():
    P = np.full((M, 120), 2.5, dtype=np.float32)
    S = oracle.harmonic_sums(P, 0, 16)
    for j, h in enumerate(oracle.harmonic_levels(16)):
        vals = S[j][~np.isnan(S[j])]
        assert vals.size and np.all(vals == 2.5 * h)


def test_domain_edges():
    """Level h covers drifts |z| <= c / h and bins r <= (n - 1 - bin0) / h only."""
    n, bin0 = 100, 10
    S = oracle.harmonic_sums(np.ones((M, n), np.float32), bin0, 4)
    assert np.all(np.isnan(S[:, :, : bin0 + 1]))                  # r <= 0
    assert not np.isnan(S[2, C + 1, bin0 + 22]) and np.isnan(S[2, C + 1, bin0 + 23])   # 10 + 4 r <= 99
    assert not np.isnan(S[2, C - 1, bin0 + 1]) and np.isnan(S[2, C - 2, bin0 + 1])     # 4 |z| <= 4
    assert not np.isnan(S[0, 0, n - 1]) and np.isnan(S[1, C, n - 1])


@pytest.mark.parametrize("cell", [(C + 2, 10 + 12), (C + 4, 10 + 24), (C - 4, 10 + 36), (C, 10 + 17)])
def test_single_cell_feeds_its_divisor_fundamentals(cell):
    """A lone unit cell at (c + w, bin0 + u) is the k-th harmonic of (r, z) = (u / k, w / k)
    for every k dividing both; S_h of those fundamentals is 1 for h >= k, 0 elsewhere."""
    y0, i0 = cell
    n, bin0, H = 80, 10, 8
    P = np.zeros((M, n), np.float32)
    P[y0, i0] = 1.0
    S = oracle.harmonic_sums(P, bin0, H)
    want = np.zeros_like(S)
    w, u = y0 - C, i0 - bin0
    for j, h in enumerate(oracle.harmonic_levels(H)):
        for k in range(1, h + 1):
            if w % k == 0 and u % k == 0:
                want[j, C + w // k, bin0 + u // k] = 1.0
    dom = _domain(M, n, bin0, H)
    want[~dom] = np.nan
    assert np.array_equal(np.isnan(S), np.isnan(want))
    assert np.array_equal(S[dom], want[dom])


def test_injected_train_sums_its_amplitudes():
    n, bin0, r0, z0 = 500, 5, 37, 1
    amps = [8.0, 4.0, 2.0, 1.0]
    P = synth.add_train(np.zeros((M, n), np.float32), bin0, r0, z0, amps)
    S = oracle.harmonic_sums(P, bin0, 4)
    assert S[0, C + z0, bin0 + r0] == 8.0
    assert S[1, C + z0, bin0 + r0] == 12.0
    assert S[2, C + z0, bin0 + r0] == 15.0


def test_candidates_are_the_crossings_of_the_sums():
    rng = np.random.default_rng(5)
    n, bin0, H = 700, 20, 8
    P = synth.noise_plane(M, n, 3)
    synth.add_train(P, bin0, 41, -1, [9.0, 9.0, 9.0, 9.0])
    thr = np.array([3.0, 5.0, 8.0, 13.0]) + rng.uniform(0, 1, 4)
    S = oracle.harmonic_sums(P, bin0, H)
    cand = oracle.harmonic_candidates(P, bin0, H, thr)
    j, y, i = np.nonzero(np.nan_to_num(S, nan=-np.inf) > thr[:, None, None])   # C order = (j, y, i)
    assert np.array_equal(cand["level"], j) and np.array_equal(cand["row"], y) and np.array_equal(cand["bin"], i)
    assert np.array_equal(cand["value"], S[j, y, i])
    assert (0, C - 1, bin0 + 41) in set(zip(cand["level"], cand["row"], cand["bin"]))


def test_noise_sum_moments():
    """Sums of h unit-exponential powers (distinct cells) have mean h and variance h: the
    default thresholds h + 6 sqrt(h) are mu + 6 sigma of each level."""
    m, n, bin0 = 33, 40000, 0
    S = oracle.harmonic_sums(synth.noise_plane(m, n, 11), bin0, 8)
    for j, h in enumerate(oracle.harmonic_levels(8)):
        v = S[j][~np.isnan(S[j])]
        assert abs(v.mean() - h) < 0.02 * h
        assert abs(v.var() - h) < 0.05 * h


def test_invalid_arguments():
    P = np.zeros((M, 50), np.float32)
    for args in [(P, 0, 3), (P, 0, 64), (P, 50, 2), (P, -1, 2), (np.zeros((8, 50), np.float32), 0, 2)]:
        with pytest.raises(ValueError):
            oracle.harmonic_sums(*args)


def test_candidate_list_truncation_and_threads():
    n, bin0, H = 900, 3, 8
    P = synth.noise_plane(M, n, 21)
    thr = [-1.0] * 4
    full = oracle.harmonic_candidates(P, bin0, H, thr)
    total = full["bin"].size
    assert total == int((~np.isnan(oracle.harmonic_sums(P, bin0, H))).sum())
    n0 = oracle.threads()
    try:
        oracle.set_threads(1)
        one = oracle.harmonic_candidates(P, bin0, H, thr)
        s1 = oracle.harmonic_sums(P, bin0, H)
        oracle.set_threads(max(2, n0))
        many = oracle.harmonic_candidates(P, bin0, H, thr)
        sm = oracle.harmonic_sums(P, bin0, H)
    finally:
        oracle.set_threads(n0)
    for k in full:
        assert np.array_equal(one[k], many[k])
    assert np.array_equal(s1, sm, equal_nan=True)
