"""GPU parity of the harmonic-summing stage (fdas_harmonic_sum) against the FP64 oracle.

The stage's own inputs are seeded planes (unit-exponential noise plus harmonic trains), so
its parity does not lean on the convolution; one test runs the whole chain from a
pulsar-like array.  The GPU adds the h harmonics in FP32 in the order k = 1, 2, ..; with
non-negative FP32 terms its error is at most gamma_{h-1} S (gamma_n = n u / (1 - n u),
u = 2^-24), the bound the sums are held to.
"""
import numpy as np
import pytest

import synth
from parity import TOL_FP32

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

BIN0 = synth.CENTRE   # 210: the delay of templates centred in the 421-tap frame
U = 2.0 ** -24


@pytest.fixture(scope="module")
def fd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1805_12280_gb300 as fd
    fd.load()
    return fd


def _gamma(h):
    h = np.asarray(h, dtype=np.float64)
    return (h - 1) * U / (1 - (h - 1) * U)


def _run(fd, P, bin0, H, thr, max_cand):
    Pd = P if isinstance(P, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(P)).cuda()
    buf, count = fd.harmonic_sum(Pd, bin0, H, list(thr), max_cand=max_cand)
    torch.cuda.synchronize()
    return fd.harmonic_to_numpy(buf, count), int(count.item())


def _sorted(got):
    """Records in (level, row, bin) order, with their level index j = log2 h."""
    lev = np.log2(got["nharm"]).astype(np.int64)
    assert np.array_equal(1 << lev, got["nharm"])
    order = np.lexsort((got["bin"], got["tpl"], lev))
    return got[order], lev[order]


@pytest.mark.parametrize("m,n,bin0,H", [(85, 5000, BIN0, 8), (85, 4500, BIN0, 32), (9, 7001, 0, 16),
                                        (1, 3000, 5, 4), (85, 2300, BIN0, 1), (85, 2048 + BIN0 + 2, BIN0, 2),
                                        (129, 20000, BIN0, 8), (131, 9000, BIN0, 4), (85, 1024 + BIN0 + 1, BIN0, 8),
                                        (3, 50000, 7, 2)])
def test_every_defined_sum(fd, oracle_mod, m, n, bin0, H):
    """Thresholds below zero make every defined S_h a record (several tiles, ragged last
    tile, staging overflow): the record set is exactly the oracle's domain, each sum within
    the FP32 summation bound.  Shapes: 129 and 131 rows (|z| up to 64 and 65), a row range
    that ends one cell past 1024 fundamentals, and a three-row plane."""
    P = synth.noise_plane(m, n, seed=41 + n)
    S = oracle_mod.harmonic_sums(P, bin0, H)
    levels = np.array(oracle_mod.harmonic_levels(H))
    defined = ~np.isnan(S)
    total = int(defined.sum())
    got, count = _run(fd, P, bin0, H, [-1.0] * levels.size, total + 64)
    assert count == total
    got, lev = _sorted(got)
    j, y, i = np.nonzero(defined)
    np.testing.assert_array_equal(lev, j)
    np.testing.assert_array_equal(got["tpl"], y)
    np.testing.assert_array_equal(got["bin"], i)
    assert np.all(got["reserved"] == 0)
    ref = S[j, y, i]
    err = np.abs(got["power"].astype(np.float64) - ref)
    assert np.all(err <= _gamma(levels[j]) * ref)


def _noise_with_trains(m, n, seed, H):
    P = synth.noise_plane(m, n, seed)
    c = (m - 1) // 2
    rng = np.random.default_rng(seed + 1)
    trains = []
    for _ in range(6):
        z = int(rng.integers(-(c // H), c // H + 1))
        r = int(rng.integers(1, (n - 1 - BIN0) // H))
        synth.add_train(P, BIN0, r, z, [4.0] * H)
        trains.append((r, z))
    return P, trains


def _compare_thresholded(fd, oracle_mod, P, H, trains):
    m = P.shape[0]
    c = (m - 1) // 2
    thr = np.array(fd.harmonic_thresholds(H))
    levels = np.array(oracle_mod.harmonic_levels(H))
    ref = oracle_mod.harmonic_candidates(P, BIN0, H, thr)
    got, count = _run(fd, P, BIN0, H, thr, ref["bin"].size + (1 << 16))
    assert count == got.size
    band = _gamma(levels[ref["level"]]) * ref["value"]
    sure = np.abs(ref["value"] - thr[ref["level"]]) > band
    key = lambda lv, t, b: set(zip(lv.tolist(), t.tolist(), b.tolist()))
    want = key(ref["level"][sure], ref["row"][sure], ref["bin"][sure])
    have = key(np.log2(got["nharm"]).astype(int), got["tpl"], got["bin"])
    assert want <= have
    in_band = key(ref["level"][~sure], ref["row"][~sure], ref["bin"][~sure])
    assert have - want <= in_band          # nothing else crosses (band cells may go either way)
    for r, z in trains:                    # every injected train crosses at its top level
        assert (levels.size - 1, c + z, BIN0 + r) in have
    return ref["bin"].size


def test_thresholded_noise_with_trains(fd, oracle_mod):
    P, trains = _noise_with_trains(85, 1 << 17, 7, 8)
    assert _compare_thresholded(fd, oracle_mod, P, 8, trains) > 0


def test_thresholded_full_plane(fd, oracle_mod):
    """The plane of the 2^22-bin, 85-template workload (1.43 GB), eight harmonics."""
    P, trains = _noise_with_trains(85, 1 << 22, 9, 8)
    assert _compare_thresholded(fd, oracle_mod, P, 8, trains) > 100_000


def test_from_a_pulsar_array(fd, oracle_mod):
    """The whole chain: the plane of an array whose signal has four harmonics, then their
    sums; the oracle takes its own FP64 plane (rounded to FP32, as stored) from the same array."""
    bank = synth.template_bank()[0]
    r, z, H = 3001.0, 2.0, 8
    x = synth.make_input(synth.pulsar(1 << 15, 7, r, z, [0.05, 0.04, 0.03, 0.02]))
    with fd.Plan(bank, n_max=x.size) as plan:
        plane = plan.convolve(torch.from_numpy(x).cuda())
        plan.status()
        thr = np.array(fd.harmonic_thresholds(H))
        got, count = _run(fd, plane, BIN0, H, thr, 1 << 20)
    p_ref = oracle_mod.direct_power(x, bank)
    P32 = p_ref.astype(np.float32)
    S = oracle_mod.harmonic_sums(P32, BIN0, H)
    levels = np.array(oracle_mod.harmonic_levels(H))
    # each of the h powers carries the plane's error (<= TOL_FP32 max P), plus FP32 rounding
    band = levels[:, None, None] * (TOL_FP32 * p_ref.max() + U * P32.max()) + _gamma(levels)[:, None, None] * np.nan_to_num(S)
    Sn = np.nan_to_num(S, nan=-np.inf)
    sure_in = set(zip(*np.nonzero(Sn > thr[:, None, None] + band)))
    maybe = set(zip(*np.nonzero(Sn > thr[:, None, None] - band)))
    have = set(zip(np.log2(got["nharm"]).astype(int).tolist(), got["tpl"].tolist(), got["bin"].tolist()))
    assert count == len(have)
    assert sure_in <= have <= maybe
    c = (bank.shape[0] - 1) // 2
    assert (3, c + int(z), BIN0 + int(r + z / 2)) in have   # the fundamental, eight harmonics


def test_no_fundamental_and_count_only(fd):
    P = torch.ones((85, BIN0 + 1), dtype=torch.float32, device="cuda")
    got, count = _run(fd, P, BIN0, 8, [-1.0] * 4, 10)            # r >= 1 does not fit
    assert count == 0 and got.size == 0
    P = torch.from_numpy(synth.noise_plane(85, 3000, 3)).cuda()
    buf = torch.full((4, 3), -7, dtype=torch.int64, device="cuda")
    count = torch.empty(1, dtype=torch.int64, device="cuda")
    fd.harmonic_sum(P, BIN0, 8, [-1.0] * 4, max_cand=0, buf=buf, count=count)
    torch.cuda.synchronize()
    assert int(count.item()) > 0 and bool((buf == -7).all())     # counted, nothing stored


def test_truncated_list_holds_members(fd, oracle_mod):
    P = synth.noise_plane(85, 6000, 5)
    H = 4
    S = oracle_mod.harmonic_sums(P, BIN0, H)
    total = int((~np.isnan(S)).sum())
    got, count = _run(fd, P, BIN0, H, [-1.0] * 3, 1000)
    assert count == total and got.size == 1000
    got, lev = _sorted(got)
    keys = set(zip(lev.tolist(), got["tpl"].tolist(), got["bin"].tolist()))
    assert len(keys) == 1000
    assert np.all(~np.isnan(S[lev, got["tpl"], got["bin"]]))


def test_plane_beyond_2_31_elements(fd):
    """Three rows of 1.6e9 bins (19.3 GB): a unit train on the z = 0 row at multiples of the
    prime r0 = 201326557 reaches cell offsets above 2^31.  With thresholds h - 1/2 the sums
    have a closed form: the fundamental j r0 collects min(h, 8 // j) units, so (h, j r0)
    crosses exactly when h j <= 8."""
    n, r0, H = 3 << 29, 201326557, 8
    assert all(r0 % d for d in range(2, int(r0 ** 0.5) + 1))
    P = torch.zeros((3, n), dtype=torch.float32, device="cuda")
    for k in range(1, H + 1):
        P[1, k * r0] = 1.0
    assert n + H * r0 > 2 ** 31
    got, count = _run(fd, P, 0, H, [h - 0.5 for h in (1, 2, 4, 8)], 1024)
    del P
    torch.cuda.empty_cache()
    want = {(h, 1, j * r0) for h in (1, 2, 4, 8) for j in range(1, H + 1) if h * j <= H}
    have = set(zip(got["nharm"].tolist(), got["tpl"].tolist(), got["bin"].tolist()))
    assert count == len(want) and have == want
    assert np.all(got["power"] == got["nharm"])


def test_row_beyond_2_31_columns(fd):
    """One row of 2^31 + 2^20 bins (8.6 GB), past the 32-bit column range: the 64-bit form
    of the kernel.  A unit train at multiples of the prime r0 = 268566509 reaches columns
    above 2^31; sums and crossings as in the three-row case."""
    n, r0, H = (1 << 31) + (1 << 20), 268566509, 8
    assert all(r0 % d for d in range(2, int(r0 ** 0.5) + 1))
    P = torch.zeros((1, n), dtype=torch.float32, device="cuda")
    for k in range(1, H + 1):
        P[0, k * r0] = 1.0
    assert H * r0 > 2 ** 31
    got, count = _run(fd, P, 0, H, [h - 0.5 for h in (1, 2, 4, 8)], 1024)
    del P
    torch.cuda.empty_cache()
    want = {(h, 0, j * r0) for h in (1, 2, 4, 8) for j in range(1, H + 1) if h * j <= H}
    have = set(zip(got["nharm"].tolist(), got["tpl"].tolist(), got["bin"].tolist()))
    assert count == len(want) and have == want
    assert np.all(got["power"] == got["nharm"])
