"""GPU tests of the fused threshold epilogue (fdas_convolve_candidates)."""
import numpy as np
import pytest

import synth
from parity import THRESHOLD, THRESHOLD_GAUSS, TOL_FP32

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def fd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1805_12280_gb300 as fd
    fd.load()
    return fd


@pytest.fixture(scope="module")
def bank():
    return synth.template_bank()[0]


def _keys(c):
    order = np.lexsort((c["bin"], c["tpl"]))
    return c[order]


@pytest.mark.parametrize("n,L,G", [(1 << 14, 2048, 85), (9001, 1024, 5), (5000, 4096, 17), (1, 2048, 85)])
def test_candidates_equal_thresholded_plane(fd, bank, n, L, G):
    x = synth.make_input(synth.single_small(n=max(n, 2), seed=31))[:n]
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    with fd.Plan(bank, n_max=max(n, 16), seg_len=L, tpl_per_cta=G) as plan:
        plane = plan.convolve(xd).cpu().numpy()
        buf, count = plan.candidates(xd, threshold=THRESHOLD, max_cand=1 << 20)
        plan.status()
        got = _keys(fd.candidates_to_numpy(buf, count))
    zi, ii = np.nonzero(plane > THRESHOLD)
    assert int(count.item()) == zi.size
    np.testing.assert_array_equal(got["tpl"], zi)                 # same set, bit-exact powers
    np.testing.assert_array_equal(got["bin"], ii)
    np.testing.assert_array_equal(got["power"], plane[zi, ii])


def test_candidates_vs_oracle(fd, oracle_mod, bank):
    x = synth.make_input(synth.single_small())
    with fd.Plan(bank, n_max=x.size) as plan:
        buf, count = plan.candidates(torch.from_numpy(x).cuda(), threshold=THRESHOLD)
        plan.status()
        got = fd.candidates_to_numpy(buf, count)
    ref = oracle_mod.direct_power(x, bank)
    band = TOL_FP32 * ref.max()
    sure = np.abs(ref - THRESHOLD) > band
    want = set(zip(*np.nonzero((ref > THRESHOLD) & sure)))
    have = set(zip(got["tpl"].tolist(), got["bin"].tolist()))
    assert want <= have                                            # every sure candidate found
    extra = have - want
    assert all(not sure[z, i] for z, i in extra)                   # the rest lie inside the band
    assert np.max(np.abs(got["power"] - ref[got["tpl"], got["bin"]])) <= band
    assert len(want) > 100


def test_gaussian_tail_threshold_set(fd, oracle_mod, bank):
    # the secondary set, T_g = -ln Q(6) = 20.74: at 2^17 points the chirp track crosses it
    # (its peak grows with N: a^2 N / 2 = 164), the noise almost never does
    x = synth.make_input(synth.single_small(n=1 << 17, seed=34))
    with fd.Plan(bank, n_max=x.size) as plan:
        xd = torch.from_numpy(x).cuda()
        plane = plan.convolve(xd).cpu().numpy()
        buf, count = plan.candidates(xd, threshold=THRESHOLD_GAUSS)
        plan.status()
        got = _keys(fd.candidates_to_numpy(buf, count))
    zi, ii = np.nonzero(plane > THRESHOLD_GAUSS)
    assert int(count.item()) == zi.size > 0
    np.testing.assert_array_equal(got["tpl"], zi)
    np.testing.assert_array_equal(got["bin"], ii)
    ref = oracle_mod.direct_power(x, bank)
    band = TOL_FP32 * ref.max()
    sure = np.abs(ref - THRESHOLD_GAUSS) > band
    assert np.array_equal((plane > THRESHOLD_GAUSS) & sure, (ref > THRESHOLD_GAUSS) & sure)
    assert (ref > THRESHOLD_GAUSS).sum() < (ref > THRESHOLD).sum() / 10


def test_candidate_overflow_and_empty(fd, bank):
    x = synth.make_input(synth.single_small(n=20000, seed=32))
    xd = torch.from_numpy(x).cuda()
    with fd.Plan(bank, n_max=x.size) as plan:
        full_buf, full_count = plan.candidates(xd, max_cand=1 << 20)
        total = int(full_count.item())
        assert total > 50
        buf, count = plan.candidates(xd, max_cand=10)          # counts everything, stores 10
        assert int(count.item()) == total
        part = fd.candidates_to_numpy(buf, count)
        assert part.size == 10 and np.unique(part[["tpl", "bin"]]).size == 10
        full = fd.candidates_to_numpy(full_buf, full_count)
        assert set(zip(part["tpl"], part["bin"])) <= set(zip(full["tpl"], full["bin"]))
        _, count0 = plan.candidates(xd, max_cand=0)             # counting only
        assert int(count0.item()) == total
        _, none = plan.candidates(xd, threshold=1e30)
        assert int(none.item()) == 0
        plan.status()


def test_candidates_reject_tensor_core_plan(fd, bank):
    with fd.Plan(bank, n_max=4096, precision=fd.FDAS_PREC_TC_FP16) as plan:
        with pytest.raises(fd.FdasError) as e:
            plan.candidates(torch.zeros(4096, dtype=torch.complex64, device="cuda"))
        assert e.value.code == fd.fdas.FDAS_ERR_UNSUPPORTED


@pytest.mark.parametrize("threshold", [0.5, -1.0])
def test_candidates_past_the_block_staging(fd, bank, threshold):
    # low thresholds put more than the staged slots of a block into the list: the rest
    # goes straight to global memory; T < 0 selects every output of the plane
    n = 20000
    x = synth.make_input(synth.single_small(n=n, seed=33))
    xd = torch.from_numpy(x).cuda()
    with fd.Plan(bank, n_max=n) as plan:
        plane = plan.convolve(xd).cpu().numpy()
        buf, count = plan.candidates(xd, threshold=threshold, max_cand=85 * n + 16)
        plan.status()
        got = _keys(fd.candidates_to_numpy(buf, count))
    zi, ii = np.nonzero(plane > threshold)
    assert int(count.item()) == zi.size and (threshold > 0 or zi.size == 85 * n)
    np.testing.assert_array_equal(got["tpl"], zi)
    np.testing.assert_array_equal(got["bin"], ii)
    np.testing.assert_array_equal(got["power"], plane[zi, ii])


@pytest.mark.parametrize("n,threshold", [(1 << 14, THRESHOLD), (9001, THRESHOLD), (1, THRESHOLD), (20000, 0.5),
                                         (3000, -1.0), (1 << 20, THRESHOLD)])
def test_two_stage_candidates_equal_its_thresholded_plane(fd, bank, n, threshold):
    # the two-stage tensor-core form's threshold epilogue: the same crossings, with the same
    # powers bit for bit, as thresholding the plane that form writes (T < 0: every output)
    x = synth.make_input(synth.single_small(n=max(n, 2), seed=35))[:n]
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    with fd.Plan(bank, n_max=max(n, 16), precision=fd.FDAS_PREC_TC_DFT2) as plan:
        plane = plan.convolve(xd).cpu().numpy()
        buf, count = plan.candidates(xd, threshold=threshold, max_cand=85 * n + 16)
        plan.status()
        got = _keys(fd.candidates_to_numpy(buf, count))
    zi, ii = np.nonzero(plane > threshold)
    assert int(count.item()) == zi.size and (threshold > 0 or zi.size == 85 * n)
    np.testing.assert_array_equal(got["tpl"], zi)
    np.testing.assert_array_equal(got["bin"], ii)
    np.testing.assert_array_equal(got["power"], plane[zi, ii])


def test_two_stage_candidates_truncation(fd, bank):
    n = 30011
    xd = torch.from_numpy(synth.make_input(synth.single_small(n=n, seed=36))).cuda()
    with fd.Plan(bank, n_max=n, precision=fd.FDAS_PREC_TC_DFT2) as plan:
        full_buf, full_count = plan.candidates(xd, threshold=3.0, max_cand=85 * n)
        total = int(full_count.item())
        assert total > 100
        buf, count = plan.candidates(xd, threshold=3.0, max_cand=10)    # counts everything, stores 10
        assert int(count.item()) == total
        part = fd.candidates_to_numpy(buf, count)
        full = fd.candidates_to_numpy(full_buf, full_count)
        assert part.size == 10 and set(zip(part["tpl"], part["bin"])) <= set(zip(full["tpl"], full["bin"]))
        _, count0 = plan.candidates(xd, threshold=3.0, max_cand=0)      # counting only
        assert int(count0.item()) == total
        plan.status()
