"""GPU parity of plans that group templates by support length (group_support=1)."""
import numpy as np
import pytest

import synth
from parity import THRESHOLD, TOL_FP32, compare

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


def _rand(n, seed):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(n) + 1j * rng.standard_normal(n)).astype(np.complex64)


def _windowed_bank(seed, M=12, K=421):
    # templates whose nonzero taps fill a window [a, a + w) of the K-tap frame
    rng = np.random.default_rng(seed)
    h = np.zeros((M, K), dtype=np.complex64)
    for z in range(M):
        w = int(rng.integers(1, K + 1))
        a = int(rng.integers(0, K - w + 1))
        h[z, a:a + w] = (rng.standard_normal(w) + 1j * rng.standard_normal(w)) / np.sqrt(2 * w)
    h[0] = 0
    h[0, K - 1] = 1.0                       # a delay by K - 1: only the last tap
    return h


def test_bank_is_split_and_matches_eq1(fd, oracle_mod, bank):
    x = synth.make_input(synth.single_small())
    with fd.Plan(bank, n_max=1 << 22, group_support=1) as plan:
        assert plan.desc.groups == 3        # 85 supports 1..421 taps, arrays of 2^22 points
        p = plan.convolve(torch.from_numpy(x).cuda()).cpu().numpy()
        plan.status()
    info = compare(p, oracle_mod.direct_power(x, bank), TOL_FP32)
    assert info["candidates"] > 100


@pytest.mark.parametrize("n", [1, 7, 300, 420, 421, 1629, 2048, 9001, 20011])
def test_shifted_supports_ragged_lengths(fd, oracle_mod, n):
    h = _windowed_bank(n)
    x = _rand(n, n + 1)
    for L in (1024, 2048, 4096):
        with fd.Plan(h, n_max=max(n, 40000), seg_len=L, tpl_per_cta=5, group_support=1) as plan:
            assert 1 <= plan.desc.groups <= 6
            out = torch.full((h.shape[0], n), -1.0, device="cuda")
            plan.convolve(torch.from_numpy(x).cuda(), out=out)
            plan.status()
            p = out.cpu().numpy()
        compare(p, oracle_mod.direct_power(x, h), TOL_FP32)
        # outputs before a template's first nonzero tap are exactly zero
        first = np.argmax(h != 0, axis=1)
        for z in range(h.shape[0]):
            assert np.all(p[z, :min(first[z], n)] == 0.0)


@pytest.mark.parametrize("n,threshold", [(30000, THRESHOLD), (3000, -1.0)])
def test_candidates_equal_thresholded_plane(fd, bank, n, threshold):
    # T < 0 also selects the zero outputs before each template's first tap
    x = synth.make_input(synth.single_small(n=n, seed=41))
    xd = torch.from_numpy(x).cuda()
    with fd.Plan(bank, n_max=1 << 22, group_support=1) as plan:
        plane = plan.convolve(xd).cpu().numpy()
        buf, count = plan.candidates(xd, threshold=threshold, max_cand=85 * n + 16)
        plan.status()
        got = fd.candidates_to_numpy(buf, count)
    got = got[np.lexsort((got["bin"], got["tpl"]))]
    zi, ii = np.nonzero(plane > threshold)
    assert int(count.item()) == zi.size > 100
    assert threshold > 0 or zi.size == 85 * n
    np.testing.assert_array_equal(got["tpl"], zi)
    np.testing.assert_array_equal(got["bin"], ii)
    np.testing.assert_array_equal(got["power"], plane[zi, ii])


def test_host_path_matches_device(fd, bank):
    x = synth.make_input(synth.single_small(n=50000, seed=42))
    with fd.Plan(bank, n_max=x.size, group_support=1) as plan:
        dev = plan.convolve(torch.from_numpy(x).cuda()).cpu().numpy()
        host = plan.convolve_host(x)
        host2 = plan.convolve_host(x[:12345])
        dev2 = plan.convolve(torch.from_numpy(x[:12345].copy()).cuda()).cpu().numpy()
        plan.status()
    np.testing.assert_array_equal(host, dev)
    np.testing.assert_array_equal(host2, dev2)


def test_time_domain_form_keeps_raw_templates(fd, bank):
    x = synth.make_input(synth.single_small(n=8000, seed=43))
    xd = torch.from_numpy(x).cuda()
    with fd.Plan(bank, n_max=x.size, group_support=1) as plan:
        a = plan.convolve(xd)
        b = plan.convolve_direct(xd)
        plan.status()
    scale = float(b.max().item())
    assert float((a - b).abs().max().item()) <= TOL_FP32 * scale


def test_batched_forms_reject_grouped_plans(fd, bank):
    x = torch.from_numpy(_rand(1000, 44)).cuda()
    with fd.Plan(bank[:10], n_max=1000, group_support=1) as plan:
        with pytest.raises(fd.FdasError) as e:
            plan.convolve_batch([x])
        assert e.value.code == fd.fdas.FDAS_ERR_UNSUPPORTED
        with pytest.raises(fd.FdasError) as e:
            fd.Server(plan, budget_bytes=1 << 24)
        assert e.value.code == fd.fdas.FDAS_ERR_UNSUPPORTED
