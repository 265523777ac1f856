"""GPU parity of the full-length frequency-domain FIR (Eq. 2) against the FP64 oracle."""
import numpy as np
import pytest

import synth
from parity import TOL_FP32, compare

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


def test_small_array_full_plane_vs_eq1(fd, oracle_mod, bank):
    x = synth.make_input(synth.single_small())
    with fd.FdFir(bank, n_max=x.size) as ff:
        assert ff.length == 1 << 21                     # smallest transform length built
        p = ff.convolve(torch.from_numpy(x).cuda()).cpu().numpy()
    info = compare(p, oracle_mod.direct_power(x, bank), TOL_FP32)
    assert info["candidates"] > 100


@pytest.mark.parametrize("n", [1, 7, 1000, 2049, 30011])
@pytest.mark.parametrize("k", [1, 5, 421])
def test_ragged_lengths_and_template_lengths(fd, oracle_mod, n, k):
    rng = np.random.default_rng(n * 7 + k)
    h = ((rng.standard_normal((3, k)) + 1j * rng.standard_normal((3, k))) / np.sqrt(2 * k)).astype(np.complex64)
    x = _rand(n, n + k)
    with fd.FdFir(h, n_max=max(n, 64)) as ff:
        out = torch.full((3, n), -1.0, device="cuda")
        ff.convolve(torch.from_numpy(x).cuda(), out=out)
        p = out.cpu().numpy()
    compare(p, oracle_mod.direct_power(x, h), TOL_FP32)


@pytest.mark.parametrize("log2p", [22, 23])
def test_long_transforms_match_overlap_save(fd, oracle_mod, bank, log2p):
    # P = 2^22 (n_max just above 2^21) and P = 2^23 (the SKA-sized array): the plane equals the
    # overlap-save plane to the FP32 tolerance, and sampled points equal Eq. (1)
    n = (1 << (log2p - 1)) + 12345 if log2p == 22 else 1 << 22
    spec = synth.single_ska() if log2p == 23 else synth.single_small(n=n, seed=51)
    x = synth.make_input(spec)
    xd = torch.from_numpy(x).cuda()
    with fd.FdFir(bank, n_max=x.size) as ff, fd.Plan(bank, n_max=x.size) as plan:
        assert ff.length == 1 << log2p
        a = ff.convolve(xd)
        b = plan.convolve(xd)
        plan.status()
        scale = float(b.max().item())
        assert float((a - b).abs().max().item()) <= TOL_FP32 * scale
        rng = np.random.default_rng(52)
        zi = rng.integers(0, 85, 2000)
        ii = np.concatenate([rng.integers(0, x.size, 1500), np.arange(250), x.size - 1 - np.arange(250)])
        got = a[torch.from_numpy(zi).cuda(), torch.from_numpy(ii).cuda()].cpu().numpy()
    ref = oracle_mod.direct_points(x, bank, zi, ii)
    assert np.max(np.abs(got - ref)) <= TOL_FP32 * scale


def test_invalid_arguments(fd, bank):
    with fd.FdFir(bank[:2], n_max=1000) as ff:
        x = torch.zeros(1001, dtype=torch.complex64, device="cuda")
        out = torch.empty(2 * 1001, dtype=torch.float32, device="cuda")
        with pytest.raises(fd.FdasError) as e:
            fd.fdas_fdfir_convolve(ff.handle, x.data_ptr(), 1001, out.data_ptr())
        assert e.value.code == fd.fdas.FDAS_ERR_INVALID_ARG
        with pytest.raises(fd.FdasError):
            fd.fdas_fdfir_convolve(ff.handle, x.data_ptr(), 100, x.data_ptr() + 400)   # overlapping
        torch.cuda.synchronize()
