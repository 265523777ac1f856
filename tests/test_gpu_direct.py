"""GPU parity of the time-domain form (Eq. 1 term by term) against the FP64 oracle."""
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


@pytest.mark.parametrize("n", [1, 100, 2047, 2048, 2049, 10000])
@pytest.mark.parametrize("k", [1, 2, 7, 8, 9, 64, 421, 1000])
def test_direct_vs_oracle(fd, oracle_mod, n, k):
    rng = np.random.default_rng(n * 7 + k)
    x = (rng.standard_normal(n) + 1j * rng.standard_normal(n)).astype(np.complex64)
    h = ((rng.standard_normal((3, k)) + 1j * rng.standard_normal((3, k))) / np.sqrt(2 * k)).astype(np.complex64)
    with fd.Plan(h, n_max=max(n, 16)) as plan:
        p = plan.convolve_direct(torch.from_numpy(x).cuda()).cpu().numpy()
        plan.status()
    compare(p, oracle_mod.direct_power(x, h), TOL_FP32)


def test_direct_full_bank_and_ols_agree(fd, oracle_mod):
    h, _ = synth.template_bank()
    x = synth.make_input(synth.single_small())
    xd = torch.from_numpy(x).cuda()
    with fd.Plan(h, n_max=x.size) as plan:
        td = plan.convolve_direct(xd).cpu().numpy()
        ols = plan.convolve(xd).cpu().numpy()
        plan.status()
    ref = oracle_mod.direct_power(x, h)
    compare(td, ref, TOL_FP32)
    assert np.max(np.abs(td - ols)) <= 2 * TOL_FP32 * ref.max()
