"""GPU parity of the tensor-core form (fp16 DFT-GEMM radix-16 passes) against the FP64 oracle."""
import numpy as np
import pytest

import synth
from parity import TOL_TC, compare

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


def _run(plan, x):
    out = plan.convolve(torch.from_numpy(np.ascontiguousarray(x)).cuda())
    plan.status()
    return out.cpu().numpy()


def test_small_array_vs_direct(fd, oracle_mod, bank):
    x = synth.make_input(synth.single_small())
    with fd.Plan(bank, n_max=x.size, precision=fd.FDAS_PREC_TC_FP16) as plan:
        assert plan.desc.precision == fd.FDAS_PREC_TC_FP16
        p = _run(plan, x)
    info = compare(p, oracle_mod.direct_power(x, bank), TOL_TC)
    # two fp16 roundings of the data (relative 2^-12 RMS each) bound the relative RMS error
    # of |y|^2 near 2 * sqrt(2) * 2^-12 = 7e-4: the result must sit inside that, and well
    # inside the 2e-3 tolerance at the maximum
    assert info["rel"] < 1e-3 and info["rrmse"] < 1e-3, info
    i = int(np.argmax(p[42 + 20]))
    assert abs(i - (int(0.3 * x.size) + 10 + 210)) <= 2


@pytest.mark.parametrize("n", [1, 7, 1627, 1628, 1629, 2048, 5000, 9001])
@pytest.mark.parametrize("G", [1, 7, 85])
def test_ragged_and_groups(fd, oracle_mod, bank, n, G):
    rng = np.random.default_rng(n * 3 + G)
    x = (rng.standard_normal(n) + 1j * rng.standard_normal(n)).astype(np.complex64)
    hs = bank[::4] if G != 85 else bank
    with fd.Plan(hs, n_max=max(n, 16), tpl_per_cta=min(G, hs.shape[0]), precision=fd.FDAS_PREC_TC_FP16) as plan:
        p = _run(plan, x)
    # fp16 data round relative to the segment's energy, which includes the outputs past n
    # that overlap-save computes and discards: for arrays shorter than a template the
    # tolerance is taken against the maximum of the untruncated convolution
    full = oracle_mod.direct_power(np.concatenate([x, np.zeros(hs.shape[1] - 1, np.complex64)]), hs)
    compare(p, oracle_mod.direct_power(x, hs), TOL_TC, scale=max(float(full.max()), 0.0))


@pytest.mark.parametrize("k", [1, 2, 64, 421, 1000, 2044])
def test_template_lengths(fd, oracle_mod, k):
    rng = np.random.default_rng(k + 7)
    n = 6000
    x = (rng.standard_normal(n) + 1j * rng.standard_normal(n)).astype(np.complex64)
    h = ((rng.standard_normal((3, k)) + 1j * rng.standard_normal((3, k))) / np.sqrt(2 * k)).astype(np.complex64)
    with fd.Plan(h, n_max=n, precision=fd.FDAS_PREC_TC_FP16) as plan:
        p = _run(plan, x)
    compare(p, oracle_mod.direct_power(x, h), TOL_TC)


def test_unsupported_options(fd, bank):
    for kw in (dict(seg_len=1024), dict(seg_len=4096), dict(autotune=1)):
        with pytest.raises(fd.FdasError) as e:
            fd.Plan(bank, n_max=1000, precision=fd.FDAS_PREC_TC_FP16, **kw)
        assert e.value.code == fd.fdas.FDAS_ERR_UNSUPPORTED


@pytest.mark.slow
def test_ska_array_vs_ols_oracle(fd, oracle_mod, bank):
    spec = synth.single_ska()
    x = synth.make_input(spec)
    with fd.Plan(bank, n_max=x.size, precision=fd.FDAS_PREC_TC_FP16) as plan:
        out = plan.convolve(torch.from_numpy(x).cuda())
        plan.status()
        p = out.cpu().numpy()
    del out
    ref = oracle_mod.ols_power(x, bank, L=2048)
    info = compare(p, ref, TOL_TC)   # at this size the band covers T: only strong candidates are tested
    assert info["rel"] < 1e-3 and info["rrmse"] < 1e-3, info
    for c in spec.chirps:
        m = 42 + int(c.z)
        i = int(round(c.r + c.z / 2)) + 210
        assert p[m, i - 3:i + 4].max() > 20 * np.median(p[m])
