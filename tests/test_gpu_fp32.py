"""GPU parity of the fused FP32 segment kernel against the FP64 oracle, through the C ABI."""
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
    h, zs = synth.template_bank()
    return h


def _run(fd, plan, x):
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    out = plan.convolve(xd)
    plan.status()
    return out.cpu().numpy()


def test_small_array_full_plane_vs_direct(fd, oracle_mod, bank):
    # N = 2^14, one chirp at 0.3 Nyquist drifting z = +20, 85 templates, L = 2048
    x = synth.make_input(synth.single_small())
    with fd.Plan(bank, n_max=x.size) as plan:
        assert (plan.desc.seg_len, plan.desc.seg_step, plan.desc.frame_len) == (2048, 1628, 421)
        p = _run(fd, plan, x)
    ref = oracle_mod.direct_power(x, bank)
    info = compare(p, ref, TOL_FP32)
    assert info["candidates"] > 100
    assert info["rrmse"] < 1e-5
    # the injected chirp is found in the z = +20 row at bin r + z/2 + 210
    i = int(np.argmax(p[42 + 20]))
    assert abs(i - (int(0.3 * x.size) + 10 + 210)) <= 2


@pytest.mark.parametrize("L", [1024, 2048, 4096])
@pytest.mark.parametrize("n", [1, 7, 419, 1000, 1627, 1628, 1629, 2048, 5000, 9001])
def test_ragged_lengths_and_segment_sizes(fd, oracle_mod, bank, L, n):
    rng = np.random.default_rng(n + L)
    x = (rng.standard_normal(n) + 1j * rng.standard_normal(n)).astype(np.complex64)
    hs = bank[::6]                                   # 15 templates, short and long
    with fd.Plan(hs, n_max=max(n, 16), seg_len=L, tpl_per_cta=4) as plan:
        p = _run(fd, plan, x)
    compare(p, oracle_mod.direct_power(x, hs), TOL_FP32)


@pytest.mark.parametrize("k", [1, 2, 5, 64, 200, 421, 1000, 2044])
def test_template_lengths(fd, oracle_mod, k):
    rng = np.random.default_rng(k)
    n = 7000
    x = (rng.standard_normal(n) + 1j * rng.standard_normal(n)).astype(np.complex64)
    h = ((rng.standard_normal((3, k)) + 1j * rng.standard_normal((3, k))) / np.sqrt(2 * k)).astype(np.complex64)
    with fd.Plan(h, n_max=n) as plan:
        d = plan.desc
        assert d.frame_len % 2 == 1 and d.seg_step % 4 == 0 and d.seg_step <= 2048 - d.frame_len + 1
        p = _run(fd, plan, x)
    compare(p, oracle_mod.direct_power(x, h), TOL_FP32)


@pytest.mark.parametrize("G", [1, 5, 17, 84, 85])
def test_templates_per_block(fd, oracle_mod, bank, G):
    x = synth.make_input(synth.single_small(n=6000, seed=4))
    with fd.Plan(bank, n_max=x.size, tpl_per_cta=G) as plan:
        p = _run(fd, plan, x)
    compare(p, oracle_mod.ols_power(x, bank), TOL_FP32)


def test_delta_and_zero_templates(fd):
    rng = np.random.default_rng(9)
    n = 5000
    x = (rng.standard_normal(n) + 1j * rng.standard_normal(n)).astype(np.complex64)
    h = np.zeros((3, 421), dtype=np.complex64)
    h[0, 0] = 1.0            # identity
    h[1, 210] = 1.0          # centred delta: 210-bin delay
    with fd.Plan(h, n_max=n) as plan:
        p = _run(fd, plan, x)
    xp = np.abs(x.astype(np.complex128)) ** 2
    np.testing.assert_allclose(p[0], xp, rtol=2e-6, atol=1e-6 * xp.max())
    assert np.all(np.abs(p[1, :210]) <= 1e-6 * xp.max())
    np.testing.assert_allclose(p[1, 210:], xp[:-210], rtol=2e-6, atol=1e-6 * xp.max())
    assert np.all(p[2] == 0.0)


def test_nan_input_stays_local(fd):
    # a NaN reaches only the outputs whose segments contain it; it is reported, not trapped
    rng = np.random.default_rng(10)
    n = 20000
    x = (rng.standard_normal(n) + 1j * rng.standard_normal(n)).astype(np.complex64)
    x[10000] = np.nan
    h, _ = synth.template_bank()
    with fd.Plan(h[40:45], n_max=n) as plan:
        p = _run(fd, plan, x)
        plan.status()
    bad = ~np.isfinite(p)
    assert bad.any()
    cols = np.nonzero(bad.any(axis=0))[0]
    assert cols.min() >= 10000 - 2 * 1628 and cols.max() < 10000 + 2 * 2048
    assert np.isfinite(p[:, :5000]).all() and np.isfinite(p[:, 16000:]).all()


def test_host_entry_point_matches_device(fd, bank):
    x = synth.make_input(synth.single_small(n=50000, seed=11))
    with fd.Plan(bank, n_max=x.size) as plan:
        p_dev = _run(fd, plan, x)
        p_host = plan.convolve_host(x)
        p_host2 = plan.convolve_host(x[:31000])      # shorter array through the same staging
        p_dev2 = _run(fd, plan, x[:31000])
    np.testing.assert_array_equal(p_host, p_dev)
    np.testing.assert_array_equal(p_host2, p_dev2)


def test_invalid_arguments(fd, bank):
    with fd.Plan(bank[:2], n_max=1000) as plan:
        x = torch.zeros(1001, dtype=torch.complex64, device="cuda")
        out = torch.empty(2 * 1001, dtype=torch.float32, device="cuda")
        with pytest.raises(fd.FdasError) as e:
            fd.fdas_convolve(plan.handle, x.data_ptr(), 1001, out.data_ptr())
        assert e.value.code == fd.fdas.FDAS_ERR_INVALID_ARG
        with pytest.raises(fd.FdasError):
            fd.fdas_convolve(plan.handle, x.data_ptr() + 8, 100, out.data_ptr())    # misaligned input
        with pytest.raises(fd.FdasError):
            fd.fdas_convolve(plan.handle, x.data_ptr(), 100, x.data_ptr() + 400)    # overlapping
        with pytest.raises(fd.FdasError):
            fd.fdas_convolve(plan.handle, x.data_ptr(), 0, out.data_ptr())
        plan.status()


@pytest.mark.slow
def test_ska_array_full_plane_vs_ols_oracle(fd, oracle_mod, bank):
    # N = 2^22, 8 chirps, 85 templates, L = 2048: the whole plane against the FP64
    # overlap-save oracle (itself pinned to Eq. 1), plus sampled points against Eq. 1.
    spec = synth.single_ska()
    x = synth.make_input(spec)
    with fd.Plan(bank, n_max=x.size) as plan:
        xd = torch.from_numpy(x).cuda()
        out = plan.convolve(xd)
        plan.status()
        p = out.cpu().numpy()
    del out
    ref = oracle_mod.ols_power(x, bank, L=2048)
    info = compare(p, ref, TOL_FP32)
    assert info["candidates"] > 1000
    rng = np.random.default_rng(12)
    zi = rng.integers(0, 85, 4000)
    ii = np.concatenate([rng.integers(0, x.size, 3000), np.arange(500), x.size - 1 - np.arange(500)])
    pts = oracle_mod.direct_points(x, bank, zi, ii)
    assert np.max(np.abs(p[zi, ii] - pts)) <= TOL_FP32 * np.max(ref)
    # each chirp is recovered in its own row
    for c in spec.chirps:
        m = 42 + int(c.z)
        i = int(round(c.r + c.z / 2)) + 210
        assert p[m, i - 3:i + 4].max() > 20 * np.median(p[m])


def test_plane_pointer_alignment_paths(fd, bank):
    # a 16-byte-aligned plane with n % 4 == 0 leaves through bulk copies from shared memory;
    # a plane that is only 4-byte aligned takes the per-thread store path: same bits
    rng = np.random.default_rng(13)
    n = 8000
    x = torch.from_numpy((rng.standard_normal(n) + 1j * rng.standard_normal(n)).astype(np.complex64)).cuda()
    with fd.Plan(bank[::9], n_max=n) as plan:
        m = plan.n_templates
        ref = plan.convolve(x)
        buf = torch.full((m * n + 4,), -1.0, dtype=torch.float32, device="cuda")
        for shift in (1, 2, 3):
            fd.fdas_convolve(plan.handle, x.data_ptr(), n, buf.data_ptr() + 4 * shift)
            plan.status()
            assert torch.equal(buf[shift:shift + m * n].view(m, n), ref)


def test_bounded_wait_timeout_is_reported(fd, oracle_mod, bank):
    # a wait for a copy that is never issued runs out after 5 ms: the status word reports it
    # once, and the context and the plan stay usable
    x = synth.make_input(synth.single_small(n=3000, seed=14))
    with fd.Plan(bank[:3], n_max=x.size) as plan:
        plan.status()
        fd.fdas_selftest_wait_timeout(plan.handle, 5.0)
        with pytest.raises(fd.FdasError) as e:
            plan.status()
        assert e.value.code == fd.fdas.FDAS_ERR_TIMEOUT
        plan.status()                                    # read and cleared
        p = _run(fd, plan, x)
    compare(p, oracle_mod.direct_power(x, bank[:3]), TOL_FP32)


@pytest.mark.slow
def test_plane_beyond_2_31_elements(fd, oracle_mod, bank):
    # 85 x (2^27 + 12345) plane = 45.6 GB: row offsets past 2^31 elements, a ragged last segment;
    # sampled points (including the last rows and bins) against Eq. (1)
    n = (1 << 27) + 12345
    g = torch.Generator().manual_seed(61)
    xc = torch.complex(torch.randn(n, generator=g), torch.randn(n, generator=g)).to(torch.complex64)
    with fd.Plan(bank, n_max=n) as plan:
        xd = xc.cuda()
        out = plan.convolve(xd)
        plan.status()
        rng = np.random.default_rng(62)
        zi = np.concatenate([rng.integers(0, 85, 1500), np.full(250, 84), np.full(250, 83)])
        ii = np.concatenate([rng.integers(0, n, 1500), n - 1 - np.arange(250), rng.integers(n - 5000, n, 250)])
        got = out[torch.from_numpy(zi).cuda(), torch.from_numpy(ii).cuda()].cpu().numpy()
        scale = float(out.max().item())
        del out, xd
    torch.cuda.empty_cache()
    ref = oracle_mod.direct_points(xc.numpy(), bank, zi, ii)
    assert np.max(np.abs(got - ref)) <= TOL_FP32 * scale
