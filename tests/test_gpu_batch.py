"""GPU tests of the batched persistent form (fdas_convolve_batch) and the autotuner."""
import numpy as np
import pytest

import synth
from parity import TOL_FP32, TOL_TC, compare

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


@pytest.mark.parametrize("L,G", [(1024, 5), (2048, 17), (2048, 85), (4096, 85)])
def test_batch_equals_single_array_path(fd, oracle_mod, bank, L, G):
    ns = [1, 5, 1627, 1628, 1629, 4000, 9001, 20011, 3, 65536]
    xs = [torch.from_numpy(_rand(n, 100 + i)).cuda() for i, n in enumerate(ns)]
    with fd.Plan(bank, n_max=max(ns), seg_len=L, tpl_per_cta=G) as plan:
        outs = plan.convolve_batch(xs)
        singles = [plan.convolve(x) for x in xs]
        plan.status()
    for x, o, s in zip(xs, outs, singles):
        assert torch.equal(o, s)          # same work items -> identical bits
    for i in (1, 4, 7):                   # and against the oracle
        x = xs[i].cpu().numpy()
        compare(outs[i].cpu().numpy(), oracle_mod.ols_power(x, bank), TOL_FP32)


def test_templates_per_block_chosen_per_call(fd, oracle_mod, bank):
    # tpl_per_cta = 0: all 85 templates per block for a full-size array, fewer for short
    # arrays (more blocks); the bits do not depend on the choice
    with fd.Plan(bank, n_max=1 << 22) as plan:
        assert plan.desc.tpl_per_cta == 0
        gs = [fd.fdas_plan_tpl_per_cta(plan.handle, 1 << k) for k in range(10, 23)]
        assert gs[-1] == 85 and gs[0] == 5
        assert all(a <= b for a, b in zip(gs, gs[1:]))           # non-decreasing in n
        ns = [1, 3000, 1 << 16, 300000]
        xs = [torch.from_numpy(_rand(n, 800 + n)).cuda() for n in ns]
        outs = plan.convolve_batch(xs)
        singles = [plan.convolve(x) for x in xs]
        plan.status()
    with fd.Plan(bank, n_max=1 << 22, tpl_per_cta=85) as fixed:
        assert fd.fdas_plan_tpl_per_cta(fixed.handle, 1 << 10) == 85
        ref = [fixed.convolve(x) for x in xs]
        fixed.status()
    for o, s, r in zip(outs, singles, ref):
        assert torch.equal(o, s) and torch.equal(s, r)
    compare(singles[2].cpu().numpy(), oracle_mod.ols_power(xs[2].cpu().numpy(), bank), TOL_FP32)


def test_batch_more_than_one_table(fd, oracle_mod, bank):
    # more arrays than fit one kernel-parameter table (120): several graph replays
    ns = [(37 * i) % 3001 + 1 for i in range(130)]
    xs = [torch.from_numpy(_rand(n, 500 + i)).cuda() for i, n in enumerate(ns)]
    hs = bank[::17]
    with fd.Plan(hs, n_max=max(ns), tpl_per_cta=2) as plan:
        outs = plan.convolve_batch(xs)
        plan.status()
    for i in (0, 64, 119, 120, 129):
        x = xs[i].cpu().numpy()
        compare(outs[i].cpu().numpy(), oracle_mod.direct_power(x, hs), TOL_FP32)


def test_persistent_grid_fills_the_gpu(fd, bank):
    # the persistent kernel runs one block per resident slot: several per SM
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    for L, per_sm in ((1024, 4), (2048, 4), (4096, 2)):
        with fd.Plan(bank, n_max=1 << 16, seg_len=L) as plan:
            assert plan.desc.batch_blocks == per_sm * sms, (L, plan.desc.batch_blocks)


def test_batch_empty_and_invalid(fd, bank):
    with fd.Plan(bank[:3], n_max=1000) as plan:
        plan.convolve_batch([])
        x = torch.zeros(500, dtype=torch.complex64, device="cuda")
        out = torch.full((3, 500), -1.0, device="cuda")
        big = torch.zeros(2000, dtype=torch.complex64, device="cuda")
        with pytest.raises(fd.FdasError) as e:
            fd.fdas_convolve_batch(plan.handle, [x.data_ptr(), big.data_ptr()], [500, 2000],
                                   [out.data_ptr(), out.data_ptr()])
        assert e.value.code == fd.fdas.FDAS_ERR_INVALID_ARG
        torch.cuda.synchronize()
        assert torch.all(out == -1.0)     # nothing was enqueued
        plan.status()


def test_repeated_batches_reuse_graph(fd, bank):
    # consecutive replays with different tables must not see stale parameters
    with fd.Plan(bank[::10], n_max=50000) as plan:
        a = [torch.from_numpy(_rand(n, 7 + n)).cuda() for n in (1000, 50000, 1)]
        b = [torch.from_numpy(_rand(n, 9 + n)).cuda() for n in (30000, 17)]
        oa = plan.convolve_batch(a)
        ob = plan.convolve_batch(b)
        oa2 = plan.convolve_batch(a)
        plan.status()
        for x, o, o2 in zip(a, oa, oa2):
            assert torch.equal(o, o2) and torch.equal(o, plan.convolve(x))
        for x, o in zip(b, ob):
            assert torch.equal(o, plan.convolve(x))


def test_autotuner(fd, oracle_mod, bank):
    # candidates (L, G) with G = 0 the per-call choice, timed on a proxy batch of 16 arrays with
    # lengths log-uniform in [tune_n_min, n_max]
    with fd.Plan(bank, n_max=1 << 17, autotune=1, tune_n_min=1 << 13) as plan:
        d = plan.desc
        assert d.tuned == 1 and d.precision == fd.FDAS_PREC_FP32
        assert d.seg_len in (1024, 2048, 4096) and d.tpl_per_cta in (0, 5, 17, 85)
        ms = np.array(d.tune_ms[:])
        assert np.all(ms > 0) and d.tune_ms_tc == 0   # every FP32 candidate ran, no tensor-core one
        idx = [1024, 2048, 4096].index(d.seg_len) * 4 + [0, 5, 17, 85].index(d.tpl_per_cta)
        assert ms[idx] == ms.min()
        x = synth.make_input(synth.single_small(n=30000, seed=3))
        out = plan.convolve(torch.from_numpy(x).cuda())
        plan.status()
    compare(out.cpu().numpy(), oracle_mod.ols_power(x, bank), TOL_FP32)
    # a second plan with the same shape reuses the cached choice
    with fd.Plan(bank, n_max=1 << 17, autotune=1, tune_n_min=1 << 13) as plan2:
        assert (plan2.desc.seg_len, plan2.desc.tpl_per_cta) == (d.seg_len, d.tpl_per_cta)


def test_autotuner_with_precision(fd, oracle_mod, bank):
    # mode 2 adds the two-stage tensor-core form: whichever wins, the plan computes a correct
    # plane at the tolerance of the chosen form, batched and single
    with fd.Plan(bank, n_max=1 << 18, autotune=2) as plan:
        d = plan.desc
        assert d.tuned == 1 and d.tune_ms_tc > 0
        best_fp32 = min(v for v in d.tune_ms[:] if v > 0)
        if d.precision == fd.FDAS_PREC_TC_DFT2:
            assert d.tune_ms_tc <= best_fp32 and d.seg_len == 2048
        else:
            assert d.precision == fd.FDAS_PREC_FP32 and best_fp32 <= d.tune_ms_tc
        x = synth.make_input(synth.single_small(n=70000, seed=4))
        xd = torch.from_numpy(x).cuda()
        out = plan.convolve(xd)
        outb = plan.convolve_batch([xd])[0]
        plan.status()
        assert torch.equal(out, outb)
    tol = TOL_TC if d.precision == fd.FDAS_PREC_TC_DFT2 else TOL_FP32
    compare(out.cpu().numpy(), oracle_mod.ols_power(x, bank), tol)


@pytest.mark.slow
def test_dedispersion_batch_sampled_vs_oracle(fd, oracle_mod, bank):
    # 64 trials with log-uniform lengths in [2^18, 2^22] (about 31 GB of planes), one chirp each
    specs = synth.batch_trials()
    xs_np = [synth.make_input(s) for s in specs]
    xs = [torch.from_numpy(x).cuda() for x in xs_np]
    with fd.Plan(bank, n_max=1 << 22) as plan:
        outs = plan.convolve_batch(xs)
        plan.status()
        for i in (0, 17, 63):               # bitwise equal to the single-array path
            assert torch.equal(outs[i], plan.convolve(xs[i]))
    rng = np.random.default_rng(77)
    for i in range(0, 64, 7):
        n = xs_np[i].size
        zi = rng.integers(0, 85, 300)
        ii = np.concatenate([rng.integers(0, n, 250), np.arange(25), n - 1 - np.arange(25)])
        got = outs[i][torch.from_numpy(zi).cuda(), torch.from_numpy(ii).cuda()].cpu().numpy()
        ref = oracle_mod.direct_points(xs_np[i], bank, zi, ii)
        c = specs[i].chirps[0]
        peak_row = 42 + int(c.z)
        scale = max(float(outs[i][peak_row].max().item()), ref.max())
        assert np.max(np.abs(got - ref)) <= TOL_FP32 * scale
