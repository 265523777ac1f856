"""GPU parity of the tensor-core forms against the FP64 oracle: the radix-16 DFT-GEMM pass
(FDAS_PREC_TC_FP16) and the two-stage form that takes the whole inverse FFT
(FDAS_PREC_TC_DFT2)."""
import numpy as np
import pytest

import synth
from parity import THRESHOLD_GAUSS, TOL_TC, compare

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


@pytest.fixture(scope="module", params=["tc_fp16", "tc_dft2"])
def prec(request, fd):
    return {"tc_fp16": fd.FDAS_PREC_TC_FP16, "tc_dft2": fd.FDAS_PREC_TC_DFT2}[request.param]


def _run(plan, x):
    out = plan.convolve(torch.from_numpy(np.ascontiguousarray(x)).cuda())
    plan.status()
    return out.cpu().numpy()


def test_small_array_vs_direct(fd, oracle_mod, bank, prec):
    x = synth.make_input(synth.single_small())
    with fd.Plan(bank, n_max=x.size, precision=prec) as plan:
        assert plan.desc.precision == prec
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
def test_ragged_and_groups(fd, oracle_mod, bank, prec, n, G):
    rng = np.random.default_rng(n * 3 + G)
    x = (rng.standard_normal(n) + 1j * rng.standard_normal(n)).astype(np.complex64)
    hs = bank[::4] if G != 85 else bank
    with fd.Plan(hs, n_max=max(n, 16), tpl_per_cta=min(G, hs.shape[0]), precision=prec) as plan:
        p = _run(plan, x)
    # fp16 data round relative to the segment's energy, which includes the outputs past n
    # that overlap-save computes and discards: only for arrays shorter than a template
    # (n < K, where the kept outputs are a small part of that energy) is the tolerance taken
    # against the maximum of the untruncated convolution; otherwise against max(P_ref)
    ref = oracle_mod.direct_power(x, hs)
    scale = None
    if n < hs.shape[1]:
        full = oracle_mod.direct_power(np.concatenate([x, np.zeros(hs.shape[1] - 1, np.complex64)]), hs)
        scale = float(full.max())
    compare(p, ref, TOL_TC, scale=scale)


@pytest.mark.parametrize("log2n", [18, 20])
def test_noise_candidates_elementwise(fd, oracle_mod, bank, prec, log2n):
    # noise only: max(P_ref) is about ln(85 N), so 2e-3 max(P_ref) is far below T = 7 and the
    # candidate rule is tested cell by cell (the band around T holds a handful of points)
    x = synth.make_input(synth.ArraySpec(n=1 << log2n, seed=40 + log2n))
    with fd.Plan(bank, n_max=x.size, precision=prec) as plan:
        p = _run(plan, x)
    ref = oracle_mod.ols_power(x, bank, L=2048)
    info = compare(p, ref, TOL_TC)
    assert TOL_TC * info["scale"] < 7.0 and info["candidates"] > 1000, info
    compare(p, ref, TOL_TC, threshold=THRESHOLD_GAUSS)


@pytest.mark.parametrize("k", [1, 2, 64, 421, 1000, 2044])
def test_template_lengths(fd, oracle_mod, prec, k):
    rng = np.random.default_rng(k + 7)
    n = 6000
    x = (rng.standard_normal(n) + 1j * rng.standard_normal(n)).astype(np.complex64)
    h = ((rng.standard_normal((3, k)) + 1j * rng.standard_normal((3, k))) / np.sqrt(2 * k)).astype(np.complex64)
    with fd.Plan(h, n_max=n, precision=prec) as plan:
        p = _run(plan, x)
    compare(p, oracle_mod.direct_power(x, h), TOL_TC)


def test_unsupported_options(fd, bank, prec):
    for kw in (dict(seg_len=1024), dict(seg_len=4096), dict(autotune=1)):
        with pytest.raises(fd.FdasError) as e:
            fd.Plan(bank, n_max=1000, precision=prec, **kw)
        assert e.value.code == fd.fdas.FDAS_ERR_UNSUPPORTED


@pytest.mark.slow
def test_ska_array_vs_ols_oracle(fd, oracle_mod, bank, prec):
    spec = synth.single_ska()
    x = synth.make_input(spec)
    with fd.Plan(bank, n_max=x.size, precision=prec) as plan:
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


def test_batched_forms_reject_the_single_pass_form(fd, bank):
    # the batched, allocation-free and served entry points have no kernel for the single-pass
    # tensor-core form: such a plan is refused before anything is enqueued (the outputs keep
    # their sentinel)
    n = 5000
    x = torch.from_numpy((np.arange(n) % 7 - 3).astype(np.complex64)).cuda()
    out = torch.full((bank.shape[0], n), -1.0, dtype=torch.float32, device="cuda")
    with fd.Plan(bank, n_max=n, precision=fd.FDAS_PREC_TC_FP16) as plan:
        for call in (fd.fdas_convolve_batch, fd.fdas_convolve_batch_noalloc):
            with pytest.raises(fd.FdasError) as e:
                call(plan.handle, [x.data_ptr()], [n], [out.data_ptr()])
            assert e.value.code == fd.fdas.FDAS_ERR_UNSUPPORTED
        with pytest.raises(fd.FdasError) as e:
            fd.fdas_server_create(plan.handle, 1 << 28)
        assert e.value.code == fd.fdas.FDAS_ERR_UNSUPPORTED
        torch.cuda.synchronize()
    assert bool((out == -1.0).all())


@pytest.mark.parametrize("gain", [1e-9, 1e-3, 1.0, 1e4])
def test_dft2_input_scale(fd, oracle_mod, bank, gain):
    # the two-stage form scales each segment's spectrum by a power of two before the fp16
    # operands: the relative error does not depend on the input's magnitude
    x = (synth.make_input(synth.single_small(n=9000, seed=3)) * np.float32(gain)).astype(np.complex64)
    with fd.Plan(bank, n_max=x.size, precision=fd.FDAS_PREC_TC_DFT2) as plan:
        p = _run(plan, x)
    ref = oracle_mod.direct_power(x, bank)
    info = compare(p, ref, TOL_TC, threshold=7.0 * gain * gain)
    assert info["rel"] < 1e-3, info


def test_dft2_zero_and_host_path(fd, oracle_mod, bank):
    # an all-zero array gives an all-zero plane; the host-buffer path (chunked launches over
    # segment ranges) gives the same bits as the device path
    with fd.Plan(bank, n_max=40000, precision=fd.FDAS_PREC_TC_DFT2) as plan:
        z = _run(plan, np.zeros(5000, np.complex64))
        assert not np.any(z)
        x = synth.make_input(synth.single_small(n=40000, seed=9))
        dev = _run(plan, x)
        host = plan.convolve_host(x)
    assert np.array_equal(dev, host)
    compare(dev, oracle_mod.ols_power(x, bank, L=2048), TOL_TC)


@pytest.mark.parametrize("m", [1, 2, 3, 85, 130])
def test_dft2_template_counts(fd, oracle_mod, m):
    # odd counts leave the second template of the last pair empty; more templates than the
    # synthetic bank use random unit-energy taps
    rng = np.random.default_rng(m)
    n, k = 7000, 200
    x = (rng.standard_normal(n) + 1j * rng.standard_normal(n)).astype(np.complex64)
    h = ((rng.standard_normal((m, k)) + 1j * rng.standard_normal((m, k))) / np.sqrt(2 * k)).astype(np.complex64)
    with fd.Plan(h, n_max=n, precision=fd.FDAS_PREC_TC_DFT2) as plan:
        p = _run(plan, x)
    compare(p, oracle_mod.direct_power(x, h), TOL_TC)


def _rand_dev(n, seed):
    rng = np.random.default_rng(seed)
    return torch.from_numpy((rng.standard_normal(n) + 1j * rng.standard_normal(n)).astype(np.complex64)).cuda()


def test_dft2_batch_noalloc_and_single_agree(fd, oracle_mod, bank):
    # the persistent batch kernel of the two-stage form runs the same items and arithmetic per
    # array as the single-array kernel: bit-identical planes, through the graph-replayed lane
    # and through the allocation-free entry point
    ns = [1, 5, 1627, 1628, 1629, 4000, 9001, 20011, 3, 65536, 300001]
    xs = [_rand_dev(n, 900 + i) for i, n in enumerate(ns)]
    with fd.Plan(bank, n_max=max(ns), precision=fd.FDAS_PREC_TC_DFT2) as plan:
        outs = plan.convolve_batch(xs)
        singles = [plan.convolve(x) for x in xs]
        na = [torch.full_like(o, -1.0) for o in outs]
        for rep in range(2):
            fd.fdas_convolve_batch_noalloc(plan.handle, [x.data_ptr() for x in xs], ns, [o.data_ptr() for o in na])
            plan.status()
            for o, s in zip(na, singles):
                assert torch.equal(o, s)
    for o, s in zip(outs, singles):
        assert torch.equal(o, s)
    for i in (2, 5, 7, 10):   # n >= K: the tolerance against max(P_ref) applies (see test_ragged_and_groups)
        x = xs[i].cpu().numpy()
        compare(outs[i].cpu().numpy(), oracle_mod.ols_power(x, bank), TOL_TC)


def test_dft2_served_same_alone_and_in_the_mix(fd, oracle_mod, bank):
    x_np = synth.make_input(synth.single_small(n=40000, seed=21))
    x = torch.from_numpy(x_np).cuda()
    with fd.Plan(bank, n_max=1 << 18, precision=fd.FDAS_PREC_TC_DFT2) as plan:
        single = plan.convolve(x).clone()
        with fd.Server(plan, budget_bytes=2 << 30, lanes=3, max_batch=8) as srv:
            t = srv.submit(x)
            alone = srv.wait(t, n=x.numel()).clone()
            srv.release(t)
            others = [_rand_dev(int(n), 700 + i) for i, n in enumerate(np.random.default_rng(6).integers(1, 1 << 18, 24))]
            tickets = [srv.submit(o) for o in others[:12]]
            tx = srv.submit(x)
            tickets += [srv.submit(o) for o in others[12:]]
            mixed = srv.wait(tx, n=x.numel()).clone()
            srv.release(tx)
            planes = [srv.wait(tk, n=o.numel()).clone() for tk, o in zip(tickets, others)]
            for tk in tickets:
                srv.release(tk)
        plan.status()
        assert torch.equal(alone, mixed) and torch.equal(alone, single)
        for i in (0, 11, 23):
            assert torch.equal(planes[i], plan.convolve(others[i]))
    compare(mixed.cpu().numpy(), oracle_mod.ols_power(x_np, bank), TOL_TC)


@pytest.mark.parametrize("n", [135_000, 137_000, 138_743, 301_000])
def test_dft2_work_shares(fd, oracle_mod, bank, n):
    # around the switch between whole template-pair groups per item (short arrays) and equal
    # shares of (segment pair, template pair) units per block: odd and even segment counts,
    # shares that start and end inside a segment pair; bits equal to the batched form, which
    # always shares units out
    rng = np.random.default_rng(n)
    x = (rng.standard_normal(n) + 1j * rng.standard_normal(n)).astype(np.complex64)
    xd = torch.from_numpy(x).cuda()
    with fd.Plan(bank, n_max=n, precision=fd.FDAS_PREC_TC_DFT2) as plan:
        p = plan.convolve(xd)
        other = torch.from_numpy(np.ascontiguousarray(x[: n // 3])).cuda()
        outs = plan.convolve_batch([other, xd])
        plan.status()
    assert torch.equal(outs[1], p)
    compare(p.cpu().numpy(), oracle_mod.ols_power(x, bank), TOL_TC)


@pytest.mark.parametrize("precision", ["fp32", "tc_dft2"])
def test_relaunches_bit_identical(fd, bank, precision):
    # the plane of one input is the same bits on every launch: a handoff between the warp roles
    # that let a consumer read a tile before its producer had written it shows up here as one
    # (segment, template) tile that differs in some launches (about one in a hundred at this size)
    prec = {"fp32": fd.FDAS_PREC_FP32, "tc_dft2": fd.FDAS_PREC_TC_DFT2}[precision]
    n = 1 << 22
    x = _rand_dev(n, 4242)
    with fd.Plan(bank, n_max=n, precision=prec) as plan:
        first = plan.convolve(x)
        again = torch.full_like(first, -1.0)
        differing = []
        for rep in range(300):
            plan.convolve(x, out=again)
            if not torch.equal(again, first):
                differing.append(rep)
        plan.status()
    assert not differing, f"launches whose plane differs from the first: {differing}"


def test_dft2_batch_and_threshold_relaunches_stable(fd, bank):
    # the same for the other two instantiations of the two-stage body: the persistent batch
    # kernel (units of several arrays shared out per block) and the threshold epilogue (the
    # records come in launch-dependent order: compared as sorted sets)
    ns = [1 << 21, (1 << 20) + 12345, 300001]
    xs = [_rand_dev(n, 5150 + i) for i, n in enumerate(ns)]
    with fd.Plan(bank, n_max=max(ns), precision=fd.FDAS_PREC_TC_DFT2) as plan:
        first = [o.clone() for o in plan.convolve_batch(xs)]
        outs = [torch.full_like(o, -1.0) for o in first]
        differing = []
        for rep in range(100):
            plan.convolve_batch(xs, outs=outs)
            if not all(torch.equal(o, f) for o, f in zip(outs, first)):
                differing.append(rep)
        assert not differing, f"batch launches whose planes differ from the first: {differing}"

        def records():   # noise of mean power 2 through unit-norm templates: ~160k crossings of 14
            buf, count = plan.candidates(xs[0], threshold=14.0, max_cand=1 << 20)
            assert int(count.item()) < buf.shape[0]   # none dropped, so the set is launch-independent
            c = fd.candidates_to_numpy(buf, count)
            return c[np.lexsort((c["bin"], c["tpl"]))]

        ref = records()
        assert ref.size > 10000
        for rep in range(30):
            np.testing.assert_array_equal(records(), ref)
        plan.status()
