"""GPU tests of the served form (continuous batching with admission by plane memory)."""
import threading
import time

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
    return torch.from_numpy((rng.standard_normal(n) + 1j * rng.standard_normal(n)).astype(np.complex64)).cuda()


@pytest.mark.parametrize("G", [17, 0])     # 0: templates per block chosen per batch
def test_result_same_alone_and_in_the_mix(fd, oracle_mod, bank, G):
    x_np = synth.make_input(synth.single_small(n=40000, seed=21))
    x = torch.from_numpy(x_np).cuda()
    with fd.Plan(bank, n_max=1 << 18, tpl_per_cta=G) as plan:
        single = plan.convolve(x).clone()
        with fd.Server(plan, budget_bytes=2 << 30, lanes=3, max_batch=8) as srv:
            t = srv.submit(x)
            alone = srv.wait(t, n=x.numel()).clone()
            srv.release(t)
            # the mix: 40 other arrays arrive from another thread while ours is in the middle
            others = [_rand(int(n), 300 + i) for i, n in enumerate(np.random.default_rng(5).integers(1, 1 << 18, 40))]
            tickets = {}

            def producer():
                for i, o in enumerate(others):
                    tickets[i] = srv.submit(o)
                    if i == 20:
                        tickets["x"] = srv.submit(x)
                    time.sleep(0.0005)
            th = threading.Thread(target=producer)
            th.start()
            th.join()
            mixed = srv.wait(tickets["x"], n=x.numel()).clone()
            other_planes = {}
            for i, o in enumerate(others):
                other_planes[i] = srv.wait(tickets[i], n=o.numel()).clone()
            for tk in tickets.values():
                srv.release(tk)
            st = srv.stats()
        plan.status()
        assert st["completed"] == 42 and st["launches"] >= 2
        # same bits alone, in the mix and through the single-array entry point
        assert torch.equal(alone, mixed) and torch.equal(alone, single)
        for i in (0, 20, 39):
            assert torch.equal(other_planes[i], plan.convolve(others[i]))
    compare(mixed.cpu().numpy(), oracle_mod.ols_power(x_np, bank), TOL_FP32)


def test_admission_waits_under_a_small_budget(fd, bank):
    n = 30000
    plane = 85 * n * 4
    with fd.Plan(bank, n_max=n) as plan:
        with fd.Server(plan, budget_bytes=2 * plane + 4096, lanes=2, max_batch=4) as srv:
            xs = [_rand(n, 40 + i) for i in range(10)]
            ref = [plan.convolve(x) for x in xs]
            tickets = [srv.submit(x) for x in xs]
            st = srv.stats()
            assert st["queued"] >= 8 and st["admission_waits"] >= 8
            for tk, r, x in zip(tickets, ref, xs):
                got = srv.wait(tk, timeout_ms=20000, n=n)
                assert torch.equal(got, r)
                srv.release(tk)              # frees memory: the next request is admitted
            st = srv.stats()
            assert st["completed"] == 10 and st["peak_bytes_in_use"] <= 2 * plane + 4096
            assert st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]
        plan.status()


def test_rejection_timeout_and_busy(fd, bank):
    n = 20000
    plane = 85 * n * 4
    with fd.Plan(bank, n_max=n) as plan:
        with fd.Server(plan, budget_bytes=plane + 1024, lanes=1) as srv:
            with fd.Server(plan, budget_bytes=plane // 2) as small:
                with pytest.raises(fd.FdasError) as e:  # its plane can never fit: rejected at once
                    small.submit(_rand(n, 1))
                assert e.value.code == fd.fdas.FDAS_ERR_REJECTED
                assert small.stats()["rejected"] == 1
            a, b = _rand(n, 2), _rand(n, 3)
            ta = srv.submit(a)
            tb = srv.submit(b)                           # waits for a's memory
            srv.wait(ta, timeout_ms=20000)
            with pytest.raises(fd.FdasError) as e:       # b cannot run until a is released
                srv.wait(tb, timeout_ms=50)
            assert e.value.code == fd.fdas.FDAS_ERR_TIMEOUT
            with pytest.raises(fd.FdasError) as e:
                srv.release(tb)
            assert e.value.code == fd.fdas.FDAS_ERR_BUSY
            srv.release(ta)
            got = srv.wait(tb, timeout_ms=20000, n=n)
            assert torch.equal(got, plan.convolve(b))
            srv.release(tb)
            with pytest.raises(fd.FdasError):
                srv.release(tb)                          # unknown ticket now
        plan.status()
