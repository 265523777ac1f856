"""The allocation-free batched entry point, fdas_convolve_batch_noalloc.

Callers such as a real-time dedispersion pipeline cannot afford a cudaMalloc (slow)
or a cudaFree (synchronises the device) while they run, and some processes hand all
device memory to another allocator up front.  For them the library offers a batched
call that allocates nothing and keeps its work counters in a fixed device array.
This test checks, through the C ABI, that two calls in a row give the same planes as
the ordinary batched call (within the FP32 tolerance used by the parity tests), and
that a batch above the documented limit is refused with a clear message.  It lives in
its own file so that pytest collects it last.
"""
import numpy as np
import pytest

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


def _inputs(ns, seed):
    rng = np.random.default_rng(seed)
    return [torch.from_numpy((rng.standard_normal(n) + 1j * rng.standard_normal(n)).astype(np.complex64)).cuda()
            for n in ns]


@pytest.mark.parametrize("G", [17, 0])     # 0: templates per block chosen per launch
def test_noalloc_batch_matches_batch_twice(fd, G):
    import synth
    bank = synth.template_bank()[0]
    ns = [1, 1629, 7000, 33333, 4096, 12]
    with fd.Plan(bank, n_max=max(ns), tpl_per_cta=G) as plan:
        for call in range(2):                           # two calls in a row share the counters
            xs = _inputs(ns, seed=40 + call)
            ref = plan.convolve_batch(xs)               # the existing entry point
            outs = [torch.full((85, n), float("nan"), device="cuda") for n in ns]
            fd.fdas_convolve_batch_noalloc(plan.handle, [x.data_ptr() for x in xs], ns,
                                           [o.data_ptr() for o in outs])
            plan.status()
            for o, r in zip(outs, ref):
                compare(o.cpu().numpy(), r.cpu().numpy(), TOL_FP32)


def test_noalloc_rejects_batches_above_the_limit(fd):
    import synth
    bank = synth.template_bank()[0][:2]
    with fd.Plan(bank, n_max=64) as plan:
        x = torch.zeros(64, dtype=torch.complex64, device="cuda")
        out = torch.full((2, 64), -1.0, device="cuda")
        count = 64 * 120 + 1
        with pytest.raises(fd.FdasError) as e:
            fd.fdas_convolve_batch_noalloc(plan.handle, [x.data_ptr()] * count, [64] * count,
                                           [out.data_ptr()] * count)
        assert e.value.code == fd.fdas.FDAS_ERR_INVALID_ARG
        assert "7680" in str(e.value)
        torch.cuda.synchronize()
        assert torch.all(out == -1.0)                   # nothing ran
        plan.status()
