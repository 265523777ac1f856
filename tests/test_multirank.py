"""Two gloo ranks on the CPU: the benchmark's replica logic (no GPU, no data exchange)."""
import importlib.util
import os
import socket

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        b = _bench()
        elapsed = 1.0 + 0.5 * rank                    # the slower rank sets the job time
        m = b.max_over_ranks(elapsed)
        spec = b.rank_array_spec(rank, log2n=12)
        q.put((rank, m, spec.seed, spec.n, b.aggregate_rate(world, 10, m)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_replicas():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    assert [r[1] for r in res] == [1.5, 1.5]                 # MAX over ranks
    assert res[0][2] != res[1][2] and res[0][3] == res[1][3] == 4096   # each rank its own array
    assert res[0][4] == pytest.approx(2 * 10 / 1.5)          # whole-job rate


def test_single_process_helpers():
    b = _bench()
    assert b.max_over_ranks(3.25) == 3.25
    assert b.aggregate_rate(1, 200, 0.2) == pytest.approx(1000.0)
    assert b.algorithmic_bytes(1 << 22, 85) == 348 * (1 << 22)
