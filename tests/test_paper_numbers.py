"""The benchmark's operation and byte accounting against numbers the paper prints."""
import importlib.util
import json
import math
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLD = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_workload.json")))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_requirement_model():
    r = GOLD["requirement"]
    t_limit = r["integration_s"] / r["dm_trials"]
    assert t_limit * 1e3 == pytest.approx(r["t_limit_ms"], abs=0.05)
    # direct-form rate 8 N K M / t_limit (one complex MAC = 8 operations)
    assert 8 * r["N"] * r["K"] * r["M"] / t_limit / 1e12 == pytest.approx(r["required_tflops"], abs=0.01)


@pytest.mark.parametrize("name", ["AOLS-2048", "AOLS-4096"])
def test_table2_clock_model(name):
    # theoretical latency: two engine passes (forward, inverse) of ceil(N / (N_FT - K)) segments,
    # N_FT / N_FT_PC clocks each, at f_max
    t = GOLD["table2_theoretical_latency_ms"]
    k = t[name]
    n, K = GOLD["requirement"]["N"], GOLD["requirement"]["K"]
    cycles = 2 * math.ceil(n / (k["N_FT"] - K)) * k["N_FT"] / t["N_FT_PC"]
    assert cycles / (k["fmax_mhz"] * 1e6) * 1e3 == pytest.approx(k["latency_ms"], rel=0.005)


def test_bench_operation_count_follows_table1():
    b = _bench()
    n, K, C = GOLD["requirement"]["N"], GOLD["requirement"]["K"], GOLD["table1"]["C"]
    L, M = 2048, 85
    # Table 1, OLS-FD, average over M filters: ceil(N/(N_FT-K)) N_FT (6 + C log2 N_FT) per filter
    lg = math.log2(L)
    table1 = M * math.ceil(n / (L - K)) * L * (6 + C * lg)
    # ours = Table 1 with the exact overlap-save step S = L-K+1, plus the forward FFT that the
    # M filters share (one per segment) and the power |y|^2 (3 operations per output)
    nseg = math.ceil(n / (L - K + 1))
    ours = b.model_flops(n, M, L, K, c=C)
    assert ours == pytest.approx(M * nseg * L * (6 + C * lg) + nseg * L * C * lg + 3 * M * n, rel=1e-12)
    assert M * nseg * L * (6 + C * lg) == pytest.approx(table1, rel=1e-3)   # step off by one: 2577 vs 2578
    assert b.algorithmic_bytes(n, M) == 8 * n + 4 * M * n


def test_paper_throughput_for_vs_baseline():
    b = _bench()
    assert b.PAPER_ARRAYS_PER_S == pytest.approx(1e3 / GOLD["multi_fpga"]["latency_ms"])
