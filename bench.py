#!/usr/bin/env python3
"""Benchmark: FDAS power planes per second on GB300 (one array of 2^22 complex64 bins,
85 templates of up to 421 taps, overlap-save with 2048-point segments, float32 plane).

One step = one full power plane (fdas_convolve: forward FFT per segment, 85 products,
inverse FFTs, discard, power, store).  Prints ONE JSON line on rank 0.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl fdas|reference]

--impl reference times the FP64 CPU oracle (the only reference this method has) on a
bounded sample of the same workload.  Under torchrun each rank processes its own
array (weak scaling, replicas: no data-path collective); rank 0 prints.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "FDAS arrays/s (85 x 2^22 float32 power plane)"
UNIT = "arrays/s"
FALLBACK_HBM_GBS = 6800.0
# Paper: three Stratix V A7 boards apply 84 x 421-tap filters to 2^22 points in
# 120 ms (Sec. 6, multiple FPGAs) -> 1 / 0.120 arrays/s.  Another machine: context.
PAPER_ARRAYS_PER_S = 1.0 / 0.120


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def local_index(dev) -> int:
    return dev.index if getattr(dev, "index", None) is not None else 0


def rank_array_spec(rank: int, log2n: int = 22):
    """Each rank processes its own dedispersion trial (replicas: no data exchange)."""
    return synth.single_ska(n=1 << log2n, seed=1 + rank)


def max_over_ranks(value: float, device=None) -> float:
    """MAX of a per-rank float over the process group (identity without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    dev = device if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(world: int, units_per_rank: int, max_elapsed_s: float) -> float:
    """Whole-job throughput: the units all ranks processed / the slowest rank's time."""
    return world * units_per_rank / max_elapsed_s


def gpu_local_cpus(device_index: int):
    """CPUs the kernel lists as local to the GPU's PCI function (None if unknown)."""
    import torch
    try:
        pr = torch.cuda.get_device_properties(device_index)
        bus = f"{pr.pci_domain_id:04x}:{pr.pci_bus_id:02x}:{pr.pci_device_id:02x}.0"
        with open(f"/sys/bus/pci/devices/{bus}/local_cpulist") as f:
            text = f.read().strip()
    except Exception:
        return None
    cpus = set()
    for part in text.split(","):
        if "-" in part:
            a, b = part.split("-")
            cpus.update(range(int(a), int(b) + 1))
        elif part:
            cpus.add(int(part))
    return sorted(cpus) or None


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def algorithmic_bytes(n: int, m: int) -> int:
    """Minimum HBM traffic of one plane: read the complex64 input once, write M*n floats."""
    return 8 * n + 4 * m * n


def model_flops(n: int, m: int, seg_len: int, tpl_len: int, c: float = 5.0) -> float:
    """Table 1 OLS-FD workload with C = 5 (Intel radix-4 engine count), M filters
    sharing one forward FFT per segment, plus the power (3 flops per point)."""
    import math
    nseg = math.ceil(n / (seg_len - tpl_len + 1))
    lg = math.log2(seg_len)
    return nseg * seg_len * (m * (6 + c * lg) + c * lg) + 3.0 * m * n


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not self.path:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) == 8:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(s):
            try:
                return float(s)
            except ValueError:
                return None
        sm = [num(r[0]) for r in rows if num(r[0]) is not None]
        mx = [num(r[1]) for r in rows if num(r[1]) is not None]
        pw = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[4 + i].lower().startswith("active")})
        loaded = [s for s in sm if mx and s >= 0.5 * max(mx)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(pw) if pw else None,
                "samples": len(rows), "reasons": reasons}


def time_oracle_sample(x, h, seg_len, target_s):
    """Time the FP64 overlap-save oracle on a prefix of the array sized for ~target_s."""
    import oracle
    oracle.build()
    n = x.size
    probe = min(n, 1 << 15)
    t0 = time.perf_counter()
    oracle.ols_power(x[:probe], h, L=seg_len)
    dt = time.perf_counter() - t0
    sample = int(min(n, max(probe, probe * target_s / max(dt, 1e-6))))
    runs, t0 = 0, time.perf_counter()
    while True:                       # repeat a whole-array sample until ~target_s of work
        oracle.ols_power(x[:sample], h, L=seg_len)
        runs += 1
        if time.perf_counter() - t0 >= target_s or sample < n:
            break
    dt = (time.perf_counter() - t0) / runs
    return sample, dt, oracle.threads(), runs


def time_oracle_harmonic(m, n_full, bin0, max_harm, thresholds, cols=1 << 20, seed=1):
    """Time the FP64 harmonic-sum oracle (C, OpenMP) on a seeded m x cols noise plane and
    scale to the m x n_full plane: the sums read a number of cells proportional to the plane."""
    import oracle
    oracle.build()
    P = synth.noise_plane(m, cols, seed)
    t0 = time.perf_counter()
    found = oracle.harmonic_candidates(P, bin0, max_harm, thresholds)
    dt = time.perf_counter() - t0
    per_array_s = dt * (n_full - 1 - bin0) / (cols - 1 - bin0)
    return {"value": 1.0 / per_array_s, "unit": "arrays/s", "cores": oracle.threads(), "kind": "oracle",
            "sample": f"FP64 harmonic-sum oracle (C, OpenMP) on a seeded {m} x {cols} noise plane "
                      f"({found['bin'].size} crossings, {dt:.2f} s), scaled by cells to {m} x {n_full}"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    spec = synth.single_ska()
    x = synth.make_input(spec)
    h, _ = synth.template_bank()
    n = x.size
    # size one step for about args.ref_step_seconds of oracle work
    probe = 1 << 14
    t0 = time.perf_counter()
    oracle.ols_power(x[:probe], h, L=args.seg_len)
    dt = time.perf_counter() - t0
    sample = int(min(n, max(probe, probe * args.ref_step_seconds / max(dt, 1e-6))))
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.ols_power(x[:sample], h, L=args.seg_len)
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    step = sum(times) / len(times)
    value = (sample / n) / step
    cores = oracle.threads()
    sample_desc = (f"FP64 overlap-save oracle on the first {sample} of {n} bins (85 templates, L={args.seg_len}) "
                   f"per step, scaled to whole arrays")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": step * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": value / PAPER_ARRAYS_PER_S, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args, n, h.shape[1]),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample_desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def workload_config(args, n, tpl_len):
    return {"workload": f"single SKA-sized array: N=2^{int(np.log2(n))} complex64, 85 templates (<= {tpl_len} taps), "
                        f"L={args.seg_len} overlap-save, {args.precision} segment FFTs, fp32 power plane",
            "n": n, "templates": 85, "tpl_len": tpl_len, "seg_len": args.seg_len,
            "tpl_per_cta": args.tpl_per_cta or "per call", "precision": args.precision,
            "l2": "no flush: each step writes the 1.43 GB plane (> 129 MB L2), evicting the 33.5 MB input"}


def run_fdas(args):
    import torch
    import paper_1805_12280_gb300 as fd

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    spec = rank_array_spec(rank, args.log2n)
    x = synth.make_input(spec)
    h, _ = synth.template_bank()
    n, m = x.size, h.shape[0]
    prec = {"tc": fd.FDAS_PREC_TC_FP16, "tc2": fd.FDAS_PREC_TC_DFT2}.get(args.precision, fd.FDAS_PREC_FP32)
    plan = fd.Plan(h, n_max=n, seg_len=args.seg_len, tpl_per_cta=args.tpl_per_cta, precision=prec)
    stream = torch.cuda.current_stream(dev)
    xd = torch.from_numpy(x).to(dev)
    out = torch.empty((m, n), dtype=torch.float32, device=dev)

    for _ in range(args.warmup):
        plan.convolve(xd, out, stream)
    plan.status(stream)
    torch.cuda.synchronize(dev)

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    gpu_index = int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[local]) \
        if os.environ.get("CUDA_VISIBLE_DEVICES", "").replace(",", "").isdigit() else local
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(gpu_index) as clocks:
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        for i in range(args.steps):
            ev[i][0].record(stream)
            plan.convolve(xd, out, stream)
            ev[i][1].record(stream)
        t_end.record(stream)
        torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    plan.status(stream)
    elapsed_ms = max_over_ranks(t_start.elapsed_time(t_end), dev)
    kern_ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
    ms_per_step = elapsed_ms / args.steps
    value = aggregate_rate(world, args.steps, elapsed_ms / 1e3)

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    e2e = None
    if not args.no_e2e:
        # host buffers on the NUMA node next to the GPU: run (and first-touch) on its local CPUs
        local = gpu_local_cpus(local_index(dev))
        saved_affinity = os.sched_getaffinity(0)
        if local and set(local) & saved_affinity:
            try:
                os.sched_setaffinity(0, set(local) & saved_affinity)
            except OSError:
                local = None
        else:
            local = None
        xh = torch.from_numpy(x).pin_memory()
        oh = torch.empty((m, n), dtype=torch.float32).pin_memory()
        xh_np, oh_np = xh.numpy(), oh.numpy()
        for _ in range(2):
            plan.convolve_host(xh_np, oh_np)
        ks = max(2, min(args.steps, 8))
        if world > 1:
            torch.distributed.barrier()
        t0 = time.perf_counter()
        for _ in range(ks):
            plan.convolve_host(xh_np, oh_np)
        dt = max_over_ranks(time.perf_counter() - t0, dev)
        e2e = {"value": aggregate_rate(world, ks, dt), "unit": UNIT, "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 4 * m * n,
               "steps": ks, "api": "fdas_convolve_host (pinned host buffers)",
               "host_cpus": f"{local[0]}-{local[-1]}" if local else "unrestricted"}
        os.sched_setaffinity(0, saved_affinity)   # the CPU baseline uses every core again
        del xh, oh

    peak, peak_kind = measured_peaks()
    alg = algorithmic_bytes(n, m)
    achieved = alg / (kern_ms / 1e3) / 1e9
    # the committed record is of the 2^22-bin, L = 2048, 85-template launch: other workloads get none
    same_workload = n == 1 << 22 and args.seg_len == 2048 and m == 85
    traffic = profile_traffic(args.precision) if same_workload else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "peak_kind": peak_kind,
                "kernel": {"fp32": f"ols_fp32_kernel<{args.seg_len}>", "tc": "ols_tc_kernel",
                           "tc2": "ols_tc2_kernel"}[args.precision],
                "algorithmic_bytes_per_launch": alg, "avg_launch_ms": kern_ms}

    # Second roofline: the paper's operation count (Table 1, C = 5) against the FP32 CUDA-core
    # peak of this GPU (SMs x 128 FP32 lanes x 2 flop per FMA x the sampled SM clock).
    flops = model_flops(n, m, args.seg_len, h.shape[1])
    roofline_alu = {"bound": "alu", "achieved": flops / (kern_ms / 1e3) / 1e12, "unit": "TFLOP/s",
                    "flops_per_launch": flops, "note": "paper operation count (Table 1, C=5); the kernel is "
                    "bound by FP32 instruction issue (see profiles/)"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sample, dt, cores, runs = time_oracle_sample(x, h, args.seg_len, args.cpu_seconds)
        cpu = {"value": (sample / n) / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"FP64 overlap-save oracle (C, OpenMP) on the first {sample} of {n} bins of the same array, "
                         f"85 templates, {runs} run(s) of {dt:.2f} s each, scaled to whole arrays"}

    forms = None
    if rank == 0 and world == 1 and not args.no_forms:
        del out
        torch.cuda.empty_cache()
        forms = {"tensor_core": bench_tc(fd, h, dev, xd), "candidates": bench_candidates(fd, h, dev, xd, x),
                 "harmonic_sum": bench_harmonic(fd, h, dev, xd, oracle_beside=not args.no_cpu_baseline),
                 "template_groups": bench_groups(fd, h, dev, xd),
                 "library_unfused_ols": bench_library_ols(h, dev, xd),
                 "full_fdfir": bench_fdfir(fd, h, dev, xd),
                 "library_full_fdfir": bench_library_fdfir(h, dev, xd),
                 "length_sweep": bench_length_sweep(fd, dev, xd),
                 "batched": bench_batch(fd, h, dev), "served": bench_serve(fd, h, dev)}

    link = host_link(dev) if rank == 0 and world == 1 and not args.no_e2e else None
    clock_summary = clocks.summary()
    sm_mhz = clock_summary.get("sm_mhz") or clock_summary.get("sm_max_mhz") or 2070.0
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    roofline_alu["peak"] = sms * 128 * 2 * sm_mhz * 1e6 / 1e12
    roofline_alu["sms"] = sms
    roofline_alu["frac"] = roofline_alu["achieved"] / roofline_alu["peak"]
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": value / PAPER_ARRAYS_PER_S, "dtype": "f32", "data": "synthetic",
                "config": workload_config(args, n, h.shape[1]),
                "tpl_per_cta_used": fd.fdas_plan_tpl_per_cta(plan.handle, n),
                "plane_gbs": 4.0 * m * n * world / (ms_per_step / 1e3) / 1e9,
                "model_tflops": model_flops(n, m, args.seg_len, h.shape[1]) * world / (ms_per_step / 1e3) / 1e12,
                "roofline": roofline, "roofline_alu": roofline_alu, "cpu_baseline": cpu, "e2e": e2e,
                "e2e_chain": ({"value": forms["candidates"]["e2e"]["arrays_per_s"], "unit": UNIT,
                               "h2d_bytes_per_step": forms["candidates"]["e2e"]["h2d_bytes"],
                               "d2h_bytes_per_step": forms["candidates"]["e2e"]["d2h_bytes"],
                               "api": "plane -> threshold candidates -> host (fdas_convolve_candidates)"}
                              if forms else None),
                "host_link": link,
                "roofline_tc": forms["tensor_core"]["tc_dft2"]["roofline"] if forms else None,
                "clocks": clock_summary,
                "forms": forms,
                "gpu_launches": args.steps,
                "vs_baseline_note": "paper: 3x Stratix V A7 FPGAs, 120 ms per 2^22 array, 84 filters (context)"}
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def _events_ms(fn, reps, stream):
    import torch
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def host_link(dev, nbytes=1 << 30, reps=5):
    """Pinned host <-> device copy rates (cudaMemcpyAsync through torch), GB/s: the ceiling of
    any end-to-end rate that moves the plane to the host."""
    import torch
    hbuf = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    dbuf = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    out = {"bytes": nbytes, "api": "torch copy_ (cudaMemcpyAsync), pinned host buffer"}
    for name, fn in (("h2d_gbs", lambda: dbuf.copy_(hbuf, non_blocking=True)),
                     ("d2h_gbs", lambda: hbuf.copy_(dbuf, non_blocking=True))):
        fn()
        ms = _events_ms(fn, reps, stream)
        out[name] = nbytes / (ms / 1e3) / 1e9
    del hbuf, dbuf
    torch.cuda.empty_cache()
    return out


def bench_tc(fd, h, dev, xd, reps=50):
    """Tensor-core form on the same array: radix-16 inverse passes as fp16 DFT-GEMMs
    (hi/lo DFT matrices, FP32 accumulation); beside it the FP32 kernel, same (L, G)."""
    import torch
    n, m = xd.numel(), h.shape[0]
    out = torch.empty((m, n), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    res = {"workload": "N=2^22, 85 templates, L=2048, G=85 (same array as the headline)"}
    for name, prec in (("tc_dft2", fd.FDAS_PREC_TC_DFT2), ("tc_fp16", fd.FDAS_PREC_TC_FP16), ("fp32", fd.FDAS_PREC_FP32)):
        with fd.Plan(h, n_max=n, precision=prec) as plan:
            for _ in range(3):
                plan.convolve(xd, out, stream)
            ms = _events_ms(lambda: plan.convolve(xd, out, stream), reps, stream)
            plan.status(stream)
        alg = algorithmic_bytes(n, m)
        res[name] = {"ms_per_array": ms, "arrays_per_s": 1e3 / ms,
                     "hbm_frac": alg / (ms / 1e3) / 1e9 / measured_peaks()[0]}
        if name == "tc_dft2":
            peak, peak_kind = measured_peaks()
            res[name]["roofline"] = {
                "bound": "hbm", "achieved": alg / (ms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                "frac": alg / (ms / 1e3) / 1e9 / peak,
                "traffic": profile_traffic("tc2") if n == 1 << 22 and m == 85 else None,
                "peak_kind": peak_kind, "kernel": "ols_tc2_kernel", "algorithmic_bytes_per_launch": alg,
                "avg_launch_ms": ms}
    res["accuracy"] = ("tests/test_gpu_tc.py: max |P - P_ref| / max P_ref < 1e-3 against the FP64 oracle "
                       "(tolerance 2e-3), strong-candidate sets identical")
    del out
    torch.cuda.empty_cache()
    return res


def bench_groups(fd, h, dev, xd, reps=50):
    """Templates grouped by support length (group_support=1): one launch per group, each with
    its own frame and step; beside it the ungrouped plan on the same array."""
    import torch
    n, m = xd.numel(), h.shape[0]
    out = torch.empty((m, n), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    res = {"workload": "N=2^22, 85 templates, L=2048, G=85 (same array as the headline)"}
    for name, grp in (("grouped", 1), ("ungrouped", 0)):
        with fd.Plan(h, n_max=n, group_support=grp) as plan:
            for _ in range(3):
                plan.convolve(xd, out, stream)
            ms = _events_ms(lambda: plan.convolve(xd, out, stream), reps, stream)
            plan.status(stream)
            res[name] = {"ms_per_array": ms, "arrays_per_s": 1e3 / ms, "launches": plan.desc.groups}
    del out
    torch.cuda.empty_cache()
    return res


def bench_candidates(fd, h, dev, xd, x_host, reps=50, threshold=7.0):
    """Fused threshold epilogue (fdas_convolve_candidates): same array, the plane is never
    written; end to end: pinned input -> device -> candidates -> host list.  The FP32 form
    (top-level keys) and the two-stage tensor-core form (`tensor_core`)."""
    import torch
    n = xd.numel()
    stream = torch.cuda.current_stream(dev)

    def run(precision, with_gauss):
        out = {}
        with fd.Plan(h, n_max=n, precision=precision) as plan:
            buf = torch.empty((1 << 22, 2), dtype=torch.int64, device=dev)
            cnt = torch.empty(1, dtype=torch.int64, device=dev)
            for _ in range(3):
                plan.candidates(xd, threshold, buf.shape[0], stream, buf, cnt)
            ms = _events_ms(lambda: plan.candidates(xd, threshold, buf.shape[0], stream, buf, cnt), reps, stream)
            ncand = int(cnt.item())
            out.update({"ms_per_array": ms, "arrays_per_s": 1e3 / ms, "candidates_per_array": ncand,
                        "candidate_bytes": 16 * ncand})
            xh = torch.from_numpy(x_host).pin_memory()
            hbuf = torch.empty((buf.shape[0], 2), dtype=torch.int64).pin_memory()
            hcnt = torch.empty(1, dtype=torch.int64).pin_memory()
            xin = torch.empty_like(xd)

            def e2e_step():
                xin.copy_(xh, non_blocking=True)
                plan.candidates(xin, threshold, buf.shape[0], stream, buf, cnt)
                hcnt.copy_(cnt, non_blocking=False)
                k = min(int(hcnt.item()), buf.shape[0])
                hbuf[:k].copy_(buf[:k], non_blocking=False)
            for _ in range(2):
                e2e_step()
            steps = 20
            t0 = time.perf_counter()
            for _ in range(steps):
                e2e_step()
            dt = (time.perf_counter() - t0) / steps
            plan.status(stream)
            out["e2e"] = {"arrays_per_s": 1.0 / dt, "h2d_bytes": 8 * n, "d2h_bytes": 8 + 16 * ncand,
                          "api": "fdas_convolve_candidates with pinned host input and candidate list"}
            if with_gauss:
                # the secondary set: the power whose exponential tail has the one-sided Gaussian
                # 6-sigma probability, T_g = -ln Q(6)
                tg = -math.log(0.5 * math.erfc(6.0 / math.sqrt(2.0)))
                ms_g = _events_ms(lambda: plan.candidates(xd, tg, buf.shape[0], stream, buf, cnt), reps, stream)
                out["gaussian_tail_threshold"] = {"threshold": tg, "ms_per_array": ms_g,
                                                  "candidates_per_array": int(cnt.item())}
            plan.status(stream)
        return out

    res = {"workload": f"N=2^22, 85 templates, L=2048, G=85, threshold {threshold:g} (6 sigma)"}
    res.update(run(fd.FDAS_PREC_FP32, True))
    res["tensor_core"] = run(fd.FDAS_PREC_TC_DFT2, True)
    return res


def bench_harmonic(fd, h, dev, xd, reps=20, oracle_beside=True):
    """Harmonic summing (fdas_harmonic_sum) of the headline array's plane: sums of 8 and 16
    harmonics at bin k r, drift k z, thresholds h + 6 sqrt(h); and the chain plane + sums."""
    import torch
    n, m = xd.numel(), h.shape[0]
    bin0 = (h.shape[1] - 1) // 2
    stream = torch.cuda.current_stream(dev)
    peak, peak_kind = measured_peaks()
    # every cell the sums read at least once: the plane from column bin0 + 1 on
    plane_bytes = 4 * m * (n - 1 - bin0)
    res = {"workload": f"plane of the N=2^22, 85-template array (1.43 GB, larger than L2), bin0={bin0}",
           "algorithmic_bytes": plane_bytes}
    with fd.Plan(h, n_max=n) as plan:
        plane = plan.convolve(xd)
        buf = torch.empty((1 << 21, 3), dtype=torch.int64, device=dev)
        cnt = torch.empty(1, dtype=torch.int64, device=dev)
        for H in (8, 16):
            thr = fd.harmonic_thresholds(H)
            run = lambda: fd.harmonic_sum(plane, bin0, H, thr, buf.shape[0], stream, buf, cnt)   # noqa: E731
            for _ in range(3):
                run()
            ms = _events_ms(run, reps, stream)
            res[f"max_harm_{H}"] = {"ms_per_array": ms, "candidates": int(cnt.item()),
                                    "plane_read_gbs": plane_bytes / (ms / 1e3) / 1e9,
                                    "hbm_frac": plane_bytes / (ms / 1e3) / 1e9 / peak,
                                    "thresholds": [round(t, 3) for t in thr]}
            traffic = profile_traffic("harmonic", f"harmonic_sum_h{H}_n2p22_traffic.json")
            if traffic:   # the bytes the launches of one call move (ncu record), at this call's duration
                res[f"max_harm_{H}"].update({"traffic": traffic, "traffic_gbs": traffic / (ms / 1e3) / 1e9,
                                             "traffic_hbm_frac": traffic / (ms / 1e3) / 1e9 / peak})

        def chain():
            plan.convolve(xd, plane, stream)
            fd.harmonic_sum(plane, bin0, 8, fd.harmonic_thresholds(8), buf.shape[0], stream, buf, cnt)
        for _ in range(3):
            chain()
        ms = _events_ms(chain, reps, stream)
        res["plane_then_sums_8"] = {"ms_per_array": ms, "arrays_per_s": 1e3 / ms}
        # end to end as a search would run it: pinned input up, plane and sums on the device,
        # the crossing count and records down (the plane never leaves the GPU)
        xh = torch.empty(n, dtype=torch.complex64).pin_memory()
        xh.copy_(xd.cpu())
        hbuf = torch.empty((buf.shape[0], 3), dtype=torch.int64).pin_memory()
        hcnt = torch.empty(1, dtype=torch.int64).pin_memory()
        xin = torch.empty_like(xd)
        thr8 = fd.harmonic_thresholds(8)

        def e2e_step():
            xin.copy_(xh, non_blocking=True)
            plan.convolve(xin, plane, stream)
            fd.harmonic_sum(plane, bin0, 8, thr8, buf.shape[0], stream, buf, cnt)
            hcnt.copy_(cnt, non_blocking=False)
            k = min(int(hcnt.item()), buf.shape[0])
            hbuf[:k].copy_(buf[:k], non_blocking=False)
            return k
        for _ in range(2):
            e2e_step()
        steps = 20
        t0 = time.perf_counter()
        for _ in range(steps):
            k = e2e_step()
        dt = (time.perf_counter() - t0) / steps
        res["plane_then_sums_8"]["e2e"] = {"arrays_per_s": 1.0 / dt, "h2d_bytes": 8 * n, "d2h_bytes": 8 + 24 * k,
                                           "api": "fdas_convolve + fdas_harmonic_sum, pinned host input, records down"}
        res["peak_kind"] = peak_kind
        plan.status(stream)
    if oracle_beside:   # the oracle beside the kernel (8 harmonics, same thresholds)
        res["max_harm_8"]["cpu_baseline"] = time_oracle_harmonic(m, n, bin0, 8, fd.harmonic_thresholds(8))
    return res


def bench_library_ols(h, dev, xd, reps=5, seg_len=2048):
    """Same-GPU library comparison (not the product path): unfused overlap-save with
    torch.fft (cuFFT) -- segment gather, batched FFT, product with all templates, batched
    inverse FFT, discard, |y|^2 -- timed with CUDA events on the same array."""
    import torch
    n, (m, k) = xd.numel(), h.shape
    S = seg_len - k + 1
    nseg = (n + S - 1) // S
    H = torch.fft.fft(torch.from_numpy(h).to(dev), n=seg_len)             # [M, L]
    pad = torch.zeros(k - 1 + nseg * S + seg_len, dtype=torch.complex64, device=dev)
    stream = torch.cuda.current_stream(dev)
    out = torch.empty((m, nseg * S), dtype=torch.float32, device=dev)
    chunk = 128                                                          # segments per step (memory)

    def run():
        pad[k - 1:k - 1 + n].copy_(xd)
        seg = pad.unfold(0, seg_len, S)[:nseg]                           # [nseg, L] views
        for c0 in range(0, nseg, chunk):
            X = torch.fft.fft(seg[c0:c0 + chunk])                        # [c, L]
            y = torch.fft.ifft(X[:, None, :] * H[None, :, :])            # [c, M, L]
            p = y[..., k - 1:].abs().square()                            # [c, M, S]
            out[:, c0 * S:(c0 + p.shape[0]) * S] = p.permute(1, 0, 2).reshape(m, -1)
    run()
    ms = _events_ms(run, reps, stream)
    del out, pad, H
    torch.cuda.empty_cache()
    return {"what": "torch.fft (cuFFT) unfused overlap-save, 128 segments per step, same array and templates",
            "ms_per_array": ms, "arrays_per_s": 1e3 / ms}


def library_full_fdfir(x, h, t_chunk=5):
    """The paper's naive FDFIR (Eq. 2) over the whole array: y = IFFT(FFT(x) . FFT(h)) with
    transforms of length 2^ceil(log2(N + K - 1)) (no segmentation), |y|^2 of the first N
    outputs; torch.fft (cuFFT on a device tensor), templates `t_chunk` at a time."""
    import torch
    n, (m, k) = x.numel(), h.shape
    nfft = 1 << int(np.ceil(np.log2(n + k - 1)))
    X = torch.fft.fft(x, n=nfft)
    out = torch.empty((m, n), dtype=torch.float32, device=x.device)
    for z0 in range(0, m, t_chunk):
        Hz = torch.fft.fft(h[z0:z0 + t_chunk], n=nfft)
        out[z0:z0 + t_chunk] = torch.fft.ifft(X[None, :] * Hz)[:, :n].abs().square()
    return out


def bench_fdfir(fd, h, dev, xd, reps=5):
    """Full-length FD-FIR (Eq. 2) through the library's own four-step kernels
    (fdas_fdfir_convolve): 2^23-point transforms of the whole array per template."""
    import torch
    n, m = xd.numel(), h.shape[0]
    out = torch.empty((m, n), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    with fd.FdFir(h, n_max=n) as ff:
        ff.convolve(xd, out, stream)
        ms = _events_ms(lambda: ff.convolve(xd, out, stream), reps, stream)
        length = ff.length
    del out
    torch.cuda.empty_cache()
    return {"what": f"fdas_fdfir_convolve: {length}-point four-step transforms (2048 x {length // 2048}) of the "
                    f"whole array, one inverse per template, same array and templates",
            "ms_per_array": ms, "arrays_per_s": 1e3 / ms, "gpu_launches_per_array": 2 + 2 * m,
            "spectra_bytes": 8 * m * length}


def bench_library_fdfir(h, dev, xd, reps=3):
    """Same-GPU library comparison (not the product path): naive full-length FDFIR."""
    import torch
    hd = torch.from_numpy(h).to(dev)
    stream = torch.cuda.current_stream(dev)
    library_full_fdfir(xd, hd)
    ms = _events_ms(lambda: library_full_fdfir(xd, hd), reps, stream)
    torch.cuda.empty_cache()
    return {"what": "torch.fft (cuFFT) naive FDFIR: 2^23-point transforms of the whole array per template, "
                    "same array and templates", "ms_per_array": ms, "arrays_per_s": 1e3 / ms}


def bench_length_sweep(fd, dev, xd, lengths=(64, 128, 256, 421)):
    """Latency against filter length (the paper's experiment, Sec. 6): 85 seeded random
    unit-energy templates of K taps on the SKA-sized array, overlap-save (L = 2048, G = 85)
    against the time-domain form (Eq. 1 term by term)."""
    import torch
    n = xd.numel()
    out = torch.empty((85, n), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    rows = []
    for K in lengths:
        rng = np.random.default_rng(5000 + K)
        hk = ((rng.standard_normal((85, K)) + 1j * rng.standard_normal((85, K))) / np.sqrt(2 * K)).astype(np.complex64)
        with fd.Plan(hk, n_max=n) as plan:
            plan.convolve(xd, out, stream)
            ms_fd = _events_ms(lambda: plan.convolve(xd, out, stream), 10, stream)
            plan.convolve_direct(xd, out, stream)
            ms_td = _events_ms(lambda: plan.convolve_direct(xd, out, stream), 3, stream)
            plan.status(stream)
        rows.append({"K": K, "ols_ms": ms_fd, "td_ms": ms_td, "td_over_ols": ms_td / ms_fd,
                     "td_tflops": 8.0 * n * K * 85 / (ms_td / 1e3) / 1e12})
    del out
    torch.cuda.empty_cache()
    return {"workload": "N=2^22, 85 random templates of K taps", "rows": rows}


def bench_batch(fd, h, dev, reps=10):
    """Batched form: 64 dedispersion trials, N log-uniform in [2^18, 2^22], one persistent
    launch per graph replay.  Rows: the FP32 plan (L = 2048, G chosen per call), the
    autotuned FP32 plan (tuned on a proxy of this length range), the autotuner free to pick
    the two-stage tensor-core form, the two-stage tensor-core plan, and the same arrays through
    the per-array paths (fdas_convolve)."""
    import torch
    specs = synth.batch_trials()
    xs = [torch.from_numpy(synth.make_input(s)).to(dev) for s in specs]
    outs = [torch.empty((h.shape[0], x.numel()), dtype=torch.float32, device=dev) for x in xs]
    total_n = sum(x.numel() for x in xs)
    stream = torch.cuda.current_stream(dev)
    alg = sum(algorithmic_bytes(x.numel(), h.shape[0]) for x in xs)
    peak = measured_peaks()[0]
    res = {"workload": "64 arrays, N log-uniform in [2^18, 2^22] (seeds 1000+i), 85 templates",
           "arrays": len(xs), "total_points": total_n, "plane_bytes": 4 * h.shape[0] * total_n,
           "algorithmic_bytes": alg}

    def row(plan):
        for _ in range(3):
            plan.convolve_batch(xs, outs, stream)
        ms = _events_ms(lambda: plan.convolve_batch(xs, outs, stream), reps, stream)
        plan.status(stream)
        d = plan.desc
        return {"seg_len": d.seg_len, "tpl_per_cta": d.tpl_per_cta or "per call", "precision": d.precision,
                "ms_per_batch": ms, "arrays_per_s": len(xs) / (ms / 1e3),
                "plane_gbs": res["plane_bytes"] / (ms / 1e3) / 1e9, "hbm_frac": alg / (ms / 1e3) / 1e9 / peak,
                "gpu_launches_per_batch": 1}

    with fd.Plan(h, n_max=1 << 22) as plan:
        res.update(row(plan))
    with fd.Plan(h, n_max=1 << 22, autotune=1, tune_n_min=1 << 18) as plan:
        res["autotuned"] = row(plan)
        res["autotuned"]["tune_ms"] = [round(v, 4) for v in plan.desc.tune_ms]
    with fd.Plan(h, n_max=1 << 22, autotune=2, tune_n_min=1 << 18) as plan:
        res["autotuned_with_precision"] = row(plan)
        res["autotuned_with_precision"]["tune_ms_tc"] = round(plan.desc.tune_ms_tc, 4)
    with fd.Plan(h, n_max=1 << 22, precision=fd.FDAS_PREC_TC_DFT2) as plan:
        res["tensor_core"] = row(plan)

        def per_array_tc():
            for x, o in zip(xs, outs):
                plan.convolve(x, o, stream)
        per_array_tc()
        ms1 = _events_ms(per_array_tc, max(2, reps // 2), stream)
        res["tensor_core"].update({"per_array_ms": ms1, "per_array_arrays_per_s": len(xs) / (ms1 / 1e3)})
    with fd.Plan(h, n_max=1 << 22) as plan:
        def per_array():
            for x, o in zip(xs, outs):
                plan.convolve(x, o, stream)
        per_array()
        ms1 = _events_ms(per_array, max(2, reps // 2), stream)
        res.update({"per_array_fp32_ms": ms1, "per_array_fp32_arrays_per_s": len(xs) / (ms1 / 1e3)})
    del xs, outs
    torch.cuda.empty_cache()
    return res


def bench_serve(fd, h, dev, rate=200.0, duration=10.0, budget=120e9, pool_size=32, stress_budget=4e9,
                stress_requests=300, precision=None):
    """Served form: Poisson arrivals at `rate`, N log-uniform in [2^16, 2^22], admission by
    plane memory within `budget`; requests cycle over `pool_size` distinct arrays.  With
    `precision` None, the FP32 plan and then the two-stage tensor-core plan."""
    if precision is None:
        res = bench_serve(fd, h, dev, rate, duration, budget, pool_size, stress_budget, stress_requests,
                          fd.FDAS_PREC_FP32)
        res["tensor_core"] = bench_serve(fd, h, dev, rate, duration, budget, pool_size, stress_budget,
                                         stress_requests, fd.FDAS_PREC_TC_DFT2)
        return res
    import queue
    import threading
    import torch
    count = int(rate * duration)
    arrivals, specs = synth.poisson_requests(count, rate_hz=rate)
    pool = [torch.from_numpy(synth.make_input(s)).to(dev) for s in specs[:pool_size]]
    res = {"workload": f"Poisson {rate:g} arrays/s for {duration:g} s ({count} requests), N log-uniform in "
                       f"[2^16, 2^22] (arrival seed 2000, {pool_size} distinct arrays 2001+i), budget "
                       f"{budget / 1e9:g} GB", "requests": count}
    with fd.Plan(h, n_max=1 << 22, precision=precision) as plan:
        stream = torch.cuda.current_stream(dev)
        outs = [torch.empty((h.shape[0], x.numel()), dtype=torch.float32, device=dev) for x in pool]

        def per_array():
            for x, o in zip(pool, outs):
                plan.convolve(x, o, stream)
        per_array()
        ms1 = _events_ms(per_array, 3, stream)
        mean_n = np.mean([x.numel() for x in pool])
        res["per_array_ms_mean"] = ms1 / len(pool)
        res["per_array_capacity_arrays_per_s"] = len(pool) / (ms1 / 1e3)
        del outs

        def run(srv, times):
            q = queue.Queue()

            def consumer():
                while True:
                    t = q.get()
                    if t is None:
                        return
                    srv.wait(t)
                    srv.release(t)
            th = threading.Thread(target=consumer)
            th.start()
            t0 = time.perf_counter()
            for i, ta in enumerate(times):
                delay = t0 + ta - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
                q.put(srv.submit(pool[i % len(pool)]))
            q.put(None)
            th.join()
            return srv.stats()

        with fd.Server(plan, budget_bytes=int(budget), lanes=2, max_batch=32) as srv:
            run(srv, np.zeros(len(pool)))                     # warm-up
            srv.reset_stats()
            st = run(srv, arrivals)
        res.update({"p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "mean_ms": st["mean_ms"],
                    "max_ms": st["max_ms"], "sustained_arrays_per_s": st["arrays_per_s"],
                    "completed": st["completed"], "launches": st["launches"],
                    "admission_waits": st["admission_waits"], "peak_plane_gb": st["peak_bytes_in_use"] / 1e9})
        with fd.Server(plan, budget_bytes=int(stress_budget), lanes=2, max_batch=32) as srv:
            run(srv, np.zeros(len(pool)))
            srv.reset_stats()
            st = run(srv, np.zeros(stress_requests))           # all at once: saturation
        res["stress"] = {"budget_gb": stress_budget / 1e9, "requests": stress_requests,
                         "arrays_per_s": st["arrays_per_s"], "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
                         "admission_waits": st["admission_waits"], "peak_plane_gb": st["peak_bytes_in_use"] / 1e9}
        res["mean_n"] = float(mean_n)
    del pool
    torch.cuda.empty_cache()
    return res


# the sources a segment kernel is compiled from, and the plan kernel that lays out the templates it reads
KERNEL_SOURCES = {"fp32": ("ols_fp32.cu", "ols_common.cuh", "fft_regs.cuh", "ptx.cuh", "tmem.cuh", "fdas_internal.cuh",
                           "plan_kernels.cu"),
                  "tc": ("ols_tc.cu", "ols_common.cuh", "fft_regs.cuh", "fft_split.cuh", "ptx.cuh", "tmem.cuh",
                         "fdas_internal.cuh", "plan_kernels.cu"),
                  "tc2": ("ols_tc2.cu", "ols_common.cuh", "fft_regs.cuh", "fft_split.cuh", "ptx.cuh", "tmem.cuh",
                          "fdas_internal.cuh", "plan_kernels.cu"),
                  "harmonic": ("harmonic.cu", "fdas_internal.cuh")}


def _code_only(text: str) -> str:
    """C/C++/CUDA source without comments and blank space (string literals kept as they are),
    so that an edit of the comments alone does not invalidate a traffic record."""
    out, i, n = [], 0, len(text)
    while i < n:
        c = text[i]
        if c == '"':                                   # string literal, escapes included
            j = i + 1
            while j < n and text[j] != '"':
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        elif text.startswith("//", i):
            i = text.find("\n", i)
            i = n if i < 0 else i
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
        else:
            out.append(c)
            i += 1
    return " ".join("".join(out).split())


def kernel_sources_sha256(precision: str) -> str:
    """Hash of the code (comments and layout excluded) of the sources a segment kernel is
    compiled from: a committed traffic record is used only while it matches."""
    import hashlib
    src = os.path.join(ROOT, "paper_1805_12280_gb300", "csrc")
    h = hashlib.sha256()
    for fn in KERNEL_SOURCES[precision]:
        with open(os.path.join(src, fn), encoding="utf-8") as f:
            h.update(_code_only(f.read()).encode())
    return h.hexdigest()


def profile_traffic(precision: str = "fp32", record: str | None = None):
    """DRAM bytes per launch (per call for the harmonic sums) from the committed ncu record,
    if it matches the kernel's sources."""
    path = os.path.join(ROOT, "profiles", record or f"ols_{precision}_L2048_n2p22_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        if d.get("kernel_sources_sha256") != kernel_sources_sha256(precision):
            return None
        return d.get("dram_bytes_per_launch")
    except Exception:
        return None


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["fdas", "reference"], default="fdas")
    ap.add_argument("--seg-len", type=int, default=2048)
    ap.add_argument("--log2n", type=int, default=22, help="array length 2^log2n (22 = the SKA-sized workload)")
    ap.add_argument("--tpl-per-cta", type=int, default=0)
    ap.add_argument("--precision", choices=["fp32", "tc", "tc2"], default="fp32",
                    help="segment-kernel arithmetic of the timed steps (tc: one radix-16 tensor-core pass; "
                         "tc2: the whole inverse FFT as two tensor-core DFT-GEMMs)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the batched and served forms")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--ref-step-seconds", type=float, default=3.0)
    args = ap.parse_args()
    if args.warmup < 3:
        log("warmup raised to 3 (timing rule)")
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_fdas(args)


if __name__ == "__main__":
    main()
