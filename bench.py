#!/usr/bin/env python3
"""Benchmark: level-blocked matrix power kernel on one GB300 (replicas across GPUs).

Workload (default): 3-D 7-point Laplacian on a 256^3 grid (n = 16,777,216, nnz =
117,047,296), FP64 values, x ~ U[-1,1) from a seeded splitmix64 stream, p = 8 powers,
one right-hand side, vectors in the matrix's own (lexicographic) row order.

One step = one mpk_apply on a plan-order plan: the persistent level-blocked kernel over all
Lp-diagram cells, with the vectors in the permuted (BFS) numbering as in the paper, where
the solver works in the permuted space.  The optional gather/scatter between the matrix's
own numbering and the plan's (an apply in original order) is timed separately and
reported as "original_order".  Levels and the plan are built once before timing (their cost
is reported).  Inputs exceed L2 (matrix 1.47 GB vs 129 MB L2), so no flush is needed.

`--workload cheb_xxz` instead times Chebyshev time propagation (the recurrence mode of the
same kernel, mpk_cheb_filter): the XXZ spin-1/2 chain, L = 24, periodic, Sz = 0 sector
(n = 2,704,156, nnz = 36,564,892), rescaled by Gershgorin bounds, a complex state held as two
real right-hand sides, degree 64 run as 8 blocks of p = 8 powers; one step = one time step.

Prints ONE JSON line (rank 0).  `--impl reference` times the CPU oracle instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Level-blocked MPK Gflop/s vs p×CSR SpMV on 1 GB300; serving p50/p99 latency"
DFMA_LANES_PER_CLK_PER_SM = 2  # GB300's FP64 FMA issue rate per SM (unit count of the roof)
SM_MAX_MHZ_FALLBACK = 2070.0   # used only if nvidia-smi gives no clock
# the level-blocked kernel, its tunables and the planner that cuts its chunks
KERNEL_SOURCES = [os.path.join(ROOT, "paper_2405_12525_gb300", "csrc", f)
                  for f in ("mpk_kernel_dev.cuh", "mpk_internal.h", "mpk_plan.cu")]
TRAFFIC_RECORD = os.path.join(ROOT, "profiles", "k_mpk_traffic.json")


def measured_profile(side: int, accum: str):
    """The committed ncu record of the level-blocked kernel for one accumulation ("f64": binary64
    sums over binary64 values; "f32": binary32 sums over bfloat16 values): DRAM bytes per launch
    and L2 hit rate.  None when the record is missing, was taken on another workload, or the
    kernel source changed since."""
    try:
        rec = json.load(open(TRAFFIC_RECORD))
        h = hashlib.sha256()
        for f in KERNEL_SOURCES:
            h.update(open(f, "rb").read())
        sha = h.hexdigest()
    except (OSError, ValueError):
        return None
    case = rec.get("records", {}).get(accum)
    if rec.get("kernel_source_sha256") != sha or not case or case.get("side") != side:
        return None
    return case


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--side", type=int, default=256, help="grid side of the 3-D Laplacian")
    ap.add_argument("--p", type=int, default=8)
    ap.add_argument("--cache-mb", type=int, default=0, help="cache budget C of the plan in MiB (0: library default)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--workload", default="laplace3d", choices=["laplace3d", "cheb_xxz", "batch_cfg3", "serving", "dlb"])
    ap.add_argument("--dlb-parts", type=int, default=4, help="row partitions of the DLB-MPK workload")
    ap.add_argument("--serve-rate", type=float, default=200.0, help="mean Poisson arrival rate (requests/s)")
    ap.add_argument("--serve-seconds", type=float, default=3.0, help="length of the arrival window (s)")
    ap.add_argument("--serve-rate2", type=float, default=10.0, help="second, sustainable arrival rate")
    ap.add_argument("--serve-shape", type=int, default=-1,
                    help="plan option `shape` of the serving plans (-1: the serving default, 0: automatic)")
    ap.add_argument("--serve-p99-ms", type=float, default=1000.0,
                    help="latency bound: the highest curve rate whose p99 stays within it is reported")
    ap.add_argument("--serve-rates", default="2,5,10,15,20,25,30,50",
                    help="arrival rates (requests/s) of the throughput-latency curve ('' for none)")
    ap.add_argument("--batch-count", type=int, default=64, help="matrices of the batch workload")
    ap.add_argument("--batch-nmax", type=float, default=2e6, help="largest matrix size of the batch workload")
    ap.add_argument("--split", action="store_true",
                    help="split bulky levels into budget-sized groups (plan option split_levels, wave-ordered units)")
    ap.add_argument("--accum", default="f64", choices=["f64", "f32"],
                    help="row-sum arithmetic: binary64, or binary32 (values then f32 or bf16; bf16 if f64 is given)")
    ap.add_argument("--values", default="f64", choices=["f64", "f32", "bf16"],
                    help="storage type of the matrix values (accumulation stays float64); the Laplacian's "
                         "{6, -1} are exact in all three")
    ap.add_argument("--xxz-L", type=int, default=24, help="chain length of the XXZ workload")
    ap.add_argument("--degree", type=int, default=64, help="Chebyshev degree of the XXZ workload")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            time.sleep(0.5)  # let the sampler start before the timed region
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        mhz, maxm, reasons = [], SM_MAX_MHZ_FALLBACK, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                mhz.append(float(parts[0]))
                maxm = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(mhz) if mhz else None, "sm_max_mhz": maxm,
                "reasons": sorted(reasons), "samples": len(mhz)}


def build_workload(side: int):
    import gen
    A = gen.laplacian_3d(side, side, side)
    X = gen.vector(A.n, 1, stream=1)
    return A, X


def algorithmic(A, p: int, m: int = 1):
    """Per-apply algorithmic quantities (FP64 values, int32 indices)."""
    flops = 2.0 * A.nnz * m * p
    a_bytes = 12.0 * A.nnz + 4.0 * (A.n + 1)
    v_bytes = 8.0 * A.n * m
    return flops, a_bytes, v_bytes


def memory_roofs(a_bytes: float, n: int, p: int, acc32: bool, hbm_gbs: float, l2_gbs: float) -> dict:
    """Memory roofs of one apply with one right-hand side (Sec. 6 roofline reasoning on this
    device's measured bandwidths).  Level-blocked, from HBM: A once, X once and every power
    written once; from L2: p passes over A and the two vectors of a power; the L2-blocked roof is
    the larger of the two times.  The plain p x SpMV moves the L2 bytes through HBM.  With
    binary32 accumulation a power also writes its binary32 copy (4 B a row) and reads the
    previous one instead of the binary64 power."""
    out_row = 8.0 + (4.0 if acc32 else 0.0)
    hbm = a_bytes + 8.0 * n + p * out_row * n
    l2 = p * (a_bytes + (4.0 if acc32 else 8.0) * n + out_row * n)
    t_hbm, t_l2 = hbm / (hbm_gbs * 1e9), l2 / (l2_gbs * 1e9)
    return {"hbm_bytes": hbm, "l2_bytes": l2, "plain_bytes": l2, "t_hbm_s": t_hbm, "t_l2_s": t_l2,
            "l2_blocked_roof_ms": max(t_hbm, t_l2) * 1e3, "plain_hbm_roof_ms": l2 / (hbm_gbs * 1e9) * 1e3}


def host_cores():
    """Logical CPUs of the host (os.cpu_count) and lscpu's model line, for the record."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                model = ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return os.cpu_count() or 1, model


def cpu_baseline(A, X, p: int, budget_s: float = 10.0):
    """The oracle as it stands on the host cores, on a bounded sample (the first powers of the same
    matrix): the serial C oracle, and the same row loop shared out over all cores (OpenMP), with
    the paper's CPU roofline (Sec. 6, P = b_s / (6 + 14 / N_nzr) flop/byte) at the host's measured
    load bandwidth as context."""
    import oracle
    cores, model = host_cores()

    def sample(fn):
        t0 = time.perf_counter()
        fn(1)
        t1 = time.perf_counter() - t0
        k = max(1, min(p, int(budget_s / max(t1, 1e-3))))
        t0 = time.perf_counter()
        r = fn(k)
        return k, time.perf_counter() - t0, r

    k1, dt1, _ = sample(lambda k: oracle.mpk(A, X, k))
    threads = [1]
    kp, dtp, _ = sample(lambda k: threads.__setitem__(0, oracle.mpk_parallel(A, X, k)[1]))
    bw = oracle.load_bandwidth(1 << 30, 5)
    nzr = A.nnz / A.n
    roof = bw / (6.0 + 14.0 / nzr) / 1e9
    par = 2.0 * A.nnz * kp / dtp / 1e9
    return {"value": par, "unit": "Gflop/s", "cores": threads[0], "kind": "oracle",
            "sample": f"oracle row loop over all {threads[0]} host threads (OpenMP, same arithmetic as the serial "
                      f"oracle) on the full matrix, {kp} of {p} powers, {dtp:.2f} s",
            "serial": {"value": 2.0 * A.nnz * k1 / dt1 / 1e9, "cores": 1,
                       "sample": f"oracle.mpk (serial C, fma per entry), {k1} of {p} powers, {dt1:.2f} s"},
            "host": {"logical_cpus": cores, "model": model, "load_bandwidth_gbs": bw / 1e9},
            "paper_cpu_roofline_gflops": roof,
            "paper_cpu_roofline_note": "Sec. 6 roofline b_s / (6 B + 14 B / N_nzr) at the host's measured load "
                                       "bandwidth (all threads summing 1 GiB)"}


def device_roofs(mpk, torch):
    """Measured on this device in this process: FP64 FMA rate (dependent chains over all SMs), load
    bandwidth from HBM (2 GiB buffer) and from L2 (64 MiB buffer), SM count and L2 size."""
    sms, l2 = mpk.device_info()
    sink_d = torch.zeros(1, dtype=torch.float64, device="cuda")
    sink_i = torch.zeros(1, dtype=torch.int32, device="cuda")

    def ms_of(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        e1.synchronize()
        return e0.elapsed_time(e1) / reps

    blocks, iters = sms * 8, 40000
    ms = ms_of(lambda: mpk.probe_dfma(blocks, iters, sink_d))
    dfma = blocks * 256 * iters * 8 * 2 / (ms * 1e-3) / 1e12
    out = {"sms": sms, "l2_bytes": l2, "fp64_fma_tflops_measured": dfma}
    for name, nbytes, reps in (("hbm_load_gbs", 2 << 30, 4), ("l2_load_gbs", 64 << 20, 60)):
        buf = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        ms = ms_of(lambda: mpk.probe_load(buf, reps, 2, sink_i))
        out[name] = reps * nbytes / (ms * 1e-3) / 1e9
        del buf
    torch.cuda.empty_cache()
    return out


def cheb_workload(L: int, degree: int):
    """XXZ chain, Gershgorin rescaling (A' = (A - c)/a) and the time-propagation coefficients
    c_0 = J_0(a dt) e^{-i c dt}, c_k = 2 (-i)^k J_k(a dt) e^{-i c dt}, with dt the largest step
    for which |J_{degree+1}(a dt)| < 1e-15 (Bessel values from scipy)."""
    import numpy as np
    import scipy.special as sp
    import gen
    A = gen.xxz_chain(L, stream=4)
    lo, hi = gen.gershgorin_bounds(A)
    a, c = (hi - lo) / 2 * 1.01, (hi + lo) / 2
    x_lo, x_hi = 0.0, float(degree)
    for _ in range(60):
        mid = 0.5 * (x_lo + x_hi)
        if abs(sp.jv(degree + 1, mid)) < 1e-15:
            x_lo = mid
        else:
            x_hi = mid
    dt = x_lo / a
    J = sp.jv(np.arange(degree + 1), a * dt)
    coef = np.array([J[0]] + [2 * (-1j) ** k * J[k] for k in range(1, degree + 1)]) * np.exp(-1j * dt * c)
    psi = gen.vector(A.n, 2, stream=5)
    psi /= np.linalg.norm(psi)
    return A, psi, a, c, dt, coef


def cheb_flops(A, degree: int, m: int = 2):
    """Per time step: degree recurrence steps, each an SpMV (2 nnz m) plus the three-term update
    (2 FMAs per element) and the complex accumulation (2 FMAs per element)."""
    return float(degree) * m * (2.0 * A.nnz + 8.0 * A.n)


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    if args.workload == "cheb_xxz":
        return run_reference_cheb(args)
    A, X = build_workload(args.side)
    import oracle
    # the oracle's row loop on all host cores (OpenMP; the serial oracle's arithmetic), the whole
    # workload per step (all p powers) unless the run would pass about two minutes, then fewer
    # powers a step
    t0 = time.perf_counter()
    _, threads = oracle.mpk_parallel(A, X, 1)
    t_power = time.perf_counter() - t0
    k = max(1, min(args.p, int(120.0 / max(1e-9, (args.warmup + args.steps) * t_power))))
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.mpk_parallel(A, X, k)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    per = statistics.mean(times)
    value = 2.0 * A.nnz * k / per / 1e9
    sample = (f"{k} of {args.p} powers of the full matrix per step, the oracle's row loop over {threads} host "
              f"threads (OpenMP)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Gflop/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"3-D 7-point Laplacian {args.side}^3, FP64, oracle sample: {k} power(s) per step",
                       "n": A.n, "nnz": A.nnz, "p": args.p},
            "cpu_baseline": {"value": value, "unit": "Gflop/s", "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "Gflop/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_reference_cheb(args):
    import oracle
    A, psi, a, c, dt, coef = cheb_workload(args.xxz_L, args.degree)
    deg = 2  # bounded sample: two recurrence steps of the same time step per step
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.cheb(A, psi, deg, coef.real.copy(), coef.imag.copy(), scale=a, shift=c)
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    per = statistics.mean(times)
    value = cheb_flops(A, deg) / per / 1e9
    line = {"impl": "reference", "metric": "Chebyshev time propagation Gflop/s (FP64) on 1 GB300", "value": value,
            "unit": "Gflop/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": per * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"XXZ chain L={args.xxz_L}, oracle sample: degree {deg} per step", "n": A.n,
                       "nnz": A.nnz},
            "cpu_baseline": {"value": value, "unit": "Gflop/s", "cores": 1, "kind": "oracle",
                             "sample": f"degree-{deg} filter of the full matrix per step (serial C oracle)"},
            "e2e": {"value": value, "unit": "Gflop/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main_cheb(args):
    """Chebyshev time propagation of the XXZ chain through mpk_cheb_filter."""
    rank, world, local = dist_env()
    import numpy as np
    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_2405_12525_gb300 as mpk
    mpk.build()
    deg, m, p = args.degree, 2, 8
    A, psi, a, c, dt, coef = cheb_workload(args.xxz_L, deg)
    flops = cheb_flops(A, deg, m)
    dA = mpk.CsrMatrix.from_host(A, is_symmetric=True)
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    L = mpk.build_levels(dA, 0)
    t_levels = time.perf_counter() - t0
    t0 = time.perf_counter()
    P = mpk.plan(dA, L, p_max=p, nrhs=m, order=mpk.ORDER_PLAN, split_levels=args.split)
    t_plan = time.perf_counter() - t0
    perm = L.perm.long()
    psi_p = torch.from_numpy(psi).cuda()[perm].contiguous()   # state in the plan's numbering
    out = torch.empty_like(psi_p)
    cr, ci = coef.real.copy(), coef.imag.copy()
    # engine choice by timing (the autotuner's rule): level-blocked staged kernel or the
    # unblocked sweep, whose results are the same bits
    tune = {}
    plans = {"staged": P, "sweep": mpk.plan(dA, L, p_max=p, nrhs=m, order=mpk.ORDER_PLAN, engine=mpk.ENGINE_SWEEP)}
    for name, Pc in plans.items():
        for _ in range(2):
            Pc.cheb_filter(psi_p, deg, cr, ci, scale=a, shift=c, out=out)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(3):
            Pc.cheb_filter(psi_p, deg, cr, ci, scale=a, shift=c, out=out)
        e1.record(stream)
        e1.synchronize()
        Pc.sync_status()
        tune[name + "_ms"] = e0.elapsed_time(e1) / 3
    chosen = min(plans, key=lambda k: tune[k + "_ms"])
    tune["chosen"] = chosen
    P = plans[chosen]
    desc = P.describe()

    def step():
        P.cheb_filter(psi_p, deg, cr, ci, scale=a, shift=c, out=out)

    def timed(fn, steps, warm):
        for _ in range(warm):
            fn()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        e1.synchronize()
        if dist:
            dist.barrier()
        return e0.elapsed_time(e1) / steps

    with ClockSampler(local) as clk:
        ms = timed(step, args.steps, args.warmup)
    P.sync_status()
    ms_max = ms
    if dist:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_max = float(t.item())
    # unitarity of the step (the expansion is truncated below 1e-15)
    o = out.double().cpu().numpy()
    norm_ratio = float(np.linalg.norm(o) / np.linalg.norm(psi))
    # context: the same number of plain SpMVs (no recurrence) on the plan's sliced copy
    Y2 = torch.empty((p + 1, A.n, m), dtype=torch.float64, device="cuda")
    ms_spmv = timed(lambda: P.spmv_powers(psi_p, p, Y=Y2), max(3, args.steps // 4), 2) * (deg / p)
    e2e = None
    if not args.no_e2e:
        hin = psi_p.cpu().pin_memory()
        hout = torch.empty_like(hin).pin_memory()
        din = torch.empty_like(psi_p)

        def e2e_step():
            din.copy_(hin, non_blocking=True)
            P.cheb_filter(din, deg, cr, ci, scale=a, shift=c, out=out)
            hout.copy_(out, non_blocking=True)

        ms_e2e = timed(e2e_step, max(3, args.steps // 4), 2)
        e2e = {"value": world * flops / (ms_e2e * 1e-3) / 1e9, "unit": "Gflop/s",
               "h2d_bytes_per_step": int(hin.numel() * 8), "d2h_bytes_per_step": int(hout.numel() * 8),
               "ms_per_step": ms_e2e}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        import oracle
        t0 = time.perf_counter()
        oracle.cheb(A, psi, 2, cr, ci, scale=a, shift=c)
        dtc = time.perf_counter() - t0
        cpu = {"value": cheb_flops(A, 2, m) / dtc / 1e9, "unit": "Gflop/s", "cores": 1, "kind": "oracle",
               "sample": f"oracle.cheb (serial C) degree 2 of the same step on the full matrix, {dtc:.2f} s"}
    sms, _ = mpk.device_info()
    peak_alu = sms * DFMA_LANES_PER_CLK_PER_SM * 2 * (clk.summary()["sm_mhz"] or SM_MAX_MHZ_FALLBACK) * 1e6 / 1e12
    achieved = flops / (ms * 1e-3) / 1e12
    if rank == 0:
        line = {
            "metric": "Chebyshev time propagation Gflop/s (FP64) on 1 GB300", "value": world * flops / (ms_max * 1e-3) / 1e9,
            "unit": "Gflop/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"XXZ spin-1/2 chain L={args.xxz_L} periodic Sz=0 (Jxy=1, Jz=0.5, h_i~U[-1,1]), "
                                   f"Gershgorin-rescaled, complex state as 2 RHS, degree {deg} as {deg // p} blocks "
                                   f"of p={p}, vectors in BFS order",
                       "n": A.n, "nnz": A.nnz, "degree": deg, "nrhs": m, "dt": dt, "scale": a, "shift": c,
                       "parallelism": f"replicas x{world}", "l2": "no flush: matrix 439 MB > L2 129 MB",
                       "levels": desc["num_levels"], "groups": desc["num_groups"], "chunks": desc["num_chunks"]},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_alu, "unit": "TFLOP/s",
                         "frac": achieved / peak_alu, "traffic": None,
                         "kernel": ("k_mpk<2,1> (recurrence mode), 8 launches per step" if chosen == "staged" else
                                    "k_sweep<2,1> (recurrence mode, unblocked), 64 launches per step"),
                         "algorithmic": "per recurrence step 2 nnz m (SpMV) + 8 n m (update, complex accumulate)"},
            "comparator": {"plain_spmv_same_count_ms": ms_spmv,
                           "note": f"{deg} plain SpMVs of the 2 RHS without the recurrence (lower bound of an unblocked "
                                   f"step)", "speedup_vs_plain_spmv": ms_spmv / ms},
            "unitarity": {"norm_ratio": norm_ratio},
            "engine_choice": tune,
            "preprocess": {"levels_ms": t_levels * 1e3, "plan_ms": t_plan * 1e3},
            "cpu_baseline": cpu, "e2e": e2e, "clocks": clk.summary(),
            "gpu_launches": args.steps * (1 + ((deg + p - 1) // p if chosen == "staged" else deg)),
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def batch_workload(count: int, nmin: float, nmax: float):
    """Config 3: `count` matrices, sizes log-uniform in [nmin, nmax]; even index a 27-point
    stencil {26, -1} stored as bfloat16 (exact), odd index a symmetric banded random graph
    (7 upper entries a row within n/100, N(0,1) values, mirrored, plus the diagonal) stored as
    float32; right-hand sides 1, 4, 8, 16 in turn, powers p ~ U{4..12}."""
    import numpy as np
    import gen
    logn = gen.uniform(gen.derive_seed(600), count, np.log(nmin), np.log(nmax))
    pu = gen.uniform(gen.derive_seed(601), count, 0.0, 1.0)
    out = []
    for i in range(count):
        n = float(np.exp(logn[i]))
        p = 4 + min(8, int(pu[i] * 9))
        m = [1, 4, 8, 16][i % 4]
        if i % 2 == 0:
            A, vt = gen.stencil27(max(3, int(round(n ** (1.0 / 3.0))))), "bf16"
        else:
            A, vt = gen.banded_random(int(n), stream=620 + i), "f32"
        out.append((A, vt, m, p))
    return out


def main_batch(args):
    """Batched uneven MPK (config 3): one launch per (value type, width) batch plan, all of a
    step's launches replayed from one CUDA graph; compared with one plan per matrix."""
    import numpy as np
    import torch
    import gen
    import paper_2405_12525_gb300 as mpk
    from paper_2405_12525_gb300 import autotune
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    mpk.build()
    t0 = time.perf_counter()
    work = batch_workload(args.batch_count, 1e4, args.batch_nmax)
    t_gen = time.perf_counter() - t0
    vt_code = {"bf16": mpk.MPK_BF16, "f32": mpk.MPK_F32}
    # blocks: 16 right-hand sides run as two blocks of 8 (same matrix, other columns)
    groups = {}
    flops = 0.0
    for i, (A, vt, m, p) in enumerate(work):
        dA = mpk.CsrMatrix.from_host(A, is_symmetric=True, value_type=vt_code[vt])
        for half in range(2 if m == 16 else 1):
            mm = 8 if m == 16 else m
            X = torch.from_numpy(gen.vector(A.n, mm, stream=700 + 2 * i + half)).cuda()
            groups.setdefault((vt, mm), []).append((dA, p, X))
        flops += 2.0 * A.nnz * m * p
    plans, tune = {}, {}
    for key, blocks in groups.items():
        B, rep = autotune.tune_batch([b[0] for b in blocks], [b[1] for b in blocks], [b[2] for b in blocks],
                                     nrhs=key[1], order=mpk.ORDER_PLAN)
        plans[key] = (B, [b[2] for b in blocks], B.apply([b[2] for b in blocks], in_place=True))
        tune[f"{key[0]}_m{key[1]}"] = {"blocks": len(blocks), "best": rep[0][1], "ms": [round(r[0], 3) for r in rep]}

    def batched_step():  # results stay in each batch plan's workspace (views), as singles write their Y
        for B, Xs, Ys in plans.values():
            B.apply(Xs, in_place=True)

    # one plan per block, applied one after the other (the same work without batching)
    singles = []
    for blocks in groups.values():
        for dA, p, X in blocks:
            P = mpk.plan(dA, mpk.build_levels(dA, 0), p_max=p, nrhs=X.shape[1], order=mpk.ORDER_PLAN)
            singles.append((P, p, X, torch.empty((p + 1, dA.n, X.shape[1]), dtype=torch.float64, device="cuda")))

    def single_step():
        for P, p, X, Y in singles:
            P.apply(X, p, Y=Y)

    def plain_step():
        for P, p, X, Y in singles:
            P.spmv_powers(X, p, Y=Y)

    stream = torch.cuda.current_stream()

    def graph_of(fn):
        fn()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            fn()
        return g

    def timed(fn, steps, warm):
        for _ in range(warm):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / steps

    g_batch = graph_of(batched_step)
    g_single = graph_of(single_step)
    with ClockSampler(local) as clk:
        ms = timed(g_batch.replay, args.steps, args.warmup)
    ms_single = timed(g_single.replay, max(3, args.steps // 2), 2)
    ms_plain = timed(plain_step, max(3, args.steps // 2), 2)
    # the batch equals the matrices run alone
    same = all(torch.equal(Y1[:, :, :], Yb) for (P, p, X, Y1), Yb in
               zip(singles, [Y for B, Xs, Ys in plans.values() for Y in Ys]))
    launches = sum(1 for _ in plans)
    line = {
        "metric": "Batched uneven MPK Gflop/s (FP64 accumulation) on 1 GB300", "value": flops / (ms * 1e-3) / 1e9,
        "unit": "Gflop/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{args.batch_count} matrices, n log-uniform in [1e4, {args.batch_nmax:.0e}]: 27-point "
                               "stencils in bfloat16 and banded random graphs in float32, RHS 1/4/8/16, p 4..12, "
                               "vectors in BFS order",
                   "total_rows": int(sum(A.n for A, _, _, _ in work)), "total_nnz": int(sum(A.nnz for A, _, _, _ in work)),
                   "batch_plans": len(plans), "generation_s": round(t_gen, 1), "autotune": tune},
        "comparator": {"one_plan_per_matrix_ms": ms_single, "plain_spmv_ms": ms_plain,
                       "speedup_vs_one_plan_per_matrix": ms_single / ms, "speedup_vs_plain": ms_plain / ms,
                       "bit_identical_to_one_plan_per_matrix": bool(same)},
        "clocks": clk.summary(), "gpu_launches": args.steps * (launches + sum(len(Xs) for B, Xs, Ys in plans.values())),
        "cpu_baseline": None, "e2e": None,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def serving_requests(mats, rate: float, seconds: float, seed: int):
    """Config 5 stream: Poisson arrivals; matrix family uniform (config 2, 3 or 4), matrix
    uniform inside it; half MPK with p ~ U{4..16}, half Chebyshev with degree ~ U{16..128};
    1..8 right-hand sides."""
    import numpy as np
    import scipy.special as sp
    import gen
    from paper_2405_12525_gb300.serving import Request
    count = int(rate * seconds * 1.5) + 16
    gaps = -np.log(gen.uniform(gen.derive_seed(seed), count, 1e-12, 1.0)) / rate
    t = np.cumsum(gaps)
    u = gen.uniform(gen.derive_seed(seed + 1), 6 * count, 0.0, 1.0).reshape(count, 6)
    fams = [[k for k in mats if k.startswith(f)] for f in ("lap", "cfg3", "xxz")]
    reqs = []
    for i in range(count):
        if t[i] > seconds:
            break
        fam = fams[min(2, int(u[i, 0] * 3))]
        name = fam[min(len(fam) - 1, int(u[i, 1] * len(fam)))]
        nrhs = 1 + min(7, int(u[i, 2] * 8))
        if u[i, 3] < 0.5:
            r = Request(i, float(t[i]), name, "mpk", 4 + min(12, int(u[i, 4] * 13)), nrhs)
        else:
            deg = 16 + min(112, int(u[i, 4] * 113))
            r = Request(i, float(t[i]), name, "cheb", deg, nrhs)
            r.coeffs = sp.jv(np.arange(deg + 1), 0.4 * deg) * np.where(np.arange(deg + 1) > 0, 2.0, 1.0)
        reqs.append(r)
    return reqs


def main_serving(args):
    """Config 5: continuous admission of mixed MPK / Chebyshev requests under a 150 GB budget."""
    import numpy as np
    import torch
    import gen
    import paper_2405_12525_gb300 as mpk
    from paper_2405_12525_gb300.serving import SERVING_SHAPE, GpuBackend, Server, request_flops
    shape = SERVING_SHAPE if args.serve_shape < 0 else args.serve_shape
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    mpk.build()
    host = {"lap256": gen.laplacian_3d(256, 256, 256), "xxz24": gen.xxz_chain(24, stream=4)}
    for i, (A, vt, m, p) in enumerate(batch_workload(8, 1e4, 2e6)):
        host[f"cfg3_{i}_{vt}"] = A
    mats = {}
    for name, A in host.items():
        lo, hi = gen.gershgorin_bounds(A)
        vt = mpk.MPK_BF16 if name.endswith("bf16") else (mpk.MPK_F32 if name.endswith("f32") else mpk.MPK_F64)
        mats[name] = (mpk.CsrMatrix.from_host(A, is_symmetric=True, value_type=vt), (hi - lo) / 2 * 1.01,
                      (hi + lo) / 2)
    pools = {}  # per matrix and width: one device block of random inputs (shared by requests)
    for name, A in host.items():
        base = torch.from_numpy(gen.vector(A.n, 8, stream=900)).cuda()
        for w in range(1, 9):
            pools[(name, w)] = base[:, :w].contiguous()
        del base
    def result_bytes(r):
        m = 1 << (r.nrhs - 1).bit_length()
        return 8 * host[r.matrix].n * m * ((r.order + 1) if r.kind == "mpk" else 1)

    def serve(rate, secs, seed, sample=0):
        reqs = serving_requests(mats, rate, secs, seed)
        for r in reqs:
            r.x = pools[(r.matrix, r.nrhs)]
            r.flops = request_flops(host[r.matrix], r)
        keep = set()
        if sample:  # a spread of kinds and matrix families whose results fit in 1 GB
            seen = set()
            for r in reqs:
                key = (r.kind, r.matrix.split("_")[0])
                if key not in seen and result_bytes(r) <= 1 << 30 and len(keep) < sample:
                    seen.add(key)
                    keep.add(r.rid)
        srv = Server(GpuBackend(mats, p_max=16, cheb_block=8, streams=8, shape=shape),
                     hbm_budget=150 * 10 ** 9, max_inflight=8, keep_results=keep or False)
        t0 = time.perf_counter()
        srv.run(reqs)
        wall = time.perf_counter() - t0
        st = srv.stats()
        st.update(rate_rps=rate, window_s=secs, wall_s=wall, rejected=len(srv.rejected))
        check = None
        if keep:
            # every sampled result against the same request run alone on the otherwise idle
            # device (plan, stream and launch as the server's, nothing else in flight)
            be = GpuBackend(mats, p_max=16, cheb_block=8, streams=1, shape=shape)
            same, worst = 0, 0.0
            kinds = []
            for r in srv.done:
                if r.rid not in keep:
                    continue
                h = be.launch(r, be.make_plan(be.plan_key(r)))
                torch.cuda.synchronize()
                alone = be.collect(r, h)
                got = r.result
                same += bool(torch.equal(got.contiguous(), alone.contiguous()))
                den = torch.linalg.vector_norm(alone.reshape(-1, alone.shape[-1]), dim=0)
                num = torch.linalg.vector_norm((got - alone).reshape(-1, alone.shape[-1]), dim=0)
                worst = max(worst, float((num / den.clamp_min(1e-300)).max()))
                kinds.append(f"{r.kind} {r.matrix} order {r.order} nrhs {r.nrhs}")
                r.result = None
                del h, alone, got
            check = {"sampled": len(kinds), "bit_identical_to_alone": same, "max_rel_diff": worst,
                     "requests": kinds,
                     "note": "served results (concurrent, 8 streams) vs the same request alone; the GPU tests "
                             "compare every served request of a smaller mix with the oracle, bit for bit"}
            del be
        for r in srv.done:
            r.result = None
        del srv
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        return st, check

    runs = {}
    check = None
    for label, rate, secs, seed in (("config", args.serve_rate, args.serve_seconds, 950),
                                    ("sustained", args.serve_rate2, max(args.serve_seconds, 10.0), 960)):
        st, chk = serve(rate, secs, seed, sample=8 if label == "config" else 0)
        runs[label] = st
        check = check or chk
    # every point draws the same request sequence (one seed); only the arrival times scale
    curve = []
    for rate in (float(x) for x in args.serve_rates.split(",") if x.strip()):
        secs = max(args.serve_seconds, min(20.0, 40.0 / rate))  # about 40 requests or more a point
        st, _ = serve(rate, secs, 970)
        curve.append({q: st.get(q) for q in ("rate_rps", "window_s", "requests", "p50_ms", "p99_ms", "mean_ms",
                                             "throughput_rps", "gflops", "max_inflight", "peak_bytes")})
    ok = [pt["rate_rps"] for pt in curve if pt.get("p99_ms") is not None and pt["p99_ms"] <= args.serve_p99_ms]
    sustainable = max(ok) if ok else None
    c = runs["config"]
    line = {
        "metric": "Serving latency p50/p99 (config 5) on 1 GB300", "value": c["p50_ms"], "unit": "ms",
        "higher_is_better": False, "n_gpus": world, "steps": c["requests"], "warmup": 0,
        "ms_per_step": c["mean_ms"], "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "Poisson arrivals of MPK (p 4..16) and Chebyshev (degree 16..128) requests, 1..8 RHS, "
                               "matrices from the 256^3 Laplacian, 8 config-3 matrices and the XXZ L=24 chain, "
                               "HBM budget 150 GB, at most 8 requests in flight on 8 streams",
                   "matrices": {k: [v.n, v.nnz] for k, v in host.items()}, "plan_shape_option": shape},
        "serving": runs, "p99_ms": c["p99_ms"], "throughput_rps": c["throughput_rps"], "gflops": c["gflops"],
        "throughput_latency_curve": curve, "per_request_check": check,
        "sustainable_rate_rps": sustainable, "sustainable_p99_bound_ms": args.serve_p99_ms,
        "clocks": None, "cpu_baseline": None, "e2e": None, "gpu_launches": None,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def main_dlb(args):
    """DLB-MPK (Alg. 2) with every partition on this device: each step loads x into the local
    vectors, runs every partition's level-capped launch, the p-1 rounds of halo exchange and
    per-level row SpMVs, and stores the powers; all of it replayed from one CUDA graph.
    Compared with TRAD (Alg. 1) on the same partitions and with the unpartitioned kernel."""
    import numpy as np
    import torch
    import paper_2405_12525_gb300 as mpk
    from paper_2405_12525_gb300.dlb import DlbMpk, mpi_overhead
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    mpk.build()
    p = args.p
    A, X = build_workload(args.side)
    flops = 2.0 * A.nnz * p
    Xd = torch.from_numpy(X).cuda()
    t0 = time.perf_counter()
    D = DlbMpk(A, args.dlb_parts, p)
    t_setup = time.perf_counter() - t0
    Y = torch.empty((p + 1, A.n, 1), dtype=torch.float64, device="cuda")
    Yt = torch.empty_like(Y)
    stream = torch.cuda.current_stream()

    def graph_of(fn):
        fn()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            fn()
        return g

    def timed(fn, steps, warm):
        for _ in range(warm):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / steps

    D.load(Xd)
    g_dlb = graph_of(D.run)
    g_trad = graph_of(D.run_trad)
    with ClockSampler(local) as clk:
        ms = timed(g_dlb.replay, args.steps, args.warmup)
    D.store(Y)
    ms_trad = timed(g_trad.replay, max(3, args.steps // 2), 2)
    D.store(Yt)
    for part in D.parts:
        part["P"].sync_status()
    same = bool(torch.equal(Y, Yt))
    # the same with X and the powers in A's own numbering (scatter into / gather from the
    # local vectors inside the step)
    g_glob = graph_of(lambda: D.apply(Xd, Y))
    ms_glob = timed(g_glob.replay, max(3, args.steps // 2), 2)
    # phase ii alone (the level-capped launches), for the split of the step
    ms_ii = timed(lambda: [part["P"].apply(part["Y"][0], p, Y=part["Y"]) for part in D.parts],
                  max(3, args.steps // 2), 2)
    # the unpartitioned level-blocked kernel on the same matrix (one launch, plan order)
    dA = mpk.CsrMatrix.from_host(A, is_symmetric=True)
    L = mpk.build_levels(dA, 0)
    P = mpk.plan(dA, L, p_max=p, order=mpk.ORDER_PLAN)
    Xp = Xd[L.perm.long()].contiguous()
    ms_one = timed(lambda: P.apply(Xp, p, Y=Yt), max(3, args.steps // 2), 2)
    n_rows_steps = sum(1 for st in D.steps if st[0] == "rows")
    launches = 1 + len(D.parts) + (p - 1) + n_rows_steps
    line = {
        "metric": "DLB-MPK Gflop/s (FP64) on 1 GB300, partitions emulated on one device", "value": flops / (ms * 1e-3) / 1e9,
        "unit": "Gflop/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"3-D 7-point Laplacian {args.side}^3, {args.dlb_parts} contiguous row partitions "
                               f"(nnz-balanced), p_m={p}, nrhs=1; x and the powers resident in the partitions' "
                               "local vectors (phases i-iii of Alg. 2 per step)",
                   "n": A.n, "nnz": A.nnz, "parts": args.dlb_parts,
                   "halo_rows": [int(part["pb"]["nh"]) for part in D.parts],
                   "local_levels": [int(part["lp"].size - 1) for part in D.parts],
                   "setup_s": round(t_setup, 2), "l2": "no flush: inputs exceed L2"},
        "overheads": {"o_dlb_local": D.overhead_local, "o_dlb": D.overhead, "o_mpi": mpi_overhead(D.problems)},
        "comparator": {"trad_ms": ms_trad, "trad_gflops": flops / (ms_trad * 1e-3) / 1e9,
                       "speedup_vs_trad": ms_trad / ms, "phase_ii_ms": ms_ii,
                       "global_numbering_ms": ms_glob,
                       "unpartitioned_lb_mpk_ms": ms_one, "unpartitioned_gflops": flops / (ms_one * 1e-3) / 1e9,
                       "bit_identical_dlb_trad": same, "trad_launches_per_step": 2 * p},
        "clocks": clk.summary(), "gpu_launches": args.steps * launches, "cpu_baseline": None, "e2e": None,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "cheb_xxz":
        return main_cheb(args)
    if args.workload == "batch_cfg3":
        return main_batch(args)
    if args.workload == "serving":
        return main_serving(args)
    if args.workload == "dlb":
        return main_dlb(args)
    rank, world, local = dist_env()
    import numpy as np
    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_2405_12525_gb300 as mpk
    mpk.build()
    p = args.p

    A, X = build_workload(args.side)
    acc32 = args.accum == "f32"
    if acc32 and args.values == "f64":
        args.values = "bf16"  # binary32 accumulation takes narrow values ({6, -1} are exact in bfloat16)
    flops, _, v_bytes = algorithmic(A, p)
    vbytes = {"f64": 8, "f32": 4, "bf16": 2}[args.values]
    a_bytes = (vbytes + 4.0) * A.nnz + 4.0 * (A.n + 1)
    vtype = {"f64": mpk.MPK_F64, "f32": mpk.MPK_F32, "bf16": mpk.MPK_BF16}[args.values]
    accum = mpk.MPK_F32 if acc32 else mpk.MPK_F64
    dA = mpk.CsrMatrix.from_host(A, is_symmetric=True, value_type=vtype)
    Xd = torch.from_numpy(X).cuda()
    stream = torch.cuda.current_stream()
    roofs = device_roofs(mpk, torch)

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    L = mpk.build_levels(dA, 0)
    t_levels = time.perf_counter() - t0
    t0 = time.perf_counter()
    cb = args.cache_mb << 20
    # headline: one kernel launch per apply, vectors in the plan's (BFS) numbering
    P = mpk.plan(dA, L, p_max=p, nrhs=1, order=mpk.ORDER_PLAN, cache_bytes=cb, accum=accum, split_levels=args.split)
    t_plan = time.perf_counter() - t0
    # the same preprocessing once more: the first calls of a process also load the library's kernel
    # modules (a one-time cost); the second pair is the cost per matrix
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    L2 = mpk.build_levels(dA, 0)
    t_levels_warm = time.perf_counter() - t0
    t0 = time.perf_counter()
    P2 = mpk.plan(dA, L2, p_max=p, nrhs=1, order=mpk.ORDER_PLAN, cache_bytes=cb, accum=accum, split_levels=args.split)
    t_plan_warm = time.perf_counter() - t0
    del P2, L2
    Po = mpk.plan(dA, L, p_max=p, nrhs=1, order=mpk.ORDER_ORIGINAL, cache_bytes=cb, accum=accum,
                  split_levels=args.split)
    desc = P.describe()
    Y = torch.empty((p + 1, A.n, 1), dtype=torch.float64, device="cuda")
    Y2 = torch.empty_like(Y)
    Xp = Xd[L.perm.long()].contiguous()   # X in the plan's numbering (input preparation)

    def timed(fn, steps, warm):
        for _ in range(warm):
            fn()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        e1.synchronize()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        return e0.elapsed_time(e1) / steps

    # ---- headline: level-blocked apply (plan order = exactly one persistent-kernel launch)
    with ClockSampler(local) as clk:
        ms = timed(lambda: P.apply(Xp, p, Y=Y), args.steps, args.warmup)
    P.sync_status()
    ms_max = ms
    if dist:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_max = float(t.item())
    value = world * flops / (ms_max * 1e-3) / 1e9

    # ---- the same powers in the matrix's own numbering (gather + kernel + permuted write)
    ms_orig = timed(lambda: Po.apply(Xd, p, Y=Y2), max(3, args.steps // 4), 2)
    Po.sync_status()
    orig_identical = bool(torch.equal(Y2[:, L.perm.long(), :], Y))
    # ---- comparators: plain p x SpMV (p separate launches), natural and BFS order.  Binary64:
    #      the row-range SpMV of the sliced copy and the plan's unblocked sweep engine; binary32
    #      accumulation: the sweep engine (the same arithmetic), in both orders.
    comps = {}
    if not acc32:
        P0 = mpk.plan(dA, None, p_max=p, nrhs=1)
        comps["plain_spmv_natural"] = timed(lambda: P0.spmv_powers(Xd, p, Y=Y2), max(3, args.steps // 4), 2)
        comps["plain_spmv_bfs"] = timed(lambda: P.spmv_powers(Xp, p, Y=Y2), max(3, args.steps // 4), 2)
        identical = bool(torch.equal(Y, Y2))   # level-blocked == back-to-back SpMV, bit for bit
        del P0
    else:
        P0 = mpk.plan(dA, None, p_max=p, nrhs=1, engine=mpk.ENGINE_SWEEP, accum=accum)
        comps["sweep_natural"] = timed(lambda: P0.apply(Xd, p, Y=Y2), max(3, args.steps // 4), 2)
        identical = True
        del P0
    Ps = mpk.plan(dA, L, p_max=p, nrhs=1, order=mpk.ORDER_PLAN, engine=mpk.ENGINE_SWEEP, accum=accum)
    comps["unblocked_sweep"] = timed(lambda: Ps.apply(Xp, p, Y=Y2), max(3, args.steps // 4), 2)
    identical = identical and bool(torch.equal(Y, Y2))
    del Ps
    # ---- comparator: plain p x CSR SpMV of the vendor library (cuSPARSE through torch's sparse
    #      CSR matmul), natural order, on the unpermuted CSR arrays (binary64 only)
    csr = None
    if not acc32:
        try:
            import warnings
            with warnings.catch_warnings():
                warnings.simplefilter("ignore")
                Acsr = torch.sparse_csr_tensor(torch.as_tensor(A.row_ptr).cuda(), torch.as_tensor(A.col).cuda(),
                                               torch.as_tensor(A.val, dtype=torch.float64).cuda(), size=(A.n, A.n))

                def csr_powers():
                    v = Xd
                    for _ in range(p):
                        v = Acsr @ v
                    return v

                ms_csr = timed(csr_powers, max(3, args.steps // 4), 2)
                v = csr_powers()
                rel = float(torch.linalg.norm(v[:, 0] - Y2[p, :, 0].index_select(0, L.iperm.long())) /
                            torch.linalg.norm(v[:, 0]))
                csr = {"ms": ms_csr, "gflops": flops / (ms_csr * 1e-3) / 1e9, "speedup": ms_csr / ms,
                       "rel_diff_power_p": rel, "library": "cuSPARSE (torch sparse CSR matmul)"}
                del Acsr, v
        except Exception as e:  # the comparator is optional; the headline does not depend on it
            csr = {"unavailable": f"{type(e).__name__}: {e}"}

    # ---- end to end through the C ABI with host buffers (mpk_apply_host: X copied in, every
    #      power stored into pinned host memory by the kernel as its units finish), plan order
    e2e = None
    if not args.no_e2e:
        Xh = Xp.cpu().pin_memory()
        Yh = torch.empty((p + 1, A.n, 1), dtype=torch.float64).pin_memory()

        def e2e_step():
            P.apply_host(Xh, p, Yh)

        ms_e2e = timed(e2e_step, max(3, args.steps // 10), 2)
        P.apply(Xp, p, Y=Y)
        torch.cuda.synchronize()
        e2e = {"value": world * flops / (ms_e2e * 1e-3) / 1e9, "unit": "Gflop/s",
               "h2d_bytes_per_step": int(Xh.numel() * 8), "d2h_bytes_per_step": int(Yh.numel() * 8),
               "ms_per_step": ms_e2e, "api": "mpk_apply_host (pinned host X and Y)",
               "bit_identical_to_device_apply": bool(torch.equal(Yh, Y.cpu()))}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(A, X, p)

    clocks = clk.summary()
    mhz = clocks["sm_mhz"] or SM_MAX_MHZ_FALLBACK
    achieved = flops / (ms * 1e-3) / 1e12
    best_name = min(comps, key=comps.get)
    best_plain = comps[best_name]
    mr = memory_roofs(a_bytes, A.n, p, acc32, roofs["hbm_load_gbs"], roofs["l2_load_gbs"])
    hbm_bytes, l2_bytes, plain_bytes = mr["hbm_bytes"], mr["l2_bytes"], mr["plain_bytes"]
    t_hbm, t_l2, roof_blocked_ms = mr["t_hbm_s"], mr["t_l2_s"], mr["l2_blocked_roof_ms"]
    bw_h = roofs["hbm_load_gbs"] * 1e9
    peak_nominal = roofs["sms"] * DFMA_LANES_PER_CLK_PER_SM * 2 * mhz * 1e6 / 1e12  # TFLOP/s
    # DRAM bytes per launch from one ncu capture of this kernel source (null once it has changed)
    prof = measured_profile(args.side, "f32" if acc32 else "f64")
    if prof and (prof.get("values") != args.values or prof.get("shape") != desc["shape"] or args.cache_mb
                 or args.split or args.p != prof.get("p")):
        prof = None  # the capture was taken on the default plan of this workload only
    traffic = prof.get("dram_bytes_per_launch") if prof else None
    if not acc32:
        roofline = {"bound": "alu", "achieved": achieved, "peak": peak_nominal, "unit": "TFLOP/s",
                    "frac": achieved / peak_nominal, "traffic": traffic,
                    "peak_note": f"{roofs['sms']} SMs x {DFMA_LANES_PER_CLK_PER_SM} FP64 FMA lanes/clk x 2 flop x "
                                 f"{mhz:.0f} MHz (median SM clock sampled during the timed region)",
                    "measured_fp64_peak": roofs["fp64_fma_tflops_measured"],
                    "frac_of_measured_fp64_peak": achieved / roofs["fp64_fma_tflops_measured"],
                    "measured_fp64_note": "FP64 FMA rate of dependent chains over all SMs (mpk_probe_dfma), this "
                                          "process; the pipe sustains ~84% of the unit-count rate"}
    else:
        achieved_gbs = hbm_bytes / (ms * 1e-3) / 1e9
        roofline = {"bound": "hbm", "achieved": achieved_gbs, "peak": roofs["hbm_load_gbs"], "unit": "GB/s",
                    "frac": achieved_gbs / roofs["hbm_load_gbs"], "traffic": traffic,
                    "peak_note": "load bandwidth from HBM measured in this process (mpk_probe_load, 2 GiB)",
                    "achieved_note": "algorithmic HBM bytes of one apply (A once, X once, p binary64 powers and "
                                     "their binary32 copies written) / kernel time"}
    roofline.update({
        "kernel": "k_mpk (persistent level-blocked kernel), one launch per step", "kernel_ms": ms,
        "algorithmic": "2 flop per stored entry per power: 2*nnz*p per launch",
        "l2_blocked_roof_ms": roof_blocked_ms, "frac_of_l2_blocked_roof": roof_blocked_ms / ms,
        "l2_blocked_roof": f"max((A_B + (p+1) V) / BW_HBM, p (A_B + 2V) / BW_L2) = max({t_hbm * 1e3:.3f}, "
                           f"{t_l2 * 1e3:.3f}) ms with BW_HBM {roofs['hbm_load_gbs']:.0f} GB/s, BW_L2 "
                           f"{roofs['l2_load_gbs']:.0f} GB/s measured in this process",
        "plain_hbm_roof_ms": plain_bytes / bw_h * 1e3,
        "effective_bandwidth_gbs": p * a_bytes / (ms * 1e-3) / 1e9,
        "effective_bandwidth_note": "p x matrix bytes / kernel time",
        "algorithmic_hbm_bytes": hbm_bytes, "algorithmic_l2_bytes": l2_bytes,
        "l2_hit_rate_profile": prof.get("l2_hit_rate") if prof else None,
        "device": roofs})
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "Gflop/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32acc" if acc32 else "f64", "data": "synthetic",
            "config": {"workload": f"3-D 7-point Laplacian {args.side}^3 lexicographic, x~U[-1,1), p={p}, nrhs=1, "
                                   f"level-blocked apply with vectors in BFS order, values {args.values}, "
                                   + ("binary32 row sums (binary64 vectors)" if acc32 else "binary64 arithmetic"),
                       "values": args.values, "accum": args.accum,
                       "n": A.n, "nnz": A.nnz, "p": p, "nrhs": 1, "parallelism": f"replicas x{world}",
                       "l2": f"no flush: inputs exceed L2 (matrix {a_bytes / 1e9:.2f} GB, L2 "
                             f"{roofs['l2_bytes'] / 1e6:.0f} MB)",
                       "levels": desc["num_levels"], "groups": desc["num_groups"], "chunks": desc["num_chunks"],
                       "shape": desc["shape"], "chunk_rows": desc["chunk_rows"], "split_levels": args.split,
                       "cache_bytes": desc["cache_bytes"], "window": desc["window"]},
            "roofline": roofline,
            "original_order": {"ms_per_step": ms_orig, "gflops": flops / (ms_orig * 1e-3) / 1e9,
                               "note": "gather X, level-blocked kernel, tiled permuted write of Y[1..p]",
                               "bit_identical_to_plan_order": orig_identical},
            "comparator": {**{k + "_gflops": flops / (v * 1e-3) / 1e9 for k, v in comps.items()},
                           **{k + "_ms": v for k, v in comps.items()},
                           "best_plain": best_name,
                           "speedup_vs_best_plain": best_plain / ms,
                           "speedup_original_order_vs_best_plain": best_plain / ms_orig,
                           "plain_hbm_gbs": plain_bytes / (best_plain * 1e-3) / 1e9,
                           "bit_identical_to_plain": identical,
                           "plain_spmv_note": "plain p x SpMV: p separate launches over this library's sliced "
                                              "(SELL-32) copy (the row-range SpMV, or the plan's unblocked sweep "
                                              "engine, whose row body is the level-blocked kernel's); best_plain "
                                              "is the fastest" + ("; binary32 accumulation in every comparator"
                                                                  if acc32 else ""),
                           "vendor_csr": csr},
            "preprocess": {"levels_ms": t_levels_warm * 1e3, "plan_ms": t_plan_warm * 1e3,
                           "spmv_equivalents": (t_levels_warm + t_plan_warm) * 1e3 / (best_plain / p),
                           "first_call": {"levels_ms": t_levels * 1e3, "plan_ms": t_plan * 1e3,
                                          "spmv_equivalents": (t_levels + t_plan) * 1e3 / (best_plain / p)},
                           "note": "levels and plan of the same matrix built twice in one process; the first "
                                   "calls also load the library's kernel modules"},
            "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
            "gpu_launches": args.steps * (2 if acc32 else 1),
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
