"""Benchmark: one step = the whole hot path on workload W2 (n=16,384 Matern 3/2 field on a
128 x 128 grid, range 0.05, nugget 1e-4, b = 0.5, a = -inf; 20,000 lattice paths = 10 shifts x
2,000 points): Matern covariance generation (Eq. 6) -> tile Cholesky -> blocked SOV sweep
(Eqs. 2-3, Algs. 2-3) -> log-domain estimate.

Metric: SOV sample-dims/s (n * paths / step time) and MVN probabilities/s (1 / step time).
Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--prec mixed|fp64|mixed_simt]
       [--impl reference]  (the CPU oracle on a bounded sample of the same workload)
Under torchrun (N > 1) the ranks split the one W2 problem by lattice paths (strong scaling):
each rank builds and factors its own copy of Sigma (the Cholesky does not divide into
independent units), sweeps its path range, and one all-gather of the per-shift pairs
(2 x 10 doubles per rank, NCCL) precedes the combine.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MVN probs/sec and SOV sample-dims/sec at n=16k, mixed vs FP64 GPU at |dP|<=1e-4"
UNIT = "sample-dims/s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


def _clock_sampler():
    try:
        return subprocess.Popen(
            ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,"
             "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", "200"],
            stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
    except Exception:
        return None


def _clock_summary(proc, gpu_index: int):
    if proc is None:
        return None
    proc.terminate()
    try:
        out, _ = proc.communicate(timeout=5)
    except Exception:
        proc.kill()
        out = ""
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in out.splitlines():
        f = [x.strip() for x in line.split(",")]
        if len(f) < 9 or not f[0].isdigit() or int(f[0]) != gpu_index:
            continue
        try:
            sm.append(float(f[1]))
            mx.append(float(f[2]))
        except ValueError:
            continue
        for k, nm in enumerate(names):
            if f[5 + k].lower().startswith("active"):
                reasons.add(nm)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
            "samples": len(sm)}


def workload(grid: int = 0):
    from paper_2405_14892_gb300 import inputs
    w = dict(inputs.WORKLOADS["W2"])
    if grid:
        w["g"] = grid
        w["name"] = f"{w['name']}-g{grid}"
    c = inputs.grid_coords(w["g"])
    a, b = inputs.limits_for(w, c.shape[0])
    return w, c, a, b


# ----------------------------------------------------------------------------- CPU oracle arm

def cpu_oracle_problem():
    """The W2 problem as the oracle sees it: covariance (closed-form Matern) and its LAPACK
    factor, built once and untimed (the factor is the input of the timed SOV sample)."""
    import oracle
    w, c, a, b = workload()
    S = oracle.matern_closed(c, w["sigma2"], w["range"], w["nu"], w["nugget"])
    L = oracle.cholesky_lapack(S)
    return w, a, b, S, L


def cpu_oracle_throughput(sample_paths: int = 48, chol_n: int = 2048, problem=None):
    """The oracle as it stands on this host's cores, on a bounded sample of W2:
    SOV on `sample_paths` paths of the full n=16,384 problem (exactly linear in the path count)
    plus the plain Cholesky loop on the leading chol_n x chol_n block (scaled by (n/chol_n)^3).
    Returns (sample-dims/s for a whole W2 step, details)."""
    import oracle
    w, a, b, S, L = problem if problem is not None else cpu_oracle_problem()
    n = S.shape[0]
    chol_n = min(chol_n, n)
    Ntot = w["Ns"] * w["M"]
    q = oracle.QMC(w["Ns"], w["M"], w["seed"])
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    oracle.sov_logw(a, b, L, q, paths=(0, sample_paths))
    t_sov = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.cholesky(S[:chol_n, :chol_n])
    t_chol = time.perf_counter() - t0
    t_step = t_chol * (n / chol_n) ** 3 + t_sov * Ntot / sample_paths
    det = {"cores": cores, "kind": "oracle",
           "sample": f"SOV: {sample_paths} of {Ntot} paths at n={n} ({t_sov:.1f} s, OpenMP over "
                     f"paths); Cholesky: plain column loop on the leading {chol_n}^2 block "
                     f"({t_chol:.1f} s, OpenMP over the rows of each column), scaled by "
                     f"(n/{chol_n})^3; all {cores} host cores; step time {t_step:.0f} s",
           "t_step_s": t_step}
    return n * Ntot / t_step, det


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    problem = cpu_oracle_problem()
    w, n = problem[0], problem[3].shape[0]
    vals = []
    det = None
    for _ in range(max(1, args.steps)):
        v, det = cpu_oracle_throughput(sample_paths=16, chol_n=1024, problem=problem)
        vals.append(v)
    v = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w["name"], "n": n, "paths": w["Ns"] * w["M"],
                       "l2": "inputs larger than L2 (n^2 FP64 = 2.1 GB)"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": det["cores"], "kind": "oracle",
                             "sample": det["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- rooflines

# kernels whose launches the library brackets with CUDA events when timing is on
TIMED_KERNELS = ("k_oz_update", "k_oz_potrf", "k_oz_trsm", "k_sov_tc", "k_syrk",
                 "k_sov_simt_f64", "k_sov_simt_f32")


# DRAM bytes per launch measured with ncu (dram__bytes_read.sum + dram__bytes_write.sum, one pass)
# on this workload itself, n = 16,384 with 20,000 paths (profiles/launches_w2_mixed.md): k_sov_tc
# 90.98 GB read + 1.42 GB written in its launch; k_oz_update 143.11 GB read + 3.11 GB written over
# the 509 launches of one factorisation.  Other sizes scale by the growth the kernels' structure
# gives: the sweep's Y re-reads as (path tiles) x n^2, the update's digit-tile reads as n^2 per
# launch.
TRAFFIC_N0 = 16384
TRAFFIC_TILES0 = 157
TRAFFIC_BYTES0 = {"k_sov_tc": 90.977e9 + 1.418e9, "k_oz_update": (143.106e9 + 3.106e9) / 509}
TRAFFIC_NOTE = {"k_oz_update": "bytes per launch, averaged over the 509 launches of one "
                               "factorisation; ncu (1 pass) at n=16384, this workload",
                "k_sov_tc": "bytes of the launch; ncu (1 pass) at n=16384 with 20,000 paths, "
                            "this workload"}


def _traffic(name, n, tiles):
    b = TRAFFIC_BYTES0.get(name)
    if b is None:
        return None
    scale = (n / TRAFFIC_N0) ** 2
    if name == "k_sov_tc":
        scale *= tiles / TRAFFIC_TILES0
    return b * scale


def chol_update_macs(n: int) -> int:
    """Multiply-adds of the left-looking trailing update of an order-n Cholesky over 64-wide block
    columns: block column j (c0 = 64 j) takes the (n - c0) x 64 panel times K = c0, i.e.
    sum_j (n - 64 j) 64 (64 j) ~ n^3/6 (so 2 x this ~ n^3/3 flops, the factorisation's work)."""
    nbc = (n + 63) // 64
    return sum((n - 64 * j) * 64 * 64 * j for j in range(1, nbc))


def sweep_far_macs(n: int, tiles: int) -> int:
    """Multiply-adds the tensor-core sweep runs on the tensor cores: super-block R (128
    dimensions) takes K = 128 R for every 128-path tile (the diagonal blocks run on CUDA cores)."""
    nsb = (n + 127) // 128
    return tiles * 128 * 128 * 128 * (nsb * (nsb - 1) // 2)


def kernel_rooflines(kt, prec, n, Ntot, peaks, peak_src, steps):
    """Achieved rate of the main kernels of the step on the METHOD's work (the Cholesky update's
    ~n^3/3 flops, the SOV limit GEMM's n(n-1) flops per path) over the kernel's launch durations, measured by the library's CUDA events on the launching stream in
    a pass of `steps` steps after the timed region.  `mma_issue_frac` is the tensor pipe's issue
    rate (the digit and slice products the kernels actually run), separately."""
    out = []
    tens_peak = peaks["bf16_tflops_sustained"]
    tens_src = f"{peak_src} bf16 dense, sustained (the kernel runs inside a long step)"
    tiles = (Ntot + 127) // 128
    ms, cnt = kt.get("k_oz_update", (0.0, 0))
    if cnt:
        fl = 2.0 * chol_update_macs(n) * steps
        ach = fl / (ms * 1e-3) / 1e12
        out.append({"kernel": "k_oz_update", "bound": "tensor", "unit": "TFLOP/s",
                    "achieved": ach, "peak": tens_peak, "frac": ach / tens_peak,
                    "mma_issue_frac": 21 * ach / tens_peak,
                    "work_flops_per_step": fl / steps, "traffic": _traffic("k_oz_update", n, tiles),
                    "traffic_note": TRAFFIC_NOTE["k_oz_update"],
                    "launches": cnt, "total_ms": ms, "launch_ms": ms / cnt,
                    "peak_source": tens_src,
                    "work": "method work: 2 sum_j (n-64j) 64 (64j) flops per factorisation "
                            "(n^3/3); each multiply-add runs as 21 BF16 digit-product MMAs "
                            "(mma_issue_frac)"})
    ms, cnt = kt.get("k_sov_tc", (0.0, 0))
    if cnt:
        fl = float(n) * (n - 1) * Ntot * cnt
        ach = fl / (ms * 1e-3) / 1e12
        issue = 2.0 * 3 * sweep_far_macs(n, tiles) * cnt / (ms * 1e-3) / 1e12
        out.append({"kernel": "k_sov_tc", "bound": "tensor", "unit": "TFLOP/s",
                    "achieved": ach, "peak": tens_peak, "frac": ach / tens_peak,
                    "mma_issue_frac": issue / tens_peak,
                    "work_flops_per_launch": fl / cnt, "traffic": _traffic("k_sov_tc", n, tiles),
                    "traffic_note": TRAFFIC_NOTE["k_sov_tc"],
                    "launches": cnt, "total_ms": ms, "launch_ms": ms / cnt,
                    "peak_source": tens_src,
                    "work": "method work: n(n-1) flops per path (the limit GEMM); the far part "
                            "runs as 3 FP16 MMAs per multiply-add (mma_issue_frac)"})
    for name in ("k_syrk", "k_sov_simt_f64", "k_sov_simt_f32"):
        ms, cnt = kt.get(name, (0.0, 0))
        if not cnt:
            continue
        if name == "k_syrk":
            fl = n ** 3 / 3.0 * (cnt / max(1, (n + 63) // 64 - 1))
            pk, src = 1.25, "nominal FP64 1.25 TFLOP/s (recipe table)"
        elif name == "k_sov_simt_f64":
            fl = float(n) * (n - 1) * Ntot * cnt
            pk, src = 1.25, "nominal FP64 1.25 TFLOP/s (recipe table)"
        else:
            fl = float(n) * (n - 1) * Ntot * cnt
            pk = 152 * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
            src = "FP32 CUDA cores: 152 SMs x 128 lanes x 2 flops x max SM clock"
        ach = fl / (ms * 1e-3) / 1e12
        out.append({"kernel": name, "bound": "alu", "unit": "TFLOP/s", "achieved": ach,
                    "peak": pk, "frac": ach / pk, "traffic": None, "launches": cnt,
                    "total_ms": ms, "launch_ms": ms / cnt, "peak_source": src})
    # the HBM view of the kernels whose DRAM traffic was measured: measured bytes per launch over
    # the average launch duration, against the measured copy bandwidth
    hbm = peaks.get("hbm_gbs", 6800.0)
    for r in out:
        if r.get("traffic"):
            gbs = r["traffic"] / (r["total_ms"] * 1e-3 / r["launches"]) / 1e9
            r["hbm_view"] = {"achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                             "peak_source": f"{peak_src} HBM copy bandwidth"}
    return out


# ----------------------------------------------------------------------------- ranks

def job_time_and_value(ms: float, units_per_rank: float, world: int, device=None):
    """Whole-job step time = the slowest rank's (max over ranks), and the job's throughput =
    units processed by all ranks / that time (under torchrun the ranks split one problem's paths,
    so each processes 1/world of its sample-dims).  Collective only when world > 1."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, world * units_per_rank / (ms * 1e-3)


# ----------------------------------------------------------------------------- GPU arm

def fp64_arm(mvn, coords, w, a_d, b_d, Ns, M, seed, n, dev, stream):
    """The plain FP64 GPU path on the same W2 step (FP64 Cholesky, FP64 sweep) on the identical
    lattice points: one untimed step (it grows the context's workspace), then one step timed with
    CUDA events on the launching stream.  Returns (ms, out3)."""
    import torch
    S = mvn.colmajor_empty(n, n, dev)
    out3 = torch.empty(3, dtype=torch.float64, device=dev)

    def step():
        mvn.mvn_matern(coords, w["sigma2"], w["range"], w["nu"], w["nugget"], out=S)
        mvn.mvn_cholesky(S, prec="fp64", check=False)
        mvn.mvn_sov(a_d, b_d, S, Ns, M, seed, prec="fp64", out3=out3)
    step()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    res = out3.cpu().numpy()
    del S
    return ms, res


def run_gpu(args):
    import torch
    import torch.distributed as dist

    import __graft_entry__
    from paper_2405_14892_gb300 import mvn

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if rank == 0 and not os.path.exists(mvn.LIB_PATH):
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
    dev = torch.device("cuda", local)
    w, c, a, b = workload(args.grid)
    n = c.shape[0]
    Ns, M = w["Ns"], w["M"]
    if args.paths:
        Ns = max(1, args.paths // M)
    Ntot = Ns * M
    seed = w["seed"]
    prec = args.prec
    from paper_2405_14892_gb300 import shard
    p0, p1 = shard.shard_range(Ntot, world, rank)
    coords = torch.tensor(c, device=dev)
    a_d = torch.tensor(a, device=dev)
    b_d = torch.tensor(b, device=dev)
    S = mvn.colmajor_empty(n, n, dev)
    out3 = torch.empty(3, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    ctx = mvn.context(local)
    pairs = torch.empty(2 * M, dtype=torch.float64, device=dev)
    all_pairs = torch.empty(2 * M * world, dtype=torch.float64, device=dev)

    def sweep():
        aa, bb = (reo["a"], reo["b"]) if args.reorder else (a_d, b_d)
        if world == 1:
            mvn.mvn_sov(aa, bb, S, Ns, M, seed, prec=prec, out3=out3)
            return
        mvn.mvn_sov_partial(aa, bb, S, Ns, M, seed, p0, p1, prec=prec, partial=pairs)
        dist.all_gather_into_tensor(all_pairs, pairs)
        mvn.mvn_sov_combine(all_pairs, Ns, M, out3=out3)

    reo = {}

    def factor():
        if args.reorder:
            # univariate variable reordering (FP64 pivoted factorisation); the sweep then runs on
            # the permuted limits
            reo["perm"], reo["a"], reo["b"], _ = mvn.mvn_cholesky_reorder(S, a_d, b_d, check=False)
        else:
            mvn.mvn_cholesky(S, prec=prec, check=False)

    def step(evs=None):
        if evs is not None:
            evs[0].record(stream)
        mvn.mvn_matern(coords, w["sigma2"], w["range"], w["nu"], w["nugget"], out=S)
        if evs is not None:
            evs[1].record(stream)
        factor()
        if evs is not None:
            evs[2].record(stream)
        sweep()
        if evs is not None:
            evs[3].record(stream)

    # launch shapes picked by the library's autotuner for this size (untimed; the JSON-lines
    # cache named by MVN_TUNE_CACHE is reused when it has this device and size)
    tuned = None if args.no_tune else mvn.mvn_autotune(n, Ntot, prec,
                                                       cache=os.environ.get("MVN_TUNE_CACHE"))
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    st, info = ctx.sync()
    if st != 0:
        raise RuntimeError(f"device error {st} info {info}: {mvn.lib().mvn_last_error(ctx.h)}")

    # ---- timed region: device clock, inputs resident in HBM, the library's per-kernel event
    # timing off (phase events only: four per step, read after the region)
    phase_ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)]
                for _ in range(args.steps)]
    clocks_proc = _clock_sampler() if rank == 0 else None
    launches0 = ctx.launches()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for k in range(args.steps):
        step(phase_ev[k])
    t_end.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    launches = ctx.launches() - launches0
    ms = t_start.elapsed_time(t_end) / args.steps
    clocks = _clock_summary(clocks_proc, local) if rank == 0 else None
    phase = {"matern": [e[0].elapsed_time(e[1]) for e in phase_ev],
             "cholesky": [e[1].elapsed_time(e[2]) for e in phase_ev],
             "sov": [e[2].elapsed_time(e[3]) for e in phase_ev]}
    ms, value = job_time_and_value(ms, n * Ntot / world, world, dev)
    st, info = ctx.sync()
    if st != 0:
        raise RuntimeError(f"device error {st} info {info}")
    res = out3.cpu().numpy()

    # ---- kernel shares: the library's CUDA events around every main launch, in a separate
    # pass after the timed region (the events add a little host work per launch)
    kt_steps = max(1, min(args.steps, 3))
    ctx.timing(True)
    for _ in range(kt_steps):
        step()
    torch.cuda.synchronize()
    ktimes = {k: ctx.kernel_time(k) for k in TIMED_KERNELS}
    ctx.timing(False)

    # ---- end to end through the C ABI with host buffers (copies inside the timed region)
    c_h = torch.tensor(c).pin_memory()
    a_h = torch.tensor(a).pin_memory()
    b_h = torch.tensor(b).pin_memory()
    res_h = torch.empty(3, dtype=torch.float64).pin_memory()
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        coords.copy_(c_h, non_blocking=True)
        a_d.copy_(a_h, non_blocking=True)
        b_d.copy_(b_h, non_blocking=True)
        step()
        res_h.copy_(out3, non_blocking=True)
        torch.cuda.synchronize()
    e2e_ms = (time.perf_counter() - t0) * 1e3 / e2e_steps
    e2e_ms, e2e_value = job_time_and_value(e2e_ms, n * Ntot / world, world, dev)
    h2d = c_h.numel() * 8 + a_h.numel() * 8 + b_h.numel() * 8
    d2h = 3 * 8

    # ---- the metric's other arm: the plain FP64 GPU path on identical lattice points
    fp64 = None
    if prec == "mixed" and not args.no_fp64_arm and not args.reorder and rank == 0:
        del S
        torch.cuda.empty_cache()
        f_ms, f_res = fp64_arm(mvn, coords, w, a_d, b_d, Ns, M, seed, n, dev, stream)
        st, info = ctx.sync()
        if st != 0:
            raise RuntimeError(f"device error {st} info {info} (FP64 arm)")
        fp64 = {"fp64_ms_per_step": f_ms, "fp64_value": n * Ntot / (f_ms * 1e-3),
                "mixed_over_fp64": f_ms / ms, "fp64_logP": float(f_res[0]),
                "fp64_P": float(f_res[1]), "fp64_err": float(f_res[2]),
                "dlogP_vs_fp64": abs(float(res[0]) - float(f_res[0])),
                "dP_vs_fp64": abs(float(res[1]) - float(f_res[1])),
                "gate": "|d log P| <= 1e-4 (relative reading of |dP| <= 1e-4; P ~ 1e-45 here)",
                "gate_ok": abs(float(res[0]) - float(f_res[0])) <= 1e-4,
                "note": "one untimed FP64 step, then one timed (CUDA events); same shift seed"}

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    peaks, peak_src = _peaks()
    sov_ms = statistics.median(phase["sov"])
    chol_ms = statistics.median(phase["cholesky"])
    rooflines = kernel_rooflines(ktimes, prec, n, Ntot, peaks, peak_src, kt_steps)
    dominant = max(rooflines, key=lambda r: r["total_ms"]) if rooflines else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "strong" if world > 1 else "weak",
        "vs_baseline": None, "dtype": {"fp64": "f64", "mixed": "f64+f32+fp16x2",
                                       "mixed_simt": "f64+f32"}[prec],
        "data": "synthetic",
        "config": {"workload": w["name"], "n": n, "paths": Ntot, "shifts": M, "points": Ns,
                   "prec": prec, "l2": "inputs larger than L2 (Sigma n^2 FP64 = 2.1 GB)",
                   "reorder": ("univariate variable reordering (FP64 pivoted Cholesky)"
                               if args.reorder else None),
                   "parallelism": (f"paths split over {world} ranks (Sigma and its factor on "
                                   f"every rank, one all-gather of per-shift pairs)"
                                   if world > 1 else "1 GPU"),
                   "launch_shapes_autotuned": tuned},
        "probs_per_sec": world / (ms * 1e-3),
        "phases_ms": {"matern": statistics.median(phase["matern"]), "cholesky": chol_ms,
                      "sov": sov_ms},
        "sov_sample_dims_per_sec": n * Ntot / (sov_ms * 1e-3),
        "logP": float(res[0]), "P": float(res[1]), "err": float(res[2]),
        "err_over_P": float(res[2]) / float(res[1]) if res[1] > 0 else None,
        "roofline": dominant,
        "rooflines": rooflines,
        "kernel_ms_per_step": {k: v[0] / kt_steps for k, v in ktimes.items() if v[1]},
        "kernel_timing_pass": f"{kt_steps} steps after the timed region, library events on",
        "e2e": {"value": e2e_value, "unit": UNIT,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "clocks": clocks,
    }
    if fp64 is not None:
        line["fp64_arm"] = fp64
    if not args.no_cpu_baseline and world == 1:
        v, det = cpu_oracle_throughput()
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": det["cores"],
                                "kind": "oracle", "sample": det["sample"]}
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="mixed", choices=["mixed", "fp64", "mixed_simt"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-arm", action="store_true",
                    help="skip the plain FP64 GPU step (about 20 s at the default size)")
    ap.add_argument("--reorder", action="store_true",
                    help="factor with the univariate variable reordering (mvn_cholesky_reorder)")
    ap.add_argument("--no-tune", action="store_true",
                    help="default launch shapes instead of the autotuner (profiling runs)")
    ap.add_argument("--workload", default="w2", choices=["w1", "w2", "w3", "w4", "w5", "w6"],
                    help="w2 (default): the contract line; the others measure the other rows")
    ap.add_argument("--grid", type=int, default=0,
                    help="override the grid side g (n = g^2; profiling runs on small cases)")
    ap.add_argument("--paths", type=int, default=0,
                    help="override the path count (multiple of the shift count; profiling runs)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "w2":
        run_gpu(args)
    else:
        import bench_workloads  # noqa: E402  (secondary rows, same timing rules)
        bench_workloads.run(args)


if __name__ == "__main__":
    main()
