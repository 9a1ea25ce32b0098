#!/usr/bin/env python
"""Benchmark: Helmholtz solves per second at a 1e-6 true relative residual.

Default workload (one step = one full solve, every row of the hot path): the
3D 256^3 periodic FD Helmholtz problem (7-point stencil, complex128
operator) in a layered medium of 6 seeded horizontal layers with c in
[1, 3] plus 10 spherical inclusions (radius 8-20 cells, +-20% contrast), a
24-cell complex-speed absorbing layer, omega for 8 points per wavelength at
min c, K = 16 symbol planes (12 real + 4 layer nodes), FGMRES(40) with the
complex64 preconditioner and FP64 Krylov work, tol 1e-6 on the true
residual.  The medium and right-hand side are resident in HBM before timing
starts; the Krylov basis (11 GB) and the symbol planes (2 GB) exceed L2, so
no flush is needed between steps.  --workload cfg2 selects the 2D 1024^2
workload, cfg1 / cfg4 the others.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl {gb300,reference}]

With N > 1 (torchrun, one rank per GPU) every rank solves its own copy:
replicas, no collective on the data path ("scaling": "weak").
--impl reference times the CPU oracle (numpy / scipy FP64) on this host's
cores: W untimed preconditioner applies, then one oracle FGMRES run of K
Arnoldi steps of the same workload; solves/s = 1 / (time per step x the
Arnoldi steps the GPU solver takes on this workload).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Helmholtz solves/s at 1e-6 true relative residual"

# name -> (problem factory, alpha, graphs, workload label, L2 note)
WORKLOADS = {
    "cfg3": ("config3", 0.3, False, "3d-256^3-layers6+incl10-layer24-ppw8-K16-fgmres40",
             "working set larger than L2 (basis 11 GB, planes 2.1 GB); no flush"),
    "cfg2": ("config2", 0.1, True, "2d-1024x1024-bumps20+gradient-layer32-ppw8-K16-fgmres40",
             "working set larger than L2 (basis 0.7 GB, planes 134 MB); no flush"),
    "cfg1": ("config1", 0.15, True, "2d-128x128-bumps3-layer16-ppw10-K8-gmres30",
             "L2-resident (17 MB working set); timed as repeated solves, not an HBM figure"),
    "cfg4": ("config4", 0.1, True, "2d-512x512-bumps3-layer16-ppw10-K12-64rhs-fgmres40",
             "working set larger than L2 (basis 11 GB for 64 rhs); no flush"),
}
DEFAULT_WORKLOAD = "cfg3"
ALPHA = 0.1
# Arnoldi steps the GPU solver takes per solve on each workload (measured on
# the GB300 by this benchmark's GPU arm; the reference arm cannot run the GPU
# and scales its per-step time by these counts)
GPU_STEPS_PER_SOLVE = {"cfg3": 95, "cfg2": 100, "cfg1": 29, "cfg4": 67}


def workload_config(p, name=DEFAULT_WORKLOAD, nrhs=1, symbol_kind=0):
    """The workload both arms run (problem and solver parameters only)."""
    fac, alpha, g_default, label, l2 = WORKLOADS[name]
    if name == "cfg3" and p.shape[0] != 256:
        label = label.replace("256^3", f"{p.shape[0]}^3")
    return {"workload": label, "grid": list(p.shape), "K": p.K, "M": p.M, "Mt": p.Mt,
            "omega": round(p.omega, 4), "restart": p.restart, "tol": p.tol, "nrhs": nrhs,
            "alpha": alpha, "symbol_kind": symbol_kind, "l2": l2}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons, pw = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
                pw.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "power_w_max": float(max(pw)), "samples": len(sm), "reasons": sorted(reasons)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except Exception:
        return {}


def dist_setup(n_gpus):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        import torch
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    return world, rank, local, dist


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(dist, x: float) -> float:
    """Largest x over the ranks (the job's time is the slowest replica's)."""
    if dist is None:
        return x
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(dist, world: int, units_per_rank: float, ms: float):
    """(slowest rank's ms, whole-job units per second)."""
    ms_max = max_over_ranks(dist, ms)
    return ms_max, world * units_per_rank / (ms_max / 1e3)


def oracle_solve_sample(p, iters: int, workers: int, alpha: float = ALPHA, med=None):
    """Bounded oracle sample: `iters` (F)GMRES Arnoldi steps of the same
    workload (oracle as it stands, FP64 numpy / scipy); med: the oracle medium
    if already built (its construction is not timed)."""
    import oracle as O
    if med is None:
        med = O.make_medium(p.c, p.zeta, None, p.omega, p.M, p.Mt, p.c_o, None, alpha)
    t0 = time.perf_counter()
    _, st = O.gmres(lambda u: O.apply_operator(med, u), p.f[0],
                    lambda v: O.apply_preconditioner(med, v, workers=workers),
                    restart=p.restart, tol=p.tol, maxit=iters)
    dt = time.perf_counter() - t0
    return dt, st["iters"]


def run_reference(args, p):
    """The reference arm: the oracle as it stands (numpy / scipy FP64, every
    host core) on the same workload.  W untimed preconditioner applies, then
    ONE oracle FGMRES run of exactly K Arnoldi steps (j = 0 .. K-1 of the
    solve, restarted every m steps as the solver does), timed as a whole;
    per-step time = that time / K.  A full oracle solve at these sizes takes
    minutes to hours, so solves/s is estimated as 1 / (per-step time x the
    Arnoldi steps the GPU solver takes on this workload)."""
    world, rank, local, dist = dist_setup(args.gpus)
    if rank != 0:
        return
    import oracle as O
    workers = os.cpu_count() or 1
    alpha = WORKLOADS[args.workload][1]
    med = O.make_medium(p.c, p.zeta, None, p.omega, p.M, p.Mt, p.c_o, None, alpha)
    iters_per_solve = args.ref_iters or GPU_STEPS_PER_SOLVE[args.workload]
    for _ in range(args.warmup):
        O.apply_preconditioner(med, p.f[0], workers=workers)
    t0 = time.perf_counter()
    _, st = O.gmres(lambda u: O.apply_operator(med, u), p.f[0],
                    lambda v: O.apply_preconditioner(med, v, workers=workers),
                    restart=p.restart, tol=p.tol, maxit=args.steps)
    dt = time.perf_counter() - t0
    steps_run = max(int(st["iters"]), 1)
    t_it = dt / steps_run
    value = 1.0 / (t_it * iters_per_solve)
    sample = (f"one oracle FGMRES({p.restart}) run of {steps_run} Arnoldi steps of one right-hand "
              f"side of the workload ({dt:.1f} s, incl. its initial and final true residual); "
              f"solves/s = 1 / (s per step x {iters_per_solve} steps per solve, the GPU solver's "
              f"step count on this workload): estimated")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * t_it, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": workload_config(p, args.workload, p.f.shape[0], args.symbol_kind),
           "impl_detail": {"precond": "complex128 (numpy / scipy.fft)", "krylov": "FP64 CGS2 (numpy)",
                           "graphs": False, "step": "one Arnoldi step of the oracle's FGMRES",
                           "warmup": "one oracle preconditioner apply per warm-up step"},
           "cpu_baseline": {"value": value, "unit": "solves/s", "cores": workers,
                            "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# DRAM traffic / algorithmic bytes of the CGS2 dot kernel in one ncu capture
# of the 3D recipe at 128^3 with the 256^3 workload's launch shapes (Arnoldi
# step j = 13: 557.2 MB read + write, 16 n (j + 2) = 503.3 MB; the right-hand
# vector is re-read by the chunks of two basis vectors per block)
DOTS_TRAFFIC_RATIO = 557.2 / 503.3
FP64_DFMA_PER_CLK_PER_SM = 2  # sm_103 (ncu: sm__sass_thread_inst_executed_op_dfma_pred_on peak)


def apply_model_bytes(p):
    """Algorithmic HBM bytes of one complex64 preconditioner apply: the
    passes' compulsory traffic with the K planes streamed once each way
    (x-forward 2s, fused last-axis pass s + Ks, inverse + weighted sum
    Ks + s + 4 B of interpolation record; 3D adds a y pass on the input and
    on every plane), for a c128 input and a c128 output."""
    s, K, n = 8, p.K, p.n * p.f.shape[0]
    per = (4 + 2 * K) * s + 4 if len(p.shape) == 2 else (6 + 4 * K) * s + 4
    return n * (per + 8)


def time_apply(plan, p, stream, reps=30, precision=1):
    """Mean time (us) of one hz_apply_preconditioner (complex64, or complex128
    with precision 0) on all the workload's right-hand sides at once, back to
    back, rotating through input/output pairs (>= 256 MB of inputs in all)
    so that the inputs are not L2-resident."""
    import torch
    n = p.n * p.f.shape[0]
    nbuf = int(min(8, max(2, -(-(256 << 20) // (16 * n)))))
    g = torch.Generator(device="cuda").manual_seed(7)
    xs = [torch.randn(n, dtype=torch.complex128, device="cuda", generator=g) for _ in range(nbuf)]
    ys = [torch.empty_like(x) for x in xs]
    for i in range(3):
        plan.apply_preconditioner(xs[i % nbuf], precision, out=ys[i % nbuf], stream=stream)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for r in range(reps):
        plan.apply_preconditioner(xs[r % nbuf], precision, out=ys[r % nbuf], stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    return 1e3 * e0.elapsed_time(e1) / reps


def plain_fp64(hz, med, p, f, stream, graphs, dist, world, plan_mixed=None, u_mixed=None,
               max_rhs=2):
    """The plain FP64 path one right-hand side at a time (complex128
    preconditioner, right GMRES): the comparison the mixed-precision batched
    solver is measured against.  One warm-up solve, then up to max_rhs
    right-hand sides solved one by one.  Also the error of the reduced-
    precision results against it: the complex64 apply of the mixed plan vs
    the complex128 apply on one random vector, and the mixed solution of
    the first right-hand side vs the FP64 one."""
    import torch
    plan = hz.Plan(med, precision=0, restart=p.restart, tol=p.tol, maxit=4000, max_nrhs=1,
                   graphs=graphs)
    plan.autotune()
    errs = {}
    if plan_mixed is not None:
        g = torch.Generator(device="cuda").manual_seed(11)
        x = torch.randn(p.n, dtype=torch.complex128, device="cuda", generator=g)
        y64 = plan.apply_preconditioner(x, 0, stream=stream)
        y32 = plan_mixed.apply_preconditioner(x, 1, stream=stream)
        torch.cuda.synchronize()
        errs["c64_apply_rel_err"] = float(torch.linalg.vector_norm(y32 - y64) /
                                          torch.linalg.vector_norm(y64))
    nr = min(f.shape[0], max_rhs)
    u = torch.zeros_like(f[:1])
    plan.solve(f[:1], u, stream=stream)
    torch.cuda.synchronize()
    barrier(dist)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    sts = []
    e0.record(stream)
    for i in range(nr):
        u.zero_()
        sts += plan.solve(f[i:i + 1], u, stream=stream)[1]
        if i == 0:
            u0 = u.clone()
    e1.record(stream)
    torch.cuda.synchronize()
    ms, value = job_rate(dist, world, nr, e0.elapsed_time(e1))
    if u_mixed is not None:
        errs["solution_rel_diff_vs_fp64"] = float(torch.linalg.vector_norm(u_mixed[:1] - u0) /
                                                  torch.linalg.vector_norm(u0))
    return {"value": value, "unit": "solves/s", "ms_per_solve": ms / nr, "rhs_sampled": nr,
            "reduced_precision_errors": errs,
            "iters": [s["iters"] for s in sts], "rel_true_resid": max(s["rel_true_resid"] for s in sts),
            "converged": all(s["converged"] for s in sts),
            "path": "precision 0: complex128 preconditioner, FP64 right GMRES, one rhs at a time"}


def run_gpu(args, p, name):
    import torch
    world, rank, local, dist = dist_setup(args.gpus)
    if world == 1:
        torch.cuda.set_device(0)
    from paper_2409_16172_gb300 import build
    if rank == 0 or world == 1:
        build.build()
    barrier(dist)
    from paper_2409_16172_gb300 import hz

    fac, alpha, graphs, label, l2 = WORKLOADS[name]
    if args.graphs >= 0:
        graphs = bool(args.graphs)
    nrhs = p.f.shape[0]
    med = hz.Medium(p.c, p.zeta, omega=p.omega, M=p.M, Mt=p.Mt, c_o=p.c_o, alpha=alpha,
                    symbol_kind=args.symbol_kind)
    plan = hz.Plan(med, precision=p.precision, restart=p.restart, tol=p.tol, maxit=4000,
                   max_nrhs=nrhs, graphs=graphs)
    tune = None
    if args.tune:
        plan.set_tune(**json.loads(args.tune))
        tune = {"set": json.loads(args.tune)}
    elif not args.no_autotune:
        tune = plan.autotune()
    f = torch.from_numpy(np.ascontiguousarray(p.f)).cuda()
    u = torch.zeros_like(f)
    stream = torch.cuda.current_stream()

    def solve(pl=plan):
        u.zero_()
        _, st = pl.solve(f, u, stream=stream)
        return st

    for _ in range(args.warmup):
        solve()
    torch.cuda.synchronize()
    fp64_probe = hz.measure_fp64_peak()
    props = torch.cuda.get_device_properties(0)
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    fp64_peak = FP64_DFMA_PER_CLK_PER_SM * 2 * props.multi_processor_count * sm_max * 1e6 / 1e12

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    hz.profile_enable(False)
    launches0 = hz.launch_count()
    barrier(dist)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    stats = [solve() for _ in range(args.steps)]
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(dist)
    launches = hz.launch_count() - launches0
    ms = ev0.elapsed_time(ev1)
    ms_max, value = job_rate(dist, world, nrhs * args.steps, ms)
    # Per-kernel CUDA events on the launching stream, in a second pass of
    # the same steps right after the timed one (events around every launch
    # would add to the timed step; graph replay carries none, so that pass
    # launches step by step)
    plan_p = plan
    if graphs:
        plan_p = hz.Plan(med, precision=p.precision, restart=p.restart, tol=p.tol, maxit=4000,
                         max_nrhs=nrhs, graphs=False)
        if args.tune:
            plan_p.set_tune(**json.loads(args.tune))
        elif tune is not None:
            plan_p.autotune()  # cached: same shapes as the timed plan
    hz.profile_enable(True)
    hz.profile_read(reset=True)
    for _ in range(max(1, min(args.steps, 3))):
        solve(plan_p)
    torch.cuda.synchronize()
    prof = hz.profile_read(reset=True)
    hz.profile_enable(False)
    clocks = sampler.stop()

    # end to end through the C ABI with host buffers: H2D of f and the
    # initial guess (pinned host memory), D2H of the solution, inside the
    # timed region; one zero initial guess per step, written before timing
    fh = torch.from_numpy(np.ascontiguousarray(p.f)).pin_memory().numpy()
    e2e_steps = max(1, min(args.steps, 5))
    uhs = [torch.zeros(p.f.shape, dtype=torch.complex128).pin_memory().numpy()
           for _ in range(e2e_steps + 1)]
    # one untimed host-buffer solve first, as the device-timed leg has its
    # warm-up solves
    plan.solve(fh, uhs.pop(), stream=stream)
    torch.cuda.synchronize()
    barrier(dist)
    t0 = time.perf_counter()
    for uh in uhs:
        plan.solve(fh, uh, stream=stream)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(dist, time.perf_counter() - t0)
    e2e_val = world * nrhs * e2e_steps / e2e_s

    ok = all(s["converged"] and s["rel_true_resid"] <= p.tol for st in stats for s in st)
    apply_us = time_apply(plan, p, stream) if p.precision == 1 else None
    plain = None
    if not args.no_plain:
        mixed = p.precision == 1
        plain = plain_fp64(hz, med, p, f, stream, graphs, dist, world,
                           plan if mixed else None, u if mixed else None)
    if rank != 0:
        return
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    hbm_src = "MEASURED_PEAKS.json hbm_gbs" if "hbm_gbs" in peaks else "fallback 6800 GB/s"
    dom = max(prof.items(), key=lambda kv: kv[1]["ms"])
    kname, d = dom
    fp64_phases = {"cgs2_dots", "cgs2_update", "stencil", "residual", "solution_update", "norm"}
    if kname in fp64_phases:
        achieved = d["flops"] / d["ms"] / 1e9  # TFLOP/s
        avg_bytes = d["bytes"] / d["launches"]
        traffic = DOTS_TRAFFIC_RATIO * avg_bytes if kname == "cgs2_dots" else None
        roof = {"kernel": kname, "bound": "alu", "achieved": achieved, "peak": fp64_peak,
                "unit": "TFLOP/s", "frac": achieved / fp64_peak, "traffic": traffic,
                "traffic_note": "bytes per launch: the DRAM read + write of one ncu-captured dot "
                                "launch (the 3D recipe at 128^3, j = 13: 557.2 MB against "
                                "503.3 MB algorithmic) "
                                "scaled to the average algorithmic bytes per launch of this phase "
                                "(the launches run j = 0..m-1, and the phase's partial-sum "
                                "launches count as launches)",
                "peak_source": f"FP64: {FP64_DFMA_PER_CLK_PER_SM} DFMA/clk/SM x 2 flops x "
                               f"{props.multi_processor_count} SMs x {sm_max:.0f} MHz "
                               f"(in-library FMA probe {fp64_probe / 1e3:.3f} TFLOP/s)",
                "launches": d["launches"], "avg_launch_us": 1e3 * d["ms"] / d["launches"],
                "hbm_gbs_achieved": d["bytes"] / d["ms"] / 1e6,
                "timing": "CUDA events per launch, profiled pass of the same steps"}
    else:
        achieved = d["bytes"] / d["ms"] / 1e6  # GB/s
        roof = {"kernel": kname, "bound": "hbm", "achieved": achieved, "peak": hbm,
                "unit": "GB/s", "frac": achieved / hbm, "traffic": None,
                "peak_source": hbm_src, "launches": d["launches"],
                "avg_launch_us": 1e3 * d["ms"] / d["launches"]}
    fft = [k for k in prof if k.startswith("fft_")]
    pb = sum(prof[k]["bytes"] for k in fft)
    pm = sum(prof[k]["ms"] for k in fft)
    n_applies = max(prof["fft_row_fwd"]["launches"], 1)
    precond = None
    if apply_us is not None:
        mb = apply_model_bytes(p)
        # traffic of the passes as they run: planes only for the (row, node)
        # or (slab, node) pairs in use
        masked = pb / n_applies
        precond = {"bound": "hbm", "achieved": mb / apply_us / 1e3, "peak": hbm, "unit": "GB/s",
                   "frac": mb / apply_us / 1e3 / hbm, "traffic": None, "peak_source": hbm_src,
                   "apply_us": apply_us, "model_bytes": mb, "masked_bytes": masked,
                   "masked_frac": masked / apply_us / 1e3 / hbm,
                   "model": "n*[(4+2K)s+4] (2D) or n*[(6+4K)s+4] (3D), s = 8 (complex64), "
                            "plus 8 B/pt for the complex128 output of the public apply",
                   "timing": "CUDA events around 30 back-to-back hz_apply_preconditioner calls, "
                             "8 rotating c128 input/output pairs (> L2)",
                   "in_solve_apply_us": 1e3 * pm / n_applies,
                   "kernels": {k: {"launches": prof[k]["launches"],
                                   "avg_us": 1e3 * prof[k]["ms"] / prof[k]["launches"],
                                   "masked_model_gbs": prof[k]["bytes"] / prof[k]["ms"] / 1e6}
                               for k in fft}}
    # The FP64 floor: every FP64 flop of a solve (stencil and residuals,
    # CGS2 dots and updates, norms, solution update) at the FP64 pipe's peak;
    # the Krylov rule that keeps these in FP64 caps solves/s at its inverse
    n_prof = max(1, min(args.steps, 3))
    fp64_flops = sum(prof[k]["flops"] for k in prof if k in fp64_phases) / n_prof
    floor_s = fp64_flops / (fp64_peak * 1e12)
    floor = {"fp64_flops_per_solve": fp64_flops, "peak_tflops": fp64_peak,
             "floor_ms_per_solve": 1e3 * floor_s,
             "ceiling_solves_per_s": world * nrhs / floor_s if floor_s > 0 else None,
             "value_over_ceiling": value * floor_s / (world * nrhs) if floor_s > 0 else None,
             "note": "FP64 flops per solve from the profiled pass (CGS2 32 n (j+1) per step, "
                     "stencil, residuals, norms, solution update) / the FP64 peak"}
    total_ms = sum(v["ms"] for v in prof.values())
    phases = {k: {"launches": v["launches"], "ms": round(v["ms"], 3),
                  "share": round(v["ms"] / total_ms, 4),
                  "gbs": round(v["bytes"] / v["ms"] / 1e6, 1) if v["ms"] else None,
                  "tflops": round(v["flops"] / v["ms"] / 1e9, 4) if v["ms"] else None}
              for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"])}

    cpu = None
    if not args.no_cpu_baseline:
        import oracle as O
        workers = os.cpu_count() or 1
        pc = p
        if nrhs > 1:  # one right-hand side of the batch; the rate is per solve
            import copy
            pc = copy.copy(p)
            pc.f = p.f[:1]
        med_o = O.make_medium(pc.c, pc.zeta, None, pc.omega, pc.M, pc.Mt, pc.c_o, None, alpha)
        # a probe of 2 steps, then samples (each stops where the oracle's
        # solve converges) until about args.cpu_seconds of oracle work
        dt, it = oracle_solve_sample(pc, 2, workers, alpha, med_o)
        while dt < args.cpu_seconds and it < 2000:
            more = int(min(max(args.cpu_seconds / max(dt / max(it, 1), 1e-9) - it, 1), 400))
            dt2, it2 = oracle_solve_sample(pc, more, workers, alpha, med_o)
            dt, it = dt + dt2, it + it2
        iters = int(np.mean([s["iters"] for s in stats[0]]))
        cpu = {"value": 1.0 / (dt / max(it, 1) * iters), "unit": "solves/s", "cores": workers,
               "kind": "oracle",
               "sample": f"{it} oracle (F)GMRES Arnoldi steps of one right-hand side of the "
                         f"workload ({dt:.1f} s); scaled by the {iters} steps of the GPU solve"}
    n = p.n
    out = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32+f64" if p.precision == 1 else "f64", "data": "synthetic",
           "config": workload_config(p, name, nrhs, args.symbol_kind),
           "impl_detail": {"precond": "complex64" if p.precision == 1 else "complex128",
                           "krylov": "FP64 CGS2", "graphs": graphs},
           "iters": [s["iters"] for s in stats[0]][:8],
           "rel_true_resid": max(s["rel_true_resid"] for s in stats[0]),
           "all_converged": ok,
           "roofline": roof, "roofline_precond": precond,
           "cpu_baseline": cpu,
           "e2e": {"value": e2e_val, "unit": "solves/s",
                   "h2d_bytes_per_step": 2 * 16 * n * nrhs, "d2h_bytes_per_step": 16 * n * nrhs},
           "gpu_launches": launches, "clocks": clocks, "phases": phases, "autotune": tune,
           "fp64_plain": plain, "fp64_floor": floor,
           "fp64_peak_tflops": fp64_peak, "fp64_probe_tflops": fp64_probe / 1e3}
    print(json.dumps(out), flush=True)


def run_example1(args):
    """The paper's Example 1 GMRES study (Section 5.1) at its own grids
    (N = 2400, 3600, 4800 by default): circular inclusion, a = 20,
    delta = 1, eta = 1/800, M = 8, PPW = 12, GMRES(10), 100 iterations.
    Runs: the paper's left form (Eqn. MainDiscretePrecond, preconditioned
    residual) with the FP64 and the complex64 preconditioner, the right /
    flexible form (true residual) with both, and no preconditioner;
    residual histories and time per step at each N, with the
    finite-difference symbol (4/h^2) sin^2(pi k / N) and with the continuous
    |xi|^2 of Eqn. 021."""
    import torch
    from paper_2409_16172_gb300 import build, synth as S
    build.build()
    from paper_2409_16172_gb300 import hz
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    its = 100
    sampler = ClockSampler(0)
    sampler.start()
    sizes = {}
    for N, sk in [(N, sk) for sk in (1, 0) for N in args.ex1_n]:
        p = S.example1(N)
        med = hz.Medium(p.c, p.zeta, p.a, omega=p.omega, M=p.M, Mt=0, c_o=1.0, alpha=0.0,
                        a_node=p.meta["a_node"], symbol_kind=sk)
        f = torch.from_numpy(np.ascontiguousarray(p.f[0])).cuda()
        runs = {}
        for key, kw in (("left_fp64", dict(precision=0, left=True)),
                        ("left_c64", dict(precision=1, left=True)),
                        ("right_fp64", dict(precision=0)), ("right_c64", dict(precision=1)),
                        ("none", dict(precision=0, no_precond=True))):
            plan = hz.Plan(med, restart=p.restart, tol=1e-14, maxit=its, **kw)
            plan.autotune()
            u = torch.zeros_like(f)
            plan.solve(f, u, stream=stream, history=its)  # warm-up
            u.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, st, H = plan.solve(f, u, stream=stream, history=its)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            h = H[0]
            runs[key] = {"resid_at_100": float(h[its - 1]), "ms_per_step": ms / its,
                         "history_every_10": [float(h[i]) for i in range(9, its, 10)],
                         "rel_true_resid": st[0]["rel_true_resid"]}
            del plan
        none = runs["none"]["resid_at_100"]
        orders = {k: math.log10(none / v["resid_at_100"]) for k, v in runs.items() if k != "none"}
        sizes[f"{N}-symbol{sk}"] = {"grid": list(p.shape), "dof": p.n, "omega": p.omega,
                                    "omega_over_pi": p.omega / math.pi, "symbol_kind": sk,
                                    "orders": orders, "runs": runs}
        del med, f
    clocks = sampler.stop()
    gaps = [v["orders"]["left_fp64"] for v in sizes.values() if v["symbol_kind"] == 1]
    first = sizes[f"{args.ex1_n[0]}-symbol1"]
    out = {"metric": "Example 1 (Section 5.1): orders of magnitude between the unpreconditioned "
                     "and the preconditioned GMRES(10) relative residual after 100 iterations "
                     "(smallest over the grids)",
           "value": min(gaps), "unit": "orders of magnitude", "n_gpus": 1, "steps": its,
           "warmup": 1, "ms_per_step": first["runs"]["left_fp64"]["ms_per_step"],
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64 (and f32 preconditioner)", "data": "synthetic",
           "config": {"workload": "example1 circular inclusion", "N": list(args.ex1_n),
                      "ppw": 12, "delta": 1.0, "eta": 1 / 800, "a": 20.0, "M": 8,
                      "restart": 10, "symbol_kind": [1, 0],
                      "value_is": "left_fp64 with the finite-difference symbol: the paper's left "
                                  "form, preconditioned residual"},
           "paper_statement": ">= 7 orders at 100 iterations (N = 2400, 3600, 4800)",
           "sizes": sizes, "clocks": clocks}
    print(json.dumps(out), flush=True)


def run_interp(args):
    """The interpolation forms Section 6 proposes, against the paper's
    piecewise-linear univariate Q_M, by FGMRES(40) steps to 1e-6 and solve
    time: (a) 2D media whose damping a(x) (omega [0.02, 0.2] and omega
    [0.005, 0.05]) does not follow c, preconditioned univariately (every node
    at the mean damping) and bivariately with Ma = 2, 3 (and 4) damping nodes,
    with the node damping regularised by alpha omega (alpha = 0.1) and not
    (alpha = 0; a > 0 everywhere); (b) the 1024^2 workload's medium with hats
    vs quadratic Lagrange polynomials vs cubic Hermite (values and
    c-derivatives) in c."""
    import torch
    from paper_2409_16172_gb300 import build, synth as S
    build.build()
    from paper_2409_16172_gb300 import hz
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    sampler = ClockSampler(0)
    sampler.start()

    def one(p, alpha=ALPHA, **mopt):
        med = hz.Medium(p.c, p.zeta, p.a, omega=p.omega, M=mopt.pop("M", p.M), Mt=p.Mt,
                        c_o=p.c_o, alpha=alpha, **mopt)
        K = med.info()["K"]
        plan = hz.Plan(med, precision=1, restart=p.restart, tol=p.tol, graphs=True)
        plan.autotune()
        f = torch.from_numpy(np.ascontiguousarray(p.f[0])).cuda()
        u = torch.zeros_like(f)
        plan.solve(f, u, stream=stream)  # warm-up (graph capture)
        times = []
        for _ in range(max(1, args.steps)):
            u.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, st = plan.solve(f, u, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        apply_us = time_apply(plan, p, stream)
        ms = float(np.median(times))
        out = {"K": K, "iters": st[0]["iters"], "converged": bool(st[0]["converged"]),
               "rel_true_resid": st[0]["rel_true_resid"], "ms_per_solve": ms,
               "solves_per_s": 1e3 / ms, "apply_us": apply_us}
        del plan, med
        return out

    N = args.int_n
    biv = {}
    for damping in ((0.02, 0.2), (0.005, 0.05)):
        pd = S.damping_problem(N=N, damping=damping)
        for alpha in (ALPHA, 0.0):
            tag = f"a/w in {list(damping)}, alpha={alpha}"
            biv[f"{tag}: univariate (a_k = mean a + alpha w)"] = one(
                pd, alpha=alpha, a_node=float(pd.a.mean()))
            for Ma in ((2, 3, 4) if alpha > 0 and damping[0] == 0.02 else (2, 3)):
                biv[f"{tag}: bivariate Ma={Ma}"] = one(pd, alpha=alpha, Ma=Ma)
    pc = S.config2() if N == 1024 else S.damping_problem(N=N)
    if N != 1024:
        pc.a = None
    basis = {}
    for M in (6, 8, 12):
        basis[f"linear M={M}"] = one(pc, M=M)
    for M in (5, 7, 11, 13):
        basis[f"quadratic M={M}"] = one(pc, M=M, basis=1)
    for M in (4, 6, 8):
        basis[f"hermite M={M}"] = one(pc, M=M, basis=2)
    clocks = sampler.stop()
    tag = "a/w in [0.005, 0.05], alpha=0.0"
    u_it = biv[f"{tag}: univariate (a_k = mean a + alpha w)"]["iters"]
    b_it = biv[f"{tag}: bivariate Ma=3"]["iters"]
    out = {"metric": "FGMRES(40) steps to 1e-6: univariate Q_M / bivariate (c, a) Q_M with "
                     "Ma = 3, damping a(x) in omega [0.005, 0.05] independent of c, alpha = 0",
           "value": u_it / max(b_it, 1), "unit": "ratio of steps", "n_gpus": 1,
           "steps": args.steps, "warmup": 1,
           "ms_per_step": biv[f"{tag}: bivariate Ma=3"]["ms_per_solve"],
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32+f64", "data": "synthetic",
           "config": {"workload": pd.name, "grid": list(pd.shape), "omega": pd.omega,
                      "damping_over_omega": [[0.02, 0.2], [0.005, 0.05]], "M": pd.M, "Mt": pd.Mt,
                      "restart": pd.restart, "alpha": ALPHA,
                      "basis_study_medium": pc.name},
           "bivariate": biv, "basis": basis, "clocks": clocks}
    print(json.dumps(out), flush=True)


def fit_beta(Ns, T_rows, d=2):
    """Order beta of T ~ M N^(d beta) log N as the paper's Table 1 computes
    it: slope / d of a least-squares line through (log N, log T) for each row
    (one M), and pooled over all rows with one intercept per row."""
    x = np.log(np.asarray(Ns, np.float64))
    rows = [float(np.polyfit(x, np.log(np.asarray(T, np.float64)), 1)[0] / d) for T in T_rows]
    X = np.zeros((len(T_rows) * len(x), 1 + len(T_rows)))
    y = np.concatenate([np.log(np.asarray(T, np.float64)) for T in T_rows])
    for r in range(len(T_rows)):
        X[r * len(x):(r + 1) * len(x), 0] = x
        X[r * len(x):(r + 1) * len(x), 1 + r] = 1.0
    pooled = float(np.linalg.lstsq(X, y, rcond=None)[0][0] / d)
    return rows, pooled


def run_complexity(args):
    """Table 1's study on the GPU: time of one Q_{N,M} apply for N = 256 ..
    2048 and M = 2, 4, 8 on the Example 1 medium (PPW 12), complex64 (the
    solver's preconditioner) and complex128, normalised to the smallest
    (N, M = 2), and the fitted order beta of T ~ M N^(2 beta) log N."""
    import torch
    from paper_2409_16172_gb300 import build, synth as S
    build.build()
    from paper_2409_16172_gb300 import hz
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    Ns, Ms = list(args.cx_n), [2, 4, 8]
    res = {}
    for prec in (1, 0):
        T = []
        for M in Ms:
            row = []
            for N in Ns:
                p = S.example1(N, M=M)
                med = hz.Medium(p.c, p.zeta, p.a, omega=p.omega, M=M, Mt=0, c_o=1.0, alpha=0.0,
                                a_node=p.meta["a_node"])
                plan = hz.Plan(med, precision=prec)
                if prec == 1:
                    plan.autotune()
                row.append(time_apply(plan, p, stream, precision=prec))
                del plan, med
            T.append(row)
        rows, pooled = fit_beta(Ns, T)
        t0 = T[0][0]
        res["c64" if prec == 1 else "c128"] = {
            "apply_us": {f"M={M}": [round(t, 2) for t in T[i]] for i, M in enumerate(Ms)},
            "normalised": {f"M={M}": [round(t / t0, 3) for t in T[i]] for i, M in enumerate(Ms)},
            "beta": {f"M={M}": round(b, 3) for M, b in zip(Ms, rows)}, "beta_pooled": round(pooled, 3)}
    out = {"metric": "Table 1 (Section 5.1): order beta of the Q_{N,M} apply time, T ~ M N^(2 beta) log N",
           "value": res["c64"]["beta_pooled"], "unit": "beta (pooled, complex64 apply)",
           "n_gpus": 1, "steps": 30, "warmup": 3, "ms_per_step": None, "higher_is_better": False,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32 / f64", "data": "synthetic",
           "config": {"workload": "example1 medium, PPW 12, a 20, delta 1", "N": Ns, "M": Ms,
                      "note": "Table 1's grids N = 180 .. 2880"},
           "paper_context": "Table 1 (MATLAB, CPU): beta 1.02 / 1.03 / 1.04 for M = 2 / 4 / 8, "
                            "pooled 1.03",
           "results": res}
    print(json.dumps(out), flush=True)


def run_spectrum(args):
    """Spectral estimates (Section 5.1, Table 2's setting: delta = 4,
    eta = 1/800, a = 20, PPW = 12): Ritz values of P_N Q_M from one Arnoldi
    cycle of 100 steps (FP64) started from a seeded random vector (the plane
    wave of Eqn. Source is nearly an eigenvector and ends the process in a
    few steps), cond estimate max|theta| / min|theta|, for M = 1 (Q_1 of
    Eqn. OneInterpPoint), 2, 4, 8, 16, 32 and without the preconditioner, at
    several N."""
    import torch
    from paper_2409_16172_gb300 import build, synth as S
    build.build()
    from paper_2409_16172_gb300 import hz
    torch.cuda.set_device(0)
    m = 100
    rows = []
    t0 = time.perf_counter()
    for N in args.spec_n:
        p = S.example1(N, delta=4.0)
        f = np.ascontiguousarray(S.random_field(np.random.Generator(np.random.PCG64(N)), p.shape))
        for M in (None, 1, 2, 4, 8, 16, 32):
            med = hz.Medium(p.c, p.zeta, p.a, omega=p.omega, M=M or 1, Mt=0, c_o=1.0, alpha=0.0,
                            a_node=p.meta["a_node"])
            plan = hz.Plan(med, precision=0, restart=m, tol=1e-14, maxit=m,
                           no_precond=M is None)
            plan.solve(f)
            H = plan.hessenberg(0)
            J = H.shape[1]
            th = np.abs(np.linalg.eigvals(H[:J, :J]))
            rows.append({"N": N, "omega_over_pi": p.omega / math.pi,
                         "M": M if M is not None else "none", "ritz_steps": J,
                         "cond_est": float(th.max() / th.min()),
                         "ritz_abs_max": float(th.max()), "ritz_abs_min": float(th.min())})
            del plan, med
    span = time.perf_counter() - t0
    out = {"metric": "Ritz-value estimate of cond(P_N Q_M) (Table 2 setting)",
           "value": next(r["cond_est"] for r in rows if r["M"] == 8), "unit": "cond estimate at M = 8, smallest N",
           "n_gpus": 1, "steps": len(rows), "warmup": 0, "ms_per_step": 1e3 * span / len(rows),
           "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": "table2-setting delta4-eta1/800-a20-ppw12", "arnoldi_steps": m,
                      "N": list(args.spec_n),
                      "note": "Table 2's grids (N = 120 .. 1920 at PPW 12, omega = 20 pi .. "
                              "320 pi)"},
           "paper_context": "Table 2 (MATLAB eigs): M = 1: 1.2e7..2.4e8, M = 8: 5.3e2..1.7e1, "
                            "M = 32: 4.9e2..1.4e1 for omega = 20 pi..320 pi",
           "rows": rows}
    print(json.dumps(out), flush=True)


def run_serving(args):
    """Serving stream: requests drawn from the serving recipe (each request
    seeded by its index) arrive with seeded exponential gaps; the server
    admits them by HBM footprint.  Requests are generated by producer
    threads ahead of their arrival times (a stream of 2000 does not fit in
    host memory at once) and only their stats are kept.  Before the stream,
    one plan per (grid, K) of the stream is autotuned (untimed, reported);
    served plans take those launch shapes from the process cache.  The plain
    FP64 path serves the first --plain-requests requests one at a time with
    the same arrival times, and the mixed-precision server serves the same
    subset, for the comparison."""
    import concurrent.futures as cf
    import queue
    import torch
    from paper_2409_16172_gb300 import build, synth as S
    build.build()
    from paper_2409_16172_gb300 import hz
    torch.cuda.set_device(0)

    pool = S.shared_media_pool(args.media_pool) if args.media_pool > 0 else None

    def request(i):
        if pool is not None:  # requests on a few shared media
            return S.shared_media_request(np.random.Generator(np.random.PCG64([16180, i])), pool)
        return S.serving_request(np.random.Generator(np.random.PCG64([16177, i])))

    gaps = np.random.Generator(np.random.PCG64(16178)).exponential(1.0 / args.rate,
                                                                    size=args.requests)
    graphs_for = (lambda q: True) if args.serve_graphs == "all" else (lambda q: q.n <= 256 * 256)
    # pre-tuning: one plan per (grid, K) seen in the first requests of the stream
    t_tune = time.perf_counter()
    keys = {}
    for i in range(min(args.requests, 200)):
        q = request(i) if len(keys) < 21 else None
        if q is None:
            break
        keys.setdefault((q.shape, q.M, q.Mt), q)
    if not args.no_pretune:
        for (shape, M, Mt), q in sorted(keys.items(), key=lambda kv: str(kv[0])):
            med = hz.Medium(q.c, q.zeta, omega=q.omega, M=M, Mt=Mt, alpha=args.serve_alpha)
            plan = hz.Plan(med, precision=1, restart=q.restart, tol=q.tol, max_nrhs=4)
            plan.autotune()
            del plan, med
    t_tune = time.perf_counter() - t_tune

    def run_stream(nreq, slots, precision, batch_slots=0):
        srv = hz.Server(max_slots=slots, autotune=0 if not args.no_pretune else -1,
                        batch_slots=batch_slots, max_bypass=args.max_bypass, order=args.order)
        out_q = queue.Queue()
        stats = []
        pool = cf.ThreadPoolExecutor(max_workers=args.gen_threads)
        futs = {}
        ahead = 2 * args.gen_threads

        def collect():
            while True:
                item = out_q.get()
                if item is None:
                    return
                t, nr = item
                done, u, st, status = srv.result(t, timeout=7200)
                stats.append((done and status == 0 and all(x["converged"] for x in st), nr,
                              max(x["iters"] for x in st)))
                del u

        col = threading.Thread(target=collect, daemon=True)
        col.start()
        for i in range(min(ahead, nreq)):
            futs[i] = pool.submit(request, i)
        t0 = time.perf_counter()
        t_next = t0
        late = 0.0
        for i in range(nreq):
            q = futs.pop(i).result()
            if i + ahead < nreq:
                futs[i + ahead] = pool.submit(request, i + ahead)
            t_next += gaps[i]
            dt = t_next - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            else:
                late = max(late, -dt)
            t = srv.submit(q.c, q.f, omega=q.omega, M=q.M, Mt=q.Mt, zeta=q.zeta, alpha=args.serve_alpha,
                           restart=q.restart, tol=q.tol, precision=precision, graphs=graphs_for(q))
            out_q.put((t, q.f.shape[0]))
            del q
        out_q.put(None)
        col.join()
        span = time.perf_counter() - t0
        st = srv.stats()
        srv.close()
        pool.shutdown()
        return span, st, stats, late

    # warm-up: two requests through a server (module loading, pools)
    srv = hz.Server(max_slots=2)
    for i in range(2):
        q = request(i)
        srv.result(srv.submit(q.c, q.f, omega=q.omega, M=q.M, Mt=q.Mt, zeta=q.zeta, alpha=args.serve_alpha,
                              restart=q.restart, tol=q.tol), timeout=600)
    srv.close()

    sampler = ClockSampler(0)
    sampler.start()
    span, st, stats, late = run_stream(args.requests, args.slots, 1, args.batch_slots)
    clocks = sampler.stop()
    unbatched = None
    if args.batch_slots > 0:
        # the same stream with every request solved on its own
        span_u, st_u, stats_u, _ = run_stream(args.requests, args.slots, 1, 0)
        unbatched = {"value": sum(x[1] for x in stats_u) / span_u, "unit": "solves/s",
                     "p50_ms": st_u["p50_ms"], "p99_ms": st_u["p99_ms"], "span_s": span_u,
                     "all_converged": all(x[0] for x in stats_u)}
    rhs = sum(x[1] for x in stats)
    ok = all(x[0] for x in stats)
    plain = None
    if args.plain_requests > 0:
        nsub = min(args.plain_requests, args.requests)
        span_m, st_m, stats_m, _ = run_stream(nsub, args.slots, 1)
        span0, st0, stats0, late0 = run_stream(nsub, 1, 0)
        rhs_sub = sum(x[1] for x in stats0)
        plain = {"requests": nsub,
                 "mixed": {"value": rhs_sub / span_m, "p50_ms": st_m["p50_ms"],
                           "p99_ms": st_m["p99_ms"], "span_s": span_m},
                 "plain_fp64": {"value": rhs_sub / span0, "unit": "solves/s",
                                "p50_ms": st0["p50_ms"], "p99_ms": st0["p99_ms"],
                                "mean_ms": st0["mean_ms"], "span_s": span0,
                                "all_converged": all(x[0] for x in stats0),
                                "generation_late_s": late0},
                 "path": "precision 0 (complex128 preconditioner, FP64 GMRES), one request "
                         "on the GPU at a time, same requests and arrival times; 'mixed' is "
                         "the mixed-precision server on the same subset"}
    wl = (f"serving-shared{args.media_pool}media-{args.requests}req" if pool is not None
          else f"serving-{args.requests}req")
    out = {"metric": METRIC + " (serving stream)", "value": rhs / span, "unit": "solves/s",
           "n_gpus": 1, "steps": args.requests, "warmup": 2,
           "ms_per_step": 1e3 * span / args.requests, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
           "config": {"workload": f"{wl}-poisson{args.rate}/s-slots{args.slots}"
                                  f"-batch{args.batch_slots}-bypass{args.max_bypass}"
                                  f"-order{args.order}-alpha{args.serve_alpha}",
                      "grids": sorted({"x".join(map(str, k[0])) for k in keys}),
                      "rhs_total": rhs, "graphs": args.serve_graphs,
                      "pretune_s": t_tune, "pretuned_keys": 0 if args.no_pretune else len(keys)},
           "latency": {"p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "mean_ms": st["mean_ms"]},
           "server": st, "all_converged": ok, "generation_late_s": late,
           "iters_max": max(x[2] for x in stats), "clocks": clocks, "fp64_plain": plain,
           "unbatched": unbatched}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--workload", choices=["cfg2", "cfg1", "cfg3", "cfg4", "serving", "example1",
                                           "spectrum", "complexity", "interp"],
                    default=DEFAULT_WORKLOAD,
                    help="cfg3 (default): the 3D 256^3 K=16 workload; cfg2: 2D 1024^2 K=16")
    ap.add_argument("--requests", type=int, default=30, help="serving: number of requests")
    ap.add_argument("--ex1-n", type=int, nargs="+", default=[2400, 3600, 4800],
                    help="example1: grid sides N (the paper's Example 1 grids)")
    ap.add_argument("--spec-n", type=int, nargs="+", default=[120, 240, 480, 960],
                    help="spectrum: grid sides N (Table 2's grids)")
    ap.add_argument("--cx-n", type=int, nargs="+", default=[180, 360, 720, 1440, 2880],
                    help="complexity: grid sides N (Table 1's grids)")
    ap.add_argument("--int-n", type=int, default=1024, help="interp: grid side N")
    ap.add_argument("--rate", type=float, default=4.0, help="serving: arrivals per second")
    ap.add_argument("--slots", type=int, default=4, help="serving: concurrent requests")
    ap.add_argument("--serve-graphs", choices=["all", "small"], default="all",
                    help="serving: captured cycle graphs for every request or only <= 256^2")
    ap.add_argument("--no-pretune", action="store_true",
                    help="serving: no autotuning before the stream (served plans keep defaults)")
    ap.add_argument("--plain-requests", type=int, default=30,
                    help="serving: requests of the plain FP64 one-at-a-time comparison (0: none)")
    ap.add_argument("--n3d", type=int, default=256,
                    help="cfg3: side of the cube (256 is the workload; smaller for profiling)")
    ap.add_argument("--restart", type=int, default=0,
                    help="override the workload's restart length m (0: the workload's own)")
    ap.add_argument("--serve-alpha", type=float, default=0.1,
                    help="serving: node damping alpha of every request")
    ap.add_argument("--order", type=int, default=1, choices=[0, 1],
                    help="serving: admission order, 0 arrival order, 1 smallest footprint first")
    ap.add_argument("--max-bypass", type=int, default=0,
                    help="serving: aging limit (times a queued request may be overtaken; 0: 2 x slots)")
    ap.add_argument("--media-pool", type=int, default=0,
                    help="serving: draw requests (1-4 sources each) on this many shared media "
                         "instead of the serving recipe's one medium per request")
    ap.add_argument("--batch-slots", type=int, default=0,
                    help="serving: batched solves of this many slots for requests on the same "
                         "medium (0: each request alone); with > 0 the unbatched stream is run too")
    ap.add_argument("--gen-threads", type=int, default=6,
                    help="serving: producer threads generating requests ahead of arrival")
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="target oracle time of the CPU-baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch shapes")
    ap.add_argument("--tune", default="",
                    help='launch shapes as JSON instead of autotuning, e.g. \'{"rowinv_mode": 1}\'')
    ap.add_argument("--symbol-kind", type=int, default=0, choices=[0, 1],
                    help="0: continuous |xi|^2 (Eqn. 021), 1: the FD-consistent discrete symbol")
    ap.add_argument("--graphs", type=int, default=-1,
                    help="1/0: force CUDA-graph cycles on/off (default: per workload)")
    ap.add_argument("--no-plain", action="store_true",
                    help="skip the plain FP64 one-rhs-at-a-time comparison solve")
    ap.add_argument("--ref-iters", type=int, default=0,
                    help="reference arm: Arnoldi steps per solve to scale by (0: the GPU "
                         "solver's measured count for the workload)")
    args = ap.parse_args()
    from paper_2409_16172_gb300 import synth as S
    if args.workload == "serving":
        run_serving(args)
        return
    if args.workload == "example1":
        run_example1(args)
        return
    if args.workload == "spectrum":
        run_spectrum(args)
        return
    if args.workload == "complexity":
        run_complexity(args)
        return
    if args.workload == "interp":
        run_interp(args)
        return
    if args.workload == "cfg3" and args.n3d != 256:
        # the same 3D recipe on a smaller cube (profiling captures)
        p = S.config3(N=args.n3d)
    else:
        p = getattr(S, WORKLOADS[args.workload][0])()
    if args.restart > 0:
        p.restart = args.restart
    if args.impl == "reference":
        run_reference(args, p)
    else:
        run_gpu(args, p, args.workload)


if __name__ == "__main__":
    main()
