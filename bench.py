#!/usr/bin/env python
"""Benchmark: ms per all-mode Poisson solve at 512 x 128 x 400 to rel-res 1e-10.

Workload: the paper's 512 x 128 x 400 annular grid (65 azimuthal modes,
Sec. 5.2), FP64 batched Fourier-mode multigrid, synthetic Poisson-count
charge densities (seeds 0 .. S-1, one per step, cycled), solved to a relative
residual of 1e-10 of the three-dimensional system.  One step = one full solve
(forward rFFT + RHS, V-cycles, inverse transform).  Each charge density is
209.7 MB and each mode vector 213 MB, larger than the 129 MB L2, so no L2
flush is needed between steps.

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle
(conjugate gradient on the 3-D operator) on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "ms per all-mode Poisson solve at 512x128x400 to rel-res 1e-10; % HBM roofline"
UNIT = "ms"
GRID = (512, 128, 400)
FALLBACK_HBM_GBS = 6800.7
# committed ncu summaries holding the level-0 smoother's DRAM bytes per launch at 512x128x400
SMOOTH_PROFILE = {"fp64": "smooth_fp64_512x128x400.md", "mixed": "smooth_fused_defect_transforms_mixed_512x128x400.md"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=4)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--precision", choices=("fp64", "mixed"), default="fp64")
    ap.add_argument("--seeds", type=int, default=10)
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-field", action="store_true", help="skip the face-field reconstruction timing")
    ap.add_argument("--no-deposit", action="store_true", help="skip the CIC deposit timing")
    ap.add_argument("--deposit-ppc", type=int, default=4, help="macro-particles per cell and species (deposit timing)")
    ap.add_argument("--no-forms", action="store_true", help="skip timing the other precision form")
    ap.add_argument("--no-batch", action="store_true", help="skip the 24-problem uneven batch")
    ap.add_argument("--no-composite", action="store_true", help="skip the channel-plume composite domain")
    ap.add_argument("--no-sequence", action="store_true", help="skip the drifting-wave sequence")
    ap.add_argument("--sequence-steps", type=int, default=200)
    ap.add_argument("--tune-cache", default=None, help="JSON file caching autotuner results")
    ap.add_argument("--learned", action="store_true", help="(default) train and evaluate the learned warm start")
    ap.add_argument("--no-learned", action="store_true", help="skip training and evaluating the learned warm start")
    ap.add_argument("--no-conv", action="store_true", help="skip timing the U-Net convolutions and inference")
    ap.add_argument("--no-tune", action="store_true", help="default schedule instead of the autotuner's")
    ap.add_argument("--schedule", default=None,
                    help='JSON of Plan settings used instead of the autotuner\'s for every form, e.g. '
                         '\'{"smooth_strip": 2, "omega": 1.2}\'')
    ap.add_argument("--learned-steps", type=int, default=40, help="evaluation steps of the learned warm start")
    ap.add_argument("--learned-epochs", type=int, default=8)
    ap.add_argument("--grid", type=int, nargs=3, metavar=("NR", "NTHETA", "NZ"), default=None,
                    help="override the 512 128 400 grid (profiling of smaller cases)")
    return ap.parse_args()


# ------------------------------------------------------------------ helpers
def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback (MEASURED_PEAKS.json absent)"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.file = None

    def start(self):
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100",
                 "-i", str(self.gpu)], stdout=self.file, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [r.strip().split(", ") for r in self.file.read().strip().splitlines() if r.strip()]
        os.unlink(self.file.name)
        sm, mx, pw, reasons = [], [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in rows:
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                pw.append(float(r[3]))
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(pw)}


def traffic_from_profile(name):
    """Per-launch DRAM bytes recorded in a committed ncu summary, or None."""
    path = os.path.join(ROOT, "profiles", name)
    try:
        for line in open(path):
            if line.startswith("dram_bytes_per_launch_full_size:"):
                return float(line.split(":")[1])
    except OSError:
        pass
    return None


def workload_config(p, seeds, tol, world):
    """The workload both arms print, identical in each (`config`)."""
    tag = "%dx%dx%d" % (p.nr, p.ntheta, p.nz)
    return {"workload": "annulus %s, %d azimuthal modes, rho seeds %s (Poisson counts, mean 27, m=8 wave), "
                        "solved to rel-res %g" % (tag, p.n_modes, seeds, tol),
            "grid_nr_ntheta_nz": [p.nr, p.ntheta, p.nz], "tol": tol,
            "parallelism": "replicas" if world > 1 else "single GPU",
            "l2": "inputs larger than L2 (rho 209.7 MB, mode vector 213 MB per step)"}


def sum_phase(infos, key):
    return {k: sum(i[key][k] for i in infos) for k in infos[0][key]}


# ------------------------------------------------------------------ CPU oracle timing
def oracle_baseline(gpu_phis, tol):
    """The oracle as it stands on the host cores: one full conjugate-gradient
    solve of the seed-0 charge density to rel-res `tol`, timed outright; then
    the same solve continued to its rounding floor (a restart from that
    solution, true residual recomputed), against which the GPU forms' seed-0
    solutions are compared element by element (rel L2, and per azimuthal mode
    normalised by the whole solution).  Also a bounded one-core sample
    (scaled by the iteration count of the full solve) and the 32x16x32 case
    solved outright."""
    import numpy as np
    import oracle
    from paper_2609_07172_gb300 import workloads as W
    p = W.c1_problem()
    g = oracle.grid_from_problem(p)
    rho = W.rho_plasma(p, 0)
    threads = oracle.get_threads()
    t0 = time.perf_counter()
    phi_tol, info = oracle.solve3d(g, rho, tol=tol, maxit=100000, stall=0)
    t_tol = time.perf_counter() - t0
    t0 = time.perf_counter()
    phi_floor, info_f = oracle.solve3d(g, rho, tol=1e-15, x0=phi_tol)
    t_floor = time.perf_counter() - t0
    per_iter = t_tol / max(info["iterations"], 1)
    # one core: a bounded sample of CG iterations, scaled by the full solve's count
    oracle.set_threads(1)
    try:
        it1 = max(2, int(3.0 / max(per_iter * threads, 1e-3)))
        t0 = time.perf_counter()
        oracle.cg_fixed_iterations(g, rho, it1)
        per_iter1 = (time.perf_counter() - t0) / it1
    finally:
        oracle.set_threads(threads)
    # the small case solved outright: to rel-res 1e-10 and to the rounding floor
    p0 = W.c0_problem()
    g0 = oracle.grid_from_problem(p0)
    rho0 = W.rho_plasma(p0, 0)
    t0 = time.perf_counter()
    oracle.solve3d(g0, rho0, tol=1e-10)
    c0_tol = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.solve3d(g0, rho0, tol=1e-15)
    c0_floor = time.perf_counter() - t0

    def modes(x):
        xh = np.fft.rfft(x, axis=1) / x.shape[1]       # numpy: comparison bookkeeping only
        return np.sqrt((np.abs(xh) ** 2).sum(axis=(0, 2)))

    ref_norm = float(np.linalg.norm(phi_floor))
    ref_modes_norm = float(np.linalg.norm(modes(phi_floor)))
    parity = {"oracle_floor": {"cg_iterations_to_tol": info["iterations"],
                               "cg_iterations_tol_to_floor": info_f["iterations"],
                               "relres_true": info_f["relres"], "seconds": t_floor,
                               "rel_l2_tol_solution_vs_floor": float(np.linalg.norm(phi_tol - phi_floor)) / ref_norm}}
    for name, arr in gpu_phis.items():
        err = float(np.linalg.norm(arr - phi_floor)) / ref_norm
        parity[name] = {"rel_l2_vs_oracle": err,
                        "per_mode_max": float(modes(arr - phi_floor).max()) / ref_modes_norm}
    return {"ms": t_tol * 1e3, "iterations": info["iterations"], "relres_true": info["relres"],
            "threads": threads, "one_thread_ms": per_iter1 * info["iterations"] * 1e3,
            "one_thread_iters_timed": it1, "c0_seconds_to_1e-10": c0_tol, "c0_seconds_to_floor": c0_floor,
            "parity": parity}


def run_reference(args):
    """The oracle as it stands on this machine's host cores, on the GPU arm's
    workload: each step a bounded sample of CG iterations (about 4 s) on that
    step's charge density (seeds cycled as in the GPU arm), scaled by the
    iterations that seed needs to reach rel-res 1e-10 (recorded by
    oracle/cg_iterations.py; the cost of an iteration does not depend on the
    data)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from oracle import cg_iterations as CI
    from paper_2609_07172_gb300 import workloads as W
    p = W.c1_problem()
    g = oracle.grid_from_problem(p)
    seeds = list(range(args.seeds))
    t0 = time.perf_counter()
    oracle.cg_fixed_iterations(g, W.rho_plasma(p, 0), 2)
    per_iter = (time.perf_counter() - t0) / 2.0
    per_step_iters = max(4, int(4.0 / max(per_iter, 1e-3)))
    vals, rhos = [], {}
    for s in range(args.warmup + args.steps):
        seed = seeds[s % len(seeds)]
        if seed not in rhos:
            rhos[seed] = W.rho_plasma(p, seed)
        t0 = time.perf_counter()
        oracle.cg_fixed_iterations(g, rhos[seed], per_step_iters)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            vals.append(dt / per_step_iters * CI.iterations(seed) * 1e3)
    ms = statistics.median(vals)
    cores = oracle.get_threads()
    recorded = sorted(int(k) for k in CI.load()["seeds"])
    sample = (f"{per_step_iters} CG iterations per step on the full 512x128x400 system (step k: seed k mod "
              f"{len(seeds)}), scaled by the iterations that seed needs to reach rel-res 1e-10 (recorded for seeds "
              f"{recorded}; others use seed 0's)")
    line = {"impl": "reference", "metric": METRIC, "value": ms, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(p, seeds, args.tol, 1),
            "cpu_baseline": {"value": ms, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": ms, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ replicas
def max_over_ranks(value, world, dist, device):
    """The largest of the ranks' values (each rank's own when world == 1)."""
    if world <= 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_ms_per_solve(ms_total_max, steps, world):
    """Whole-job time per solve: `world` replicas each solved `steps` problems
    in at most `ms_total_max` (the slowest rank's time)."""
    return ms_total_max / (steps * world)


# ------------------------------------------------------------------ GPU arm
def time_form(plan, rhos, phi, steps, warmup, tol, world, dist, sampler=None):
    """Warm up, then time `steps` solves on the plan's stream; returns (ms total, infos, clocks)."""
    import torch
    for w in range(warmup):
        plan.solve(rhos[w % len(rhos)], phi, tol=tol)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    infos = []
    ev[0].record(plan.stream)
    for k in range(steps):
        _, info = plan.solve(rhos[k % len(rhos)], phi, tol=tol)
        infos.append(info)
        ev[k + 1].record(plan.stream)
    torch.cuda.synchronize()
    clocks = sampler.stop() if sampler else None
    if world > 1:
        dist.barrier()
    # per-solve times (each solve returns its info, so the steps do not overlap)
    for k, info in enumerate(infos):
        info["ms_event"] = ev[k].elapsed_time(ev[k + 1])
    return ev[0].elapsed_time(ev[-1]), infos, clocks


def percentiles(infos):
    xs = sorted(i["ms_event"] for i in infos)
    q = lambda f: xs[min(len(xs) - 1, int(round(f * (len(xs) - 1))))]
    return {"p10": q(0.1), "p50": q(0.5), "p90": q(0.9)}


def roofline(infos, prec_fp64, fp64_tflops, hbm_peak, hbm_src, traffic):
    """Roofline of the dominant kernel class from the library's PROFILE events
    and its algorithmic byte / flop accounting over the timed solves."""
    ms = sum_phase(infos, "ms_phase")
    by = sum_phase(infos, "bytes_phase")
    fl = sum_phase(infos, "flops_phase")
    n = sum_phase(infos, "launches_phase")
    dom = max(ms, key=ms.get)
    gbs = by[dom] / (ms[dom] * 1e-3) / 1e9 if ms[dom] > 0 else None
    tfs = fl[dom] / (ms[dom] * 1e-3) / 1e12 if ms[dom] > 0 else None
    per_launch_bytes = by[dom] / max(n[dom], 1)
    out = {"kernel_class": dom, "launches": n[dom], "ms_per_launch": ms[dom] / max(n[dom], 1),
           "algorithmic_bytes_per_launch": per_launch_bytes,
           "algorithmic_flops_per_launch": fl[dom] / max(n[dom], 1)}
    if prec_fp64:
        out.update({"bound": "alu", "achieved": tfs, "peak": fp64_tflops, "unit": "TFLOP/s",
                    "frac": tfs / fp64_tflops if tfs else None,
                    "peak_source": "measured: FP64 FMA throughput probe (pic_poisson_measure_fma_peaks) on this GPU",
                    "hbm_achieved_gbs": gbs, "hbm_peak_gbs": hbm_peak,
                    "hbm_frac": gbs / hbm_peak if gbs else None})
    else:
        out.update({"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
                    "frac": gbs / hbm_peak if gbs else None, "peak_source": hbm_src,
                    "fp64_tflops": tfs})
    out["traffic"] = traffic
    return out


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2609_07172_gb300 import FP64, MIXED, Plan, binding as B, measure_fma_peaks, query
    from paper_2609_07172_gb300 import workloads as W

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    B.load(build_if_missing=True)
    # wall seconds of each leg of this run (setup and tuning included), for the record
    legs, t_leg = {}, [time.perf_counter()]

    def leg(name):
        now = time.perf_counter()
        legs[name] = round(now - t_leg[0], 2)
        t_leg[0] = now

    prec = FP64 if args.precision == "fp64" else MIXED
    p = W.annulus(*args.grid) if args.grid else W.c1_problem()
    q = query(p, precision=prec)
    seeds = [rank * 1000 + s for s in range(args.seeds)]
    rhos = [torch.from_numpy(W.rho_plasma(p, s)).to(dev) for s in seeds]
    phi = torch.empty(p.shape, dtype=torch.float64, device=dev)
    fp64_gflops, fp32_gflops = measure_fma_peaks()
    hbm_peak, hbm_src = measured_peaks()
    tag = "%dx%dx%d" % (p.nr, p.ntheta, p.nz)

    # schedule (sweeps, FP32 inner cycles, smoother block size) picked by the
    # autotuner on this problem, outside the timed region (cached with --tune-cache)
    def tuned_kw(precision):
        if args.schedule:
            return json.loads(args.schedule), None
        if args.no_tune:
            return {}, None
        from paper_2609_07172_gb300 import autotune
        t = autotune([p], [rhos[0]], tol=args.tol, precision=precision, graph=True, repeats=2,
                     cache=args.tune_cache)
        return {k: t[k] for k in ("pre_sweeps", "post_sweeps", "inner_cycles", "smooth_threads", "smooth_strip",
                                  "omega", "smooth_fused", "fmg", "inner_first") if k in t}, t

    kw, tuned = tuned_kw(prec)
    schedules = {args.precision: kw}
    # headline: each solve one CUDA graph (device-side convergence loop)
    plan = Plan(p, precision=prec, graph=True, **kw)
    ms_total, infos, clocks = time_form(plan, rhos, phi, args.steps, args.warmup, args.tol, world, dist,
                                        ClockSampler(local))
    ms_total = max_over_ranks(ms_total, world, dist, dev)
    ms_local = ms_total / args.steps
    ms_per_solve = job_ms_per_solve(ms_total, args.steps, world)
    cycles = [i["cycles"] for i in infos]
    by = sum_phase(infos, "bytes_phase")
    solve_gbs = sum(by.values()) / len(infos) / (ms_local * 1e-3) / 1e9
    # profiled pass: the same solves through the host-driven loop with CUDA events
    # around every launch, for per-kernel-class times and the roofline
    pplan = Plan(p, precision=prec, profile=True, **kw)
    ms_prof, pinfos, _ = time_form(pplan, rhos, phi, args.steps, 2, args.tol, world, dist)
    pplan.close()
    ms_ph = sum_phase(pinfos, "ms_phase")
    # DRAM bytes of a level-0 half-sweep at 512x128x400 (ncu, scaled from 512x128x200 where valid)
    traffic = traffic_from_profile(SMOOTH_PROFILE[args.precision]) if tag == "512x128x400" else None
    sched = {"pre_sweeps": kw.get("pre_sweeps", 2), "post_sweeps": kw.get("post_sweeps", 2),
             "inner_cycles": kw.get("inner_cycles", 2), "smooth_threads": kw.get("smooth_threads", 256),
             "smooth_strip": kw.get("smooth_strip", 0), "omega": kw.get("omega", 1.0),
             "smooth_fused": kw.get("smooth_fused", 0), "fmg": kw.get("fmg", 0),
             "inner_first": kw.get("inner_first", 0)}

    line = {"metric": METRIC, "value": ms_per_solve, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_local, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if prec == FP64 else "f32+f64",
            "data": "synthetic",
            "config": workload_config(p, seeds, args.tol, world),
            "solver": {"form": "%s batched GMG" % args.precision, "levels": q["levels"], "schedule": sched,
                       "driver": "one CUDA graph per solve (PIC_POISSON_GRAPH)"},
            "status": sorted({i["status"] for i in infos}),
            "cycles": {"min": min(cycles), "max": max(cycles), "median": statistics.median(cycles)},
            "ms_per_solve_percentiles": percentiles(infos),
            "rel_res_max": max(i["rel_res"] for i in infos),
            "gpu_launches": int(sum(i["launches"] for i in infos)),
            "phase_ms_per_solve": {k: v / len(pinfos) for k, v in ms_ph.items()},
            "roofline": dict(roofline(pinfos, prec == FP64, fp64_gflops / 1e3, hbm_peak, hbm_src, traffic),
                             timed_region="profiled pass: the same %d solves through the host-driven loop with "
                                          "CUDA events around every launch" % args.steps),
            "hbm_roofline_solve": {"achieved_gbs": solve_gbs, "peak_gbs": hbm_peak, "frac": solve_gbs / hbm_peak,
                                   "algorithmic_bytes_per_solve": sum(by.values()) / len(infos),
                                   "peak_source": hbm_src},
            "fma_peaks_gflops": {"fp64": fp64_gflops, "fp32": fp32_gflops},
            "clocks": clocks,
            "host_loop_profiled_ms_per_solve": ms_prof / args.steps}
    if tuned:
        line["autotune"] = {"candidates": len(tuned.get("tried", [])), "best_ms": tuned.get("ms")}
    leg("headline (tuning, timed and profiled solves)")

    # ---- end to end through the C ABI with host buffers (pinned), copies inside the timed region
    if not args.no_e2e:
        # one pinned host buffer per field, reused every step as a particle code
        # reuses its deposit and field arrays (the transfers are of the full
        # arrays each step)
        rho_h = rhos[0].cpu().pin_memory()
        phi_h = torch.empty(p.shape, dtype=torch.float64).pin_memory()
        ne = max(3, args.steps // 4)

        def host_ms(hplan):
            for _ in range(2):
                hplan.solve_host(rho_h, phi_h, tol=args.tol)
            if world > 1:
                dist.barrier()
            t0 = time.perf_counter()
            for k in range(ne):
                hplan.solve_host(rho_h, phi_h, tol=args.tol)
            return job_ms_per_solve(max_over_ranks((time.perf_counter() - t0) * 1e3, world, dist, dev), ne, world)

        # default path: the transforms read rho_h and write phi_h in place over
        # the CPU-GPU link; for comparison, the same call through device staging copies
        e2e_ms = host_ms(plan)
        with Plan(p, precision=prec, graph=True, host_staged=True, **kw) as splan:
            staged_ms = host_ms(splan)
        nbytes = p.nr * p.ntheta * p.nz * 8
        line["e2e"] = {"value": e2e_ms, "unit": UNIT, "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
                       "steps": ne, "api": "pic_poisson_solve_host (pinned host buffers, read and written in place "
                                           "by the transforms)",
                       "staged_ms_per_solve": staged_ms}
        leg("e2e")
    ref_phi = phi.clone()
    # seed-0 solutions for the element-wise comparison with the oracle (cpu_baseline leg)
    want_parity = not args.no_cpu_baseline and rank == 0 and world == 1 and tag == "512x128x400"
    gpu_phis = {}
    if want_parity:
        for label, t in (("tol", args.tol), ("floor", 0.0)):
            plan.solve(rhos[0], phi, tol=t)
            torch.cuda.synchronize()
            gpu_phis["%s_%s" % (args.precision, label)] = phi.cpu().numpy()
        leg("seed-0 solves for the oracle comparison")

    # ---- face-field reconstruction of the solved potential (the PIC step after the solve)
    if not args.no_field:
        er, ea, ez = plan.face_field(phi)
        for _ in range(3):
            plan.face_field(phi, er, ea, ez)
        st = torch.cuda.current_stream()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(10)]
        torch.cuda.synchronize()
        for a, b in evs:
            a.record(plan.stream)
            plan.face_field(phi, er, ea, ez)
            b.record(plan.stream)
        torch.cuda.synchronize()
        fms = statistics.median(a.elapsed_time(b) for a, b in evs)
        cells = p.nr * p.ntheta * p.nz
        fbytes = 8.0 * (cells + er.numel() + ea.numel() + ez.numel())   # phi read once, three face arrays written
        fp64_instr = 6.0 * cells                                         # one subtraction, one multiplication per face
        line["face_field"] = {"ms": fms, "achieved_gbs": fbytes / fms / 1e6, "peak_gbs": hbm_peak,
                              "hbm_frac": fbytes / fms / 1e6 / hbm_peak,
                              "fp64_issue_frac": fp64_instr / (fms * 1e-3) / (fp64_gflops * 1e9 / 2.0),
                              "bound": "alu (FP64: 6 instructions per cell)",
                              "algorithmic_bytes": fbytes, "launches": len(evs)}
        del er, ea, ez
        leg("face field")

    # ---- CIC deposit of two species and projection to rho (the PIC step before the solve)
    if not args.no_deposit and args.deposit_ppc > 0:
        line["deposit"] = run_deposit(args, plan, p)
        leg("deposit")
    plan.close()

    # ---- the other form on the same GPU and inputs (mixed FP32/FP64 when the headline is FP64)
    if not args.no_forms:
        other = MIXED if prec == FP64 else FP64
        name = "mixed" if other == MIXED else "fp64"
        kw2, _ = tuned_kw(other)
        schedules[name] = kw2
        plan2 = Plan(p, precision=other, graph=True, **kw2)
        steps2 = max(4, args.steps // 2)
        phi2 = torch.empty_like(phi)
        ms2, infos2, _ = time_form(plan2, rhos, phi2, steps2, 2, args.tol, world, dist)
        plan2.solve(rhos[(args.steps - 1) % len(rhos)], phi2, tol=args.tol)
        torch.cuda.synchronize()
        diff = float(torch.linalg.vector_norm(phi2 - ref_phi) / torch.linalg.vector_norm(ref_phi))
        if want_parity:
            for label, t in (("tol", args.tol), ("floor", 0.0)):
                plan2.solve(rhos[0], phi2, tol=t)
                torch.cuda.synchronize()
                gpu_phis["%s_%s" % (name, label)] = phi2.cpu().numpy()
        plan2.close()
        pplan2 = Plan(p, precision=other, profile=True, **kw2)
        _, pinfos2, _ = time_form(pplan2, rhos, phi2, steps2, 1, args.tol, world, dist)
        pplan2.close()
        by2 = sum_phase(infos2, "bytes_phase")
        ms2_solve = ms2 / steps2
        gbs2 = sum(by2.values()) / len(infos2) / (ms2_solve * 1e-3) / 1e9
        c2 = [i["cycles"] for i in infos2]
        line["forms"] = {name: {
            "ms_per_solve": ms2_solve, "steps": steps2, "ms_per_solve_percentiles": percentiles(infos2), "dtype": "f32+f64" if other == MIXED else "f64",
            "schedule": kw2 or "defaults", "cycles_median": statistics.median(c2),
            "outer_iterations_median": statistics.median([i["outer_iterations"] for i in infos2]),
            "rel_res_max": max(i["rel_res"] for i in infos2),
            "rel_l2_vs_headline_phi": diff,
            "phase_ms_per_solve": {k: v / len(pinfos2) for k, v in sum_phase(pinfos2, "ms_phase").items()},
            "roofline": roofline(pinfos2, other == FP64, fp64_gflops / 1e3, hbm_peak, hbm_src,
                                 traffic_from_profile(SMOOTH_PROFILE[name])
                                 if tag == "512x128x400" else None),
            "hbm_roofline_solve": {"achieved_gbs": gbs2, "peak_gbs": hbm_peak, "frac": gbs2 / hbm_peak}}}
        leg("other form")

    if not args.no_composite:
        line["composite_channel_plume"] = run_composite(args, schedules, world, dist)
        leg("composite and axial-mesh workloads")
    if not args.no_batch:
        line["batch_uneven"] = run_batch(args, dev, hbm_peak, fp64_gflops / 1e3)
        leg("uneven batch")
    if not args.no_sequence:
        line["sequence"] = run_sequence(args, dev, p, schedules)
        leg("sequence")
    if not args.no_conv:
        line["learned_conv"] = run_conv(args, dev, p, ms_per_solve / max(statistics.median(cycles), 1))
        leg("tcgen05 convolution")
    if not args.no_learned:
        try:
            line["learned_warm_start"] = run_learned(args, dev, p)
        except RuntimeError as exc:   # reported, not fatal to the benchmark line
            line["learned_warm_start"] = {"error": str(exc)}
        leg("learned warm start")

    if not args.no_cpu_baseline and rank == 0 and world == 1:
        det = oracle_baseline(gpu_phis, args.tol)
        line["cpu_baseline"] = {"value": det["ms"], "unit": UNIT, "cores": det["threads"], "kind": "oracle",
                                "sample": "one full FP64 oracle CG solve of the 512x128x400 system (rho seed 0) "
                                          "to rel-res %g, run outright: %d iterations, true rel-res %.3g"
                                          % (args.tol, det["iterations"], det["relres_true"]),
                                "one_thread": {"value": det["one_thread_ms"], "unit": UNIT, "cores": 1,
                                               "sample": "%d CG iterations on one core, scaled by the %d of "
                                                         "the full solve" % (det["one_thread_iters_timed"],
                                                                             det["iterations"])},
                                "c0_32x16x32_s": {"to_rel_res_1e-10": det["c0_seconds_to_1e-10"],
                                                  "to_floor": det["c0_seconds_to_floor"],
                                                  "cores": det["threads"]}}
        if gpu_phis:
            line["rel_l2_vs_oracle"] = dict(det["parity"], note=(
                "seed 0; GPU forms solved to rel-res %g (tol) and to their rounding floor (floor), each "
                "against the oracle's CG solution continued to its floor; per_mode_max: largest per-mode "
                "error norm over the whole solution's norm" % args.tol))
        leg("CPU oracle")
    line["leg_seconds"] = legs
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_composite(args, schedules, world, dist):
    """The channel-plume composite domain (two patches of the bounding annulus,
    grounded exposed faces, charge only inside) at 512 x 128 x 384: the
    headline grid with 384 axial cells, so that the exit plane at nz / 2 stays
    on a coarse face down to a small dense coarsest level.  FP64 and mixed
    solves to the benchmark tolerance, each one CUDA graph, each with the
    autotuner's schedule for that problem and form (_time_forms).  Then the
    same for a non-uniform axial mesh on the headline grid."""
    import torch
    from paper_2609_07172_gb300 import FP64, MIXED, Plan, workloads as W
    import numpy as np
    p = W.channel_plume(512, 128, 384)
    out = {"workload": "channel_plume_512x128x384", "active_cells_rz": int(p.active_cells().sum()),
           "patches": [list(q) for q in p.patches]}
    out.update(_time_forms(args, schedules, world, dist, p, 900))
    # a non-uniform axial mesh on the headline grid: each cell 1.002 times as
    # tall as the one below it (the top cell 2.2 times the bottom one)
    q = W.annulus(512, 128, 400)
    w = 1.002 ** np.arange(q.nz)
    q = q.with_z_faces(q.z0 + (q.z1 - q.z0) * np.r_[0.0, np.cumsum(w)] / w.sum())
    out["axial_stretched_512x128x400"] = dict(_time_forms(args, schedules, world, dist, q, 950),
                                              ratio=1.002)
    return out


def _time_forms(args, schedules, world, dist, p, seed0):
    """FP64 and mixed graph solves of problem p to the benchmark tolerance,
    each with the autotuner's schedule for this problem (cached with
    --tune-cache; with --schedule or --no-tune: the headline forms' settings
    without the fused smoother)."""
    import torch
    from paper_2609_07172_gb300 import FP64, MIXED, Plan, workloads as W
    rhos = [W.rho_plasma_torch(p, seed0 + s) for s in range(4)]
    phi = torch.empty(p.shape, dtype=torch.float64, device="cuda")
    out = {}
    for name, prec in (("fp64", FP64), ("mixed", MIXED)):
        if args.schedule or args.no_tune:
            kw = dict(schedules.get(name) or {})
            kw["smooth_fused"] = 0
        else:
            from paper_2609_07172_gb300 import autotune
            t = autotune([p], [rhos[0]], tol=args.tol, precision=prec, graph=True, repeats=2,
                         cache=args.tune_cache)
            kw = {k: t[k] for k in ("pre_sweeps", "post_sweeps", "inner_cycles", "smooth_threads", "smooth_strip",
                                    "omega", "smooth_fused", "fmg", "inner_first") if k in t}
        with Plan(p, precision=prec, graph=True, **kw) as plan:
            steps = max(4, args.steps // 4)
            ms, infos, _ = time_form(plan, rhos, phi, steps, 2, args.tol, world, dist)
        # one profiled host-loop solve: where the time goes (CUDA events
        # around every launch; not the timed figure above)
        with Plan(p, precision=prec, profile=True, **kw) as plan:
            _, pinfo = plan.solve(rhos[0], phi, tol=args.tol)
        out[name] = {"ms_per_solve": ms / steps, "steps": steps, "schedule": kw,
                     "cycles_median": statistics.median(i["cycles"] for i in infos),
                     "rel_res_max": max(i["rel_res"] for i in infos),
                     "status": sorted({i["status"] for i in infos}),
                     "profiled_phase_ms": {k: v for k, v in pinfo["ms_phase"].items() if v > 0}}
    del rhos, phi
    torch.cuda.empty_cache()
    return out


def run_deposit(args, plan, p):
    """Ions and electrons, args.deposit_ppc per cell each, uniformly inside
    their cells and in cell-major order (as a periodically sorted particle
    array), deposited to the nodes and projected to rho; CUDA events."""
    import torch
    ppc = args.deposit_ppc
    cells = p.nr * p.ntheta * p.nz
    dr, dz, da = (p.r_out - p.r_in) / p.nr, (p.z1 - p.z0) / p.nz, p.theta_span / p.ntheta
    gen = torch.Generator(device="cuda").manual_seed(11)

    def species():
        c = torch.arange(cells * ppc, device="cuda", dtype=torch.int64) // ppc
        i, rest = c % p.nr, c // p.nr
        j, k = rest % p.ntheta, rest // p.ntheta
        u = torch.rand((3, c.numel()), device="cuda", dtype=torch.float64, generator=gen)
        return (p.r_in + (i + u[0]) * dr, (j + u[1]) * da, p.z0 + (k + u[2]) * dz)

    ions, elec = species(), species()
    w, e = 1e8, 1.602176634e-19
    ni = torch.zeros(plan.node_shape(), dtype=torch.float64, device="cuda")
    ne = torch.zeros_like(ni)
    rho = torch.empty(p.shape, dtype=torch.float64, device="cuda")

    def step():
        ni.zero_()
        ne.zero_()
        plan.deposit(*ions, w, ni)
        plan.deposit(*elec, w, ne)
        plan.project(ni, e, rho)
        plan.project(ne, -e, rho, accumulate=True)

    for _ in range(2):
        step()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(5)]
    torch.cuda.synchronize()
    for a, b in evs:
        a.record(plan.stream)
        step()
        b.record(plan.stream)
    torch.cuda.synchronize()
    ms = statistics.median(a.elapsed_time(b) for a, b in evs)
    n = 2 * cells * ppc
    # charge check: the projected charge of the equal ion and electron counts is zero up to rounding
    rc = p.r_in + (torch.arange(p.nr, device="cuda", dtype=torch.float64) + 0.5) * dr
    qsum = float((rho * (rc * dr * da * dz)).sum())
    out = {"ms": ms, "particles": n, "particles_per_s": n / (ms * 1e-3), "per_cell_per_species": ppc,
           "order": "cell-major (sorted)", "kernels": "k_deposit x2 (warp-aggregated FP64 atomics), k_project x2",
           "net_charge_over_ion_charge": qsum / (e * w * cells * ppc)}
    del ions, elec, ni, ne, rho
    torch.cuda.empty_cache()
    return out


def run_batch(args, dev, hbm_peak, fp64_tflops):
    """24 independent problems of uneven sizes (seed 3) in one batched, autotuned,
    graph-captured plan vs one graph-captured plan per problem."""
    import torch
    from paper_2609_07172_gb300 import FP64, BatchPlan, Plan, autotune
    from paper_2609_07172_gb300 import workloads as W
    probs = W.uneven_batch(3)
    problems = [p for p, _ in probs]
    rhos = [torch.from_numpy(W.rho_plasma(p, s)).to(dev) for p, s in probs]
    tuned = autotune(problems, rhos, tol=args.tol, precision=FP64, graph=True, repeats=2, cache=args.tune_cache)
    kw = {k: tuned[k] for k in ("pre_sweeps", "post_sweeps", "inner_cycles", "smooth_threads", "smooth_strip",
                                "omega", "smooth_fused", "fmg", "inner_first") if k in tuned}
    bp = BatchPlan(problems, graph=True, **kw)
    phis = [torch.empty_like(r) for r in rhos]
    for _ in range(2):
        bp.solve(rhos, phis, tol=args.tol)
    steps = max(3, args.steps // 8)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(steps):
        _, infos = bp.solve(rhos, phis, tol=args.tol)
    e1.record()
    torch.cuda.synchronize()
    ms_batch = e0.elapsed_time(e1) / steps
    launches = infos[0]["launches"]
    bp.close()
    # the same batch through the host loop with events around every launch:
    # the sum of its kernels' device times, against the graph's wall time (the
    # gaps between launches are what one persistent launch would save)
    pbp = BatchPlan(problems, profile=True, **kw)
    _, pinf = pbp.solve(rhos, phis, tol=args.tol)
    kernel_ms = sum(pinf[0]["ms_phase"].values())
    pbp.close()
    plans = [Plan(q, graph=True, **kw) for q in problems]
    # each problem's own algorithmic bytes and flops (its own cycle count): the
    # work the batch has to do, for its roofline
    alg_bytes = alg_flops = 0.0
    for pl, r, f in zip(plans, rhos, phis):
        _, inf1 = pl.solve(r, f, tol=args.tol)
        alg_bytes += sum(inf1["bytes_phase"].values())
        alg_flops += sum(inf1["flops_phase"].values())
    torch.cuda.synchronize()
    e0.record()
    for _ in range(steps):
        for pl, r, f in zip(plans, rhos, phis):
            pl.solve(r, f, tol=args.tol)
    e1.record()
    torch.cuda.synchronize()
    ms_each = e0.elapsed_time(e1) / steps
    for pl in plans:
        pl.close()
    # the same batch in the mixed form (FP32 V-cycles in FP64 defect
    # correction), autotuned on the batch
    from paper_2609_07172_gb300 import MIXED
    try:
        mt = autotune(problems, rhos, tol=args.tol, precision=MIXED, graph=True, repeats=2, cache=args.tune_cache)
        mkw = {k: mt[k] for k in ("pre_sweeps", "post_sweeps", "inner_cycles", "smooth_threads", "smooth_strip",
                                  "omega", "smooth_fused", "fmg", "inner_first") if k in mt}
        mbp = BatchPlan(problems, precision=MIXED, graph=True, **mkw)
        for _ in range(2):
            mbp.solve(rhos, phis, tol=args.tol)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(steps):
            _, minfos = mbp.solve(rhos, phis, tol=args.tol)
        e1.record()
        torch.cuda.synchronize()
        ms_mixed = e0.elapsed_time(e1) / steps
        mbp.close()
        mixed = {"ms_per_batch": ms_mixed, "cycles": minfos[0]["cycles"],
                 "outer_iterations": minfos[0]["outer_iterations"],
                 "rel_res_max": max(i["rel_res"] for i in minfos), "autotuned": dict(mkw, ms=mt.get("ms")),
                 "status": sorted({i["status"] for i in minfos})}
    except RuntimeError as exc:   # reported, not fatal to the benchmark line
        mixed = {"error": str(exc)}
    return {"workload": "24 problems, N_r in {64..512}, N_theta in {16..128}, N_z in {64,200,400} (seed 3), "
                        "FP64, rel-res %g" % args.tol,
            "cells_total": int(sum(q.nr * q.ntheta * q.nz for q in problems)),
            "ms_per_batch": ms_batch, "ms_one_plan_per_problem": ms_each, "steps": steps,
            "cycles": infos[0]["cycles"], "rel_res_max": max(i["rel_res"] for i in infos),
            "launches_per_batch": launches, "autotuned": dict(kw, ms=tuned.get("ms")),
            "kernel_ms_per_batch": kernel_ms,
            "gap_ms_per_batch": ms_batch - kernel_ms,
            "roofline": {"algorithmic_bytes_per_batch": alg_bytes, "algorithmic_flops_per_batch": alg_flops,
                         "achieved_gbs": alg_bytes / (ms_batch * 1e-3) / 1e9, "peak_gbs": hbm_peak,
                         "hbm_frac": alg_bytes / (ms_batch * 1e-3) / 1e9 / hbm_peak,
                         "fp64_tflops": alg_flops / (ms_batch * 1e-3) / 1e12, "fp64_peak_tflops": fp64_tflops,
                         "fp64_frac": alg_flops / (ms_batch * 1e-3) / 1e12 / fp64_tflops,
                         "note": "the sum of each problem's own algorithmic bytes and FP64 flops (its own cycles) "
                                 "over the batched solve's time"},
            "autotune_candidates": len(tuned.get("tried", [])) or None,
            "mixed": mixed}


def run_sequence(args, dev, p, schedules):
    """Drifting m = 8 wave (one azimuthal cell per step) at the headline grid,
    solved back to back with the previous step's mode-space iterate as initial
    guess (pic_poisson_get_modes, then pic_poisson_solve_modes; with fmg the
    full-multigrid start runs on the guess's correction equation),
    against the zero initial guess, both graph-captured with the form's tuned
    schedule."""
    import torch
    from paper_2609_07172_gb300 import FP64, MIXED, Plan
    from paper_2609_07172_gb300 import workloads as W
    out = {"workload": "%dx%dx%d drifting m=8 wave, %d steps, GPU-drawn Poisson counts (seeded)"
                       % (p.nr, p.ntheta, p.nz, args.sequence_steps), "tol": args.tol}
    for name, prec in (("fp64", FP64), ("mixed", MIXED)):
        kw = schedules.get(name, {})
        warm = Plan(p, precision=prec, graph=True, **kw)
        zero = Plan(p, precision=prec, graph=True, **kw)
        phi = torch.zeros(p.shape, dtype=torch.float64, device=dev)
        tmp = torch.empty_like(phi)
        uh = torch.zeros(warm.mode_shape, dtype=torch.float64, device=dev)
        ms_w = ms_z = 0.0
        cyc_w, cyc_z = [], []
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for t in range(args.sequence_steps):
            rho = W.drifting_rho_torch(p, t, device=dev)
            torch.cuda.synchronize()
            e0.record()
            # the previous step's mode-space iterate as the initial guess (no transform of phi)
            _, iw = warm.solve_modes(rho, uh, phi, tol=args.tol)
            warm.get_modes(uh)
            e1.record()
            torch.cuda.synchronize()
            if t > 0:
                ms_w += e0.elapsed_time(e1)
                cyc_w.append(iw["cycles"])
            if t % 20 == 1:                      # zero-guess reference on a sample of steps
                e0.record()
                _, iz = zero.solve(rho, tmp, tol=args.tol)
                e1.record()
                torch.cuda.synchronize()
                ms_z += e0.elapsed_time(e1)
                cyc_z.append(iz["cycles"])
        n = args.sequence_steps - 1
        out[name] = {"schedule": kw or "defaults",
                     "ms_per_step_prev_guess": ms_w / n, "cycles_per_step_prev_guess": sum(cyc_w) / n,
                     "ms_per_step_zero_guess": ms_z / len(cyc_z), "cycles_per_step_zero_guess":
                         sum(cyc_z) / len(cyc_z), "zero_guess_sampled_steps": len(cyc_z)}
        warm.close()
        zero.close()
    return out


def run_conv(args, dev, p, ms_per_cycle):
    """The U-Net's convolutions at the warm start's size (65 modes on the
    256 x 200 grid and its three coarser levels): tcgen05 implicit GEMM
    (pic_nn_conv3x3) against the legacy mma.sync kernel, CUDA events, median
    of 10; then the whole warm-start inference (residual, restriction, pack,
    U-Net, unpack, prolongation, minimal-residual step; random weights -- the
    cost does not depend on them) with each, against one V-cycle."""
    import torch
    from paper_2609_07172_gb300 import Plan, learned as LW
    from paper_2609_07172_gb300.unet import P as TP, UNet, _ok, _st, nn_lib
    lib = nn_lib()
    n = p.ntheta // 2 + 1
    h0, w0 = p.nz // 2, p.nr // 2
    layers = [("e0", 0, 16, 16), ("e1", 1, 16, 32), ("e2", 2, 32, 64), ("b1", 3, 64, 128), ("b2", 3, 128, 64),
              ("d2", 2, 128, 32), ("d1", 1, 64, 16), ("d0", 0, 32, 16), ("out", 0, 16, 16)]
    g = torch.Generator(device=dev).manual_seed(17)
    out = {}
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(10)]
    st = torch.cuda.current_stream()
    for name, lv, cin, cout in layers:
        h, w = h0 >> lv, w0 >> lv
        x = torch.randn(n, h, w, cin, device=dev, generator=g).to(torch.bfloat16)
        wt = (torch.randn(9, cout, cin, device=dev, generator=g) / (9 * cin) ** 0.5).to(torch.bfloat16)
        b = torch.randn(cout, device=dev, generator=g)
        y = torch.empty(n, h, w, cout, dtype=torch.bfloat16, device=dev)
        rec = {"shape": [n, h, w, cin, cout]}
        for entry, key in (("pic_nn_conv3x3", "tcgen05"), ("pic_nn_conv3x3_mma_sync", "mma_sync")):
            f = getattr(lib, entry)
            for _ in range(3):
                _ok(f(TP(x), cin, TP(wt), TP(b), TP(y), None, cout, n, h, w, 1, _st()))
            torch.cuda.synchronize()
            for a, e in evs:
                a.record(st)
                _ok(f(TP(x), cin, TP(wt), TP(b), TP(y), None, cout, n, h, w, 1, _st()))
                e.record(st)
            torch.cuda.synchronize()
            rec[key + "_us"] = statistics.median(a.elapsed_time(e) for a, e in evs) * 1e3
        pix = n * h * w
        rec["algorithmic_bytes"] = 2.0 * pix * (cin + cout) + 2.0 * 9 * cin * cout
        rec["flops"] = 2.0 * pix * cout * 9 * cin
        t = rec["tcgen05_us"] * 1e-6
        rec["tcgen05_gbs"] = rec["algorithmic_bytes"] / t / 1e9
        rec["tcgen05_tflops"] = rec["flops"] / t / 1e12
        out[name] = rec
        del x, wt, b, y
    st_err = conv_tc_status(lib)
    # the whole warm-start inference with each convolution path
    plan = Plan(p, graph=True)
    net = UNet(seed=0)
    ws = LW.WarmStart(net, 1.0, p, plan)
    from paper_2609_07172_gb300 import workloads as W
    bhat = plan.forward(W.drifting_rho_torch(p, 0))
    u = torch.zeros(plan.mode_shape, dtype=torch.float64, device=dev)
    inf = {}
    for entry, key in (("pic_nn_conv3x3", "tcgen05"), ("pic_nn_conv3x3_mma_sync", "mma_sync")):
        net.conv_entry = entry
        for _ in range(2):
            ws.guess(bhat, u)
        torch.cuda.synchronize()
        a, e = evs[0]
        a.record(st)
        for _ in range(5):
            ws.guess(bhat, u)
        e.record(st)
        torch.cuda.synchronize()
        inf[key + "_ms"] = a.elapsed_time(e) / 5
    plan.close()
    dom = max(out, key=lambda k: out[k]["tcgen05_us"])
    return {"layers": out, "tc_wait_status": st_err, "warm_start_inference": inf,
            "solve_ms_per_cycle": ms_per_cycle,
            "dominant_layer": dom,
            "note": "65 samples (modes) per layer on the 256x200 grid and its coarser levels; algorithmic bytes = "
                    "input + output activations + weights in BF16; flops = 2 x pixels x cout x 9 cin"}


def conv_tc_status(lib):
    import ctypes
    st = ctypes.c_int(-1)
    lib.pic_nn_conv_tc_status(ctypes.byref(st))
    return st.value


def run_learned(args, dev, p):
    """Learned warm start: train the U-Net on 3000 (residual, correction) pairs from
    plain solves of a 256x64x200 drifting-wave sequence (seed 7), then solve the
    drifting sequence at the headline grid from the learned guess vs the
    previous-step guess (inference, extra transform and step included)."""
    import torch
    from paper_2609_07172_gb300 import learned as LW, workloads as W
    from paper_2609_07172_gb300.unet import UNet
    t0 = time.perf_counter()
    pt = W.annulus(256, 64, 200)
    steps = -(-3000 // pt.n_modes)
    X, Y, gain = LW.training_pairs(pt, steps=steps, seed=7, limit=3000)
    t_data = time.perf_counter() - t0
    net = UNet(seed=0)
    t0 = time.perf_counter()
    losses = LW.train(net, X, Y, epochs=args.learned_epochs, batch=16, lr=1e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    del X, Y
    res = LW.evaluate_sequence(net, gain, p, steps=args.learned_steps, tol=args.tol, coarse=True, gpu_inputs=True,
                               bound=True,
                               seed=3)
    # inference alone (pack, U-Net, unpack, prolongation, minimal-residual step)
    plan = None
    from paper_2609_07172_gb300 import Plan
    plan = Plan(p, graph=True)
    ws = LW.WarmStart(net, gain, p, plan)
    rho = W.drifting_rho_torch(p, 0)
    bhat = plan.forward(rho)
    u = torch.zeros(plan.mode_shape, dtype=torch.float64, device=dev)
    ws.guess(bhat, u)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(5):
        ws.guess(bhat, u)
    e1.record()
    torch.cuda.synchronize()
    inf_ms = e0.elapsed_time(e1) / 5
    plan.close()
    return {"train": {"grid": "256x64x200 drifting m=8 wave, seed 7", "pairs": 3000, "params": net.n_params(),
                      "epochs": args.learned_epochs, "batch": 16, "data_s": t_data, "train_s": t_train,
                      "loss_epoch_mean": losses},
            "eval": {k: v for k, v in res.items() if k != "records"},
            "warm_start_ms": inf_ms,
            "note": "learned = forward transform + residual of the previous iterate + U-Net on the 2:1 restricted "
                    "residual (65 modes at 256x200) + prolongation + minimal-residual step, then the solve; "
                    "prev = solve from the previous-step modes; both graph-captured FP64 to rel-res %g" % args.tol}


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
