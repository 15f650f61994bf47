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


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=4)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--precision", choices=("fp64", "mixed"), default="fp64")
    ap.add_argument("--seeds", type=int, default=4)
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--extra-forms", action="store_true", help="also time the mixed-precision form")
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


def v_bytes(nr, nz, nm, word=8):
    return nr * nz * nm * 2 * word


def algorithmic_model(q, info_list, pre, post, word=8, grid=GRID):
    """Compulsory HBM bytes per solve and FP64 flops of the smoother class.

    Per level l (V_l = one complex mode vector of the level): a red-black half
    sweep reads the other colour of u and this colour of b and writes this
    colour of u (1.5 V_l, 8 flops per real component); residual + restriction
    reads u, b and writes coarse b and u (2.5 V_l); prolongation reads coarse
    u and reads/writes u (2.25 V_l); forward / inverse transforms move one
    real 3-D array and one mode vector each.
    """
    nm = q["n_modes"]
    L = q["levels"]
    V = [v_bytes(q["nr"][l], q["nz"][l], nm, word) for l in range(L)]
    X = grid[0] * grid[1] * grid[2] * 8
    tot_bytes, sm_bytes, sm_flops, sm_launches = 0.0, 0.0, 0.0, 0
    for info in info_list:
        c = info["cycles"]
        b = 2.0 * (X + V[0])   # forward + inverse
        # level 0: pre-smoothing once per residual check (c + 1 checks), post once per cycle
        half0 = 2 * pre * (c + 1) + 2 * post * c
        sweeps = {0: half0}
        for l in range(1, L - 1):
            sweeps[l] = 2 * (pre + post) * c
        for l, h in sweeps.items():
            sm_bytes += h * 1.5 * V[l]
            sm_flops += h * (V[l] / (2 * word)) / 2 * 16     # updated complex entries x 16 flops
            sm_launches += h
        b += sm_bytes_total(sweeps, V)
        b += (c + 1) * 2.5 * V[0] + sum(c * 2.5 * V[l] for l in range(1, L - 1))
        b += sum(c * 2.25 * V[l] for l in range(0, L - 1))
        b += c * 2 * V[L - 1]
        tot_bytes += b
    return tot_bytes, sm_bytes, sm_flops, sm_launches


def sm_bytes_total(sweeps, V):
    return sum(h * 1.5 * V[l] for l, h in sweeps.items())


def traffic_from_profile(name):
    """Per-launch DRAM bytes recorded in a committed ncu summary, or None."""
    path = os.path.join(ROOT, "profiles", name)
    try:
        for line in open(path):
            if line.startswith("dram_bytes_per_fine_launch:"):
                return float(line.split(":")[1])
    except OSError:
        pass
    return None


# ------------------------------------------------------------------ CPU oracle timing
def oracle_sample(max_seconds=20.0, min_iters=20):
    """Time oracle CG iterations on the full workload; returns (ms per solve, details)."""
    import numpy as np  # noqa: F401
    import oracle
    from paper_2609_07172_gb300 import workloads as W
    rec_path = os.path.join(ROOT, "oracle", "c1_cg_iterations.json")
    with open(rec_path) as f:
        rec = json.load(f)
    p = W.c1_problem()
    g = oracle.grid_from_problem(p)
    rho = W.rho_plasma(p, 0)
    t0 = time.perf_counter()
    oracle.cg_fixed_iterations(g, rho, 2)
    t_two = time.perf_counter() - t0
    iters = max(min_iters, int(max_seconds / max(t_two / 2.0, 1e-3)))
    t0 = time.perf_counter()
    oracle.cg_fixed_iterations(g, rho, iters)
    dt = time.perf_counter() - t0
    per_iter = dt / iters
    ms = per_iter * rec["iterations"] * 1e3
    return ms, {"iters_timed": iters, "seconds": dt, "per_iter_ms": per_iter * 1e3,
                "iters_to_tol": rec["iterations"], "threads": oracle.get_threads()}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from paper_2609_07172_gb300 import workloads as W
    rec = json.load(open(os.path.join(ROOT, "oracle", "c1_cg_iterations.json")))
    p = W.c1_problem()
    g = oracle.grid_from_problem(p)
    rho = W.rho_plasma(p, 0)
    per_step_iters = 8
    vals = []
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.cg_fixed_iterations(g, rho, per_step_iters)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            vals.append(dt / per_step_iters * rec["iterations"] * 1e3)
    ms = statistics.median(vals)
    cores = oracle.get_threads()
    sample = (f"{per_step_iters} CG iterations per step on the full 512x128x400 system (seed 0), "
              f"scaled by the {rec['iterations']} iterations the oracle needs to reach rel-res 1e-10")
    line = {"impl": "reference", "metric": METRIC, "value": ms, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "annulus 512x128x400, 65 modes, rho seed 0", "tol": 1e-10},
            "cpu_baseline": {"value": ms, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": ms, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm
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

    prec = FP64 if args.precision == "fp64" else MIXED
    p = W.annulus(*args.grid) if args.grid else W.c1_problem()
    q = query(p, precision=prec)
    seeds = [rank * 1000 + s for s in range(args.seeds)]
    rhos = [torch.from_numpy(W.rho_plasma(p, s)).to(dev) for s in seeds]
    phi = torch.empty(p.shape, dtype=torch.float64, device=dev)
    fp64_gflops, fp32_gflops = measure_fma_peaks()

    plan = Plan(p, precision=prec, profile=True)
    stream = plan.stream
    for w in range(args.warmup):
        plan.solve(rhos[w % len(rhos)], phi, tol=args.tol)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    infos = []
    e0.record(stream)
    for k in range(args.steps):
        _, info = plan.solve(rhos[k % len(rhos)], phi, tol=args.tol)
        infos.append(info)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    if world > 1:
        dist.barrier()
    ms_total = e0.elapsed_time(e1)
    if world > 1:
        t = torch.tensor([ms_total], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_total = float(t.item())
    ms_per_solve = ms_total / (args.steps * world)
    ms_local = ms_total / args.steps
    statuses = sorted({i["status"] for i in infos})
    cycles = [i["cycles"] for i in infos]
    rel = [i["rel_res"] for i in infos]

    # ---- roofline of the dominant kernel class (level-0 + coarse smoother half-sweeps)
    hbm_peak, hbm_src = measured_peaks()
    word = 8 if prec == FP64 else 4
    ph_ms = {k: sum(i["ms_phase"][k] for i in infos) for k in infos[0]["ms_phase"]}
    ph_n = {k: sum(i["launches_phase"][k] for i in infos) for k in infos[0]["launches_phase"]}
    dominant = max(ph_ms, key=ph_ms.get)
    tot_bytes, sm_bytes, sm_flops, sm_launches = algorithmic_model(q, infos, 2, 2, word, (p.nr, p.ntheta, p.nz))
    sm_ms = ph_ms["smooth"]
    sm_gbs = sm_bytes / (sm_ms * 1e-3) / 1e9 if sm_ms > 0 else None
    sm_tflops = sm_flops / (sm_ms * 1e-3) / 1e12 if sm_ms > 0 else None
    fp64_tf = fp64_gflops / 1e3
    if prec == FP64:
        roof = {"bound": "alu", "achieved": sm_tflops, "peak": fp64_tf, "unit": "TFLOP/s",
                "frac": sm_tflops / fp64_tf if sm_tflops else None,
                "traffic": traffic_from_profile("smooth_fp64_512x128x400.md"),
                "kernel": "k_smooth<double> (red-black Gauss-Seidel half-sweep, all levels)",
                "peak_source": "FP64 FMA throughput measured live by pic_poisson_measure_fma_peaks",
                "hbm_achieved_gbs": sm_gbs, "hbm_peak_gbs": hbm_peak,
                "hbm_frac": sm_gbs / hbm_peak if sm_gbs else None,
                "launches": ph_n["smooth"], "model_launches": sm_launches}
    else:
        roof = {"bound": "hbm", "achieved": sm_gbs, "peak": hbm_peak, "unit": "GB/s",
                "frac": sm_gbs / hbm_peak if sm_gbs else None,
                "traffic": traffic_from_profile("smooth_fp32_512x128x400.md"),
                "kernel": "k_smooth<float>", "peak_source": hbm_src}
    solve_gbs = tot_bytes / len(infos) / (ms_local * 1e-3) / 1e9

    line = {"metric": METRIC, "value": ms_per_solve, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_local, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if prec == FP64 else "f32+f64",
            "data": "synthetic",
            "config": {"workload": "annulus %dx%dx%d, %d azimuthal modes, %s batched GMG V(2,2), "
                                   "rho seeds %s (Poisson counts, mean 27, m=8 wave)"
                                   % (p.nr, p.ntheta, p.nz, p.n_modes, args.precision, seeds),
                       "grid_nr_ntheta_nz": [p.nr, p.ntheta, p.nz], "tol": args.tol, "levels": q["levels"],
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "l2": "inputs larger than L2 (rho 209.7 MB, mode vector 213 MB per step)"},
            "status": statuses, "cycles": {"min": min(cycles), "max": max(cycles),
                                           "median": statistics.median(cycles)},
            "rel_res_max": max(rel),
            "gpu_launches": int(sum(i["launches"] for i in infos)),
            "phase_ms_per_solve": {k: v / len(infos) for k, v in ph_ms.items()},
            "dominant_phase": dominant,
            "roofline": roof,
            "hbm_roofline_solve": {"achieved_gbs": solve_gbs, "peak_gbs": hbm_peak, "frac": solve_gbs / hbm_peak,
                                   "bytes_per_solve": tot_bytes / len(infos), "peak_source": hbm_src},
            "fma_peaks_gflops": {"fp64": fp64_gflops, "fp32": fp32_gflops},
            "clocks": clocks}

    # ---- end to end through the C ABI with host buffers (pinned), copies inside the timed region
    if not args.no_e2e:
        rho_h = [r.cpu().pin_memory() for r in rhos]
        phi_h = torch.empty(p.shape, dtype=torch.float64).pin_memory()
        plan.solve_host(rho_h[0], phi_h, tol=args.tol)
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        ne = max(3, args.steps // 4)
        for k in range(ne):
            plan.solve_host(rho_h[k % len(rho_h)], phi_h, tol=args.tol)
        e2e_ms = (time.perf_counter() - t0) * 1e3 / ne
        if world > 1:
            t = torch.tensor([e2e_ms], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_ms = float(t.item()) / world
        nbytes = p.nr * p.ntheta * p.nz * 8
        line["e2e"] = {"value": e2e_ms, "unit": UNIT, "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
                       "steps": ne}

    if args.extra_forms and prec == FP64:
        line["forms"] = {}
    plan.close()

    if not args.no_cpu_baseline and rank == 0 and world == 1:
        ms, det = oracle_sample()
        line["cpu_baseline"] = {"value": ms, "unit": UNIT, "cores": det["threads"], "kind": "oracle",
                                "sample": "%d CG iterations (%.1f s) of the FP64 oracle on the full 512x128x400 "
                                          "system, scaled by the %d iterations it needs to reach rel-res 1e-10"
                                          % (det["iters_timed"], det["seconds"], det["iters_to_tol"])}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
