"""Record how many oracle CG iterations a full-size solve needs, per seed.

Runs the FP64 oracle's conjugate gradient on the 512 x 128 x 400 annulus
from a zero guess until the relative residual reaches 1e-10, for the charge
densities of the given seeds, and writes the iteration counts and final
residuals to ``oracle/c1_cg_iterations.json`` (one entry per seed; existing
entries of other seeds are kept).  The reference arm of the benchmark times
a bounded number of oracle iterations per step and scales by the step's
seed's count.  Calls only the oracle and the seeded input generator.

Usage: python oracle/cg_iterations.py [seed ...]   (default: 0 .. 9)
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2609_07172_gb300 import workloads as W  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c1_cg_iterations.json")


def load():
    try:
        with open(OUT) as f:
            rec = json.load(f)
    except OSError:
        rec = {}
    if "seeds" not in rec:   # the single-seed layout: its seed 0 entry
        old = rec
        rec = {"workload": "annulus 512x128x400", "tol": 1e-10, "seeds": {}}
        if "iterations" in old:
            rec["seeds"]["0"] = {k: old[k] for k in ("iterations", "relres_recursive", "relres_true", "threads",
                                                     "seconds") if k in old}
    return rec


def iterations(seed):
    """Iterations seed `seed` needs (the seed-0 count if that seed is not recorded)."""
    seeds = load()["seeds"]
    return int(seeds.get(str(seed), seeds["0"])["iterations"])


def main(seeds, tol=1e-10):
    p = W.c1_problem()
    g = oracle.grid_from_problem(p)
    for seed in seeds:
        rho = W.rho_plasma(p, seed)
        t0 = time.time()
        phi, info = oracle.solve3d(g, rho, tol=tol, maxit=100000, stall=0)
        dt = time.time() - t0
        rec = load()
        rec["seeds"][str(seed)] = {"iterations": info["iterations"], "relres_recursive": info["relres_recursive"],
                                   "relres_true": info["relres"], "threads": oracle.get_threads(), "seconds": dt}
        with open(OUT, "w") as f:
            json.dump(rec, f, indent=1, sort_keys=True)
        print(seed, json.dumps(rec["seeds"][str(seed)]), flush=True)


if __name__ == "__main__":
    main([int(a) for a in sys.argv[1:]] or list(range(10)))
