"""Record how many oracle CG iterations a full-size solve needs.

Runs the FP64 oracle's conjugate gradient on the 512 x 128 x 400 annulus
(charge density seed 0) from a zero guess until the relative residual
reaches 1e-10, and writes the iteration count and final residuals to
``oracle/c1_cg_iterations.json``.  The CPU-baseline leg of the benchmark
times a bounded number of oracle iterations and scales by this count.
Calls only the oracle and the seeded input generator.
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


def main(seed=0, tol=1e-10):
    p = W.c1_problem()
    g = oracle.grid_from_problem(p)
    rho = W.rho_plasma(p, seed)
    t0 = time.time()
    phi, info = oracle.solve3d(g, rho, tol=tol, maxit=100000, stall=0)
    dt = time.time() - t0
    rec = {"workload": "annulus 512x128x400, rho seed %d" % seed, "tol": tol,
           "iterations": info["iterations"], "relres_recursive": info["relres_recursive"],
           "relres_true": info["relres"], "threads": oracle.get_threads(), "seconds": dt}
    with open(OUT, "w") as f:
        json.dump(rec, f, indent=1)
    print(json.dumps(rec))


if __name__ == "__main__":
    main()
