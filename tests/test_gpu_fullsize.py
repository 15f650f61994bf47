"""Parity at the full 512 x 128 x 400 workload, in the configurations the
benchmark times (needs a GPU).

  * Element-wise parity at the rounding floor (Sec. 5's CPU/GPU agreement;
    Eq. evaluation_field_metrics): the oracle's conjugate gradient solves
    the 3-D system to its floor on the host cores (a few minutes), then once
    more from that solution (a restart recomputes the true residual and
    refines it), and every form of the library solved with tol <= 0 must
    match it to rel L2 <= 1e-12 (FP64) or <= 1e-10 (mixed, fused and not,
    in 3-D and per azimuthal mode normalised by the whole solution).
  * At the benchmark's stop (rel-res 1e-10) the 3-D residual of the returned
    potential, recomputed by the oracle's own operator in physical space, is
    below the tolerance and agrees with the value the library reports
    (Parseval); the error of these solutions against the oracle's floor
    solution is reported (it is bounded only by the condition number times
    the residual).
  * The right-hand side of sampled (r, z) columns equals the plain DFT of the
    oracle's 3-D right-hand side (Eq. azimuthal_dft with 1/N).
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import fields as F
from helpers import rel_l2, to_modes
from paper_2609_07172_gb300 import FP64, MIXED, Plan, binding as B, workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-10
# schedules of the kind the autotuner picks for this grid (the bench tunes its own)
FORMS = {
    "fp64": dict(precision=FP64, pre_sweeps=1, post_sweeps=2, smooth_threads=64),
    "fp64_fmg": dict(precision=FP64, pre_sweeps=2, post_sweeps=1, smooth_threads=128, fmg=1),
    "mixed": dict(precision=MIXED, pre_sweeps=2, post_sweeps=2, inner_cycles=3, smooth_threads=128,
                  smooth_strip=2),
    "mixed_fused": dict(precision=MIXED, pre_sweeps=2, post_sweeps=2, inner_cycles=3, smooth_fused=1),
}


@pytest.fixture(scope="module")
def full():
    p = W.c1_problem()
    rho = W.rho_plasma(p, seed=0)
    return p, oracle.grid_from_problem(p), rho


@pytest.fixture(scope="module")
def solutions(full):
    p, g, rho = full
    out = {}
    for name, kw in FORMS.items():
        with Plan(p, graph=True, **kw) as plan:
            phi, info = plan.solve(torch.from_numpy(rho).cuda(), tol=TOL)
        out[name] = (phi.cpu().numpy(), info)
    return out


@pytest.fixture(scope="module")
def oracle_floor(full):
    """The oracle's solution at its rounding floor: CG to a recursive rel-res
    of 1e-15, then a restart from that solution (true residual recomputed)."""
    p, g, rho = full
    phi, info = oracle.solve3d(g, rho, tol=1e-15)
    phi, info2 = oracle.solve3d(g, rho, tol=1e-15, x0=phi)
    print("oracle floor: %d + %d CG iterations, true rel-res %.3e"
          % (info["iterations"], info2["iterations"], info2["relres"]))
    return phi, info2


@pytest.mark.parametrize("name", list(FORMS))
def test_full_size_floor_matches_oracle(full, oracle_floor, name):
    p, g, rho = full
    ref, _ = oracle_floor
    with Plan(p, graph=True, **FORMS[name]) as plan:
        phi, info = plan.solve(torch.from_numpy(rho).cuda(), tol=0.0)
    got = phi.cpu().numpy()
    assert info["status"] == B.OK, info
    err = rel_l2(got, ref)
    print("%s: tol 0, %d cycles, rel-res %.3e, rel L2 vs oracle %.3e" % (name, info["cycles"], info["rel_res"], err))
    if FORMS[name]["precision"] == FP64:
        assert err <= 1e-12, (name, err)
    else:
        assert err <= 1e-10, (name, err)
        e = to_modes(got - ref)
        per_mode = np.sqrt((e ** 2).sum(axis=(0, 1, 3))) / np.linalg.norm(to_modes(ref))
        assert per_mode.max() <= 1e-10, (name, per_mode.max())
    assert oracle.relres(g, rho, got) <= 1e-12


def test_full_size_tol_solutions_error_vs_oracle(full, solutions, oracle_floor):
    """Reported, not bounded: a 1e-10 residual bounds the error only by the
    condition number (~2e5 here) times 1e-10."""
    ref, _ = oracle_floor
    for name, (phi, info) in solutions.items():
        err = rel_l2(phi, ref)
        print("%s: tol %g, %d cycles, rel-res %.3e, rel L2 vs oracle floor %.3e"
              % (name, TOL, info["cycles"], info["rel_res"], err))
        assert np.isfinite(err)


@pytest.mark.parametrize("name", list(FORMS))
def test_full_size_residual_by_the_oracle(full, solutions, name):
    p, g, rho = full
    phi, info = solutions[name]
    assert info["status"] == B.OK, info
    rel = oracle.relres(g, rho, phi)
    assert rel <= TOL * 1.05, (name, rel)
    assert rel == pytest.approx(info["rel_res"], rel=1e-3), (name, rel, info["rel_res"])


def test_full_size_forms_agree(solutions):
    ref = solutions["fp64"][0]
    nrm = np.linalg.norm(ref)
    for name in ("fp64_fmg", "mixed", "mixed_fused"):
        assert np.linalg.norm(solutions[name][0] - ref) / nrm <= 1e-9, name
    # fused and separate half-sweeps are the same arithmetic
    assert np.array_equal(solutions["mixed"][0], solutions["mixed_fused"][0])


def test_full_size_rhs_matches_dft_of_oracle_rhs(full):
    p, g, rho = full
    b3 = oracle.rhs3d(g, rho)                       # (nz, ntheta, nr), oracle arithmetic
    with Plan(p) as plan:
        bh = plan.forward(torch.from_numpy(rho).cuda())   # (nz, nr, nm, 2) mode layout
        b = bh.cpu().numpy()
    rng = np.random.default_rng(5)
    ks = rng.integers(0, p.nz, 24)
    is_ = rng.integers(0, p.nr, 24)
    n = p.ntheta
    j = np.arange(n)
    for k, i in zip(ks, is_):
        col = b3[k, :, i]
        for m in range(p.n_modes):
            ref = (col * np.exp(-2j * np.pi * m * j / n)).sum() / n
            got = b[k, i, m, 0] + 1j * b[k, i, m, 1]
            assert abs(got - ref) <= 1e-12 * (np.abs(col).max() + 1e-300), (k, i, m, got, ref)


def test_full_size_face_field_flux_balance_is_the_solver_residual(full, solutions):
    """E = -grad phi of the returned potential: each cell's outward face fluxes
    minus its charge is dalpha (A phi - b) of that cell, so the imbalance's
    norm relative to dalpha ||b|| is the solve's relative residual."""
    p, g, rho = full
    phi, info = solutions["fp64"]
    with Plan(p) as plan:
        e = plan.face_field(torch.from_numpy(phi).cuda())
        torch.cuda.synchronize()
    res, _ = F.gauss_residual(g, rho, *[x.cpu().numpy() for x in e])
    b = oracle.rhs3d(g, rho)
    rel = np.linalg.norm(res) / (p.theta_span / p.ntheta * np.linalg.norm(b))
    assert rel == pytest.approx(oracle.relres(g, rho, phi), rel=1e-3)
    assert rel <= TOL * 1.05
