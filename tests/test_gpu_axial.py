"""Non-uniform axial meshes vs the FP64 oracle (needs a GPU).

With axial faces given, every row has its own widths and centre distances,
so the library builds per-row coefficient tables (south and north couplings
apart) and solves the coarsest level densely; the oracle applies the same
finite-volume system from the same face arrays.  Bar: relative L2 against the
oracle's converged solution <= 1e-12 (FP64) or 1e-10 (mixed).
"""
import numpy as np
import pytest
import torch

import oracle
from helpers import cond_estimate, rel_l2, with_bias_walls
from paper_2609_07172_gb300 import FP64, MIXED, BatchPlan, Plan, binding as B, workloads as W

pytestmark = pytest.mark.gpu

TOL = {FP64: 1e-12, MIXED: 1e-10}


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _sz(p, ratio):
    w = ratio ** np.arange(p.nz)
    return p.with_z_faces(p.z0 + (p.z1 - p.z0) * np.r_[0.0, np.cumsum(w)] / w.sum())


CASES = {
    "growing_64x16x48": lambda: _sz(with_bias_walls(W.annulus(64, 16, 48)), 1.04),
    "shrinking_96x8x40": lambda: _sz(W.annulus(96, 8, 40, phi_r_out=-30.0), 0.96),
    "stretched_r_and_z": lambda: _sz(W.annulus(64, 8, 64).with_r_faces(
        W.stretched_radial_faces(0.02, 0.05, 64, 1.03)), 1.03),
    "semi_coarsened_32x8x200": lambda: _sz(W.annulus(32, 8, 200), 1.005),
    "channel_plume_stretched_z": lambda: _sz(W.channel_plume(64, 16, 48), 1.03),
}


@pytest.fixture(scope="module")
def refs():
    out = {}
    for name, make in CASES.items():
        p = make()
        g = oracle.grid_from_problem(p)
        rho = W.rho_plasma(p, seed=71)
        out[name] = (p, g, rho, oracle.solve3d(g, rho, tol=1e-15)[0])
    return out


@pytest.mark.parametrize("graph", [False, True], ids=["hostloop", "graph"])
@pytest.mark.parametrize("precision", [FP64, MIXED], ids=["fp64", "mixed"])
@pytest.mark.parametrize("name", list(CASES))
def test_axial_mesh_matches_oracle(refs, name, precision, graph):
    p, g, rho, ref = refs[name]
    with Plan(p, precision=precision, graph=graph) as plan:
        phi, info = plan.solve(dev(rho), tol=0.0)
    got = phi.cpu().numpy()
    assert info["status"] == B.OK, info
    assert rel_l2(got, ref) <= TOL[precision], info
    assert oracle.relres(g, rho, got) <= 1e-12


@pytest.mark.parametrize("kw", [dict(fmg=1, pre_sweeps=2, post_sweeps=1), dict(smooth_strip=2),
                                dict(smooth_strip=4, omega=1.15)], ids=["fmg", "strip2", "strip4_sor"])
def test_axial_mesh_settings(refs, kw):
    p, g, rho, ref = refs["growing_64x16x48"]
    with Plan(p, graph=True, **kw) as plan:
        phi, info = plan.solve(dev(rho), tol=0.0)
    assert info["status"] == B.OK
    assert rel_l2(phi.cpu().numpy(), ref) <= 1e-12


@pytest.mark.parametrize("precision", [FP64, MIXED], ids=["fp64", "mixed"])
def test_axial_mesh_stops_at_tol_with_the_oracles_residual(precision):
    p = _sz(W.annulus(128, 32, 96), 1.01)
    g = oracle.grid_from_problem(p)
    rho = W.rho_plasma(p, seed=72)
    with Plan(p, precision=precision, graph=True) as plan:
        phi, info = plan.solve(dev(rho), tol=1e-10)
    assert info["status"] == B.OK and info["rel_res"] <= 1e-10
    assert info["cycles"] <= 24, info
    true = oracle.relres(g, rho, phi.cpu().numpy())
    assert true == pytest.approx(info["rel_res"], rel=1e-6, abs=1e-14)


def test_strongly_stretched_mesh_converges_to_tol():
    """Cells stretched 1.03 per cell in both r and z (cell aspect varying
    about 6-fold over the grid): the point smoother loses part of its
    effect, so a cycle may reduce the residual by less than half.  A given
    tolerance is reached, with the oracle's own residual, and the error
    against the oracle's floor solution obeys the bound a residual gives,
    ||e|| / ||phi|| <= kappa(A) * rel-res, with kappa from the oracle's
    operator."""
    p = _sz(W.annulus(64, 8, 64).with_r_faces(W.stretched_radial_faces(0.02, 0.05, 64, 1.03)), 1.03)
    g = oracle.grid_from_problem(p)
    rho = W.rho_plasma(p, seed=73)
    ref, _ = oracle.solve3d(g, rho, tol=1e-15)
    kappa = cond_estimate(g)
    for precision in (FP64, MIXED):
        with Plan(p, precision=precision, graph=True, max_cycles=400) as plan:
            phi, info = plan.solve(dev(rho), tol=1e-10)
        got = phi.cpu().numpy()
        true = oracle.relres(g, rho, got)
        err = rel_l2(got, ref)
        print(precision, info["cycles"], info["rel_res0"], info["rel_res"], true, err, kappa)
        assert info["status"] == B.OK and info["rel_res"] <= 1e-10, info
        assert true <= 1.05e-10
        assert err <= kappa * true + 1e-12


def test_batch_mixes_axial_meshes_patches_and_plain():
    probs = [_sz(W.annulus(32, 8, 24), 1.05), with_bias_walls(W.annulus(40, 8, 24)),
             W.channel_plume(32, 8, 24), _sz(W.channel_plume(64, 8, 48), 0.97)]
    rhos = [W.rho_plasma(q, seed=80 + i) for i, q in enumerate(probs)]
    with BatchPlan(probs, graph=True) as bp:
        phis, infos = bp.solve([dev(r) for r in rhos], tol=0.0)
    for q, r, phi, info in zip(probs, rhos, phis, infos):
        ref, _ = oracle.solve3d(oracle.grid_from_problem(q), r, tol=1e-15)
        assert info["status"] == B.OK, info
        assert rel_l2(phi.cpu().numpy(), ref) <= 1e-12


@pytest.mark.parametrize("precision", [FP64, MIXED], ids=["fp64", "mixed"])
def test_uniform_faces_take_the_dense_coarsest_solve_and_agree(precision):
    """Axial faces given at the uniform positions: the plan builds per-row
    tables and solves the coarsest level densely (the 2 N_m right-hand sides
    through the two GEMMs of the dense solve: 34 of them, a partial column
    tile, over 120 coarsest cells, a partial row tile), while the plan without
    faces takes the separable solve and the mode-local bottom.  Two
    independent coarsest solvers, the same discrete system: at the floor the
    potentials agree with each other and with the oracle."""
    p = with_bias_walls(W.annulus(96, 32, 80))
    q = p.with_z_faces(np.linspace(p.z0, p.z1, p.nz + 1))
    rho = W.rho_plasma(p, seed=73)
    with Plan(p, precision=precision) as a:
        phi_a, ia = a.solve(dev(rho), tol=0.0)
    with Plan(q, precision=precision) as b:
        phi_b, ib = b.solve(dev(rho), tol=0.0)
    assert ia["status"] == B.OK and ib["status"] == B.OK
    got_a, got_b = phi_a.cpu().numpy(), phi_b.cpu().numpy()
    assert rel_l2(got_b, got_a) <= TOL[precision]
    g = oracle.grid_from_problem(q)
    ref = oracle.solve3d(g, rho, tol=1e-15)[0]
    assert rel_l2(got_b, ref) <= TOL[precision]
