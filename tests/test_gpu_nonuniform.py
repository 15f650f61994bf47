"""Non-uniform radial meshes (appendix face conductances on arbitrary
radial faces) against the oracle, which takes the same face array (needs a
GPU)."""
import numpy as np
import pytest
import torch

import oracle
from oracle import fields as F
from helpers import rel_l2, with_bias_walls
from paper_2609_07172_gb300 import FP64, MIXED, BatchPlan, Plan, binding as B, workloads as W

pytestmark = pytest.mark.gpu

TOL = {FP64: 1e-12, MIXED: 1e-10}


def stretched(nr, nt, nz, ratio, **kw):
    p = W.annulus(nr, nt, nz, **kw)
    return p.with_r_faces(W.stretched_radial_faces(p.r_in, p.r_out, nr, ratio))


CASES = {
    "s64x16x48": lambda: stretched(64, 16, 48, 1.03),
    "s32x8x32_bias": lambda: with_bias_walls(stretched(32, 8, 32, 1.05)),
    "s96x4x24_shrinking": lambda: stretched(96, 4, 24, 0.98),
    "s40x8x200_semi": lambda: stretched(40, 8, 200, 1.04),
}


def _rho(p, seed):
    return np.random.default_rng(seed).normal(size=p.shape) * 1e-6


@pytest.mark.parametrize("precision", [FP64, MIXED], ids=["fp64", "mixed"])
@pytest.mark.parametrize("name", list(CASES))
def test_nonuniform_solve_matches_oracle(name, precision):
    p = CASES[name]()
    g = oracle.grid_from_problem(p)
    rho = _rho(p, 3)
    ref, _ = oracle.solve3d(g, rho, tol=1e-15)
    with Plan(p, precision=precision) as plan:
        phi, info = plan.solve(torch.from_numpy(rho).cuda(), tol=0.0)
    got = phi.cpu().numpy()
    assert info["status"] == B.OK, info
    assert rel_l2(got, ref) <= TOL[precision], info
    assert oracle.relres(g, rho, got) <= 1e-12


def test_nonuniform_full_multigrid_start_matches_oracle():
    p = with_bias_walls(stretched(64, 16, 48, 1.03))
    g = oracle.grid_from_problem(p)
    rho = _rho(p, 6)
    ref, _ = oracle.solve3d(g, rho, tol=1e-15)
    with Plan(p, fmg=1, graph=True) as plan:
        phi, info = plan.solve(torch.from_numpy(rho).cuda(), tol=0.0)
    assert info["status"] == B.OK
    assert rel_l2(phi.cpu().numpy(), ref) <= TOL[FP64], info


def test_nonuniform_fused_smoother_matches_oracle():
    p = stretched(64, 16, 48, 1.03)
    g = oracle.grid_from_problem(p)
    rho = _rho(p, 4)
    ref, _ = oracle.solve3d(g, rho, tol=1e-15)
    with Plan(p, precision=MIXED, smooth_fused=1, pre_sweeps=2, post_sweeps=2) as plan:
        phi, info = plan.solve(torch.from_numpy(rho).cuda(), tol=0.0)
    assert rel_l2(phi.cpu().numpy(), ref) <= TOL[MIXED], info


def test_nonuniform_face_field_matches_oracle():
    p = with_bias_walls(stretched(32, 8, 32, 1.05))
    g = oracle.grid_from_problem(p)
    rho = _rho(p, 5)
    phi, _ = oracle.solve3d(g, rho, tol=1e-15)
    with Plan(p) as plan:
        got = plan.face_field(torch.from_numpy(phi).cuda())
        torch.cuda.synchronize()
    for e, want in zip(got, F.face_field(g, phi)):
        assert np.abs(e.cpu().numpy() - want).max() <= 1e-12 * np.abs(want).max()
    res, scale = F.gauss_residual(g, rho, *[x.cpu().numpy() for x in got])
    assert np.abs(res).max() <= 1e-11 * scale


def test_batch_mixes_uniform_and_nonuniform_problems():
    probs = [W.annulus(32, 8, 32), stretched(64, 16, 48, 1.03), stretched(32, 4, 16, 0.97)]
    rhos = [_rho(p, 10 + i) for i, p in enumerate(probs)]
    refs = [oracle.solve3d(oracle.grid_from_problem(p), r, tol=1e-15)[0] for p, r in zip(probs, rhos)]
    with BatchPlan(probs) as bp:
        phis, infos = bp.solve([torch.from_numpy(r).cuda() for r in rhos], tol=0.0)
    for phi, ref, info in zip(phis, refs, infos):
        assert info["status"] == B.OK
        assert rel_l2(phi.cpu().numpy(), ref) <= TOL[FP64]


def test_invalid_faces_are_rejected():
    p = W.annulus(8, 4, 8)
    bad = W.stretched_radial_faces(p.r_in, p.r_out, p.nr, 1.1)
    bad[3] = bad[2]   # not strictly increasing
    with pytest.raises(B.PicPoissonError):
        Plan(p.with_r_faces(bad))
