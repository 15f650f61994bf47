"""Mixed-precision form vs the FP64 oracle (needs a GPU).

FP32 V-cycles inside an FP64 defect-correction loop: the residual of the 3-D
system, the iterate update and the norms stay FP64, so the solve reaches the
same FP64 residual; the bar is relative L2 <= 1e-10 in phi against the FP64
oracle, and the error is reported per azimuthal mode (normalised by the whole
solution's norm, so tiny modes do not blow up) and for the 3-D potential.
"""
import numpy as np
import pytest
import torch

import oracle
from helpers import narrow_span, rel_l2, small_rin, to_modes, with_bias_walls
from paper_2609_07172_gb300 import MIXED, Plan, binding as B, workloads as W

pytestmark = pytest.mark.gpu

MIXED_TOL = 1e-10


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def cases():
    out = [pytest.param(with_bias_walls(W.annulus(nr, nt, nz)), id=f"annulus{nr}x{nt}x{nz}")
           for nr, nt, nz in [(32, 16, 32), (40, 8, 24), (64, 32, 48), (15, 4, 9), (128, 64, 64)]]
    out.append(pytest.param(narrow_span(), id="narrow_span"))
    out.append(pytest.param(small_rin(), id="small_rin"))
    return out


@pytest.mark.parametrize("p", cases())
def test_mixed_floor_matches_fp64_oracle(p):
    g = oracle.grid_from_problem(p)
    rho = W.rho_plasma(p, seed=1)
    ref, _ = oracle.solve3d(g, rho, tol=1e-15)
    with Plan(p, precision=MIXED) as plan:
        phi, info = plan.solve(dev(rho), tol=0.0)
    got = phi.cpu().numpy()
    assert info["status"] == B.OK
    assert rel_l2(got, ref) <= MIXED_TOL, info
    assert oracle.relres(g, rho, got) <= 1e-12       # FP64 defect reaches the FP64 floor
    # per-mode errors, normalised by the whole solution
    e = to_modes(got - ref)
    nrm = np.linalg.norm(to_modes(ref))
    per_mode = np.sqrt((e ** 2).sum(axis=(0, 1, 3))) / nrm
    assert per_mode.max() <= MIXED_TOL


@pytest.mark.parametrize("tol", [1e-6, 1e-10])
def test_mixed_stop_at_tolerance(tol):
    p = with_bias_walls(W.annulus(96, 16, 40))
    g = oracle.grid_from_problem(p)
    rho = W.rho_plasma(p, seed=2)
    with Plan(p, precision=MIXED) as plan:
        phi, info = plan.solve(dev(rho), tol=tol)
    assert info["status"] == B.OK and info["rel_res"] <= tol
    assert info["outer_iterations"] >= 1 and info["cycles"] >= info["outer_iterations"]
    true = oracle.relres(g, rho, phi.cpu().numpy())
    assert true == pytest.approx(info["rel_res"], rel=1e-6, abs=1e-14)


@pytest.mark.parametrize("inner", [1, 3])
def test_mixed_inner_cycles(inner):
    p = W.annulus(64, 16, 64)
    g = oracle.grid_from_problem(p)
    rho = W.rho_plasma(p, seed=3)
    ref, _ = oracle.solve3d(g, rho, tol=1e-15)
    with Plan(p, precision=MIXED, inner_cycles=inner) as plan:
        phi, info = plan.solve(dev(rho), tol=0.0)
    assert info["cycles"] == inner * info["outer_iterations"]
    assert rel_l2(phi.cpu().numpy(), ref) <= MIXED_TOL


def test_mixed_tiny_charge_is_scaled():
    """A right-hand side near the FP32 underflow range still converges (power-of-two scaling)."""
    p = W.annulus(32, 8, 32, phi_z0=0.0)
    rho = W.rho_plasma(p, seed=4) * 1e-30
    g = oracle.grid_from_problem(p)
    ref, _ = oracle.solve3d(g, rho, tol=1e-15)
    with Plan(p, precision=MIXED) as plan:
        phi, info = plan.solve(dev(rho), tol=1e-12)
    assert info["status"] == B.OK
    assert rel_l2(phi.cpu().numpy(), ref) <= MIXED_TOL
