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


@pytest.mark.parametrize("scale", [1e-30, 1e-120, 1e100])
def test_mixed_tiny_charge_is_scaled(scale):
    """Right-hand sides far outside the FP32 range still converge: the FP32
    correction problem and the double-float transform both scale by powers
    of two.  (The residual norms are FP64 sums of squares, so right-hand
    sides must stay within about 1e-150 .. 1e150 in either form.)"""
    p = W.annulus(32, 8, 32, phi_z0=0.0)   # every wall at 0 V: phi is linear in rho
    rho1 = W.rho_plasma(p, seed=4)
    rho = rho1 * scale
    g = oracle.grid_from_problem(p)
    ref = oracle.solve3d(g, rho1, tol=1e-15)[0] * scale
    with Plan(p, precision=MIXED) as plan:
        phi, info = plan.solve(dev(rho), tol=1e-12)
    assert info["status"] == B.OK
    assert rel_l2(phi.cpu().numpy() / scale, ref / scale) <= MIXED_TOL


FUSED_CASES = [(64, 32, 48), (96, 16, 40), (256, 8, 32), (64, 8, 400), (40, 8, 24), (512, 128, 64)]


@pytest.mark.parametrize("sweeps", [(1, 1), (1, 2), (2, 1), (2, 2)])
@pytest.mark.parametrize("dims", FUSED_CASES, ids=[f"{a}x{b}x{c}" for a, b, c in FUSED_CASES])
def test_fused_smoother_matches_oracle(dims, sweeps):
    """The fused FP32 smoother (all sweeps of a pre- or post-smoothing in one
    wavefront pass) reaches the oracle's solution: several column tiles and row
    ranges, semi-coarsened levels (64x8x400, 256x8x32) and 65 modes in mode
    groups (512x128x64)."""
    p = with_bias_walls(W.annulus(*dims))
    g = oracle.grid_from_problem(p)
    rho = W.rho_plasma(p, seed=31)
    ref, _ = oracle.solve3d(g, rho, tol=1e-15)
    with Plan(p, precision=MIXED, smooth_fused=1, pre_sweeps=sweeps[0], post_sweeps=sweeps[1]) as plan:
        phi, info = plan.solve(dev(rho), tol=0.0)
    assert info["status"] == B.OK
    assert rel_l2(phi.cpu().numpy(), ref) <= MIXED_TOL, info


BITWISE_CASES = [(96, 32, 72), (512, 128, 64), (256, 64, 200)]


@pytest.mark.parametrize("sweeps", [(1, 2), (2, 2)])
@pytest.mark.parametrize("dims", BITWISE_CASES, ids=[f"{a}x{b}x{c}" for a, b, c in BITWISE_CASES])
def test_fused_smoother_is_bitwise_the_separate_half_sweeps(dims, sweeps):
    """Fusing changes where values live and when they move, not the arithmetic:
    the solve is bitwise identical to separate half-sweeps, cycle for cycle.
    The larger cases give each block long row ranges, so most row steps take
    the kernel's interior body (no range, wall-row or class tests) and the
    rest its general body."""
    p = with_bias_walls(W.annulus(*dims))
    rho = dev(W.rho_plasma(p, seed=32))
    out = []
    for fused in (0, 1):
        with Plan(p, precision=MIXED, smooth_fused=fused, pre_sweeps=sweeps[0], post_sweeps=sweeps[1],
                  inner_cycles=2, graph=bool(fused)) as plan:
            phi, info = plan.solve(rho, tol=1e-10)
        out.append((phi.cpu(), info["cycles"], info["outer_iterations"]))
    assert out[0][1:] == out[1][1:]
    assert torch.equal(out[0][0], out[1][0])


def test_fused_smoother_rejects_unsupported_schedules():
    p = W.annulus(64, 16, 48)
    for kw in (dict(pre_sweeps=3, post_sweeps=2), dict(pre_sweeps=0, post_sweeps=2), dict(omega=1.2)):
        with pytest.raises(B.PicPoissonError):
            Plan(p, precision=MIXED, smooth_fused=1, **kw)
    with pytest.raises(B.PicPoissonError):
        Plan(p, smooth_fused=1)   # FP64 form


@pytest.mark.parametrize("fused", [0, 1], ids=["halfsweeps", "fused"])
@pytest.mark.parametrize("inner,first", [(1, 3), (3, 5), (2, 6)])
def test_mixed_larger_first_correction(inner, first, fused):
    """inner_first FP32 V-cycles on the first correction, inner_cycles on the
    later ones: the loop reaches the oracle's floor, its cycle count is
    first + inner (outer - 1), and the graph (an if node ahead of the while
    node) gives the host loop's iterate bit for bit."""
    p = with_bias_walls(W.annulus(96, 16, 40))
    g = oracle.grid_from_problem(p)
    rho = W.rho_plasma(p, seed=33)
    ref, _ = oracle.solve3d(g, rho, tol=1e-15)
    kw = dict(precision=MIXED, inner_cycles=inner, inner_first=first, smooth_fused=fused, pre_sweeps=2,
              post_sweeps=2)
    out = {}
    for graph in (False, True):
        with Plan(p, graph=graph, **kw) as plan:
            out[graph] = plan.solve(dev(rho), tol=0.0)
    (pa, ia), (pg, ig) = out[False], out[True]
    assert ia["status"] == ig["status"] == B.OK
    assert ia["outer_iterations"] >= 2
    assert ia["cycles"] == first + inner * (ia["outer_iterations"] - 1)
    for k in ("cycles", "outer_iterations", "rel_res", "launches", "bytes_phase"):
        assert ia[k] == ig[k], k
    assert torch.equal(pa, pg)
    assert rel_l2(pg.cpu().numpy(), ref) <= MIXED_TOL


def test_mixed_larger_first_correction_saves_a_defect():
    """At tol 1e-10 a first correction of inner + 2 cycles needs no more FP32
    cycles than plain inner-cycle corrections and no more FP64 defects."""
    p = with_bias_walls(W.annulus(128, 32, 96))
    g = oracle.grid_from_problem(p)
    rho = dev(W.rho_plasma(p, seed=34))
    res = {}
    for first in (0, 5):
        with Plan(p, precision=MIXED, inner_cycles=3, inner_first=first, graph=True) as plan:
            phi, info = plan.solve(rho, tol=1e-10)
        assert info["status"] == B.OK and info["rel_res"] <= 1e-10
        assert oracle.relres(g, rho.cpu().numpy(), phi.cpu().numpy()) <= 1.05e-10
        res[first] = info
    assert res[5]["outer_iterations"] <= res[0]["outer_iterations"]
    assert res[5]["launches_phase"]["defect"] <= res[0]["launches_phase"]["defect"]


@pytest.mark.parametrize("graph", [False, True], ids=["hostloop", "graph"])
def test_mixed_larger_first_correction_skipped_when_converged(graph):
    """An initial iterate that already meets tol stops at the first test: the
    if node of the larger first pass and the while node both stay closed."""
    p = with_bias_walls(W.annulus(64, 16, 48))
    rho = dev(W.rho_plasma(p, seed=35))
    with Plan(p, precision=MIXED) as plan:
        phi0, _ = plan.solve(rho, tol=1e-13)
    with Plan(p, precision=MIXED, inner_cycles=2, inner_first=4, initial_guess=True, graph=graph) as plan:
        phi = phi0.clone()
        phi, info = plan.solve(rho, phi, tol=1e-10)
        assert info["status"] == B.OK and info["cycles"] == 0 and info["outer_iterations"] == 0
        assert info["rel_res"] <= 1e-10
        # a looser start runs the first pass and then the loop
        phi = (phi0 * 0.9).contiguous()
        phi, info = plan.solve(rho, phi, tol=1e-10)
        assert info["status"] == B.OK and info["rel_res"] <= 1e-10
        assert info["cycles"] >= 4 and (info["cycles"] - 4) % 2 == 0


def test_mixed_larger_first_correction_in_an_uneven_batch():
    from paper_2609_07172_gb300 import BatchPlan
    probs = [with_bias_walls(W.annulus(*d)) for d in [(32, 16, 32), (96, 16, 40), (15, 4, 9), (64, 32, 48)]]
    rhos = [W.rho_plasma(q, seed=36 + i) for i, q in enumerate(probs)]
    with BatchPlan(probs, precision=MIXED, inner_cycles=2, inner_first=4, graph=True) as bp:
        phis, infos = bp.solve([dev(r) for r in rhos], tol=0.0)
    for q, r, phi, info in zip(probs, rhos, phis, infos):
        ref, _ = oracle.solve3d(oracle.grid_from_problem(q), r, tol=1e-15)
        assert info["status"] == B.OK, info
        assert info["cycles"] == 4 + 2 * (info["outer_iterations"] - 1)
        assert rel_l2(phi.cpu().numpy(), ref) <= MIXED_TOL
