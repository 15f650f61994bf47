"""CUDA path vs the FP64 CPU oracle, element by element (needs a GPU).

Every step of the path is called through the C ABI (ctypes binding): the
forward transform + right-hand side (a-1), the mode operator / residual
(a-3/a-4/a-7 arithmetic), the inverse transform (a-8) and the full solve.
Sizes span several FFT tiles (32 columns), ragged tails (nr not a multiple of
32), single-level grids, N_theta = 2 .. 128, and stress geometries where the
azimuthal shift lambda_m mu dominates.  Tolerance: relative L2 <= 1e-12 in
phi for the FP64 path (the FP64 parity bound); transforms and residuals agree
to rounding (1e-13 of the largest entry).
"""
import numpy as np
import pytest
import torch

import oracle
from helpers import (discrete_manufactured_rho, from_modes, narrow_span, rel_l2, small_rin, to_modes,
                     with_bias_walls)
from paper_2609_07172_gb300 import Plan, PicPoissonError, binding as B, workloads as W

pytestmark = pytest.mark.gpu

DIMS = [(32, 16, 32), (40, 8, 24), (96, 16, 40), (64, 32, 48), (15, 4, 9), (48, 2, 16), (128, 64, 64)]
FP64_TOL = 1e-12


def problems():
    out = []
    for nr, nt, nz in DIMS:
        out.append(pytest.param(with_bias_walls(W.annulus(nr, nt, nz)), id=f"annulus{nr}x{nt}x{nz}"))
    out.append(pytest.param(narrow_span(), id="narrow_span"))
    out.append(pytest.param(small_rin(), id="small_rin"))
    # strongly anisotropic cells: z-only and r-only semi-coarsening
    out.append(pytest.param(W.annulus(64, 8, 400), id="aniso_z"))
    out.append(pytest.param(W.annulus(256, 8, 32), id="aniso_r"))
    return out


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.mark.parametrize("p", problems())
def test_forward_transform_and_rhs(p):
    g = oracle.grid_from_problem(p)
    rho = W.rho_plasma(p, seed=5)
    expect = to_modes(oracle.rhs3d(g, rho))
    with Plan(p) as plan:
        got = plan.forward(dev(rho)).cpu().numpy()
    scale = np.abs(expect).max()
    np.testing.assert_allclose(got, expect, rtol=0, atol=1e-13 * scale)
    assert np.all(got[:, :, 0, 1] == 0.0)
    if p.ntheta >= 2:
        assert np.all(got[:, :, p.ntheta // 2, 1] == 0.0)


@pytest.mark.parametrize("p", problems())
def test_inverse_transform(p):
    rng = np.random.default_rng(3)
    xm = rng.standard_normal((p.nz, p.nr, p.ntheta // 2 + 1, 2))
    expect = from_modes(xm, p.ntheta)      # imaginary parts of m = 0, N/2 are ignored
    with Plan(p) as plan:
        got = plan.inverse(dev(xm)).cpu().numpy()
    np.testing.assert_allclose(got, expect, rtol=0, atol=1e-13 * np.abs(expect).max())


@pytest.mark.parametrize("p", problems())
def test_mode_operator_matches_3d_operator(p):
    """b_hat - A_m u_hat on the GPU equals (1/N) DFT of the oracle's b - A_3D phi."""
    g = oracle.grid_from_problem(p)
    rng = np.random.default_rng(7)
    rho = W.rho_plasma(p, seed=9)
    phi = rng.standard_normal(p.shape) * 50.0
    r3 = oracle.rhs3d(g, rho) - oracle.apply3d(g, phi)
    expect = to_modes(r3)
    with Plan(p) as plan:
        bhat = plan.forward(dev(rho))
        r, rel = plan.mode_residual(dev(to_modes(phi)), bhat)
        got = r.cpu().numpy()
    np.testing.assert_allclose(got, expect, rtol=0, atol=1e-12 * np.abs(expect).max())
    rn, bn = oracle.residual(g, rho, phi)
    assert rel == pytest.approx(rn / bn, rel=1e-10)


@pytest.mark.parametrize("p", problems())
def test_solve_matches_oracle_at_floor(p):
    g = oracle.grid_from_problem(p)
    rho = W.rho_plasma(p, seed=1)
    ref, oinfo = oracle.solve3d(g, rho, tol=1e-15)
    with Plan(p) as plan:
        phi, info = plan.solve(dev(rho), tol=0.0)
    got = phi.cpu().numpy()
    assert info["status"] == B.OK
    err = rel_l2(got, ref)
    assert err <= FP64_TOL, (err, info, oinfo)
    assert oracle.relres(g, rho, got) <= 1e-12


def test_c0_discrete_manufactured():
    p = W.c0_problem()
    phi_ex = W.c0_phi_exact(p)
    rho = discrete_manufactured_rho(p, phi_ex)
    with Plan(p) as plan:
        phi, info = plan.solve(dev(rho), tol=0.0)
    assert rel_l2(phi.cpu().numpy(), phi_ex) <= FP64_TOL


@pytest.mark.parametrize("sweeps", [(1, 1), (0, 2), (2, 0), (3, 1), (1, 0), (2, 2)])
def test_sweep_schedules_match_oracle(sweeps):
    """Every smoothing schedule (including the red-only residual, black-only
    prolongation and fused first-red variants and their full counterparts)
    converges to the oracle's solution."""
    p = with_bias_walls(W.annulus(64, 32, 48))
    g = oracle.grid_from_problem(p)
    rho = W.rho_plasma(p, seed=12)
    ref, _ = oracle.solve3d(g, rho, tol=1e-15)
    with Plan(p, pre_sweeps=sweeps[0], post_sweeps=sweeps[1]) as plan:
        phi, info = plan.solve(dev(rho), tol=0.0)
    assert info["status"] == B.OK
    assert rel_l2(phi.cpu().numpy(), ref) <= FP64_TOL, info


@pytest.mark.parametrize("strip", [1, 2, 4])
@pytest.mark.parametrize("dims", [(64, 32, 48), (96, 16, 38), (40, 8, 14)])
def test_smoother_strips_match_oracle(strip, dims):
    """The strip smoother (each thread updates `strip` same-parity rows) gives
    the oracle's solution, FP64 and mixed, including strips that run past the
    last row (nz = 38 and 14: ragged tails at every level) and levels with
    fewer rows of one parity than the strip."""
    p = with_bias_walls(W.annulus(*dims))
    g = oracle.grid_from_problem(p)
    rho = W.rho_plasma(p, seed=13)
    ref, _ = oracle.solve3d(g, rho, tol=1e-15)
    for prec, tol in ((B.FP64, FP64_TOL), (B.MIXED, 1e-10)):
        with Plan(p, precision=prec, smooth_strip=strip) as plan:
            phi, info = plan.solve(dev(rho), tol=0.0)
        assert info["status"] == B.OK
        assert rel_l2(phi.cpu().numpy(), ref) <= tol, (prec, info)


@pytest.mark.parametrize("omega", [1.15, 1.3])
@pytest.mark.parametrize("strip", [0, 2])
def test_over_relaxed_smoother_matches_oracle(omega, strip):
    """Red-black SOR (u <- u + omega (u_GS - u)) converges to the same discrete
    solution, FP64 and mixed, with both smoother mappings."""
    p = with_bias_walls(W.annulus(64, 32, 48))
    g = oracle.grid_from_problem(p)
    rho = W.rho_plasma(p, seed=15)
    ref, _ = oracle.solve3d(g, rho, tol=1e-15)
    for prec, tol in ((B.FP64, FP64_TOL), (B.MIXED, 1e-10)):
        with Plan(p, precision=prec, omega=omega, smooth_strip=strip, pre_sweeps=1, post_sweeps=1) as plan:
            phi, info = plan.solve(dev(rho), tol=0.0)
        assert info["status"] == B.OK
        assert rel_l2(phi.cpu().numpy(), ref) <= tol, (prec, info)


def test_omega_outside_0_2_is_rejected():
    with pytest.raises(PicPoissonError):
        Plan(W.annulus(32, 8, 32), omega=2.0)


def test_smoother_strip_is_deterministic_and_matches_one_entry_mapping():
    """Strips change only the work assignment: every update reads the same
    values, so the result is bitwise identical to one entry per thread."""
    p = with_bias_walls(W.annulus(96, 16, 40))
    rho = dev(W.rho_plasma(p, seed=14))
    out = []
    for strip in (0, 1, 2, 4):
        with Plan(p, smooth_strip=strip) as plan:
            phi, info = plan.solve(rho, tol=1e-10)
        out.append((phi.cpu(), info["cycles"]))
    for phi, cyc in out[1:]:
        assert cyc == out[0][1]
        assert torch.equal(phi, out[0][0])


@pytest.mark.parametrize("tol", [1e-6, 1e-10])
def test_stop_at_tolerance_reports_true_residual(tol):
    p = with_bias_walls(W.annulus(64, 32, 48))
    g = oracle.grid_from_problem(p)
    rho = W.rho_plasma(p, seed=2)
    with Plan(p) as plan:
        phi, info = plan.solve(dev(rho), tol=tol)
    assert info["status"] == B.OK
    assert info["rel_res"] <= tol
    true = oracle.relres(g, rho, phi.cpu().numpy())
    assert true == pytest.approx(info["rel_res"], rel=1e-6, abs=1e-14)


def test_zero_problem_gives_zero():
    p = W.annulus(32, 8, 16, phi_z0=0.0)
    with Plan(p) as plan:
        phi, info = plan.solve(torch.zeros(p.shape, dtype=torch.float64, device="cuda"), tol=1e-10)
    assert info["status"] == B.OK and info["rel_res"] == 0.0
    assert torch.count_nonzero(phi).item() == 0


def test_nonfinite_rho_is_reported():
    p = W.c0_problem()
    rho = np.zeros(p.shape)
    rho[3, 2, 1] = np.nan
    with Plan(p) as plan:
        with pytest.raises(PicPoissonError) as ei:
            plan.solve(dev(rho))
    assert ei.value.status == B.ENONFINITE


def test_not_converged_is_reported():
    p = W.annulus(64, 16, 64)
    rho = W.rho_plasma(p, seed=4)
    with Plan(p, max_cycles=1) as plan:
        phi, info = plan.solve(dev(rho), tol=1e-14)
    assert info["status"] == B.ENOTCONVERGED
    assert info["cycles"] == 1 and info["rel_res"] > 1e-14


def test_initial_guess_exact_solution_needs_no_cycle():
    p = W.annulus(64, 16, 48)
    rho = W.rho_plasma(p, seed=6)
    with Plan(p) as plan:
        phi, _ = plan.solve(dev(rho), tol=0.0)
    with Plan(p, initial_guess=True) as plan:
        phi2 = phi.clone()
        phi2, info = plan.solve(dev(rho), phi2, tol=1e-10)
    assert info["cycles"] == 0 and info["rel_res0"] < 1e-12
    assert rel_l2(phi2.cpu().numpy(), phi.cpu().numpy()) < 1e-13


def test_deterministic_and_host_entry_point_agree():
    p = W.annulus(96, 16, 40)
    rho = W.rho_plasma(p, seed=8)
    with Plan(p) as plan:
        a, _ = plan.solve(dev(rho), tol=1e-10)
        b, _ = plan.solve(dev(rho), tol=1e-10)
        rho_h = torch.from_numpy(rho).pin_memory()
        phi_h = torch.empty(p.shape, dtype=torch.float64).pin_memory()
        info = plan.solve_host(rho_h, phi_h, tol=1e-10)          # mapped pinned buffers, read in place
        phi_p = torch.zeros(p.shape, dtype=torch.float64)
        info_p = plan.solve_host(torch.from_numpy(rho.copy()), phi_p, tol=1e-10)   # pageable: staged
    with Plan(p, host_staged=True, graph=True) as plan:
        phi_s = torch.zeros(p.shape, dtype=torch.float64).pin_memory()
        info_s = plan.solve_host(rho_h, phi_s, tol=1e-10)       # pinned, forced through staging
        phi_g = torch.zeros(p.shape, dtype=torch.float64).pin_memory()
    with Plan(p, graph=True) as plan:
        info_g = plan.solve_host(rho_h, phi_g, tol=1e-10)       # in place, inside the captured graph
    assert torch.equal(a, b)
    for ph, inf in ((phi_h, info), (phi_p, info_p), (phi_s, info_s), (phi_g, info_g)):
        assert torch.equal(a.cpu(), ph)
        assert inf["status"] == B.OK


def test_profile_counts_launches():
    p = W.annulus(64, 16, 64)
    rho = W.rho_plasma(p, seed=4)
    with Plan(p, profile=True) as plan:
        _, info = plan.solve(dev(rho), tol=1e-10)
    lp, ms = info["launches_phase"], info["ms_phase"]
    assert lp["forward"] == 1 and lp["inverse"] == 1
    assert lp["smooth"] > 0 and ms["smooth"] > 0
    assert info["launches"] == sum(lp.values())


@pytest.mark.parametrize("dims", [(64, 16, 400), (512, 16, 64), (512, 128, 400)])
def test_convergence_rate_independent_of_cell_aspect(dims):
    """Semi-coarsening keeps coarse cells near-isotropic, so strongly
    anisotropic grids converge in about as many cycles as the paper's grid."""
    p = W.annulus(*dims)
    rho = W.rho_plasma(p, seed=3)
    with Plan(p) as plan:
        _, info = plan.solve(dev(rho), tol=1e-10)
    assert info["status"] == B.OK and info["cycles"] <= 12, info["cycles"]


BOTTOM_CASES = [(64, 32, 48), (96, 16, 40), (64, 8, 400), (256, 8, 32), (512, 128, 64), (40, 8, 24)]


@pytest.mark.parametrize("prec", [B.FP64, B.MIXED], ids=["fp64", "mixed"])
@pytest.mark.parametrize("dims", BOTTOM_CASES, ids=[f"{a}x{b}x{c}" for a, b, c in BOTTOM_CASES])
def test_local_bottom_is_bitwise_the_level_kernels(dims, prec):
    """The mode-local bottom (the level above the coarsest and the coarsest
    solve in one block per mode and part) runs the level kernels' operations
    in their order: same cycles, bitwise the same potential, including
    semi-coarsened bottoms (64x8x400, 256x8x32)."""
    p = with_bias_walls(W.annulus(*dims))
    rho = dev(W.rho_plasma(p, seed=41))
    out = []
    for lb in (-1, 0):
        with Plan(p, precision=prec, local_bottom=lb, pre_sweeps=1, post_sweeps=2) as plan:
            phi, info = plan.solve(rho, tol=1e-10)
        assert info["status"] == B.OK
        out.append((phi.cpu(), info["cycles"]))
    assert out[0][1] == out[1][1]
    assert torch.equal(out[0][0], out[1][0])


@pytest.mark.parametrize("dims", [(64, 32, 48), (96, 16, 40), (64, 8, 400), (256, 8, 32), (40, 8, 24)])
def test_full_multigrid_start_matches_oracle(dims):
    """A solve started by a full-multigrid pass converges to the oracle's
    solution and reaches a given tolerance in no more cycles than from zero."""
    p = with_bias_walls(W.annulus(*dims))
    g = oracle.grid_from_problem(p)
    rho = W.rho_plasma(p, seed=43)
    ref, _ = oracle.solve3d(g, rho, tol=1e-15)
    with Plan(p, fmg=1) as plan:
        phi, info = plan.solve(dev(rho), tol=0.0)
    assert info["status"] == B.OK
    assert rel_l2(phi.cpu().numpy(), ref) <= FP64_TOL, info
    cyc = []
    for f in (0, 1):
        with Plan(p, fmg=f, graph=True) as plan:
            _, info = plan.solve(dev(rho), tol=1e-10)
        assert info["status"] == B.OK and info["rel_res"] <= 1e-10
        cyc.append(info["cycles"])
    assert cyc[1] <= cyc[0], cyc


def test_full_multigrid_needs_fp64():
    with pytest.raises(PicPoissonError):
        Plan(W.annulus(32, 8, 32), precision=B.MIXED, fmg=1)


@pytest.mark.parametrize("graph", [False, True], ids=["hostloop", "graph"])
@pytest.mark.parametrize("dims", [(64, 32, 48), (64, 8, 400), (40, 8, 24)])
def test_full_multigrid_start_from_a_given_iterate(dims, graph):
    """fmg with an initial iterate runs the full-multigrid pass on the
    correction equation: the solve still reaches the oracle's solution, and a
    tolerance in no more cycles than the same guess without it."""
    p = with_bias_walls(W.annulus(*dims))
    g = oracle.grid_from_problem(p)
    rho = W.rho_plasma(p, seed=44)
    ref, _ = oracle.solve3d(g, rho, tol=1e-15)
    guess = oracle.solve3d(g, W.rho_plasma(p, seed=45), tol=1e-8)[0]   # a neighbouring step's solution
    with Plan(p, fmg=1, initial_guess=True, graph=graph) as plan:
        phi, info = plan.solve(dev(rho), dev(guess), tol=0.0)
    assert info["status"] == B.OK
    assert rel_l2(phi.cpu().numpy(), ref) <= FP64_TOL, info
    cyc = []
    for f in (0, 1):
        with Plan(p, fmg=f, initial_guess=True, graph=graph) as plan:
            _, info = plan.solve(dev(rho), dev(guess), tol=1e-10)
        assert info["status"] == B.OK and info["rel_res"] <= 1e-10
        cyc.append(info["cycles"])
    assert cyc[1] <= cyc[0], cyc
    # the mode-layout initial iterate takes the same start
    with Plan(p, fmg=1, graph=graph) as plan:
        uh = dev(to_modes(guess))       # the guess in mode layout
        phi_m, info_m = plan.solve_modes(dev(rho), uh, tol=0.0)
    assert info_m["status"] == B.OK
    assert rel_l2(phi_m.cpu().numpy(), ref) <= FP64_TOL


@pytest.mark.parametrize("kw", [dict(precision=B.FP64), dict(precision=B.MIXED),
                                dict(precision=B.MIXED, smooth_fused=1, pre_sweeps=2, post_sweeps=2)],
                         ids=["fp64", "mixed", "mixed_fused"])
def test_largest_azimuthal_resolution_matches_oracle(kw):
    """N_theta = 256, the largest the plan takes: 129 modes (the transforms'
    longest columns, nine mode groups of the fused smoother)."""
    p = with_bias_walls(W.annulus(32, 256, 24))
    g = oracle.grid_from_problem(p)
    rho = W.rho_plasma(p, seed=46)
    ref, _ = oracle.solve3d(g, rho, tol=1e-15)
    with Plan(p, graph=True, **kw) as plan:
        phi, info = plan.solve(dev(rho), tol=0.0)
    assert info["status"] == B.OK
    assert rel_l2(phi.cpu().numpy(), ref) <= (FP64_TOL if kw["precision"] == B.FP64 else 1e-10), info
