"""Composite domains (union of rectangular patches) vs the FP64 oracle (needs a GPU).

Sec. 2.2: the active r-z cross-section is a union of patches; faces between
an active and an inactive cell are Dirichlet faces at the exposed-face
potential; coarsening keeps every patch edge on a coarse face (Sec. 3.2,
protected faces) and the coarsest level is solved densely.  The bar is the
one of the plain annulus: relative L2 against the oracle's converged solution
<= 1e-12 (FP64) or 1e-10 (mixed), phi exactly 0 outside the patches, and the
reported residual equal to the oracle's.
"""
import numpy as np
import pytest
import torch

import oracle
from helpers import rel_l2, with_bias_walls
from paper_2609_07172_gb300 import FP64, MIXED, BatchPlan, Plan, binding as B, workloads as W

pytestmark = pytest.mark.gpu

TOL = {FP64: 1e-12, MIXED: 1e-10}


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _stretched(p):
    return p.with_r_faces(W.stretched_radial_faces(p.r_in, p.r_out, p.nr, 1.02))


CASES = {
    "channel_plume_32x8x24": lambda: W.channel_plume(32, 8, 24),
    "channel_plume_64x16x48": lambda: W.channel_plume(64, 16, 48, phi_r_out=-20.0),
    "channel_plume_stretched": lambda: _stretched(W.channel_plume(64, 8, 48)),
    "three_patches_exposed_40V": lambda: with_bias_walls(W.annulus(48, 8, 40)).with_patches(
        [(0, 24, 0, 16), (0, 48, 16, 32), (32, 48, 32, 40)], 40.0),
    "island_128x32x64": lambda: W.annulus(128, 32, 64).with_patches(
        [(32, 96, 16, 48), (96, 112, 24, 32)], -15.0),
}


@pytest.fixture(scope="module")
def refs():
    out = {}
    for name, make in CASES.items():
        p = make()
        g = oracle.grid_from_problem(p)
        rho = W.rho_plasma(p, seed=51)
        out[name] = (p, g, rho, oracle.solve3d(g, rho, tol=1e-15)[0])
    return out


@pytest.mark.parametrize("graph", [False, True], ids=["hostloop", "graph"])
@pytest.mark.parametrize("precision", [FP64, MIXED], ids=["fp64", "mixed"])
@pytest.mark.parametrize("name", list(CASES))
def test_composite_domain_matches_oracle(refs, name, precision, graph):
    p, g, rho, ref = refs[name]
    with Plan(p, precision=precision, graph=graph) as plan:
        phi, info = plan.solve(dev(rho), tol=0.0)
    got = phi.cpu().numpy()
    assert info["status"] == B.OK, info
    assert rel_l2(got, ref) <= TOL[precision], info
    assert oracle.relres(g, rho, got) <= 1e-12
    assert np.all(got.transpose(0, 2, 1)[~p.active_cells()] == 0.0)


@pytest.mark.parametrize("kw", [dict(fmg=1, pre_sweeps=2, post_sweeps=1), dict(smooth_strip=2),
                                dict(omega=1.2), dict(smooth_threads=64)],
                         ids=["fmg", "strip2", "sor", "threads64"])
def test_composite_domain_settings(refs, kw):
    p, g, rho, ref = refs["three_patches_exposed_40V"]
    with Plan(p, graph=True, **kw) as plan:
        phi, info = plan.solve(dev(rho), tol=0.0)
    assert info["status"] == B.OK
    assert rel_l2(phi.cpu().numpy(), ref) <= 1e-12


@pytest.mark.parametrize("precision", [FP64, MIXED], ids=["fp64", "mixed"])
def test_composite_domain_stops_at_tol_with_the_oracles_residual(precision):
    p = W.channel_plume(128, 32, 96)
    g = oracle.grid_from_problem(p)
    rho = W.rho_plasma(p, seed=52)
    with Plan(p, precision=precision, graph=True) as plan:
        phi, info = plan.solve(dev(rho), tol=1e-10)
    assert info["status"] == B.OK and info["rel_res"] <= 1e-10
    assert info["cycles"] <= 20, info
    true = oracle.relres(g, rho, phi.cpu().numpy())
    assert true == pytest.approx(info["rel_res"], rel=1e-6, abs=1e-14)


def test_charge_outside_the_patches_is_ignored():
    p = W.channel_plume(32, 8, 24)
    rho = W.rho_plasma(p, seed=53)
    noise = np.random.default_rng(9).normal(size=p.shape) * np.abs(rho).max()
    outside = np.broadcast_to(~p.active_cells()[:, None, :], p.shape)
    with Plan(p) as plan:
        a, _ = plan.solve(dev(rho), tol=1e-12)
        b, _ = plan.solve(dev(rho + noise * outside), tol=1e-12)
    assert torch.equal(a, b)


def test_initial_guess_outside_the_patches_is_ignored():
    p = W.channel_plume(64, 8, 48)
    rho = dev(W.rho_plasma(p, seed=54))
    with Plan(p) as plan:
        ref, info0 = plan.solve(rho, tol=1e-12)
    junk = torch.from_numpy(np.random.default_rng(2).normal(size=p.shape) * 1e3).cuda()
    outside = torch.from_numpy(np.broadcast_to(~p.active_cells()[:, None, :], p.shape).copy()).cuda()
    guess = torch.where(outside, junk, 0.5 * ref).contiguous()
    with Plan(p, initial_guess=True) as plan:
        phi, info = plan.solve(rho, guess, tol=1e-12)
    assert info["status"] == B.OK
    assert rel_l2(phi.cpu().numpy(), ref.cpu().numpy()) <= 1e-10
    assert torch.all(phi[outside] == 0)


@pytest.mark.parametrize("precision", [FP64, MIXED], ids=["fp64", "mixed"])
def test_batch_mixes_composite_and_plain_problems(precision):
    probs = [W.channel_plume(32, 8, 24), with_bias_walls(W.annulus(40, 8, 24)),
             W.annulus(64, 16, 48).with_patches([(0, 32, 0, 48), (32, 64, 16, 32)], 12.0),
             _stretched(W.channel_plume(64, 8, 48))]
    rhos = [W.rho_plasma(q, seed=60 + i) for i, q in enumerate(probs)]
    with BatchPlan(probs, precision=precision, graph=True) as bp:
        phis, infos = bp.solve([dev(r) for r in rhos], tol=0.0)
    for q, r, phi, info in zip(probs, rhos, phis, infos):
        ref, _ = oracle.solve3d(oracle.grid_from_problem(q), r, tol=1e-15)
        assert info["status"] == B.OK, info
        assert rel_l2(phi.cpu().numpy(), ref) <= TOL[precision]


@pytest.mark.parametrize("graph", [False, True], ids=["hostloop", "graph"])
@pytest.mark.parametrize("name", list(CASES))
def test_composite_domain_fused_smoother_matches_oracle(refs, name, graph):
    """The fused FP32 smoother on per-row coefficient classes (south and north
    couplings apart, the restriction's face conductances per class)."""
    p, g, rho, ref = refs[name]
    with Plan(p, precision=MIXED, smooth_fused=1, pre_sweeps=2, post_sweeps=2, graph=graph) as plan:
        phi, info = plan.solve(dev(rho), tol=0.0)
    got = phi.cpu().numpy()
    assert info["status"] == B.OK, info
    assert rel_l2(got, ref) <= TOL[MIXED], info
    assert oracle.relres(g, rho, got) <= 1e-12
    assert np.all(got.transpose(0, 2, 1)[~p.active_cells()] == 0.0)


def test_fused_smoother_batch_mixes_composite_and_plain(refs):
    """A batch of composite and plain problems: the per-row variant keeps the
    three-class path for the plain ones."""
    names = ["channel_plume_64x16x48", "island_128x32x64"]
    probs = [refs[n][0] for n in names] + [with_bias_walls(W.annulus(64, 16, 48))]
    rhos = [refs[n][2] for n in names] + [W.rho_plasma(probs[-1], seed=52)]
    ref_plain, _ = oracle.solve3d(oracle.grid_from_problem(probs[-1]), rhos[-1], tol=1e-15)
    refs_all = [refs[n][3] for n in names] + [ref_plain]
    with BatchPlan(probs, precision=MIXED, smooth_fused=1, pre_sweeps=2, post_sweeps=1, graph=True) as bp:
        phis, infos = bp.solve([dev(r) for r in rhos], tol=0.0)
    for phi, ref, info in zip(phis, refs_all, infos):
        assert info["status"] == B.OK, info
        assert rel_l2(phi.cpu().numpy(), ref) <= TOL[MIXED]


def test_fused_smoother_refused_on_axial_faces_only():
    w = 1.02 ** np.arange(24)
    q = W.annulus(32, 8, 24)
    q = q.with_z_faces(q.z0 + (q.z1 - q.z0) * np.r_[0.0, np.cumsum(w)] / w.sum())
    with pytest.raises(B.PicPoissonError):
        Plan(q, precision=MIXED, smooth_fused=1)
    with Plan(W.channel_plume(32, 8, 24), precision=MIXED, smooth_fused=1):
        pass


def test_autotune_on_a_composite_domain(tmp_path):
    """The tuner tries the fused smoother on a composite domain too and
    returns a working schedule."""
    from paper_2609_07172_gb300 import autotune
    p = W.channel_plume(64, 16, 48)
    rho = dev(W.rho_plasma(p, seed=55))
    best = autotune([p], [rho], tol=1e-10, precision=MIXED, graph=True, repeats=1)
    assert any(t["fused"] for t in best["tried"])
    kw = {k: best[k] for k in ("pre_sweeps", "post_sweeps", "inner_cycles", "smooth_threads", "smooth_strip",
                               "omega", "inner_first", "smooth_fused")}
    with Plan(p, precision=MIXED, graph=True, **kw) as plan:
        phi, info = plan.solve(rho, tol=1e-10)
    assert info["status"] == B.OK and info["rel_res"] <= 1e-10
