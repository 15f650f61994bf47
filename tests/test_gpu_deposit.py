"""Cloud-in-cell deposit (warp-aggregated) and charge projection on the GPU
against the oracle's plain scatter-add (needs a GPU)."""
import numpy as np
import pytest
import torch

import oracle
from oracle import deposit as D
from helpers import narrow_span, small_rin
from paper_2609_07172_gb300 import BatchPlan, Plan, binding as B, workloads as W

pytestmark = pytest.mark.gpu

W0 = 1e8
E = 1.602176634e-19

def _stretch_z(p, ratio):
    w = ratio ** np.arange(p.nz)
    return p.with_z_faces(p.z0 + (p.z1 - p.z0) * np.r_[0.0, np.cumsum(w)] / w.sum())


CASES = {
    "c0": W.c0_problem,
    "small_rin": small_rin,
    "narrow_span": narrow_span,
    "ragged": lambda: W.annulus(38, 4, 19),
    "stretched_r": lambda: W.annulus(40, 8, 24).with_r_faces(W.stretched_radial_faces(0.02, 0.05, 40, 1.06)),
    "stretched_z": lambda: _stretch_z(W.annulus(24, 4, 40), 0.95),
    "channel_plume": lambda: W.channel_plume(32, 8, 24),
    "channel_plume_stretched": lambda: _stretch_z(W.channel_plume(48, 4, 32).with_r_faces(
        W.stretched_radial_faces(0.02, 0.05, 48, 1.04)), 1.04),
}


def _faces(p):
    rf = np.asarray(p.r_faces) if p.r_faces is not None else p.r_in + (p.r_out - p.r_in) * np.arange(p.nr + 1) / p.nr
    zf = np.asarray(p.z_faces) if p.z_faces is not None else p.z0 + (p.z1 - p.z0) * np.arange(p.nz + 1) / p.nz
    return rf, zf


def _particles(p, n, seed, sort):
    rng = np.random.default_rng(seed)
    r = rng.uniform(p.r_in, p.r_out, n)
    a = rng.uniform(0.0, p.theta_span, n)
    z = rng.uniform(p.z0, p.z1, n)
    r[:5] = p.r_out + 1.0          # outside: deposit nothing
    a[5] = -0.1
    if sort:   # cell-major order, as a periodically sorted particle array
        rf, zf = _faces(p)
        ir = np.searchsorted(rf, r, side="right")
        ia = np.floor(a / p.theta_span * p.ntheta)
        iz = np.searchsorted(zf, z, side="right")
        o = np.lexsort((ir, ia, iz))
        r, a, z = r[o], a[o], z[o]
    return r, a, z


def _inside(p, r, a, z):
    """Particles the deposit takes: inside the grid and, on a composite domain, in an active cell."""
    rf, zf = _faces(p)
    ir = np.searchsorted(rf, r, side="right") - 1
    iz = np.searchsorted(zf, z, side="right") - 1
    ok = (ir >= 0) & (ir < p.nr) & (iz >= 0) & (iz < p.nz) & (a >= 0) & (a < p.theta_span)
    if getattr(p, "patches", None):
        act = p.active_cells()
        ok[ok] = act[iz[ok], ir[ok]]
    return int(ok.sum())


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.mark.parametrize("sort", [False, True], ids=["unsorted", "sorted"])
@pytest.mark.parametrize("name", list(CASES))
def test_deposit_and_projection_match_oracle(name, sort):
    p = CASES[name]()
    g = oracle.grid_from_problem(p)
    n = 20 * p.nr * p.nz + 37
    ri, ai, zi = _particles(p, n, 1, sort)
    re, ae, ze = _particles(p, n, 2, sort)
    with Plan(p) as plan:
        ni = plan.deposit(_dev(ri), _dev(ai), _dev(zi), W0)
        ne = plan.deposit(_dev(re), _dev(ae), _dev(ze), W0)
        rho = plan.project(ni, E)
        rho = plan.project(ne, -E, rho, accumulate=True)
        torch.cuda.synchronize()
    want_i = D.deposit(g, ri, ai, zi, W0)
    got_i = ni.cpu().numpy()
    assert np.abs(got_i - want_i).max() <= 1e-12 * np.abs(want_i).max()
    want_rho = D.project(g, want_i, E) + D.project(g, D.deposit(g, re, ae, ze, W0), -E)
    scale = np.abs(D.project(g, want_i, E)).max()
    assert np.abs(rho.cpu().numpy() - want_rho).max() <= 1e-12 * scale
    # the deposited number: the particles inside (active cells of a composite domain)
    assert (got_i * D.node_volumes(g)[:, None, :]).sum() == pytest.approx(W0 * _inside(p, ri, ai, zi), rel=1e-12)
    if getattr(p, "patches", None):   # no charge outside the patches
        act = np.broadcast_to(p.active_cells()[:, None, :], want_rho.shape)
        assert np.all(rho.cpu().numpy()[~act] == 0.0)


def test_deposit_adds_and_empty_is_a_no_op():
    p = W.annulus(16, 8, 12)
    r, a, z = _particles(p, 3000, 3, True)
    with Plan(p) as plan:
        n1 = plan.deposit(_dev(r), _dev(a), _dev(z), W0)
        n2 = plan.deposit(_dev(r), _dev(a), _dev(z), W0, n1.clone())
        e = torch.empty(0, dtype=torch.float64, device="cuda")
        n3 = plan.deposit(e, e, e, W0, n1.clone())
        torch.cuda.synchronize()
    assert torch.allclose(n2, 2 * n1, rtol=1e-14, atol=0)
    assert torch.equal(n3, n1)


def test_deposit_needs_a_single_problem_plan():
    probs = [W.annulus(16, 4, 16), W.annulus(32, 8, 16)]
    with BatchPlan(probs) as bp:
        x = torch.zeros(4, dtype=torch.float64, device="cuda")
        nodes = torch.zeros((17, 4, 17), dtype=torch.float64, device="cuda")
        st = B.load().pic_poisson_deposit(bp._plan, *[B.ctypes.c_void_p(t.data_ptr()) for t in (x, x, x)], 4, W0,
                                          B.ctypes.c_void_p(nodes.data_ptr()))
        assert st == B.EINVAL


def test_particles_on_faces_of_a_stretched_mesh():
    """Particles placed exactly on radial and axial faces of a stretched
    mesh: the cell is the one whose lower face they sit on, as in the
    oracle's search over the faces."""
    p = _stretch_z(W.annulus(24, 4, 20).with_r_faces(W.stretched_radial_faces(0.02, 0.05, 24, 1.08)), 1.07)
    g = oracle.grid_from_problem(p)
    rf, zf = _faces(p)
    rng = np.random.default_rng(9)
    r = np.r_[rf[:-1], rng.choice(rf[:-1], 200)]
    z = np.r_[rng.choice(zf[:-1], rf.size - 1), zf[rng.integers(0, p.nz, 200)]]
    a = rng.uniform(0.0, p.theta_span, r.size)
    with Plan(p) as plan:
        got = plan.deposit(_dev(r), _dev(a), _dev(z), W0).cpu().numpy()
    want = D.deposit(g, r, a, z, W0)
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()
