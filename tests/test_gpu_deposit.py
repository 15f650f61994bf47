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

CASES = {
    "c0": W.c0_problem,
    "small_rin": small_rin,
    "narrow_span": narrow_span,
    "ragged": lambda: W.annulus(38, 4, 19),
}


def _particles(p, n, seed, sort):
    rng = np.random.default_rng(seed)
    r = rng.uniform(p.r_in, p.r_out, n)
    a = rng.uniform(0.0, p.theta_span, n)
    z = rng.uniform(p.z0, p.z1, n)
    r[:5] = p.r_out + 1.0          # outside: deposit nothing
    a[5] = -0.1
    if sort:   # cell-major order, as a periodically sorted particle array
        ir = np.floor((r - p.r_in) / (p.r_out - p.r_in) * p.nr)
        ia = np.floor(a / p.theta_span * p.ntheta)
        iz = np.floor((z - p.z0) / (p.z1 - p.z0) * p.nz)
        o = np.lexsort((ir, ia, iz))
        r, a, z = r[o], a[o], z[o]
    return r, a, z


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
    # the deposited number: all particles but the six outside
    assert (got_i * D.node_volumes(g)[:, None, :]).sum() == pytest.approx(W0 * (n - 6), rel=1e-12)


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
