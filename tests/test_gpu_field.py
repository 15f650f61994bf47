"""Face-field reconstruction (E = -grad phi on the cell faces) on the GPU
against the oracle's definition (needs a GPU)."""
import numpy as np
import pytest
import torch

import oracle
from oracle import fields as F
from helpers import narrow_span, small_rin, with_bias_walls
from paper_2609_07172_gb300 import BatchPlan, Plan, binding as B, workloads as W

pytestmark = pytest.mark.gpu

CASES = {
    "c0": W.c0_problem,
    "bias_walls": lambda: with_bias_walls(W.annulus(40, 8, 24)),
    "small_rin": small_rin,
    "narrow_span": narrow_span,
    "ragged": lambda: W.annulus(37 * 2, 4, 19),
    "one_cell_wide": lambda: W.annulus(1, 2, 3),
}


@pytest.mark.parametrize("name", list(CASES))
def test_face_field_matches_oracle(name):
    p = CASES[name]()
    g = oracle.grid_from_problem(p)
    rho = W.rho_plasma(p, seed=3)
    phi, _ = oracle.solve3d(g, rho, tol=1e-15)
    with Plan(p) as plan:
        got = plan.face_field(torch.from_numpy(phi).cuda())
        torch.cuda.synchronize()
    for e, want in zip(got, F.face_field(g, phi)):
        e = e.cpu().numpy()
        assert e.shape == want.shape
        assert np.abs(e - want).max() <= 1e-12 * np.abs(want).max()


def test_field_of_the_library_solution_obeys_the_discrete_gauss_law():
    p = with_bias_walls(W.annulus(64, 16, 48))
    g = oracle.grid_from_problem(p)
    rho = W.rho_plasma(p, seed=4)
    with Plan(p) as plan:
        phi, info = plan.solve(torch.from_numpy(rho).cuda(), tol=0.0)
        e = plan.face_field(phi)
        torch.cuda.synchronize()
    res, scale = F.gauss_residual(g, rho, *[x.cpu().numpy() for x in e])
    assert np.abs(res).max() <= 1e-11 * scale


def test_face_field_needs_a_single_problem_plan():
    probs = [W.annulus(16, 4, 16), W.annulus(32, 8, 16)]
    with BatchPlan(probs) as bp:
        phi = torch.zeros(probs[0].shape, dtype=torch.float64, device="cuda")
        er = torch.empty((16, 4, 17), dtype=torch.float64, device="cuda")
        ea = torch.empty((16, 4, 16), dtype=torch.float64, device="cuda")
        ez = torch.empty((17, 4, 16), dtype=torch.float64, device="cuda")
        st = B.load().pic_poisson_face_field(bp._plan, *[B.ctypes.c_void_p(t.data_ptr()) for t in (phi, er, ea, ez)])
        assert st == B.EINVAL
