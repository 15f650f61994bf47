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

def _stretch_z(p, ratio):
    w = ratio ** np.arange(p.nz)
    return p.with_z_faces(p.z0 + (p.z1 - p.z0) * np.r_[0.0, np.cumsum(w)] / w.sum())


def _channel_plume_stretched(nr, nt, nz, ratio, pe=40.0):
    """The channel-plume topology (Sec. 2.2) on faces stretched in r and z, exposed faces at pe."""
    p = W.channel_plume(nr, nt, nz)
    p = _stretch_z(p.with_r_faces(W.stretched_radial_faces(p.r_in, p.r_out, nr, ratio)), ratio)
    return p.with_patches(p.patches, phi_exposed=pe)


CASES = {
    "c0": W.c0_problem,
    "stretched_r": lambda: W.annulus(48, 8, 32).with_r_faces(W.stretched_radial_faces(0.02, 0.05, 48, 1.04)),
    "stretched_z": lambda: _stretch_z(with_bias_walls(W.annulus(40, 8, 36)), 1.05),
    "channel_plume": lambda: W.channel_plume(64, 8, 48).with_patches(W.channel_plume(64, 8, 48).patches,
                                                                      phi_exposed=25.0),
    "channel_plume_stretched": lambda: _channel_plume_stretched(64, 8, 48, 1.03),
    "three_patches": lambda: W.annulus(48, 4, 40).with_patches([(0, 16, 0, 20), (16, 48, 8, 40), (0, 8, 24, 40)],
                                                              phi_exposed=-12.0),
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


@pytest.mark.parametrize("name", ["c0_bias", "channel_plume_stretched"])
def test_field_of_the_library_solution_obeys_the_discrete_gauss_law(name):
    p = with_bias_walls(W.annulus(64, 16, 48)) if name == "c0_bias" else _channel_plume_stretched(64, 8, 48, 1.03)
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
