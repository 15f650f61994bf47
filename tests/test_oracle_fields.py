"""Pins of the oracle's face-field reconstruction (CPU).

The discrete Gauss law ties the reconstructed face field to the oracle's own
finite-volume system: for its solution, every cell's outward face fluxes sum
to rho V / eps0 (appendix "Cell integration and face fluxes"), so a wrong
distance, area, wall value or sign fails it.  A linear potential gives the
closed-form field.
"""
import numpy as np
import pytest

import oracle
from oracle import fields as F
from helpers import narrow_span, small_rin, with_bias_walls
from paper_2609_07172_gb300 import workloads as W


def _nonuniform_grid():
    rng = np.random.default_rng(11)
    r_faces = 0.02 + np.cumsum(np.r_[0.0, rng.uniform(0.5, 1.5, 10)]) * 2e-3
    z_faces = np.cumsum(np.r_[0.0, rng.uniform(0.5, 1.5, 9)]) * 3e-3
    return oracle.Grid(r_faces, z_faces, 8, 2 * np.pi, 8.8541878128e-12, 20.0, -10.0, 300.0, 0.0)


CASES = {
    "annulus": lambda: oracle.grid_from_problem(W.annulus(12, 8, 10)),
    "bias_walls": lambda: oracle.grid_from_problem(with_bias_walls(W.annulus(10, 4, 12))),
    "small_rin": lambda: oracle.grid_from_problem(small_rin(8, 8, 8)),
    "narrow_span": lambda: oracle.grid_from_problem(narrow_span(8, 4, 8)),
    "nonuniform": _nonuniform_grid,
}


@pytest.mark.parametrize("name", list(CASES))
def test_gauss_law_holds_for_the_oracle_solution(name):
    g = CASES[name]()
    rng = np.random.default_rng(5)
    rho = rng.normal(size=g.shape) * 1e-6
    phi, _ = oracle.solve3d(g, rho, tol=1e-15)
    res, scale = F.gauss_residual(g, rho, *F.face_field(g, phi))
    assert np.abs(res).max() <= 1e-11 * scale


def test_linear_potential_gives_the_closed_form_field():
    p = W.annulus(10, 8, 12)
    zc = p.z_centres()
    L = p.z1 - p.z0
    bias = 300.0 * (1.0 - (zc - p.z0) / L)
    g = oracle.grid_from_problem(p.with_r_wall_data(bias, bias))
    phi = np.broadcast_to(bias[:, None, None], g.shape).copy()
    er, ea, ez = F.face_field(g, phi)
    assert np.abs(ez - 300.0 / L).max() <= 1e-9 * 300.0 / L   # every axial face, walls included
    assert np.abs(er).max() == 0.0 and np.abs(ea).max() == 0.0


def test_a_wrong_arc_length_fails_the_gauss_law():
    """A planted mistake (the azimuthal distance taken at the outer face radius
    instead of the centre) must be caught by the pin."""
    g = oracle.grid_from_problem(small_rin(8, 8, 8)).homogeneous()   # the charge alone drives the field
    rho = np.random.default_rng(6).normal(size=g.shape) * 1e-6
    phi, _ = oracle.solve3d(g, rho, tol=1e-15)
    er, ea, ez = F.face_field(g, phi)
    rc = 0.5 * (g.r_faces[:-1] + g.r_faces[1:])
    ea_wrong = ea * rc / g.r_faces[1:]
    res, scale = F.gauss_residual(g, rho, er, ea_wrong, ez)
    assert np.abs(res).max() > 1e-3 * scale


# ---------------------------------------------------------------- composite domains, stretched faces

def _channel_plume_stretched(nr=16, nt=4, nz=12, ratio=1.06):
    """The channel-plume topology (Sec. 2.2) on faces stretched in r and z,
    with exposed faces at 40 V."""
    p = W.channel_plume(nr, nt, nz)
    p = p.with_r_faces(W.stretched_radial_faces(p.r_in, p.r_out, nr, ratio))
    w = ratio ** np.arange(nz)
    p = p.with_z_faces(p.z0 + (p.z1 - p.z0) * np.r_[0.0, np.cumsum(w)] / w.sum())
    return p.with_patches(p.patches, phi_exposed=40.0)


@pytest.mark.parametrize("stretched", [False, True], ids=["uniform", "stretched"])
def test_gauss_law_on_a_composite_domain(stretched):
    p = _channel_plume_stretched() if stretched else W.channel_plume(16, 4, 12).with_patches(
        W.channel_plume(16, 4, 12).patches, phi_exposed=40.0)
    g = oracle.grid_from_problem(p)
    rho = W.rho_plasma(p, seed=31)
    phi, _ = oracle.solve3d(g, rho, tol=1e-15)
    er, ea, ez = F.face_field(g, phi)
    res, scale = F.gauss_residual(g, rho, er, ea, ez)
    assert np.abs(res).max() <= 1e-11 * scale
    # no field where no active cell is
    act = g.active.astype(bool)
    assert np.all(ea[:, :, :][np.broadcast_to(~act[:, None, :], ea.shape)] == 0.0)


def test_exposed_faces_differenced_as_interior_faces_fail_the_gauss_law():
    """A planted mistake: the face between an active and an inactive cell
    differenced centre to centre against the inactive cell's phi = 0, as if
    it were an interior face."""
    p = _channel_plume_stretched()
    g = oracle.grid_from_problem(p)
    rho = W.rho_plasma(p, seed=32)
    phi, _ = oracle.solve3d(g, rho, tol=1e-15)
    plain = oracle.Grid(g.r_faces, g.z_faces, g.ntheta, g.L_alpha, g.eps0, g.phi_rin, g.phi_rout,
                        g.phi_z0, g.phi_z1)
    er, ea, ez = F.face_field(plain, phi)
    res, scale = F.gauss_residual(g, rho, er, ea, ez)
    assert np.abs(res).max() > 1e-3 * scale


def test_all_active_composite_field_is_the_plain_field():
    p = W.annulus(10, 4, 8)
    g = oracle.grid_from_problem(p)
    ga = oracle.Grid(g.r_faces, g.z_faces, g.ntheta, g.L_alpha, g.eps0, g.phi_rin, g.phi_rout, g.phi_z0,
                     g.phi_z1, np.ones((g.nz, g.nr), dtype=bool), 77.0)
    phi = np.random.default_rng(3).normal(size=g.shape)
    for a, b in zip(F.face_field(g, phi), F.face_field(ga, phi)):
        np.testing.assert_array_equal(a, b)
