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
