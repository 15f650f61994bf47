"""Pins of the oracle's composite domain (CPU).

The active cross-section is a union of rectangular patches; a face between an
active and an inactive cell is a Dirichlet face at the exposed-face potential,
with the centre-to-face distance, like a wall face (Sec. 2.2 and the
appendix's "Dirichlet faces").  So a single patch is the same discrete
problem as the plain grid built on that patch's own faces, with each wall the
bounding wall where the patch touches it and the exposed potential elsewhere:
the masked solve must equal that independent grid's solve.  A wrong distance,
conductance, wall value or sign on an exposed face breaks the equality.
"""
import numpy as np
import pytest

import oracle
from helpers import with_bias_walls
from paper_2609_07172_gb300 import workloads as W


def _nonuniform(p):
    return p.with_r_faces(W.stretched_radial_faces(p.r_in, p.r_out, p.nr, 1.06))


def _subgrid(g, patch, v):
    i0, i1, k0, k1 = patch
    return oracle.Grid(g.r_faces[i0:i1 + 1], g.z_faces[k0:k1 + 1], g.ntheta, g.L_alpha, g.eps0,
                       g.phi_rin[k0:k1] if i0 == 0 else v,
                       g.phi_rout[k0:k1] if i1 == g.nr else v,
                       g.phi_z0[i0:i1] if k0 == 0 else v,
                       g.phi_z1[i0:i1] if k1 == g.nz else v)


PATCHES = [
    ("interior", (3, 9, 2, 8)),        # every face exposed
    ("inner_wall", (0, 5, 3, 10)),     # touches the inner r wall
    ("anode", (4, 8, 0, 6)),           # touches z = 0 (the 300 V wall)
    ("outer_top", (6, 12, 5, 12)),     # touches the outer r wall and z = L
]


@pytest.mark.parametrize("nonuniform", [False, True], ids=["uniform", "stretched"])
@pytest.mark.parametrize("name,patch", PATCHES, ids=[n for n, _ in PATCHES])
def test_single_patch_is_the_plain_problem_on_its_own_faces(name, patch, nonuniform):
    p = with_bias_walls(W.annulus(12, 8, 12))
    if nonuniform:
        p = _nonuniform(p)
    v = 37.5
    pm = p.with_patches([patch], v)
    g = oracle.grid_from_problem(pm)
    rho = W.rho_plasma(pm, seed=7)
    phi, info = oracle.solve3d(g, rho, tol=1e-15)
    assert info["converged"]
    i0, i1, k0, k1 = patch
    sub = _subgrid(g, patch, v)
    phi_s, _ = oracle.solve3d(sub, rho[k0:k1, :, i0:i1], tol=1e-15)
    got = phi[k0:k1, :, i0:i1]
    assert np.abs(got - phi_s).max() <= 1e-11 * np.abs(phi_s).max()
    # inactive cells are not unknowns: held at zero
    mask = pm.active_cells()
    assert np.all(phi.transpose(0, 2, 1)[~mask] == 0.0)


def test_patch_covering_everything_is_the_unmasked_grid():
    p = with_bias_walls(W.annulus(10, 4, 8))
    g0 = oracle.grid_from_problem(p)
    g1 = oracle.grid_from_problem(p.with_patches([(0, 10, 0, 8)], 123.0))
    rng = np.random.default_rng(3)
    x = rng.normal(size=g0.shape)
    assert np.array_equal(oracle.apply3d(g0, x), oracle.apply3d(g1, x))
    assert np.array_equal(oracle.rhs3d(g0, x), oracle.rhs3d(g1, x))
    # two abutting patches are one domain: the shared interface is not a face of the mask
    g2 = oracle.grid_from_problem(p.with_patches([(0, 10, 0, 3), (0, 10, 3, 8)], 123.0))
    assert np.array_equal(oracle.apply3d(g0, x), oracle.apply3d(g2, x))


def test_constant_potential_on_the_channel_plume():
    """Every wall and exposed face at V and no charge: phi = V on every active cell."""
    v = -42.0
    p = W.channel_plume(16, 8, 12, phi_r_in=v, phi_r_out=v, phi_z0=v, phi_z1=v)
    p = p.with_patches(p.patches, v)
    g = oracle.grid_from_problem(p)
    phi, _ = oracle.solve3d(g, np.zeros(p.shape), tol=1e-15)
    mask = p.active_cells()
    a = phi.transpose(0, 2, 1)
    assert np.abs(a[mask] - v).max() <= 1e-12 * abs(v)
    assert np.all(a[~mask] == 0.0)


def test_channel_plume_rows_couple_only_active_cells():
    """The operator's row of an active cell reads no inactive value, and an
    inactive cell's row is the identity: A applied to a field that is nonzero
    only on inactive cells is that field itself."""
    p = W.channel_plume(16, 8, 12)
    g = oracle.grid_from_problem(p)
    mask = np.broadcast_to(p.active_cells()[:, None, :], p.shape)
    rng = np.random.default_rng(4)
    x = rng.normal(size=p.shape) * (~mask)
    ax = oracle.apply3d(g, x)
    assert np.array_equal(ax, x)
