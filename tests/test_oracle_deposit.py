"""Pins of the oracle's cloud-in-cell deposit and charge projection (CPU).

The CIC weights of a particle sum to one and the projection's octant shares
of a cell sum to one, so the deposited number and the projected charge are
conserved exactly; a particle on a node or at a cell centre has a closed-form
deposit; a constant nodal density projects to a constant charge density.
"""
import numpy as np
import pytest

import oracle
from oracle import deposit as D
from helpers import small_rin
from paper_2609_07172_gb300 import workloads as W

W0 = 1e8


def _nonuniform_grid():
    rng = np.random.default_rng(12)
    r_faces = 0.003 + np.cumsum(np.r_[0.0, rng.uniform(0.5, 1.5, 7)]) * 1e-3
    z_faces = np.cumsum(np.r_[0.0, rng.uniform(0.5, 1.5, 6)]) * 2e-3
    return oracle.Grid(r_faces, z_faces, 8, 2 * np.pi, 8.8541878128e-12, 0.0, 0.0, 0.0, 0.0)


GRIDS = {
    "annulus": lambda: oracle.grid_from_problem(W.annulus(10, 8, 9)),
    "small_rin": lambda: oracle.grid_from_problem(small_rin(8, 4, 8)),
    "nonuniform": _nonuniform_grid,
}


def _particles(g, n, seed, outside=0):
    rng = np.random.default_rng(seed)
    rf, zf = g.r_faces, g.z_faces
    r = rng.uniform(rf[0], rf[-1], n)
    z = rng.uniform(zf[0], zf[-1], n)
    a = rng.uniform(0.0, g.L_alpha, n)
    if outside:
        r[:outside] = rf[-1] + 1e-3
    return r, a, z


@pytest.mark.parametrize("name", list(GRIDS))
def test_deposit_and_projection_conserve_charge(name):
    g = GRIDS[name]()
    r, a, z = _particles(g, 4000, 1, outside=7)
    nodes = D.deposit(g, r, a, z, W0)
    inside = 4000 - 7
    assert (nodes * D.node_volumes(g)[:, None, :]).sum() == pytest.approx(W0 * inside, rel=1e-13)
    rho = D.project(g, nodes, -1.602176634e-19)
    assert (rho * D.cell_volumes(g)).sum() == pytest.approx(-1.602176634e-19 * W0 * inside, rel=1e-13)


def test_particle_on_a_node_and_at_a_cell_centre():
    g = GRIDS["annulus"]()
    rf, zf, da = g.r_faces, g.z_faces, g.L_alpha / g.ntheta
    vol = D.node_volumes(g)
    # on node (c=3, j=2, a=4): everything there
    nodes = D.deposit(g, [rf[4]], [2 * da], [zf[3]], W0)
    want = np.zeros_like(nodes)
    want[3, 2, 4] = W0 / vol[3, 4]
    assert np.allclose(nodes, want, rtol=1e-14, atol=0)
    # at the centre of cell (k=2, j=5, i=6): an eighth to each corner
    nodes = D.deposit(g, [0.5 * (rf[6] + rf[7])], [5.5 * da], [0.5 * (zf[2] + zf[3])], W0)
    for c in (2, 3):
        for j in (5, 6):
            for a_ in (6, 7):
                assert nodes[c, j % g.ntheta, a_] == pytest.approx(W0 / 8 / vol[c, a_], rel=1e-14)
    assert np.count_nonzero(nodes) == 8


def test_constant_nodal_density_projects_to_constant_charge():
    g = GRIDS["nonuniform"]()
    nodes = np.full((g.nz + 1, g.ntheta, g.nr + 1), 3.0)
    rho = D.project(g, nodes, 2.0)
    assert np.allclose(rho, 6.0, rtol=1e-15, atol=0)


def test_equal_radial_shares_would_break_conservation():
    """A planted mistake (splitting a cell's charge evenly between its inner
    and outer nodes, ignoring the r weighting) must fail the conservation pin
    near the axis."""
    g = GRIDS["small_rin"]()
    r, a, z = _particles(g, 2000, 2)
    nodes = D.deposit(g, r, a, z, W0)
    n = nodes
    ns = n + np.roll(n, -1, axis=1)
    nzs = ns[:-1] + ns[1:]
    rho_wrong = 0.25 * 0.5 * (nzs[:, :, :-1] + nzs[:, :, 1:])
    total = (rho_wrong * D.cell_volumes(g)).sum()
    assert abs(total / (W0 * 2000) - 1.0) > 1e-4


# ---------------------------------------------------------------- composite domains, stretched faces

def _composite_grid(stretch):
    p = W.channel_plume(16, 4, 12)
    if stretch:
        p = p.with_r_faces(W.stretched_radial_faces(p.r_in, p.r_out, 16, 1.06))
        w = 1.06 ** np.arange(12)
        p = p.with_z_faces(p.z0 + (p.z1 - p.z0) * np.r_[0.0, np.cumsum(w)] / w.sum())
    return oracle.grid_from_problem(p)


@pytest.mark.parametrize("stretch", [False, True], ids=["uniform", "stretched"])
def test_composite_deposit_conserves_the_charge_of_active_cells(stretch):
    g = _composite_grid(stretch)
    r, a, z = _particles(g, 6000, 3, outside=5)
    ir = np.searchsorted(g.r_faces, r, side="right") - 1
    iz = np.searchsorted(g.z_faces, z, side="right") - 1
    inb = (ir >= 0) & (ir < g.nr) & (iz >= 0) & (iz < g.nz)
    n_active = int(g.active.astype(bool)[iz[inb], ir[inb]].sum())
    assert 0 < n_active < 6000 - 5
    nodes = D.deposit(g, r, a, z, W0)
    assert (nodes * D.node_volumes(g)[:, None, :]).sum() == pytest.approx(W0 * n_active, rel=1e-13)
    rho = D.project(g, nodes, 1.602176634e-19)
    assert (rho * D.cell_volumes(g)).sum() == pytest.approx(1.602176634e-19 * W0 * n_active, rel=1e-13)
    act = np.broadcast_to(g.active.astype(bool)[:, None, :], rho.shape)
    assert np.all(rho[~act] == 0.0)


def test_composite_with_full_node_volumes_breaks_conservation():
    """A planted mistake: nodes on an exposed face keep their whole control
    volume (the inactive octants included)."""
    g = _composite_grid(True)
    r, a, z = _particles(g, 6000, 4)
    nodes = D.deposit(g, r, a, z, W0)
    plain = oracle.Grid(g.r_faces, g.z_faces, g.ntheta, g.L_alpha, g.eps0, 0.0, 0.0, 0.0, 0.0)
    wrong = nodes * D.node_volumes(g)[:, None, :] / D.node_volumes(plain)[:, None, :]
    rho = D.project(g, wrong, 1.0)
    ir = np.searchsorted(g.r_faces, r, side="right") - 1
    iz = np.searchsorted(g.z_faces, z, side="right") - 1
    n_active = int(g.active.astype(bool)[iz, ir].sum())
    assert abs((rho * D.cell_volumes(g)).sum() / (W0 * n_active) - 1.0) > 1e-3


def test_all_active_composite_deposit_is_the_plain_deposit():
    g = oracle.grid_from_problem(W.annulus(10, 8, 9))
    ga = oracle.Grid(g.r_faces, g.z_faces, g.ntheta, g.L_alpha, g.eps0, 0.0, 0.0, 0.0, 0.0,
                     np.ones((g.nz, g.nr), dtype=bool))
    r, a, z = _particles(g, 3000, 5)
    np.testing.assert_allclose(D.deposit(ga, r, a, z, W0), D.deposit(g, r, a, z, W0), rtol=1e-14, atol=0)
