"""FP64 cloud-in-cell deposit and charge projection on the oracle's grid
(test infrastructure only: the tests, the smoke check and the benchmark's CPU
leg may import it; the product library never does).

Deposit (Sec. "Warp-aggregated cylindrical CIC deposition", Eqs. cic_weights
and particle_cic_update), one species of macro-particles of weight W: a
particle in cell (i, j, k) at normalised position (xi, eta, zeta) in [0,1)^3
within the cell adds

    n_nu += W / V_nu * w_r w_alpha w_z,   w^(0) = 1 - t, w^(1) = t,

to each of the cell's eight corner nodes nu (node index a in [0, nr] at the
radial face r_a, j periodic in alpha, c in [0, nz] at the axial face z_c).
V_nu is the node's cylindrical control volume: from the centre of the cell
below to the centre of the cell above in r and in z (cut at the walls), a
full dalpha in alpha, with the exact radial integral of r dr.  Particles
outside the domain deposit nothing.  A plain scatter-add, particle by
particle (no aggregation).

Projection (Sec. 2: "a volume-consistent projection to cell-centred charge";
the paper gives no formula, this is the reading): each node's control volume
is split into the octants that lie in its adjacent cells, and an octant's
charge goes to its cell,

    rho_q = charge * sum over the corners nu of q of n_nu V_(nu in q) / V_q,

so sum_q rho_q V_q = charge * sum_nu n_nu V_nu = charge * W * (particles
deposited): charge is conserved by construction.

Composite domain (Sec. 2.2, a union of rectangular patches; the reading):
particles in inactive cells deposit nothing, a node's control volume counts
only its octants in active cells, and inactive cells get no charge; the
conservation identity then holds over the active cells.  Non-uniform faces
need nothing more: offsets within a cell use its own faces, the node
intervals run between the neighbouring centres, and a cell's axial octant
share stays 1/2 (face to centre is half the cell).
"""
from __future__ import annotations

import numpy as np


def _centres(f):
    return 0.5 * (f[:-1] + f[1:])


def _node_extents(f):
    """Lower and upper ends of each node's control interval along one axis."""
    c = _centres(f)
    return np.r_[f[0], c], np.r_[c, f[-1]]


def node_volumes(g):
    """V_nu, shape (nz+1, nr+1) (the same for every alpha node).

    Composite domain (g.active set): only the octants of the node's control
    volume that lie in active cells count, V_nu = sum over its active
    neighbour cells q of V(nu in q), so that the projection below conserves
    the charge deposited in active cells exactly (no particle sits in an
    inactive cell, and no charge is projected there)."""
    rf, zf = g.r_faces, g.z_faces
    da = g.L_alpha / g.ntheta
    if g.active is None:
        rlo, rhi = _node_extents(rf)
        zlo, zhi = _node_extents(zf)
        # the integral of r dr, (rhi^2 - rlo^2) / 2, factored (no cancellation far from the axis)
        return da * (zhi - zlo)[:, None] * ((rhi - rlo) * (rhi + rlo) / 2)[None, :]
    rc, zc = _centres(rf), _centres(zf)
    nr, nz = rf.size - 1, zf.size - 1
    # the half cells next to each face: cell i's part toward its lower face (lo) and its upper face (hi)
    vr_lo = (rc - rf[:-1]) * (rc + rf[:-1]) / 2
    vr_hi = (rf[1:] - rc) * (rf[1:] + rc) / 2
    hz = np.diff(zf) / 2
    act = g.active.astype(bool)
    vol = np.zeros((nz + 1, nr + 1))
    for k in range(nz):
        for i in range(nr):
            if not act[k, i]:
                continue
            for c, vz in ((k, hz[k]), (k + 1, hz[k])):
                vol[c, i] += da * vz * vr_lo[i]
                vol[c, i + 1] += da * vz * vr_hi[i]
    return vol


def deposit(g, r, alpha, z, weight):
    """Nodal number density (nz+1, ntheta, nr+1) of particles at (r, alpha, z)."""
    r, alpha, z = (np.asarray(x, dtype=np.float64) for x in (r, alpha, z))
    rf, zf = g.r_faces, g.z_faces
    nr, nz, nt = rf.size - 1, zf.size - 1, g.ntheta
    da = g.L_alpha / nt
    nodes = np.zeros((nz + 1, nt, nr + 1))
    ir = np.searchsorted(rf, r, side="right") - 1
    iz = np.searchsorted(zf, z, side="right") - 1
    ia = np.floor(alpha / da).astype(np.int64)
    ok = (ir >= 0) & (ir < nr) & (iz >= 0) & (iz < nz) & (ia >= 0) & (ia < nt)
    if g.active is not None:   # a particle in an inactive cell of a composite domain deposits nothing
        ok[ok] = g.active.astype(bool)[iz[ok], ir[ok]]
    ir, iz, ia = ir[ok], iz[ok], ia[ok]
    xr = (r[ok] - rf[ir]) / (rf[ir + 1] - rf[ir])
    xz = (z[ok] - zf[iz]) / (zf[iz + 1] - zf[iz])
    xa = alpha[ok] / da - ia
    vol = node_volumes(g)
    for dz_, wz in ((0, 1.0 - xz), (1, xz)):
        for da_, wa in ((0, 1.0 - xa), (1, xa)):
            for dr_, wr in ((0, 1.0 - xr), (1, xr)):
                c, a, j = iz + dz_, ir + dr_, (ia + da_) % nt
                np.add.at(nodes, (c, j, a), weight * wr * wa * wz / vol[c, a])
    return nodes


def project(g, nodes, charge):
    """Cell-centred charge density (nz, ntheta, nr) from nodal number density."""
    rf, zf = g.r_faces, g.z_faces
    rc = _centres(rf)
    # radial share of the cell's lower / upper corner nodes: the exact r dr
    # integrals of the half cells over the cell's
    r0, r1 = rf[:-1], rf[1:]
    whole = (r1 - r0) * (r1 + r0)
    flo = (rc - r0) * (rc + r0) / whole
    fhi = (r1 - rc) * (r1 + rc) / whole
    n = np.asarray(nodes, dtype=np.float64)
    ns = n + np.roll(n, -1, axis=1)              # the two alpha nodes of a cell
    nzs = ns[:-1] + ns[1:]                       # and its two z nodes
    rho = charge * 0.25 * (flo * nzs[:, :, :-1] + fhi * nzs[:, :, 1:])
    if g.active is not None:   # composite domain: no charge in inactive cells
        rho = np.where(np.broadcast_to(g.active.astype(bool)[:, None, :], rho.shape), rho, 0.0)
    return rho


def cell_volumes(g):
    rf, zf = g.r_faces, g.z_faces
    da = g.L_alpha / g.ntheta
    return da * np.diff(zf)[:, None, None] * ((rf[1:] - rf[:-1]) * (rf[1:] + rf[:-1]) / 2)[None, None, :]
