"""FP64 face-field reconstruction on the oracle's grid (test infrastructure
only: the tests, the smoke check and the benchmark's CPU leg may import it;
the product library never does).

E = -grad phi on every cell face of the three-dimensional grid (Sec. 2: the
particle-in-cell cycle keeps the electric field on cell faces), written from
the definition with numpy on the oracle's own face coordinates:

  radial face between cells i-1 and i:  E_r = (phi_(i-1) - phi_i) / (r_i - r_(i-1))
  inner / outer wall faces:             E_r = (phi_wall - phi_0) / (r_0 - r_in),
                                         E_r = (phi_(nr-1) - phi_wall) / (r_out - r_(nr-1))
  azimuthal face j+1/2 (periodic):      E_a = (phi_j - phi_(j+1)) / (r_i dalpha)
  axial faces:                          as radial, with the z0 / z1 wall values

with cell centres at face midpoints (non-uniform faces included) and the
distances of the operator's face conductances (appendix Eqs. interior_face_conductances,
dirichlet_face_conductances: centre to centre between cells, centre to face
on a Dirichlet wall).

gauss_residual() is the discrete Gauss law that pins it: for the solution of
the oracle's system (appendix "Cell integration and face fluxes"), the
outward face fluxes of every cell, area times E.n with areas r_f dalpha dz
(radial faces), dr dz (azimuthal) and r dr dalpha (axial, the midpoint area of
the conductance G_z = r dr / dz), sum to rho r dr dalpha dz / eps0.
"""
from __future__ import annotations

import numpy as np


def _centres(f):
    return 0.5 * (f[:-1] + f[1:])


def face_field(g, phi):
    """(E_r (nz, nt, nr+1), E_alpha (nz, nt, nr), E_z (nz+1, nt, nr)) from phi (nz, nt, nr).

    Composite domain (g.active set; Sec. 2.2): a face between an active and
    an inactive cell is a Dirichlet face at phi_exposed, differenced from the
    active cell's centre to the face like a wall face; a face with no active
    cell on either side (including a wall face of an inactive cell) carries
    no field, E = 0.
    """
    phi = np.asarray(phi, dtype=np.float64)
    rf, zf = g.r_faces, g.z_faces
    rc, zc = _centres(rf), _centres(zf)
    nz, nt, nr = phi.shape
    da = g.L_alpha / nt
    er = np.empty((nz, nt, nr + 1))
    er[:, :, 1:nr] = (phi[:, :, :-1] - phi[:, :, 1:]) / (rc[1:] - rc[:-1])
    er[:, :, 0] = (g.phi_rin[:, None] - phi[:, :, 0]) / (rc[0] - rf[0])
    er[:, :, nr] = (phi[:, :, -1] - g.phi_rout[:, None]) / (rf[-1] - rc[-1])
    ea = (phi - np.roll(phi, -1, axis=1)) / (rc * da)
    ez = np.empty((nz + 1, nt, nr))
    ez[1:nz] = (phi[:-1] - phi[1:]) / (zc[1:] - zc[:-1])[:, None, None]
    ez[0] = (g.phi_z0[None, :] - phi[0]) / (zc[0] - zf[0])
    ez[nz] = (phi[-1] - g.phi_z1[None, :]) / (zf[-1] - zc[-1])
    if g.active is None:
        return er, ea, ez
    act = g.active.astype(bool)                          # (nz, nr)
    pe = g.phi_exposed
    # radial faces a = 1 .. nr-1 between cells a-1 (west) and a (east)
    for k in range(nz):
        for a in range(nr + 1):
            w = a > 0 and act[k, a - 1]
            e = a < nr and act[k, a]
            if a == 0 or a == nr:                        # wall faces: only an active cell has one
                if not (w or e):
                    er[k, :, a] = 0.0
            elif w and not e:                            # exposed face east of cell a-1
                er[k, :, a] = (phi[k, :, a - 1] - pe) / (rf[a] - rc[a - 1])
            elif e and not w:                            # exposed face west of cell a
                er[k, :, a] = (pe - phi[k, :, a]) / (rc[a] - rf[a])
            elif not (w or e):
                er[k, :, a] = 0.0
    ea[~np.broadcast_to(act[:, None, :], ea.shape)] = 0.0
    for c in range(nz + 1):
        for i in range(nr):
            s = c > 0 and act[c - 1, i]
            n = c < nz and act[c, i]
            if c == 0 or c == nz:
                if not (s or n):
                    ez[c, :, i] = 0.0
            elif s and not n:
                ez[c, :, i] = (phi[c - 1, :, i] - pe) / (zf[c] - zc[c - 1])
            elif n and not s:
                ez[c, :, i] = (pe - phi[c, :, i]) / (zc[c] - zf[c])
            elif not (s or n):
                ez[c, :, i] = 0.0
    return er, ea, ez


def gauss_residual(g, rho, er, ea, ez):
    """Per cell: sum of outward face fluxes minus rho V / eps0, and a scale
    to make it relative: the largest sum of absolute flux terms and source
    (the fluxes of wall potentials can dwarf the charge).  In a composite
    domain only active cells are unknowns; the residual of the others is 0."""
    rf, zf = g.r_faces, g.z_faces
    rc = _centres(rf)
    dr, dz = np.diff(rf), np.diff(zf)
    nz, nt, nr = ea.shape
    da = g.L_alpha / nt
    ar = rf[None, :] * da * dz[:, None]                  # (nz, nr+1) radial face areas
    terms = [er[:, :, 1:] * ar[:, None, 1:], -er[:, :, :-1] * ar[:, None, :-1]]
    aa = dr[None, :] * dz[:, None]                       # (nz, nr) azimuthal face areas
    terms += [ea * aa[:, None, :], -np.roll(ea, 1, axis=1) * aa[:, None, :]]
    az = (rc * dr * da)[None, None, :]                   # axial face areas
    terms += [ez[1:] * az, -ez[:-1] * az]
    src = np.asarray(rho, dtype=np.float64) * (rc * dr * da)[None, None, :] * dz[:, None, None] / g.eps0
    flux = sum(terms)
    scale = sum(np.abs(t) for t in terms) + np.abs(src)
    res = flux - src
    if g.active is not None:
        keep = np.broadcast_to(g.active.astype(bool)[:, None, :], res.shape)
        res = np.where(keep, res, 0.0)
        scale = np.where(keep, scale, 0.0)
    return res, float(scale.max())
