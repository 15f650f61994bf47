"""Seeded synthetic inputs for the cylindrical field solve.

This module describes problems (grid sizes, geometry, wall potentials) and
draws charge densities.  It holds none of the solver's arithmetic: no
conductances, transforms or multigrid.  Both the CUDA library's binding and
the CPU oracle take a :class:`Problem` and build their own discretisations
from its parameters.

Workloads (the paper's 512 x 128 x 400 annulus of Sec. 5.2 and the smaller
and uneven cases built around it):

* :func:`annulus` -- r in [0.02, 0.05] m, z in [0, 0.03] m, full 2*pi annulus,
  phi = 0 V on both r walls, 300 V at z = 0 and 0 V at z = L.
* :func:`c0_phi_exact` -- the smooth manufactured potential
  sin(pi (r - r_in)/(r_out - r_in)) sin(pi z / L) (1 + 0.3 cos 2 theta) plus the
  z-linear bias 300 (1 - z / L), sampled at cell centres.
* :func:`rho_plasma` -- rho = e (n_i - n_e) from per-cell Poisson macroparticle
  counts (mean 27 per species, macroparticle weight 1e8), a Gaussian axial
  ionisation profile, and an m = 8 azimuthal ion-density wave of 5 %
  amplitude (rho = e (n_i - n_e), Eq. electrostatic_system).
* :func:`channel_plume` -- the composite channel-plume domain (two patches of
  the bounding annulus, grounded exposed faces); charge is zero outside it.
* :func:`uneven_batch` -- 24 independent problems of mixed sizes.
* :func:`drifting_rho` -- the same plasma with the m = 8 wave advanced by one
  azimuthal cell per step.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
import math

import numpy as np

EPS0 = 8.8541878128e-12        # vacuum permittivity, F/m (CODATA 2018)
E_CHARGE = 1.602176634e-19     # elementary charge, C (exact SI value)


@dataclass(frozen=True)
class Problem:
    """One cylindrical Poisson problem on a uniform (r, theta, z) cell grid.

    Arrays are laid out (nz, ntheta, nr), r fastest.  Wall potentials are
    azimuthally invariant.  ``phi_r_in_z`` / ``phi_r_out_z`` optionally give the
    inner / outer r-wall potential per axial cell (length nz); when None the
    scalar value applies along the whole wall.
    """
    nr: int
    ntheta: int
    nz: int
    r_in: float = 0.02
    r_out: float = 0.05
    z0: float = 0.0
    z1: float = 0.03
    theta_span: float = 2.0 * math.pi
    phi_r_in: float = 0.0
    phi_r_out: float = 0.0
    phi_z0: float = 300.0
    phi_z1: float = 0.0
    eps0: float = EPS0
    phi_r_in_z: tuple | None = field(default=None, compare=False)
    phi_r_out_z: tuple | None = field(default=None, compare=False)
    r_faces: tuple | None = field(default=None, compare=False)   # nr + 1 radial faces; None: uniform
    z_faces: tuple | None = field(default=None, compare=False)   # nz + 1 axial faces; None: uniform
    # composite domain (Sec. 2.2): active cells are the union of patches (i0, i1, k0, k1), cells
    # i0 <= i < i1, k0 <= k < k1; None: the whole annulus.  Exposed patch faces are at phi_exposed.
    patches: tuple | None = field(default=None, compare=False)
    phi_exposed: float = 0.0

    @property
    def shape(self):
        return (self.nz, self.ntheta, self.nr)

    @property
    def n_modes(self):
        return self.ntheta // 2 + 1

    def r_centres(self):
        if self.r_faces is not None:
            f = np.asarray(self.r_faces, dtype=np.float64)
            return 0.5 * (f[:-1] + f[1:])
        dr = (self.r_out - self.r_in) / self.nr
        return self.r_in + (np.arange(self.nr) + 0.5) * dr

    def z_centres(self):
        if self.z_faces is not None:
            f = np.asarray(self.z_faces, dtype=np.float64)
            return 0.5 * (f[:-1] + f[1:])
        dz = (self.z1 - self.z0) / self.nz
        return self.z0 + (np.arange(self.nz) + 0.5) * dz

    def theta_centres(self):
        da = self.theta_span / self.ntheta
        return (np.arange(self.ntheta) + 0.5) * da

    def with_r_faces(self, faces):
        """The same problem on a non-uniform radial mesh (faces[0] and faces[-1] become the walls)."""
        f = tuple(float(v) for v in faces)
        return replace(self, r_faces=f, r_in=f[0], r_out=f[-1])

    def with_z_faces(self, faces):
        """The same problem on a non-uniform axial mesh (faces[0] and faces[-1] become the walls)."""
        f = tuple(float(v) for v in faces)
        return replace(self, z_faces=f, z0=f[0], z1=f[-1])

    def with_patches(self, patches, phi_exposed: float = 0.0):
        """The same bounding annulus restricted to a union of rectangular cell patches."""
        return replace(self, patches=tuple(tuple(int(v) for v in q) for q in patches), phi_exposed=float(phi_exposed))

    def active_cells(self) -> np.ndarray:
        """(nz, nr) boolean mask of the cells the patches cover (all True without patches)."""
        if not self.patches:
            return np.ones((self.nz, self.nr), dtype=bool)
        a = np.zeros((self.nz, self.nr), dtype=bool)
        for (i0, i1, k0, k1) in self.patches:
            a[k0:k1, i0:i1] = True
        return a

    def with_r_wall_data(self, phi_r_in_z, phi_r_out_z):
        return replace(self, phi_r_in_z=tuple(float(v) for v in phi_r_in_z),
                       phi_r_out_z=tuple(float(v) for v in phi_r_out_z))


def stretched_radial_faces(r_in: float, r_out: float, nr: int, ratio: float) -> np.ndarray:
    """nr + 1 radial faces from r_in to r_out, each cell `ratio` times as wide as the one inside it."""
    w = ratio ** np.arange(nr)
    return r_in + (r_out - r_in) * np.r_[0.0, np.cumsum(w)] / w.sum()


def annulus(nr: int, ntheta: int, nz: int, **kw) -> Problem:
    """The paper-scale annular geometry and wall potentials at any resolution."""
    return Problem(nr=nr, ntheta=ntheta, nz=nz, **kw)


def channel_plume(nr: int, ntheta: int, nz: int, **kw) -> Problem:
    """Channel-plume composite domain of the paper's topology (Sec. 2.2): an
    annular channel, radial cells [nr/4, nr/2), over the lower half of the
    axis (its base on the 300 V wall at z = 0), opening into a plume that
    fills the whole radial extent over the upper half.  Exposed channel and
    exit-plane faces are grounded (0 V)."""
    p = annulus(nr, ntheta, nz, **kw)
    return p.with_patches(((nr // 4, nr // 2, 0, nz // 2), (0, nr, nz // 2, nz)), 0.0)


def c0_problem() -> Problem:
    """Tiny case: 32 x 16 x 32 cells, 9 azimuthal modes."""
    return annulus(32, 16, 32)


def c1_problem() -> Problem:
    """Paper-scale case: 512 x 128 x 400 cells, 65 azimuthal modes (Sec. 5.2)."""
    return annulus(512, 128, 400)


def c0_phi_exact(p: Problem) -> np.ndarray:
    """Manufactured potential sampled at cell centres, shape (nz, ntheta, nr)."""
    r = p.r_centres()
    z = p.z_centres()
    th = p.theta_centres()
    L = p.z1 - p.z0
    S = np.sin(np.pi * (r - p.r_in) / (p.r_out - p.r_in))
    Z = np.sin(np.pi * (z - p.z0) / L)
    T = 1.0 + 0.3 * np.cos(2.0 * th)
    bias = 300.0 * (1.0 - (z - p.z0) / L)
    return Z[:, None, None] * T[None, :, None] * S[None, None, :] + bias[:, None, None]


def rho_plasma(p: Problem, seed, wave_phase: float = 0.0, mean_count: float = 27.0,
               weight: float = 1e8, wave_m: int = 8, wave_amp: float = 0.05,
               profile_centre: float = 0.5, profile_width: float = 0.15) -> np.ndarray:
    """Charge density from Poisson macroparticle counts, shape (nz, ntheta, nr).

    Ion counts are drawn first, then electron counts, each over the whole
    array in C order, from ``numpy.random.default_rng(seed)``.  The expected
    count per species is ``mean_count * g(z)`` with g a unit-mean Gaussian
    axial profile (centre ``profile_centre * L``, width ``profile_width * L``);
    ions carry the extra factor 1 + wave_amp cos(wave_m (theta - wave_phase)).
    Number density is count * weight / cell volume (r dr dtheta dz).
    """
    rng = np.random.default_rng(seed)
    L = p.z1 - p.z0
    z = p.z_centres() - p.z0
    G = np.exp(-((z - profile_centre * L) ** 2) / (2.0 * (profile_width * L) ** 2))
    g = G / G.mean()
    th = p.theta_centres()
    lam_e = np.broadcast_to((mean_count * g)[:, None, None], p.shape)
    wave = 1.0 + wave_amp * np.cos(wave_m * (th - wave_phase))
    lam_i = (mean_count * g)[:, None, None] * wave[None, :, None] * np.ones((1, 1, p.nr))
    n_i = rng.poisson(lam_i)
    n_e = rng.poisson(lam_e)
    dr = (p.r_out - p.r_in) / p.nr
    dz = L / p.nz
    da = p.theta_span / p.ntheta
    vol = p.r_centres() * dr * da * dz
    rho = (E_CHARGE * weight) * (n_i - n_e).astype(np.float64) / vol[None, None, :]
    if p.patches:
        rho *= p.active_cells()[:, None, :]   # no charge outside the composite domain
    return rho


def uneven_batch(seed: int = 3, count: int = 24):
    """Independent problems of uneven sizes with their charge densities' seeds.

    Sizes are drawn from ``default_rng(seed)``: for each problem an index into
    N_r in {64,128,256,512}, then N_theta in {16,32,64,128}, then N_z in
    {64,200,400}.  Problem ``p`` draws its charge density with seed
    ``seed * 1000 + p``.
    """
    rng = np.random.default_rng(seed)
    nrs, nts, nzs = (64, 128, 256, 512), (16, 32, 64, 128), (64, 200, 400)
    out = []
    for p in range(count):
        nr = nrs[int(rng.integers(len(nrs)))]
        nt = nts[int(rng.integers(len(nts)))]
        nz = nzs[int(rng.integers(len(nzs)))]
        out.append((annulus(nr, nt, nz), seed * 1000 + p))
    return out


def drifting_rho(p: Problem, t: int, base_seed: int = 3) -> np.ndarray:
    """Step ``t`` of a drifting-wave sequence: the m = 8 wave advanced by t cells."""
    da = p.theta_span / p.ntheta
    return rho_plasma(p, [base_seed, t], wave_phase=t * da)


def rho_plasma_torch(p: Problem, seed: int, wave_phase: float = 0.0, device="cuda", mean_count: float = 27.0,
                     weight: float = 1e8, wave_m: int = 8, wave_amp: float = 0.05, profile_centre: float = 0.5,
                     profile_width: float = 0.15):
    """The rho_plasma recipe drawn on the GPU with a seeded torch generator.

    Same distribution as :func:`rho_plasma` (not the same samples: torch's
    generator replaces numpy's).  Used for long sequences of full-size inputs
    whose host-side generation would dominate a benchmark.
    """
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    L = p.z1 - p.z0
    z = torch.as_tensor(p.z_centres() - p.z0, device=device)
    G = torch.exp(-((z - profile_centre * L) ** 2) / (2.0 * (profile_width * L) ** 2))
    gz = G / G.mean()
    th = torch.as_tensor(p.theta_centres(), device=device)
    lam_e = (mean_count * gz)[:, None, None].expand(p.nz, p.ntheta, p.nr).contiguous()
    wave = 1.0 + wave_amp * torch.cos(wave_m * (th - wave_phase))
    lam_i = lam_e * wave[None, :, None]
    n_i = torch.poisson(lam_i, generator=g)
    n_e = torch.poisson(lam_e, generator=g)
    dr = (p.r_out - p.r_in) / p.nr
    dz = L / p.nz
    da = p.theta_span / p.ntheta
    vol = torch.as_tensor(p.r_centres() * dr * da * dz, device=device)
    rho = (E_CHARGE * weight) * (n_i - n_e) / vol[None, None, :]
    if p.patches:
        rho = rho * torch.as_tensor(p.active_cells(), device=device)[:, None, :]
    return rho


def drifting_rho_torch(p: Problem, t: int, base_seed: int = 3, device="cuda"):
    """GPU-drawn step ``t`` of the drifting-wave sequence (see :func:`drifting_rho`)."""
    da = p.theta_span / p.ntheta
    return rho_plasma_torch(p, base_seed * 1_000_003 + t, wave_phase=t * da, device=device)
