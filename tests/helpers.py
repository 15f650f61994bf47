"""Shared test helpers: FFT bookkeeping for comparisons and oracle-derived inputs.

numpy's FFT serves only to move oracle results into mode space for
element-wise comparison; it is a library routine, not part of either side.
"""
import math

import numpy as np

import oracle
from paper_2609_07172_gb300 import workloads as W


def to_modes(x3d):
    """(nz, ntheta, nr) real -> (nz, nr, nm, 2) mode layout of (1/N) rfft along theta."""
    n = x3d.shape[1]
    xh = np.fft.rfft(x3d, axis=1) / n          # (nz, nm, nr)
    xh = np.transpose(xh, (0, 2, 1))           # (nz, nr, nm)
    return np.ascontiguousarray(np.stack([xh.real, xh.imag], axis=-1))


def from_modes(xm, ntheta):
    """(nz, nr, nm, 2) mode layout -> (nz, ntheta, nr) via the unscaled inverse."""
    xh = xm[..., 0] + 1j * xm[..., 1]
    xh = np.transpose(xh, (0, 2, 1))
    return np.fft.irfft(xh, n=ntheta, axis=1) * ntheta


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def discrete_manufactured_rho(p, phi_ex):
    """rho for which the oracle's discrete system has phi_ex as its solution."""
    g = oracle.grid_from_problem(p)
    bD = oracle.rhs3d(g, np.zeros(p.shape))
    s = oracle.rhs3d(g.homogeneous(), np.ones(p.shape))
    return (oracle.apply3d(g, phi_ex) - bD) / s


def narrow_span(nr=32, ntheta=16, nz=32):
    """The paper's production sector: r from 100 m, span 6.39918e-5 rad (Sec. 2.2).

    The radial width is nr / 1024 m (31.25 mm at nr = 32) instead of the
    paper's 25.6 mm so that every face r_in + i dr is exactly representable:
    at r / dr ~ 1e5 a non-representable width makes the two sides' face
    differences disagree at ~1e-11, which is geometry rounding, not solver error.
    """
    return W.Problem(nr=nr, ntheta=ntheta, nz=nz, r_in=100.0, r_out=100.0 + nr / 1024.0, z0=0.0, z1=0.02,
                     theta_span=6.39918e-5, phi_r_in=0.0, phi_r_out=0.0, phi_z0=200.0, phi_z1=0.0)


def small_rin(nr=32, ntheta=16, nz=32):
    """Annulus close to the axis, where lambda_m mu / D0 is large."""
    return W.Problem(nr=nr, ntheta=ntheta, nz=nz, r_in=0.002, r_out=0.005, z0=0.0, z1=0.003,
                     phi_r_in=10.0, phi_r_out=-5.0, phi_z0=300.0, phi_z1=0.0)


def with_bias_walls(p):
    """r-wall potentials that vary with z (exercises the per-cell b^D table)."""
    zc = p.z_centres()
    bias = 300.0 * (1.0 - (zc - p.z0) / (p.z1 - p.z0))
    return p.with_r_wall_data(bias, 0.5 * bias)


def cond_estimate(g, iters=60, seed=0):
    """Upper estimate of the 2-norm condition number of the oracle's 3-D
    operator A (SPD): lambda_max by power iteration on A (a Rayleigh quotient
    from below, so raised by 25 % for the power iteration's slow convergence
    at the top of the spectrum), lambda_min
    by inverse iteration with the oracle's CG solves (from above, lowered by
    1 %).  The operator is the homogeneous one; wall data only enter b."""
    h = g.homogeneous()
    s = oracle.rhs3d(h, np.ones(g.shape))          # b = s rho on the homogeneous grid
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(g.shape)
    for _ in range(iters):
        y = oracle.apply3d(h, x)
        x = y / np.linalg.norm(y)
    lmax = float(np.vdot(x, oracle.apply3d(h, x)))
    x = rng.standard_normal(g.shape)
    for _ in range(8):
        y, _ = oracle.solve3d(h, x / s, tol=1e-13)  # A y = x
        x = y / np.linalg.norm(y)
    lmin = float(np.vdot(x, oracle.apply3d(h, x)))
    return 1.25 * lmax / (0.99 * lmin)
