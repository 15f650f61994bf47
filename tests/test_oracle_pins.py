"""Pins of the FP64 CPU oracle against what the paper and mathematics fix.

Each test checks the oracle against something other than itself: exact
numbers printed in the paper's appendix, the closed-form discrete azimuthal
eigenvalue, dense LAPACK solves, a closed-form solution, and the second-order
convergence of an analytically manufactured potential.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2609_07172_gb300 import workloads as W


def unit_grid(r_faces, z_faces, ntheta=8, L=2 * math.pi, eps0=1.0):
    return oracle.Grid(r_faces, z_faces, ntheta, L, eps0, 0.0, 0.0, 0.0, 0.0)


def lam(m, n, L):
    """Exact discrete azimuthal eigenvalue, Eq. discrete_azimuthal_eigenvalue."""
    da = L / n
    return 4.0 / da ** 2 * math.sin(math.pi * m / n) ** 2


# ---------------------------------------------------------------- worked examples

def test_worked_stencil_coefficients(golden):
    g0 = golden("worked_stencil.txt")
    # 3 x 3 r-z cells with unit spacing; the centre cell has r = 2, faces 1.5 / 2.5
    g = unit_grid([0.5, 1.5, 2.5, 3.5], [-0.5, 0.5, 1.5, 2.5], eps0=W.EPS0)
    c = oracle.cell_coeffs(g, 1, 1)
    assert c["G"][0] == pytest.approx(g0["G_r_minus"][0], rel=1e-15)
    assert c["G"][1] == pytest.approx(g0["G_r_plus"][0], rel=1e-15)
    assert c["G"][2] == pytest.approx(g0["G_z_minus"][0], rel=1e-15)
    assert c["G"][3] == pytest.approx(g0["G_z_plus"][0], rel=1e-15)
    assert not c["dirichlet"].any()
    assert c["mu"] == pytest.approx(g0["mu"][0], rel=1e-15)
    assert c["s"] * W.EPS0 == pytest.approx(g0["s_times_eps0"][0], rel=1e-15)
    assert c["D0"] == pytest.approx(g0["D0_interior"][0], rel=1e-15)


def test_worked_stencil_matrix_row_every_mode(golden):
    """Row of A_m for the worked cell: (8 + 0.5 lambda_m), -1.5, -2.5, -2, -2."""
    g0 = golden("worked_stencil.txt")
    n, L = 8, 2 * math.pi
    g = unit_grid([0.5, 1.5, 2.5, 3.5], [-0.5, 0.5, 1.5, 2.5], ntheta=n, L=L)
    rng = np.random.default_rng(1)
    f = rng.standard_normal((3, 3))  # (k, i)
    j = np.arange(n)
    for m in range(n // 2 + 1):
        for basis in (np.cos, np.sin):
            v = basis(2 * math.pi * m * j / n)
            phi = f[:, None, :] * v[None, :, None]
            out = oracle.apply3d(g, phi)
            row = ((g0["D0_interior"][0] + g0["mu"][0] * lam(m, n, L)) * f[1, 1]
                   - g0["G_r_minus"][0] * f[1, 0] - g0["G_r_plus"][0] * f[1, 2]
                   - g0["G_z_minus"][0] * f[0, 1] - g0["G_z_plus"][0] * f[2, 1])
            np.testing.assert_allclose(out[1, :, 1], row * v, rtol=0, atol=1e-12)


def test_worked_stencil_dirichlet_east(golden):
    g0 = golden("worked_stencil.txt")
    # two radial cells: the second (r = 2) has its east face on the wall r = 2.5
    g = oracle.Grid([0.5, 1.5, 2.5], [-0.5, 0.5, 1.5, 2.5], 4, 2 * math.pi, W.EPS0,
                    0.0, 7.0, 0.0, 0.0)
    c = oracle.cell_coeffs(g, 1, 1)
    assert c["dirichlet"][1] and not c["dirichlet"][0]
    assert c["G"][1] == pytest.approx(g0["GD_r_plus"][0], rel=1e-15)
    assert c["D0"] == pytest.approx(g0["D0_dirichlet_east"][0], rel=1e-15)
    # right-hand side: s rho + 5 phi^D_E with rho = 1, phi^D_E = 7
    rho = np.ones(g.shape)
    b = oracle.rhs3d(g, rho)
    expect = g0["s_times_eps0"][0] / W.EPS0 * 1.0 + g0["rhs_dirichlet_factor"][0] * 7.0
    np.testing.assert_allclose(b[1, :, 1], expect, rtol=1e-15)


def test_two_cell_shifted_family_golden(golden):
    """The appendix's two-cell example built as cells of a grid and assembled
    by the oracle's 3-D operator.

    The paper gives the two cells only through their numbers: a shared face
    of conductance 2, mode-independent diagonals 8 and 9 "including their
    other faces", mu = 0.5 and 0.4, lambda = 3.  Two axially adjacent cells
    of one radial column, with radial neighbours on both sides and axial
    neighbours above and below, realise them (the geometry below follows
    from the appendix's conductance formulas); the 2 x 2 block of the
    oracle's A_0 and A_m on those cells, read off apply3d with theta-constant
    and cos(2 pi m j / N) inputs, must be the printed matrices."""
    g0 = golden("two_cell.txt")
    A0_paper = np.array(g0["A0"]).reshape(2, 2)
    Am_paper = np.array(g0["Am"]).reshape(2, 2)
    mu1, mu2 = g0["M"]
    lam_m = g0["lambda"][0]
    G, D1, D2 = -A0_paper[0, 1], A0_paper[0, 0], A0_paper[1, 1]
    # column of width a at centre c; heights h1, h2 = (mu2 / mu1) h1:
    #   mu1 = a h1 / c and G = c a / ((h1 + h2) / 2) give a^2 = mu1 G (1 + mu2/mu1) / 2
    h1 = 1.0
    h2 = mu2 / mu1 * h1
    a = math.sqrt(mu1 * G * (h1 + h2) / (2 * h1))
    c = a * h1 / mu1
    r1, r2 = c - a / 2, c + a / 2
    # radial conductances per unit height X = r1/(c - c_w) + r2/(c_e - c), split evenly;
    # the axial neighbours' conductances c a / d fill the rest of each diagonal
    X = 5.0
    cw = c - r1 / (X / 2)
    ce = c + r2 / (X / 2)
    r0, r3 = 2 * cw - r1, 2 * ce - r2
    ds = c * a / (D1 - G - h1 * X)
    dn = c * a / (D2 - G - h2 * X)
    h0, h3 = 2 * ds - h1, 2 * dn - h2
    assert 0 < r0 < r1 and r3 > r2 and h0 > 0 and h3 > 0
    z = np.cumsum([0.0, h0, h1, h2, h3])
    # lambda_m = 4 sin^2(pi m / N) / dalpha^2 = lam_m at N = 4, m = 1
    n, m = 4, 1
    dalpha = 2 * math.sin(math.pi * m / n) / math.sqrt(lam_m)
    g = oracle.Grid([r0, r1, r2, r3], z, n, n * dalpha, W.EPS0, 0.0, 0.0, 0.0, 0.0)
    cells = [(1, 1), (1, 2)]                     # (i, k): the two cells, k = 1 below k = 2
    assert oracle.cell_coeffs(g, 1, 1)["mu"] == pytest.approx(mu1, rel=1e-14)
    assert oracle.cell_coeffs(g, 1, 2)["mu"] == pytest.approx(mu2, rel=1e-14)
    j = np.arange(n)
    for mode, expect in ((0, A0_paper), (m, Am_paper)):
        v = np.cos(2 * math.pi * mode * j / n)
        block = np.zeros((2, 2))
        for col, (i, k) in enumerate(cells):
            f = np.zeros((g.nz, g.nr))
            f[k, i] = 1.0
            out = oracle.apply3d(g, f[:, None, :] * v[None, :, None])
            for row, (ii, kk) in enumerate(cells):
                block[row, col] = out[kk, 0, ii]        # v_0 = 1
        np.testing.assert_allclose(block, expect, rtol=1e-13, atol=1e-13 * np.abs(expect).max())


# ---------------------------------------------------------------- eigenvalue identity

@pytest.mark.parametrize("n", [4, 8, 16])
def test_discrete_eigenvalue_identity(n):
    """A_3D (f (x) v_m) = (A_0 f + lambda_m mu f) (x) v_m with the exact discrete
    eigenvalue; the continuous k_m^2 must fail (Eq. discrete_azimuthal_eigenvalue)."""
    rng = np.random.default_rng(n)
    r_faces = 0.3 + np.cumsum(np.r_[0.0, rng.uniform(0.05, 0.2, 7)])
    z_faces = np.cumsum(np.r_[0.0, rng.uniform(0.05, 0.2, 5)])
    L = 0.7
    g = unit_grid(r_faces, z_faces, ntheta=n, L=L)
    nz, nr = z_faces.size - 1, r_faces.size - 1
    f = rng.standard_normal((nz, nr))
    flat = f[:, None, :] * np.ones((1, n, 1))
    A0f = oracle.apply3d(g, flat)[:, 0, :]   # theta-constant: no angular term
    rc = 0.5 * (r_faces[1:] + r_faces[:-1])
    mu = np.diff(z_faces)[:, None] * np.diff(r_faces)[None, :] / rc[None, :]
    j = np.arange(n)
    worst_wrong = 0.0
    for m in range(n // 2 + 1):
        for basis in (np.cos, np.sin):
            v = basis(2 * math.pi * m * j / n)
            if np.abs(v).max() < 1e-8:   # sin at m = 0 and m = N/2 vanishes
                continue
            out = oracle.apply3d(g, f[:, None, :] * v[None, :, None])
            expect = (A0f + lam(m, n, L) * mu * f)[:, None, :] * v[None, :, None]
            scale = np.abs(expect).max()
            np.testing.assert_allclose(out, expect, rtol=0, atol=1e-13 * scale)
            km2 = (2 * math.pi * m / L) ** 2
            wrong = (A0f + km2 * mu * f)[:, None, :] * v[None, :, None]
            worst_wrong = max(worst_wrong, np.abs(out - wrong).max() / scale)
    assert worst_wrong > 1e-3


# ---------------------------------------------------------------- dense direct solves

def dense_matrix(g):
    n = int(np.prod(g.shape))
    A = np.empty((n, n))
    e = np.zeros(n)
    for c in range(n):
        e[c] = 1.0
        A[:, c] = oracle.apply3d(g, e).ravel()
        e[c] = 0.0
    return A


@pytest.mark.parametrize("dims", [(6, 4, 6), (8, 8, 8), (10, 16, 12)])
def test_cg_matches_dense_solve(dims):
    nr, nt, nz = dims
    p = W.annulus(nr, nt, nz, phi_r_in=-20.0, phi_r_out=45.0)
    g = oracle.grid_from_problem(p)
    rho = W.rho_plasma(p, seed=11)
    A = dense_matrix(g)
    assert np.array_equal(A, A.T)            # conductances shared by both cells of a face
    assert np.linalg.eigvalsh(A).min() > 0   # SPD: every plane touches a Dirichlet wall
    b = oracle.rhs3d(g, rho).ravel()
    x_dense = np.linalg.solve(A, b)
    x_cg, info = oracle.solve3d(g, rho, tol=1e-15)
    err = np.linalg.norm(x_cg.ravel() - x_dense) / np.linalg.norm(x_dense)
    assert err < 1e-13, (err, info)


# ---------------------------------------------------------------- closed forms

def test_linear_bias_is_exact():
    """rho = 0 with the z-linear wall data: phi = 300 (1 - z / L) at cell centres."""
    p0 = W.annulus(24, 8, 20)
    zc = p0.z_centres()
    bias = 300.0 * (1.0 - (zc - p0.z0) / (p0.z1 - p0.z0))
    p = p0.with_r_wall_data(bias, bias)
    g = oracle.grid_from_problem(p)
    phi_exact = np.broadcast_to(bias[:, None, None], p.shape)
    rho = np.zeros(p.shape)
    assert oracle.relres(g, rho, phi_exact) < 1e-14
    phi, info = oracle.solve3d(g, rho, tol=1e-15)
    np.testing.assert_allclose(phi, phi_exact, rtol=1e-12, atol=1e-10)


@pytest.mark.parametrize("ratio", [1.15, 0.8])
def test_linear_bias_is_exact_on_a_stretched_axial_mesh(ratio):
    """A potential linear in z is reproduced exactly by the cell-centred
    finite volumes on any axial spacing: every z face carries the same flux
    r dr c (the conductance's 1 / distance cancels the difference), the wall
    faces included.  A conductance or volume built from a uniform dz, or a
    wall distance of half the wrong cell, breaks it."""
    p0 = W.annulus(12, 8, 14)
    w = ratio ** np.arange(p0.nz)
    zf = p0.z0 + (p0.z1 - p0.z0) * np.r_[0.0, np.cumsum(w)] / w.sum()
    p0 = p0.with_z_faces(zf)
    zc = p0.z_centres()
    bias = 300.0 * (1.0 - (zc - p0.z0) / (p0.z1 - p0.z0))
    p = p0.with_r_wall_data(bias, bias)
    g = oracle.grid_from_problem(p)
    phi_exact = np.broadcast_to(bias[:, None, None], p.shape)
    rho = np.zeros(p.shape)
    assert oracle.relres(g, rho, phi_exact) < 1e-14
    phi, info = oracle.solve3d(g, rho, tol=1e-15)
    np.testing.assert_allclose(phi, phi_exact, rtol=1e-12, atol=1e-10)
    # the same field on a uniform mesh's centres is not a solution here
    zu = p0.z0 + (np.arange(p0.nz) + 0.5) * (p0.z1 - p0.z0) / p0.nz
    wrong = np.broadcast_to((300.0 * (1.0 - (zu - p0.z0) / (p0.z1 - p0.z0)))[:, None, None], p.shape)
    assert oracle.relres(g, rho, wrong) > 1e-3


def test_c0_discrete_manufactured():
    """C0: rho from the discrete operator reproduces the sampled potential."""
    p = W.c0_problem()
    g = oracle.grid_from_problem(p)
    phi_ex = W.c0_phi_exact(p)
    bD = oracle.rhs3d(g, np.zeros(p.shape))
    s = oracle.rhs3d(g.homogeneous(), np.ones(p.shape))
    rho = (oracle.apply3d(g, phi_ex) - bD) / s
    phi, info = oracle.solve3d(g, rho, tol=1e-15)
    err = np.linalg.norm(phi - phi_ex) / np.linalg.norm(phi_ex)
    assert err < 1e-12, (err, info)


def analytic_case(n_r, n_t, n_z):
    p0 = W.annulus(n_r, n_t, n_z)
    r = p0.r_centres()
    z = p0.z_centres()
    th = p0.theta_centres()
    L = p0.z1 - p0.z0
    a = math.pi / (p0.r_out - p0.r_in)
    bz = math.pi / L
    S = np.sin(a * (r - p0.r_in))
    dS = a * np.cos(a * (r - p0.r_in))
    Z = np.sin(bz * (z - p0.z0))
    T = 1.0 + 0.3 * np.cos(2 * th)
    bias = 300.0 * (1.0 - (z - p0.z0) / L)
    phi = Z[:, None, None] * T[None, :, None] * S[None, None, :] + bias[:, None, None]
    # Laplacian in cylindrical coordinates, Eq. cylindrical_poisson; bias is harmonic
    lap = (Z[:, None, None] * T[None, :, None] * ((-a * a * S + dS / r) - bz * bz * S)[None, None, :]
           + Z[:, None, None] * (-1.2 * np.cos(2 * th))[None, :, None] * (S / r ** 2)[None, None, :])
    rho = -p0.eps0 * lap
    p = p0.with_r_wall_data(bias, bias)
    return p, rho, phi


def test_second_order_convergence():
    errs2, errsinf = [], []
    for n in (16, 32, 64):
        p, rho, phi_ex = analytic_case(n, n, n)
        g = oracle.grid_from_problem(p)
        phi, info = oracle.solve3d(g, rho, tol=1e-14)
        d = phi - phi_ex
        errs2.append(np.sqrt(np.mean(d ** 2)))
        errsinf.append(np.abs(d).max())
    o2 = [math.log2(errs2[i] / errs2[i + 1]) for i in range(2)]
    oi = [math.log2(errsinf[i] / errsinf[i + 1]) for i in range(2)]
    assert min(o2) > 1.9, (errs2, o2)
    assert min(oi) > 1.9, (errsinf, oi)
