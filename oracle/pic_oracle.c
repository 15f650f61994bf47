/*
 * FP64 CPU oracle for the cylindrical electrostatic field solve.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or constant generator with the CUDA library; it applies the
 * three-dimensional seven-point finite-volume operator directly, with no
 * Fourier transform, and solves it by plain conjugate gradient.
 *
 * Grid conventions (all arrays row-major, r fastest):
 *   cell (i, j, k): i in [0,nr) radial, j in [0,ntheta) azimuthal (periodic),
 *   k in [0,nz) axial; linear index (k*ntheta + j)*nr + i.
 *   r_faces[0..nr], z_faces[0..nz] are the cell faces; cell centres are face
 *   midpoints (cell geometry, appendix "Cell integration and face fluxes").
 *
 * Operator, written cell by cell (Sec. 3.1 angular difference; appendix
 * Eqs. interior_face_conductances, dirichlet_face_conductances,
 * integrated_mode_shift, integrated_charge_rhs, boundary_rhs_appendix):
 *   (A phi)_ijk = sum over interior r/z faces  G_f (phi_ijk - phi_nbr)
 *              + sum over Dirichlet r/z faces G^D_f phi_ijk
 *              + mu_ik (2 phi_ijk - phi_i,j+1,k - phi_i,j-1,k) / dalpha^2
 *   b_ijk       = s_ik rho_ijk + sum over Dirichlet faces G^D_f phi^D_f
 * with mu = dr dz / r, s = r dr dz / eps0, dalpha = L_alpha / ntheta.
 * The r-z part is the finite-volume integral of the "times r" mode equation
 * (Eq. mode_poisson) over the cell; the angular part is the seven-point
 * second difference of Sec. 3.1 multiplied by the same cell factor mu.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int nr, ntheta, nz;
    const double *r_faces;  /* nr+1 radial faces, r_faces[0] > 0 */
    const double *z_faces;  /* nz+1 axial faces */
    double L_alpha;         /* azimuthal period */
    double eps0;            /* vacuum permittivity */
    const double *phi_rin;  /* nz values: Dirichlet potential on the inner r wall, per axial cell */
    const double *phi_rout; /* nz values: outer r wall */
    const double *phi_z0;   /* nr values: lower z wall, per radial cell */
    const double *phi_z1;   /* nr values: upper z wall */
    const unsigned char *active; /* nz*nr cell flags (k-major), or NULL: every cell active.  The active
                                    cells are the composite domain's union of patches (Sec. 2.2) */
    double phi_exposed;     /* Dirichlet potential of an exposed face: a face between an active and an
                               inactive cell */
} oracle_grid;

typedef struct {
    int iterations;
    int converged;          /* 1 if the recursive residual reached tol */
    double relres_recursive;
    double relres_true;     /* ||b - A phi|| / ||b|| recomputed from phi */
    double bnorm;
} oracle_cg_info;

static int g_threads = 0;

void oracle_set_threads(int n) { g_threads = n; }

int oracle_get_threads(void) {
#ifdef _OPENMP
    return g_threads > 0 ? g_threads : omp_get_max_threads();
#else
    return 1;
#endif
}

static int nthreads(void) { return oracle_get_threads(); }

static double rc(const oracle_grid *g, int i) { return 0.5 * (g->r_faces[i] + g->r_faces[i + 1]); }
static double zc(const oracle_grid *g, int k) { return 0.5 * (g->z_faces[k] + g->z_faces[k + 1]); }
static double drw(const oracle_grid *g, int i) { return g->r_faces[i + 1] - g->r_faces[i]; }
static double dzw(const oracle_grid *g, int k) { return g->z_faces[k + 1] - g->z_faces[k]; }
static int act(const oracle_grid *g, int i, int k) { return !g->active || g->active[(size_t)k * g->nr + i]; }

/*
 * Coefficients of cell (i,k), appendix Eqs. interior_face_conductances and
 * dirichlet_face_conductances: a face between two active cells uses the
 * centre-to-centre distance; a face on the domain wall, or between an active
 * and an inactive cell (an exposed patch face, Sec. 2.2), is a Dirichlet face
 * and uses the centre-to-face distance.  An inactive cell has all-zero
 * coefficients (it is not an unknown of the system).
 * out[0..3] = conductance of the W (r-), E (r+), S (z-), N (z+) face
 * out[4..7] = 1 if that face is a Dirichlet face, else 0
 * out[8] = mu (Eq. mode_mass_coefficient), out[9] = s (Eq. mode_rhs),
 * out[10] = D0, the sum of the four face conductances (Eq. base_diagonal_with_boundary)
 */
void oracle_cell_coeffs(const oracle_grid *g, int i, int k, double *out) {
    const double r = rc(g, i), z = zc(g, k), dr = drw(g, i), dz = dzw(g, k);
    const double rm = g->r_faces[i], rp = g->r_faces[i + 1];
    double gw, ge, gs, gn;
    int dw = 0, de = 0, ds = 0, dn = 0;
    if (!act(g, i, k)) {
        for (int a = 0; a < 11; ++a) out[a] = 0.0;
        return;
    }
    if (i > 0 && act(g, i - 1, k)) gw = rm * dz / (r - rc(g, i - 1));
    else { gw = rm * dz / (r - rm); dw = 1; }
    if (i < g->nr - 1 && act(g, i + 1, k)) ge = rp * dz / (rc(g, i + 1) - r);
    else { ge = rp * dz / (rp - r); de = 1; }
    if (k > 0 && act(g, i, k - 1)) gs = r * dr / (z - zc(g, k - 1));
    else { gs = r * dr / (z - g->z_faces[k]); ds = 1; }
    if (k < g->nz - 1 && act(g, i, k + 1)) gn = r * dr / (zc(g, k + 1) - z);
    else { gn = r * dr / (g->z_faces[k + 1] - z); dn = 1; }
    out[0] = gw; out[1] = ge; out[2] = gs; out[3] = gn;
    out[4] = dw; out[5] = de; out[6] = ds; out[7] = dn;
    out[8] = dr * dz / r;
    out[9] = r * dr * dz / g->eps0;
    out[10] = gw + ge + gs + gn;
}

/* out = A phi (homogeneous: the Dirichlet values themselves enter only b).
   An inactive cell's row is the identity (its value is held at zero by b = 0). */
void oracle_apply(const oracle_grid *g, const double *phi, double *out) {
    const int nr = g->nr, nt = g->ntheta, nz = g->nz;
    const double da = g->L_alpha / nt;
    const double inv_da2 = 1.0 / (da * da);
#pragma omp parallel for schedule(static) num_threads(nthreads())
    for (int k = 0; k < nz; ++k) {
        double c[11];
        for (int i = 0; i < nr; ++i) {
            oracle_cell_coeffs(g, i, k, c);
            if (!act(g, i, k)) {
                for (int j = 0; j < nt; ++j) out[((size_t)k * nt + j) * nr + i] = phi[((size_t)k * nt + j) * nr + i];
                continue;
            }
            for (int j = 0; j < nt; ++j) {
                const int jp = (j + 1) % nt, jm = (j + nt - 1) % nt;
                const size_t q = ((size_t)k * nt + j) * nr + i;
                const double p = phi[q];
                double acc = 0.0;
                /* W and E faces */
                if (c[4] != 0.0) acc += c[0] * p;
                else acc += c[0] * (p - phi[q - 1]);
                if (c[5] != 0.0) acc += c[1] * p;
                else acc += c[1] * (p - phi[q + 1]);
                /* S and N faces: neighbours one axial plane away */
                if (c[6] != 0.0) acc += c[2] * p;
                else acc += c[2] * (p - phi[q - (size_t)nt * nr]);
                if (c[7] != 0.0) acc += c[3] * p;
                else acc += c[3] * (p - phi[q + (size_t)nt * nr]);
                /* periodic angular second difference times mu */
                const double pj = phi[((size_t)k * nt + jp) * nr + i];
                const double mj = phi[((size_t)k * nt + jm) * nr + i];
                acc += c[8] * (2.0 * p - pj - mj) * inv_da2;
                out[q] = acc;
            }
        }
    }
}

/* b = s rho + sum over Dirichlet faces of G^D phi^D (appendix Eq. full_finite_volume_row);
   a face on the bounding wall takes that wall's potential, an exposed patch face
   phi_exposed; an inactive cell has b = 0. */
void oracle_rhs(const oracle_grid *g, const double *rho, double *b) {
    const int nr = g->nr, nt = g->ntheta, nz = g->nz;
#pragma omp parallel for schedule(static) num_threads(nthreads())
    for (int k = 0; k < nz; ++k) {
        double c[11];
        for (int i = 0; i < nr; ++i) {
            oracle_cell_coeffs(g, i, k, c);
            double bd = 0.0;
            if (c[4] != 0.0) bd += c[0] * (i == 0 ? g->phi_rin[k] : g->phi_exposed);
            if (c[5] != 0.0) bd += c[1] * (i == nr - 1 ? g->phi_rout[k] : g->phi_exposed);
            if (c[6] != 0.0) bd += c[2] * (k == 0 ? g->phi_z0[i] : g->phi_exposed);
            if (c[7] != 0.0) bd += c[3] * (k == nz - 1 ? g->phi_z1[i] : g->phi_exposed);
            for (int j = 0; j < nt; ++j) {
                const size_t q = ((size_t)k * nt + j) * nr + i;
                b[q] = c[9] * rho[q] + bd;
            }
        }
    }
}

static double dot(const double *a, const double *b, size_t n) {
    double s = 0.0;
#pragma omp parallel for reduction(+ : s) schedule(static) num_threads(nthreads())
    for (long long q = 0; q < (long long)n; ++q) s += a[q] * b[q];
    return s;
}

/* ||b - A phi||_2 and ||b||_2 for the system defined by rho and the wall data. */
void oracle_residual(const oracle_grid *g, const double *rho, const double *phi, double *rnorm, double *bnorm) {
    const size_t n = (size_t)g->nr * g->ntheta * g->nz;
    double *b = (double *)malloc(n * sizeof(double));
    double *ap = (double *)malloc(n * sizeof(double));
    oracle_rhs(g, rho, b);
    oracle_apply(g, phi, ap);
    double rr = 0.0, bb = 0.0;
#pragma omp parallel for reduction(+ : rr, bb) schedule(static) num_threads(nthreads())
    for (long long q = 0; q < (long long)n; ++q) {
        const double d = b[q] - ap[q];
        rr += d * d;
        bb += b[q] * b[q];
    }
    *rnorm = sqrt(rr);
    *bnorm = sqrt(bb);
    free(b);
    free(ap);
}

/*
 * Plain conjugate gradient on A phi = b (A is symmetric positive definite:
 * conductances are shared by the two cells of a face, the angular coupling is
 * symmetric, and every connected r-z plane touches a Dirichlet wall).
 * phi holds the initial guess on entry and the iterate on exit.  Stops when
 * the recursive relative residual falls to tol, after maxit iterations, or
 * when the recursive residual has not reached a new minimum for `stall`
 * iterations (stall <= 0 disables that test).
 */
int oracle_cg(const oracle_grid *g, const double *rho, double *phi, double tol, int maxit, int stall,
              oracle_cg_info *info) {
    const size_t n = (size_t)g->nr * g->ntheta * g->nz;
    double *b = (double *)malloc(n * sizeof(double));
    double *r = (double *)malloc(n * sizeof(double));
    double *p = (double *)malloc(n * sizeof(double));
    double *ap = (double *)malloc(n * sizeof(double));
    if (!b || !r || !p || !ap) {
        free(b); free(r); free(p); free(ap);
        return 2;
    }
    oracle_rhs(g, rho, b);
    oracle_apply(g, phi, ap);
#pragma omp parallel for schedule(static) num_threads(nthreads())
    for (long long q = 0; q < (long long)n; ++q) {
        r[q] = b[q] - ap[q];
        p[q] = r[q];
    }
    const double bnorm = sqrt(dot(b, b, n));
    double rr = dot(r, r, n);
    double best = rr;
    int since_best = 0, it = 0, converged = 0;
    const double stop = (tol * bnorm) * (tol * bnorm);
    if (bnorm == 0.0 || rr <= stop) converged = 1;
    while (!converged && it < maxit) {
        oracle_apply(g, p, ap);
        const double pap = dot(p, ap, n);
        if (!(pap > 0.0)) break;
        const double alpha = rr / pap;
        double rr_new = 0.0;
#pragma omp parallel for reduction(+ : rr_new) schedule(static) num_threads(nthreads())
        for (long long q = 0; q < (long long)n; ++q) {
            phi[q] += alpha * p[q];
            r[q] -= alpha * ap[q];
            rr_new += r[q] * r[q];
        }
        ++it;
        if (rr_new <= stop) { rr = rr_new; converged = 1; break; }
        if (rr_new < best) { best = rr_new; since_best = 0; }
        else if (stall > 0 && ++since_best >= stall) { rr = rr_new; break; }
        const double beta = rr_new / rr;
        rr = rr_new;
#pragma omp parallel for schedule(static) num_threads(nthreads())
        for (long long q = 0; q < (long long)n; ++q) p[q] = r[q] + beta * p[q];
    }
    double rn, bn;
    oracle_residual(g, rho, phi, &rn, &bn);
    if (info) {
        info->iterations = it;
        info->converged = converged;
        info->relres_recursive = bnorm > 0.0 ? sqrt(rr) / bnorm : 0.0;
        info->relres_true = bn > 0.0 ? rn / bn : rn;
        info->bnorm = bn;
    }
    free(b); free(r); free(p); free(ap);
    return 0;
}

/*
 * Time `iters` conjugate-gradient iterations at full size without any stop
 * test (the cost of one iteration does not depend on the data).  Used only to
 * time the oracle on a bounded sample of a large workload.
 */
int oracle_cg_fixed(const oracle_grid *g, const double *rho, double *phi, int iters, double *relres_out) {
    oracle_cg_info info;
    memset(&info, 0, sizeof info);
    int rc_ = oracle_cg(g, rho, phi, 0.0, iters, 0, &info);
    if (relres_out) *relres_out = info.relres_recursive;
    return rc_;
}
