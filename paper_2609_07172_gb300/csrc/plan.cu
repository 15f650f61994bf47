// Plan construction: descriptor validation, multigrid hierarchy, per-level
// coefficient tables (step a-2), coarsest-level factors, device workspace and
// the launch tables that let one kernel launch serve a batch of problems.
#include <algorithm>
#include <cstddef>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>

#include <type_traits>

#include "plan.h"
#include "symeig.h"

namespace pp {

static thread_local char g_err[512];

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
}
void clear_error() { g_err[0] = 0; }
const char *last_error_text() { return g_err; }

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr double kEps0 = 8.8541878128e-12;   // F/m, CODATA 2018
constexpr int kMaxNtheta = 256;
constexpr int kMaxCoarseCells = 4096;
constexpr int kMaxCoarseNz = 64;
constexpr unsigned kKnownFlags =
    PIC_POISSON_USE_INITIAL_GUESS | PIC_POISSON_PROFILE | PIC_POISSON_GRAPH | PIC_POISSON_HOST_STAGED;

int resolve(const pic_poisson_desc *in, pic_poisson_desc *d) {
    if (!in) {
        set_error("desc is NULL");
        return PIC_POISSON_EINVAL;
    }
    *d = *in;
    // face arrays, where given, replace r_in / r_out or z0 / z1 (checked below)
    if (!std::isfinite(d->theta_span) || (!d->r_faces && !(std::isfinite(d->r_in) && std::isfinite(d->r_out))) ||
        (!d->z_faces && !(std::isfinite(d->z0) && std::isfinite(d->z1)))) {
        set_error("r_in, r_out, z0, z1 and theta_span must be finite (theta_span <= 0 selects 2 pi)");
        return PIC_POISSON_EINVAL;
    }
    if (d->theta_span <= 0) d->theta_span = 2.0 * kPi;
    if (d->eps0 <= 0) d->eps0 = kEps0;
    if (d->max_cycles <= 0) d->max_cycles = 200;
    if (d->pre_sweeps < 0) d->pre_sweeps = 2;
    if (d->post_sweeps < 0) d->post_sweeps = 2;
    if (d->inner_cycles <= 0) d->inner_cycles = 2;
    if (d->inner_first <= d->inner_cycles || d->precision != PIC_POISSON_MIXED) d->inner_first = d->inner_cycles;
    if (d->smooth_threads <= 0) d->smooth_threads = MG_THREADS;
    if (d->smooth_strip < 0) d->smooth_strip = 0;
    if (d->omega <= 0) d->omega = 1.0;
    if (d->smooth_fused < 0) d->smooth_fused = 0;
    if (d->fmg != 0 && (d->fmg != 1 || d->precision != PIC_POISSON_FP64)) {
        set_error("fmg must be 0, or 1 with precision PIC_POISSON_FP64 (got %d)", d->fmg);
        return PIC_POISSON_EINVAL;
    }
    if (d->local_bottom != 0 && d->local_bottom != -1) {
        set_error("local_bottom must be 0 or -1 (got %d)", d->local_bottom);
        return PIC_POISSON_EINVAL;
    }
    if (d->smooth_fused > 1) {
        set_error("smooth_fused must be 0 or 1 (got %d)", d->smooth_fused);
        return PIC_POISSON_EINVAL;
    }
    if (!(d->omega < 2.0)) {
        set_error("omega must be in (0, 2) (got %g)", d->omega);
        return PIC_POISSON_EINVAL;
    }
    if (d->smooth_strip != 0 && d->smooth_strip != 1 && d->smooth_strip != 2 && d->smooth_strip != 4) {
        set_error("smooth_strip must be <= 0, 1, 2 or 4 (got %d)", d->smooth_strip);
        return PIC_POISSON_EINVAL;
    }
    if (d->smooth_threads != 64 && d->smooth_threads != 128 && d->smooth_threads != 256 && d->smooth_threads != 512) {
        set_error("smooth_threads must be 64, 128, 256 or 512 (got %d)", d->smooth_threads);
        return PIC_POISSON_EINVAL;
    }
    if (d->nr < 1 || d->nz < 1) {
        set_error("nr and nz must be >= 1 (got %d, %d)", d->nr, d->nz);
        return PIC_POISSON_EINVAL;
    }
    if (d->ntheta < 2 || d->ntheta > kMaxNtheta || (d->ntheta & (d->ntheta - 1))) {
        set_error("ntheta must be a power of two in [2, %d] (got %d)", kMaxNtheta, d->ntheta);
        return PIC_POISSON_EINVAL;
    }
    if (d->r_faces && d->nr >= 1) {   // given faces define the radial walls
        for (int a = 0; a <= d->nr; ++a)
            if (!std::isfinite(d->r_faces[a]) || (a > 0 && !(d->r_faces[a] > d->r_faces[a - 1]))) {
                set_error("r_faces must be nr + 1 finite, strictly increasing values");
                return PIC_POISSON_EINVAL;
            }
        d->r_in = d->r_faces[0];
        d->r_out = d->r_faces[d->nr];
    }
    if (d->z_faces && d->nz >= 1) {   // given faces define the axial walls
        for (int a = 0; a <= d->nz; ++a)
            if (!std::isfinite(d->z_faces[a]) || (a > 0 && !(d->z_faces[a] > d->z_faces[a - 1]))) {
                set_error("z_faces must be nz + 1 finite, strictly increasing values");
                return PIC_POISSON_EINVAL;
            }
        d->z0 = d->z_faces[0];
        d->z1 = d->z_faces[d->nz];
    }
    if (!(d->r_in > 0) || !(d->r_out > d->r_in) || !(d->z1 > d->z0) || !std::isfinite(d->r_out) ||
        !std::isfinite(d->z0) || !std::isfinite(d->z1)) {
        set_error("need 0 < r_in < r_out and z0 < z1 (finite)");
        return PIC_POISSON_EINVAL;
    }
    if (d->precision != PIC_POISSON_FP64 && d->precision != PIC_POISSON_MIXED) {
        set_error("precision must be PIC_POISSON_FP64 or PIC_POISSON_MIXED");
        return PIC_POISSON_EINVAL;
    }
    if (d->pre_sweeps + d->post_sweeps == 0 || d->pre_sweeps > 64 || d->post_sweeps > 64 || d->inner_cycles > 64 ||
        d->inner_first > 64) {
        set_error("need 0 < pre_sweeps + post_sweeps, sweeps <= 64, inner_cycles and inner_first <= 64");
        return PIC_POISSON_EINVAL;
    }
    if (d->flags & ~kKnownFlags) {
        set_error("unknown flag bits 0x%x", d->flags & ~kKnownFlags);
        return PIC_POISSON_EINVAL;
    }
    if (d->n_patches < 0 || d->n_patches > PIC_POISSON_MAX_PATCHES || (d->n_patches > 0 && !d->patches)) {
        set_error("n_patches must be in [0, %d] with a patches array", PIC_POISSON_MAX_PATCHES);
        return PIC_POISSON_EINVAL;
    }
    for (int a = 0; a < d->n_patches; ++a) {
        const int *x = d->patches + 4 * a;
        if (!(0 <= x[0] && x[0] < x[1] && x[1] <= d->nr && 0 <= x[2] && x[2] < x[3] && x[3] <= d->nz)) {
            set_error("patch %d (%d, %d, %d, %d) must be non-empty and inside the %d x %d grid", a, x[0], x[1],
                      x[2], x[3], d->nr, d->nz);
            return PIC_POISSON_EINVAL;
        }
        for (int b2 = 0; b2 < a; ++b2) {
            const int *y = d->patches + 4 * b2;
            if (x[0] < y[1] && y[0] < x[1] && x[2] < y[3] && y[2] < x[3]) {
                set_error("patches %d and %d overlap", b2, a);
                return PIC_POISSON_EINVAL;
            }
        }
    }
    if (d->n_patches > 0 && !std::isfinite(d->phi_exposed)) {
        set_error("a composite domain needs a finite phi_exposed");
        return PIC_POISSON_EINVAL;
    }
    if (d->z_faces && d->smooth_fused) {
        set_error("a non-uniform axial mesh needs smooth_fused = 0");
        return PIC_POISSON_EINVAL;
    }
    if (d->n_patches == 0) d->patches = nullptr;
    const double n = (double)d->nr * d->nz * (d->ntheta / 2 + 1);
    if (n > 2.0e9) {
        set_error("too many mode entries (nr*nz*(ntheta/2+1) = %.0f > 2e9)", n);
        return PIC_POISSON_EINVAL;
    }
    return PIC_POISSON_OK;
}

// Coarsening that keeps coarse cells near-isotropic (the point smoother only
// smooths well when neither direction's coupling dominates: G_z / G_r =
// (dr / dz)^2).  From a level with cell aspect dr / dz: above sqrt(2) halve
// only N_z, below 1/sqrt(2) halve only N_r, otherwise halve both; a halved
// count must be even and at least 8, and the level being coarsened needs an
// even N_r (it is smoothed red-black).  Stop when the preferred step is not
// possible; the coarsest level is solved directly.  A composite domain's
// patch boundaries are protected faces (Sec. 3.2): a direction is halved only
// while every patch boundary in it lies on a face of the coarser level, so no
// coarse cell straddles a patch edge.
int hierarchy(const pic_poisson_desc &d, int *nr, int *nz, int *levels) {
    int L = 1, r = d.nr, z = d.nz;
    nr[0] = r;
    nz[0] = z;
    const double Lr = d.r_out - d.r_in, Lz = d.z1 - d.z0, s2 = std::sqrt(2.0);
    int sr = 1, sz = 1;   // level-0 cells per cell of the current level
    auto aligned = [&](int axis, int scale) {
        for (int a = 0; a < d.n_patches; ++a) {
            const int *x = d.patches + 4 * a + 2 * axis;
            if (x[0] % scale || x[1] % scale) return false;
        }
        return true;
    };
    while (L < PIC_POISSON_MAX_LEVELS && r % 2 == 0) {
        const double aspect = (Lr / r) / (Lz / z);
        const bool can_r = r >= 8 && aligned(0, 2 * sr), can_z = z % 2 == 0 && z >= 8 && aligned(1, 2 * sz);
        int r2 = r, z2 = z;
        if (aspect > s2) {
            if (!can_z) break;
            z2 = z / 2;
        } else if (aspect < 1.0 / s2) {
            if (!can_r) break;
            r2 = r / 2;
        } else {
            if (!(can_r && can_z)) break;
            r2 = r / 2;
            z2 = z / 2;
        }
        if (r2 != r) sr *= 2;
        if (z2 != z) sz *= 2;
        r = r2;
        z = z2;
        nr[L] = r;
        nz[L] = z;
        ++L;
    }
    *levels = L;
    if (d.n_patches > 0 || d.z_faces) {   // dense coarsest solve over the active cells
        long act = d.n_patches > 0 ? 0 : (long)r * z;
        for (int a = 0; a < d.n_patches; ++a) {
            const int *x = d.patches + 4 * a;
            act += (long)((x[1] - x[0]) / sr) * ((x[3] - x[2]) / sz);
        }
        if (act > PIC_POISSON_MAX_DENSE) {
            set_error("the coarsest level %d x %d of this composite domain or non-uniform axial mesh has %ld "
                      "active cells (> %d): use counts and patch boundaries with more factors of two",
                      r, z, act, PIC_POISSON_MAX_DENSE);
            return PIC_POISSON_EINVAL;
        }
        return PIC_POISSON_OK;
    }
    if (z > kMaxCoarseNz || (long)r * z > kMaxCoarseCells) {
        set_error("coarsest level %d x %d (r x z) exceeds the direct-solve limit (nz <= %d, cells <= %d); "
                  "use cell counts with more factors of two",
                  r, z, kMaxCoarseNz, kMaxCoarseCells);
        return PIC_POISSON_EINVAL;
    }
    return PIC_POISSON_OK;
}

double wall_rin(const pic_poisson_desc &d, int k) { return d.phi_r_in_z ? d.phi_r_in_z[k] : d.phi_r_in; }
double wall_rout(const pic_poisson_desc &d, int k) { return d.phi_r_out_z ? d.phi_r_out_z[k] : d.phi_r_out; }

// Exact discrete azimuthal eigenvalue, Eq. discrete_azimuthal_eigenvalue.
double lambda_m(const pic_poisson_desc &d, int m) {
    const double da = d.theta_span / d.ntheta;
    const double s = std::sin(kPi * m / d.ntheta);
    return 4.0 / (da * da) * s * s;
}

// Coefficients of one uniform level (appendix Eqs. interior_face_conductances,
// dirichlet_face_conductances, mode_mass_coefficient), rediscretised on the
// level's own cells.
// Uniform radial faces r_in + (r_out - r_in) a / nr.
std::vector<double> uniform_faces(const pic_poisson_desc &d, int nr) {
    std::vector<double> f(nr + 1);
    for (int a = 0; a <= nr; ++a) f[a] = d.r_in + (d.r_out - d.r_in) * a / nr;
    return f;
}

// Coefficients of one level on radial faces rf (appendix Eqs.
// interior_face_conductances, dirichlet_face_conductances,
// mode_mass_coefficient): a radial face between two cells uses the
// centre-to-centre distance, a wall face the centre-to-wall distance; cell
// centres are face midpoints.
void build_level(const pic_poisson_desc &d, const std::vector<double> &rf, int nz, int nm, LevelHost &h) {
    const int nr = (int)rf.size() - 1;
    h.nr = nr;
    h.nz = nz;
    h.rf = rf;
    h.dr = (rf[nr] - rf[0]) / nr;
    h.dz = (d.z1 - d.z0) / nz;
    const double dz = h.dz;
    h.rc.assign(nr, 0.0);
    h.drc.assign(nr, 0.0);
    for (int i = 0; i < nr; ++i) {
        h.rc[i] = 0.5 * (rf[i] + rf[i + 1]);
        h.drc[i] = rf[i + 1] - rf[i];
    }
    h.cw.assign(nr, 0.0);
    h.ce.assign(nr, 0.0);
    h.cz.assign(nr, 0.0);
    h.d0r.assign(nr, 0.0);
    h.mu.assign(nr, 0.0);
    for (int i = 0; i < nr; ++i) {
        const double rm = rf[i], rp = rf[i + 1], rc = h.rc[i], dr = h.drc[i];
        const double gw = (i > 0) ? rm * dz / (rc - h.rc[i - 1]) : rm * dz / (rc - rm);
        const double ge = (i < nr - 1) ? rp * dz / (h.rc[i + 1] - rc) : rp * dz / (rp - rc);
        h.cw[i] = (i > 0) ? gw : 0.0;
        h.ce[i] = (i < nr - 1) ? ge : 0.0;
        h.d0r[i] = gw + ge;
        h.cz[i] = rc * dr / dz;
        h.mu[i] = dr * dz / rc;
    }
    h.ncls = std::min(nz, 3);
    if (nz == 1) h.tz = {4.0};
    else if (nz == 2) h.tz = {3.0, 3.0};
    else h.tz = {3.0, 2.0, 3.0};
    const size_t nt = (size_t)h.ncls * nr * nm;
    h.diag.assign(nt, 0.0);
    h.invd.assign(nt, 0.0);
    h.hw.assign(nt, 0.0);
    h.he.assign(nt, 0.0);
    h.hz.assign(nt, 0.0);
    for (int c = 0; c < h.ncls; ++c)
        for (int i = 0; i < nr; ++i)
            for (int m = 0; m < nm; ++m) {
                const size_t t = ((size_t)c * nr + i) * nm + m;
                const double dg = h.d0r[i] + h.tz[c] * h.cz[i] + lambda_m(d, m) * h.mu[i];
                // smoother tables carry the over-relaxation factor: with
                // omega b / diag and omega G / diag the update is
                // u <- (1 - omega) u + (omega b_hat + sum omega h u)
                const double w = d.omega > 0 ? d.omega : 1.0;
                h.diag[t] = dg;
                h.invd[t] = w / dg;
                h.hw[t] = w * h.cw[i] / dg;
                h.he[t] = w * h.ce[i] / dg;
                h.hz[t] = w * h.cz[i] / dg;
            }
}

// Face conductances of active cell (i, k) of level h (appendix Eqs.
// interior_face_conductances, dirichlet_face_conductances): g[0..3] of the W,
// E, S, N faces and dir[0..3] = 1 for a Dirichlet face -- a wall face or, in a
// composite domain, an exposed face (the neighbour is inactive), both at the
// centre-to-face distance.
void cell_faces(const LevelHost &h, int i, int k, double *g, int *dir) {
    auto on = [&](int ii, int kk) { return h.act.empty() || h.act[(size_t)kk * h.nr + ii] != 0; };
    const double rm = h.rf[i], rp = h.rf[i + 1], rc = h.rc[i];
    dir[0] = !(i > 0 && on(i - 1, k));
    dir[1] = !(i < h.nr - 1 && on(i + 1, k));
    dir[2] = !(k > 0 && on(i, k - 1));
    dir[3] = !(k < h.nz - 1 && on(i, k + 1));
    if (h.zc.empty()) {   // uniform axial spacing
        g[0] = dir[0] ? rm * h.dz / (rc - rm) : h.cw[i];
        g[1] = dir[1] ? rp * h.dz / (rp - rc) : h.ce[i];
        g[2] = dir[2] ? 2.0 * h.cz[i] : h.cz[i];
        g[3] = dir[3] ? 2.0 * h.cz[i] : h.cz[i];
        return;
    }
    // non-uniform axial faces: the row's own width and centre distances
    const double dz = h.dzc[k], zc = h.zc[k], ar = rc * h.drc[i];
    g[0] = rm * dz / (dir[0] ? rc - rm : rc - h.rc[i - 1]);
    g[1] = rp * dz / (dir[1] ? rp - rc : h.rc[i + 1] - rc);
    g[2] = ar / (dir[2] ? zc - h.zf[k] : zc - h.zc[k - 1]);
    g[3] = ar / (dir[3] ? h.zf[k + 1] - zc : h.zc[k + 1] - zc);
}

// mu of cell (i, k) (Eq. mode_mass_coefficient) and its s (Eq. mode_rhs) times eps0.
double mu_cell(const LevelHost &h, int i, int k) {
    return h.zc.empty() ? h.mu[i] : h.drc[i] * h.dzc[k] / h.rc[i];
}
double s_eps0_cell(const LevelHost &h, int i, int k) {
    return h.rc[i] * h.drc[i] * (h.zc.empty() ? h.dz : h.dzc[k]);
}

// Per-row level tables (a composite domain or a non-uniform axial mesh):
// rows are grouped into classes by their active pattern and their
// neighbours' (each distinct pattern one class; on a non-uniform axial mesh
// every row is its own class); an inactive cell gets zero diag, invd and h
// entries (the smoother leaves its u = 0 and the residual kernels skip it),
// an active cell the diagonal of its own faces, exposed ones Dirichlet, and
// no coupling across a Dirichlet face.  South and north couplings are kept
// apart (hz and hn; ccs and ccn), as the axial distances may differ.
void build_rowwise_tables(const pic_poisson_desc &d, int nm, LevelHost &h) {
    const int nr = h.nr, nz = h.nz;
    std::map<std::vector<unsigned char>, int> seen;
    std::vector<int> rep;
    h.rcls.assign(nz, 0);
    if (h.act.empty()) h.act.assign((size_t)nr * nz, 1);
    for (int k = 0; k < nz; ++k) {
        if (!h.zc.empty()) {   // every row its own class
            h.rcls[k] = k;
            rep.push_back(k);
            continue;
        }
        std::vector<unsigned char> sig(nr);
        for (int i = 0; i < nr; ++i) {
            const unsigned char a = h.act[(size_t)k * nr + i];
            const unsigned char sb = k > 0 ? h.act[(size_t)(k - 1) * nr + i] : 0;
            const unsigned char nb = k < nz - 1 ? h.act[(size_t)(k + 1) * nr + i] : 0;
            sig[i] = (unsigned char)(a | (sb << 1) | (nb << 2));
        }
        auto it = seen.find(sig);
        if (it == seen.end()) {
            it = seen.emplace(sig, (int)rep.size()).first;
            rep.push_back(k);
        }
        h.rcls[k] = it->second;
    }
    h.ncls = (int)rep.size();
    const size_t nt = (size_t)h.ncls * nr * nm;
    h.diag.assign(nt, 0.0);
    h.invd.assign(nt, 0.0);
    h.hw.assign(nt, 0.0);
    h.he.assign(nt, 0.0);
    h.hz.assign(nt, 0.0);
    h.hn.assign(nt, 0.0);
    h.d0c.assign((size_t)h.ncls * nr, 0.0);
    for (auto *v : {&h.ccw, &h.cce, &h.ccs, &h.ccn}) v->assign((size_t)h.ncls * nr, 0.0);
    const double w = d.omega > 0 ? d.omega : 1.0;
    for (int c = 0; c < h.ncls; ++c) {
        const int k = rep[c];
        for (int i = 0; i < nr; ++i) {
            if (!h.act[(size_t)k * nr + i]) continue;
            double g[4];
            int dir[4];
            cell_faces(h, i, k, g, dir);
            const double d0 = g[0] + g[1] + g[2] + g[3], mu = mu_cell(h, i, k);
            const size_t ci = (size_t)c * nr + i;
            h.d0c[ci] = d0;
            h.ccw[ci] = dir[0] ? 0.0 : g[0];
            h.cce[ci] = dir[1] ? 0.0 : g[1];
            h.ccs[ci] = dir[2] ? 0.0 : g[2];
            h.ccn[ci] = dir[3] ? 0.0 : g[3];
            for (int m = 0; m < nm; ++m) {
                const size_t t = ci * nm + m;
                const double dg = d0 + lambda_m(d, m) * mu;
                h.diag[t] = dg;
                h.invd[t] = w / dg;
                h.hw[t] = w * h.ccw[ci] / dg;
                h.he[t] = w * h.cce[ci] / dg;
                h.hz[t] = w * h.ccs[ci] / dg;
                h.hn[t] = w * h.ccn[ci] / dg;
            }
        }
    }
}

// Level-0 active flags [nz][nr] of a composite domain (empty: no patches).
std::vector<unsigned char> patch_mask(const pic_poisson_desc &d) {
    std::vector<unsigned char> a;
    if (d.n_patches == 0) return a;
    a.assign((size_t)d.nr * d.nz, 0);
    for (int p = 0; p < d.n_patches; ++p) {
        const int *x = d.patches + 4 * p;
        for (int k = x[2]; k < x[3]; ++k)
            for (int i = x[0]; i < x[1]; ++i) a[(size_t)k * d.nr + i] = 1;
    }
    return a;
}

// Dense factors of a composite domain's coarsest level: the symmetric
// A_0 (face conductances, no azimuthal term) over the active cells, scaled
// S = M^(-1/2) A_0 M^(-1/2) with M = diag(mu), and S = Q Lambda Q^T, so
// that A_m^(-1) = M^(-1/2) Q (Lambda + lambda_m)^(-1) Q^T M^(-1/2) for every
// mode from one factorisation.
int dense_factors(const ProblemPlan &q, std::vector<int> &aidx, std::vector<int> &amap, std::vector<double> &Q,
                  std::vector<double> &QT, std::vector<double> &lam, std::vector<double> &isq,
                  std::vector<double> &lamm) {
    const LevelHost &h = q.lv[q.L - 1];
    const int nr = h.nr, nz = h.nz;
    amap.assign((size_t)nr * nz, -1);
    aidx.clear();
    for (int k = 0; k < nz; ++k)
        for (int i = 0; i < nr; ++i)
            if (h.act[(size_t)k * nr + i]) {
                amap[(size_t)k * nr + i] = (int)aidx.size();
                aidx.push_back(k * nr + i);
            }
    const int n = (int)aidx.size();
    isq.assign(n, 0.0);
    for (int a = 0; a < n; ++a) isq[a] = 1.0 / std::sqrt(mu_cell(h, aidx[a] % nr, aidx[a] / nr));
    std::vector<double> S((size_t)n * n, 0.0);
    for (int a = 0; a < n; ++a) {
        const int k = aidx[a] / nr, i = aidx[a] % nr;
        double g[4];
        int dir[4];
        cell_faces(h, i, k, g, dir);
        S[(size_t)a * n + a] = (g[0] + g[1] + g[2] + g[3]) * isq[a] * isq[a];
        const int nb[4] = {dir[0] ? -1 : amap[(size_t)k * nr + i - 1], dir[1] ? -1 : amap[(size_t)k * nr + i + 1],
                           dir[2] ? -1 : amap[(size_t)(k - 1) * nr + i], dir[3] ? -1 : amap[(size_t)(k + 1) * nr + i]};
        for (int f = 0; f < 4; ++f)
            if (nb[f] >= 0) S[(size_t)a * n + nb[f]] = -g[f] * isq[a] * isq[nb[f]];
    }
    if (!sym_eig_cached(S, n, Q, lam)) {
        set_error("the coarsest level's dense eigendecomposition did not converge");
        return PIC_POISSON_EINVAL;
    }
    QT.assign((size_t)n * n, 0.0);
    for (int a = 0; a < n; ++a)
        for (int j = 0; j < n; ++j) QT[(size_t)j * n + a] = Q[(size_t)a * n + j];
    lamm.assign(q.nm, 0.0);
    for (int m = 0; m < q.nm; ++m) lamm[m] = lambda_m(q.d, m);
    return PIC_POISSON_OK;
}

// Coarsest-level factors: axial eigenbasis (closed form for the uniform
// cell-centred Dirichlet operator: V_kj ~ sin(pi (j+1)(k+1/2)/nz), eigenvalue
// 4 sin^2(pi (j+1) / (2 nz))) and the Thomas factorisation of the radial
// tridiagonal system of every (mode, axial eigenvector).
void coarse_factors(const ProblemPlan &pp_, std::vector<double> &V, std::vector<double> &e, std::vector<double> &piv,
                    std::vector<double> &cpr) {
    const LevelHost &h = pp_.lv[pp_.L - 1];
    const int nr = h.nr, nz = h.nz, nm = pp_.nm;
    V.assign((size_t)nz * nz, 0.0);
    std::vector<double> lam_z(nz);
    for (int j = 0; j < nz; ++j) {
        const int p = j + 1;
        const double nrm = (p < nz) ? std::sqrt(2.0 / nz) : std::sqrt(1.0 / nz);
        for (int k = 0; k < nz; ++k) V[(size_t)k * nz + j] = nrm * std::sin(kPi * p * (k + 0.5) / nz);
        const double s = std::sin(kPi * p / (2.0 * nz));
        lam_z[j] = 4.0 * s * s;
    }
    e.assign(nr, 0.0);
    for (int i = 0; i + 1 < nr; ++i) e[i] = -h.ce[i];
    piv.assign((size_t)nm * nz * nr, 0.0);
    cpr.assign((size_t)nm * nz * nr, 0.0);
    for (int m = 0; m < nm; ++m) {
        const double lm = lambda_m(pp_.d, m);
        for (int j = 0; j < nz; ++j) {
            double *pv = &piv[((size_t)m * nz + j) * nr];
            double *cp = &cpr[((size_t)m * nz + j) * nr];
            double prev_c = 0.0;
            for (int i = 0; i < nr; ++i) {
                const double di = h.d0r[i] + lm * h.mu[i] + lam_z[j] * h.cz[i];
                const double den = di - (i > 0 ? e[i - 1] * prev_c : 0.0);
                pv[i] = 1.0 / den;
                cp[i] = (i + 1 < nr) ? e[i] * pv[i] : 0.0;
                prev_c = cp[i];
            }
        }
    }
}

// Bump allocator over one device allocation (sizing pass when base == nullptr).
struct Carver {
    char *base = nullptr;
    size_t off = 0;
    template <class T> T *take(size_t count) {
        off = (off + 255) & ~(size_t)255;
        T *p = base ? (T *)(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

// Device address of the convergence loop's per-problem stop flags, for the
// kernels' early exit; null for a single problem, whose loop simply ends.
const int *ctrl_done(const pic_poisson_plan_s &P) {
    if (P.n < 2) return nullptr;
    return reinterpret_cast<const int *>(reinterpret_cast<const char *>(P.ctrl) + offsetof(Ctrl, done));
}

// Axial faces of level l: the given ones, or uniform ones from z0, z1.
std::vector<double> level_zfaces(const ProblemPlan &q, int l) {
    const LevelHost &h = q.lv[l];
    if (!h.zf.empty()) return h.zf;
    std::vector<double> f(h.nz + 1);
    for (int a = 0; a <= h.nz; ++a) f[a] = q.d.z0 + (q.d.z1 - q.d.z0) * a / h.nz;
    f[h.nz] = q.d.z1;
    return f;
}

// Bins of a cell lookup over faces f[0..n]: as many as make each bin no wider
// than half the narrowest cell (so a bin meets at most two cells), at least n.
int lookup_bins(const std::vector<double> &f) {
    const int n = (int)f.size() - 1;
    double wmin = INFINITY;
    for (int a = 0; a < n; ++a) wmin = std::min(wmin, f[a + 1] - f[a]);
    const double nb = std::ceil(2.0 * (f[n] - f[0]) / wmin);
    return (int)std::min(std::max(nb, (double)n), 1048576.0);
}

// The cell holding the lower end of each bin: max{a < n : f[a] <= f0 + b w}.
std::vector<int> lookup_table(const std::vector<double> &f, int nb) {
    const int n = (int)f.size() - 1;
    std::vector<int> t(nb);
    int a = 0;
    for (int b = 0; b < nb; ++b) {
        const double x = f[0] + (f[n] - f[0]) * b / nb;
        while (a + 1 < n && f[a + 1] <= x) ++a;
        t[b] = a;
    }
    return t;
}

int setup_problem(ProblemPlan &q, const pic_poisson_desc &d) {
    q.d = d;
    if (d.phi_r_in_z) {
        q.rin_z.assign(d.phi_r_in_z, d.phi_r_in_z + d.nz);
        q.d.phi_r_in_z = q.rin_z.data();
    }
    if (d.phi_r_out_z) {
        q.rout_z.assign(d.phi_r_out_z, d.phi_r_out_z + d.nz);
        q.d.phi_r_out_z = q.rout_z.data();
    }
    q.uniform_r = !d.r_faces;
    q.rf0 = d.r_faces ? std::vector<double>(d.r_faces, d.r_faces + d.nr + 1) : uniform_faces(d, d.nr);
    q.d.r_faces = q.rf0.data();
    q.patches.assign(d.patches, d.patches + 4 * d.n_patches);
    if (d.z_faces) q.zf0.assign(d.z_faces, d.z_faces + d.nz + 1);
    q.d.z_faces = q.zf0.empty() ? nullptr : q.zf0.data();
    q.d.patches = q.patches.empty() ? nullptr : q.patches.data();
    int nr[PIC_POISSON_MAX_LEVELS], nz[PIC_POISSON_MAX_LEVELS];
    int rc = hierarchy(q.d, nr, nz, &q.L);
    if (rc) return rc;
    q.nm = d.ntheta / 2 + 1;
    q.lv.resize(q.L);
    const std::vector<unsigned char> act0 = patch_mask(q.d);
    std::vector<double> rf = q.rf0;   // a level halved in r keeps every other face
    std::vector<double> zf = q.zf0;   // non-uniform axial faces (empty: uniform)
    for (int l = 0; l < q.L; ++l) {
        if (l > 0 && nr[l] != nr[l - 1]) {
            std::vector<double> c(nr[l] + 1);
            for (int a = 0; a <= nr[l]; ++a) c[a] = rf[2 * a];
            rf.swap(c);
        }
        if (l > 0 && nz[l] != nz[l - 1] && !zf.empty()) {   // likewise in z
            std::vector<double> c(nz[l] + 1);
            for (int a = 0; a <= nz[l]; ++a) c[a] = zf[2 * a];
            zf.swap(c);
        }
        LevelHost &h = q.lv[l];
        build_level(q.d, rf, nz[l], q.nm, h);
        if (!zf.empty()) {
            h.zf = zf;
            h.zc.assign(nz[l], 0.0);
            h.dzc.assign(nz[l], 0.0);
            for (int k = 0; k < nz[l]; ++k) {
                h.zc[k] = 0.5 * (zf[k] + zf[k + 1]);
                h.dzc[k] = zf[k + 1] - zf[k];
            }
        }
        if (!act0.empty()) {   // protected faces: each coarse cell lies in one patch or none
            const int sr = d.nr / nr[l], sz = d.nz / nz[l];
            h.act.assign((size_t)nr[l] * nz[l], 0);
            for (int k = 0; k < nz[l]; ++k)
                for (int i = 0; i < nr[l]; ++i) h.act[(size_t)k * nr[l] + i] = act0[(size_t)(k * sz) * d.nr + i * sr];
        }
        if (!act0.empty() || !zf.empty()) build_rowwise_tables(q.d, q.nm, h);
    }
    q.nact = 0;
    if (!act0.empty() || !zf.empty())
        for (unsigned char a : q.lv[q.L - 1].act) q.nact += a;
    return PIC_POISSON_OK;
}

template <class T, class V> void carve_level(const LevelHost &h, int nm, int nt, Carver &c, LevelDev<T> &v) {
    v.nr = h.nr;
    v.nz = h.nz;
    v.nm = nm;
    v.ncls = h.ncls;
    v.rnm = fdiv_rcp((unsigned)nm);
    v.rnr = fdiv_rcp((unsigned)h.nr);
    v.rhr = fdiv_rcp((unsigned)h.nr / 2);
    v.nt = nt;
    v.init = 0;
    const size_t n = (size_t)h.nr * h.nz * nm, ntab = (size_t)h.ncls * h.nr * nm;
    v.u = c.take<V>(n);
    v.b = c.take<V>(n);
    v.bh = c.take<V>(n);
    v.cw = c.take<T>(h.nr);
    v.ce = c.take<T>(h.nr);
    v.cz = c.take<T>(h.nr);
    v.invd = c.take<T>(ntab);
    v.diag = c.take<T>(ntab);
    v.hw = c.take<T>(ntab);
    v.he = c.take<T>(ntab);
    v.hz = c.take<T>(ntab);
    v.rcls = h.rcls.empty() ? nullptr : c.take<int>(h.nz);
    v.holes = std::find(h.act.begin(), h.act.end(), (unsigned char)0) != h.act.end() ? 1 : 0;
    const bool rw = !h.rcls.empty();
    v.hn = rw ? c.take<T>(ntab) : nullptr;
    const size_t nc = (size_t)h.ncls * h.nr;
    v.ccw = rw ? c.take<T>(nc) : nullptr;
    v.cce = rw ? c.take<T>(nc) : nullptr;
    v.ccs = rw ? c.take<T>(nc) : nullptr;
    v.ccn = rw ? c.take<T>(nc) : nullptr;
}

template <class T> void carve_coarse(const ProblemPlan &q, Carver &c, CoarseDev<T> &cd) {
    const LevelHost &h = q.lv[q.L - 1];
    const size_t nf = (size_t)q.nm * h.nz * h.nr;
    cd.nr = h.nr;
    cd.nz = h.nz;
    cd.nm = q.nm;
    cd.nact = q.nact;
    if (q.nact > 0) {   // composite domain: dense solve (coarse_factors' tables are not used)
        const size_t na = (size_t)q.nact;
        cd.V = cd.e = cd.piv = cd.cpr = nullptr;
        cd.aidx = c.take<int>(na);
        cd.amap = c.take<int>((size_t)h.nr * h.nz);
        cd.Q = c.take<float>(na * na);
        cd.QT = c.take<float>(na * na);
        cd.lam = c.take<float>(na);
        cd.isq = c.take<float>(na);
        cd.lamm = c.take<float>(q.nm);
        cd.Y = c.take<float>(na * 2 * q.nm);
        cd.Z = c.take<float>(na * 2 * q.nm);
        cd.up = c.take<double>(2 * (size_t)q.nm);
        return;
    }
    cd.aidx = cd.amap = nullptr;
    cd.Q = cd.QT = cd.lam = cd.isq = cd.lamm = nullptr;
    cd.Y = cd.Z = nullptr;
    cd.up = nullptr;
    cd.V = c.take<T>((size_t)h.nz * h.nz);
    cd.e = c.take<T>(h.nr);
    cd.piv = c.take<T>(nf);
    cd.cpr = c.take<T>(nf);
}

template <class T> void carve_hier(pic_poisson_plan_s &P, Carver &c, Hier<T> &H) {
    const int nl = std::max(P.Lmax - 1, 0);
    H.smooth.assign(nl, nullptr);
    H.restr.assign(nl, nullptr);
    H.prolong.assign(nl, nullptr);
    H.fpre.assign(nl, nullptr);
    H.fpost.assign(nl, nullptr);
    H.rhs.assign(nl, nullptr);
    H.interp.assign(nl, nullptr);
    for (int l = 0; l < nl; ++l) {
        H.smooth[l] = c.take<LaunchTab<T>>(1);
        H.restr[l] = c.take<LaunchTab<T>>(1);
        H.prolong[l] = c.take<LaunchTab<T>>(1);
        if (H.fused) {
            H.fpre[l] = c.take<FusedTab>(1);
            H.fpost[l] = c.take<FusedTab>(1);
        }
        if (P.shared.fmg) {
            H.rhs[l] = c.take<LaunchTab<T>>(1);
            H.interp[l] = c.take<LaunchTab<T>>(1);
        }
    }
    H.coarse = c.take<CoarseTab<T>>(1);
    H.dense = c.take<DenseTab<T>>(1);
    H.bottom = c.take<BottomTab<T>>(1);
}

// Lay out (or size) the whole device workspace.
void carve(pic_poisson_plan_s &P, Carver &c) {
    const bool mixed = P.shared.precision == PIC_POISSON_MIXED;
    size_t g_restr0 = 0, g_single = 0, g_defect = 0, g_fft = 0, g_api = 0;
    for (int p = 0; p < P.n; ++p) {
        ProblemPlan &q = P.pr[p];
        const int nt = q.d.ntheta;
        q.dl.assign(mixed ? 1 : q.L, LevelDev<double>{});
        q.fl.assign(mixed ? q.L : 0, LevelDev<float>{});
        for (int l = 0; l < (int)q.dl.size(); ++l) {
            carve_level<double, double2>(q.lv[l], q.nm, nt, c, q.dl[l]);
            q.dl[l].relax = 1.0 - q.d.omega;
        }
        for (int l = 0; l < (int)q.fl.size(); ++l) {
            carve_level<float, float2>(q.lv[l], q.nm, nt, c, q.fl[l]);
            q.fl[l].relax = (float)(1.0 - q.d.omega);
        }
        q.u2.assign(q.fl.size(), nullptr);
        if (P.h32.fused)
            for (int l = 0; l + 1 < (int)q.fl.size(); ++l)
                q.u2[l] = c.take<float2>((size_t)q.lv[l].nr * q.lv[l].nz * q.nm);
        if (mixed) carve_coarse(q, c, q.cf);
        else carve_coarse(q, c, q.cd);
        const int M = nt / 2;
        q.tw = (const double *)c.take<double2>(std::max(M / 2, 1));
        q.tw2 = (const double *)c.take<double2>(M + 1);
        q.twf = c.take<float4>(std::max(M / 2, 1));
        q.tw2f = c.take<float4>(M + 1);
        q.s0 = c.take<double>(q.lv[0].act.empty() ? q.lv[0].nr : (size_t)q.lv[0].nr * q.lv[0].nz);
        q.bD0 = c.take<double>((size_t)q.lv[0].nr * q.lv[0].nz);
        q.mask0 = q.lv[0].act.empty() ? nullptr : c.take<double>((size_t)q.lv[0].nr * q.lv[0].nz);
        q.fwin = c.take<double>(q.lv[0].nz);
        q.fwout = c.take<double>(q.lv[0].nz);
        q.finv_rda = c.take<double>(q.lv[0].nr);
        q.finv_rd = c.take<double>(q.lv[0].nr + 1);
        q.dep_inv_vr = c.take<double>(q.lv[0].nr + 1);
        q.dep_inv_vz = c.take<double>(q.lv[0].nz + 1);
        q.dep_flo = c.take<double>(q.lv[0].nr);
        q.dep_fhi = c.take<double>(q.lv[0].nr);
        q.finv_zd = c.take<double>(q.lv[0].nz + 1);
        q.finv_half = c.take<double>(2 * (size_t)q.lv[0].nr + 2 * (size_t)q.lv[0].nz);
        q.act0 = q.lv[0].act.empty() ? nullptr : c.take<unsigned char>(q.lv[0].act.size());
        q.dep_inv_v2 = q.lv[0].act.empty() ? nullptr : c.take<double>((size_t)(q.lv[0].nr + 1) * (q.lv[0].nz + 1));
        q.dep_rf = c.take<double>(q.lv[0].nr + 1);
        q.dep_zf = c.take<double>(q.lv[0].nz + 1);
        q.dep_inv_wr = c.take<double>(q.lv[0].nr);
        q.dep_inv_wz = c.take<double>(q.lv[0].nz);
        q.dep_nrbin = lookup_bins(q.lv[0].rf);
        q.dep_nzbin = lookup_bins(level_zfaces(q, 0));
        q.dep_rbin = c.take<int>(q.dep_nrbin);
        q.dep_zbin = c.take<int>(q.dep_nzbin);
        const LevelHost &h0 = q.lv[0];
        const size_t n0 = (size_t)h0.nr * h0.nz * q.nm;
        g_fft += (size_t)h0.nz * ((h0.nr + FFT_TI - 1) / FFT_TI);
        if (q.L > 1) g_restr0 += mg_blocks((size_t)q.lv[1].nr * q.lv[1].nz * q.nm);
        else g_single += mg_blocks(n0);
        g_defect += mg_blocks(n0);
        if (p == 0) g_api = mg_blocks(n0);
    }
    P.fwd = c.take<FFTTab>(1);
    P.guess = c.take<FFTTab>(1);
    P.inv = c.take<FFTTab>(1);
    P.api_fft = c.take<FFTTab>(1);
    if (mixed) carve_hier(P, c, P.h32);
    else carve_hier(P, c, P.h64);
    P.res_single = c.take<LaunchTab<double>>(1);
    P.api_res = c.take<LaunchTab<double>>(1);
    P.defect = c.take<DefectTab>(1);
    P.ctrl = c.take<Ctrl>(1);
    P.npartials = std::max(std::max(g_restr0 + g_single, g_defect), 2 * g_api) + 64;
    P.npartials_fwd = g_fft + 64;
    P.partials = c.take<double>(P.npartials);
    P.partials_fwd = c.take<double>(P.npartials_fwd);
    // at most one chunk per PSUM_CHUNK partials plus one per problem
    P.partials2 = c.take<double>(P.npartials / PSUM_CHUNK + (size_t)P.n + 64);
    P.psum = c.take<PsumTab>(1);
    P.dsum = c.take<double>(8);
}

template <class T> void to_dev(const std::vector<double> &src, const T *dst, cudaStream_t st, cudaError_t &err) {
    if (err != cudaSuccess || src.empty()) return;
    std::vector<T> conv(src.begin(), src.end());
    err = cudaMemcpyAsync((void *)dst, conv.data(), conv.size() * sizeof(T), cudaMemcpyHostToDevice, st);
    if (err == cudaSuccess) err = cudaStreamSynchronize(st);
}

void ints_to_dev(const std::vector<int> &src, const int *dst, cudaStream_t st, cudaError_t &err) {
    if (err != cudaSuccess || src.empty() || !dst) return;
    err = cudaMemcpyAsync((void *)dst, src.data(), src.size() * sizeof(int), cudaMemcpyHostToDevice, st);
    if (err == cudaSuccess) err = cudaStreamSynchronize(st);
}

template <class X> void blob_to_dev(const X &src, X *dst, cudaStream_t st, cudaError_t &err) {
    if (err != cudaSuccess || !dst) return;
    err = cudaMemcpyAsync(dst, &src, sizeof(X), cudaMemcpyHostToDevice, st);
    if (err == cudaSuccess) err = cudaStreamSynchronize(st);
}

template <class T> void upload_level(const LevelHost &h, const LevelDev<T> &v, cudaStream_t st, cudaError_t &err) {
    ints_to_dev(h.rcls, v.rcls, st, err);
    to_dev(h.hn, v.hn, st, err);
    to_dev(h.ccw, v.ccw, st, err);
    to_dev(h.cce, v.cce, st, err);
    to_dev(h.ccs, v.ccs, st, err);
    to_dev(h.ccn, v.ccn, st, err);
    to_dev(h.cw, v.cw, st, err);
    to_dev(h.ce, v.ce, st, err);
    to_dev(h.cz, v.cz, st, err);
    to_dev(h.invd, v.invd, st, err);
    to_dev(h.diag, v.diag, st, err);
    to_dev(h.hw, v.hw, st, err);
    to_dev(h.he, v.he, st, err);
    to_dev(h.hz, v.hz, st, err);
}

// Launch tables of one precision's hierarchy.  views(q) is problem q's level list.
template <class T, class Views, class Coarse>
void build_hier(pic_poisson_plan_s &P, Hier<T> &H, Views views, Coarse coarse, cudaStream_t st, cudaError_t &err) {
    const int nl = std::max(P.Lmax - 1, 0);
    const int pre = P.shared.pre_sweeps, post = P.shared.post_sweeps;
    H.g_smooth.assign(nl, 0);
    H.g_restr.assign(nl, 0);
    H.g_prolong.assign(nl, 0);
    H.strip.assign(nl, 1);
    H.g_fpre.assign(nl, 0);
    H.g_fpost.assign(nl, 0);
    H.fres.assign(nl, 0);
    for (int l = 0; l < nl; ++l) {
        LaunchTab<T> ts{}, tr{}, tp{};
        FusedTab fa{}, fb{};
        ts.done = tr.done = tp.done = fa.done = fb.done = ctrl_done(P);
        int nprob = 0;
        bool res = H.fused;   // restriction fused into pre-smoothing: every pair of levels halves r and z
        for (int p = 0; p < P.n; ++p)
            if (l < P.pr[p].smoothed()) {
                ++nprob;
                const LevelHost &a = P.pr[p].lv[l], &b = P.pr[p].lv[l + 1];
                res = res && b.nr * 2 == a.nr && b.nz * 2 == a.nz;
            }
        H.fres[l] = res;
        // fused smoother blocks per problem: one wave of two blocks per SM
        const int target = std::max(1, 2 * 152 / std::max(nprob, 1));
        // smoother strip (0: one entry per thread); a strip longer than the
        // level's rows of one parity is cut to the next power of two that fits
        int strip = P.shared.smooth_strip;
        int zmax = 0;
        for (int p = 0; p < P.n; ++p)
            if (l < P.pr[p].smoothed()) zmax = std::max(zmax, (views(P.pr[p])[l].nz + 1) / 2);
        while (strip > 1 && strip > zmax) strip >>= 1;
        H.strip[l] = strip;
        for (int p = 0; p < P.n; ++p) {
            const ProblemPlan &q = P.pr[p];
            if (l >= q.smoothed()) continue;
            const std::vector<LevelDev<T>> &v = views(q);
            LevelDev<T> f = v[l];
            f.init = (l + 1 == q.L - 1) ? 0 : (pre > 0 ? 2 : 1);
            const size_t half = (size_t)f.nz * (f.nr / 2) * f.nm, full = (size_t)f.nz * f.nr * f.nm;
            const size_t coarse_n = (size_t)v[l + 1].nz * v[l + 1].nr * f.nm;
            ts.pid[ts.n] = tr.pid[tr.n] = tp.pid[tp.n] = p;
            ts.f[ts.n] = f;
            ts.f[ts.n].strip = strip;
            ts.start[ts.n + 1] = ts.start[ts.n] + (strip == 0 ? mg_blocks(half, P.shared.smooth_threads)
                                                             : smooth_blocks(f.nr, f.nz, f.nm, strip,
                                                                             P.shared.smooth_threads));
            ++ts.n;
            tr.f[tr.n] = f;
            tr.c[tr.n] = v[l + 1];
            tr.start[tr.n + 1] = tr.start[tr.n] + mg_blocks(coarse_n);
            tp.f[tp.n] = f;
            tp.c[tp.n] = v[l + 1];
            tp.start[tp.n + 1] = tp.start[tp.n] + mg_blocks(post > 0 && P.shared.omega == 1.0 ? half : full);
            if constexpr (std::is_same<T, float>::value) {
                if (H.fused) {
                    // pre-smoothing u -> u2; the restriction reads u2 and the
                    // prolongation corrects u2; post-smoothing u2 -> u
                    tr.f[tr.n].u = q.u2[l];
                    tp.f[tp.n].u = q.u2[l];
                    unsigned nb = 0;
                    FusedProb a{};
                    a.L = f;
                    a.C = v[l + 1];
                    a.init = f.init;
                    a.in = f.u;
                    a.out = q.u2[l];
                    fused_shape(f.nr, f.nz, f.nm, 2 * pre, res, target, a, nb);
                    fa.pid[fa.n] = p;
                    fa.p[fa.n] = a;
                    fa.start[fa.n + 1] = fa.start[fa.n] + nb;
                    ++fa.n;
                    FusedProb b{};
                    b.L = f;
                    b.in = q.u2[l];
                    b.out = f.u;
                    // post-smoothing holds fewer registers: three blocks per SM on level 0
                    fused_shape(f.nr, f.nz, f.nm, 2 * post, false, l == 0 ? target * 3 / 2 : target, b, nb);
                    fb.pid[fb.n] = p;
                    fb.p[fb.n] = b;
                    fb.start[fb.n + 1] = fb.start[fb.n] + nb;
                    ++fb.n;
                }
            }
            ++tr.n;
            ++tp.n;
        }
        H.g_smooth[l] = ts.start[ts.n];
        H.g_restr[l] = tr.start[tr.n];
        H.g_prolong[l] = tp.start[tp.n];
        if (ts.n == 0) {
            H.smooth[l] = H.restr[l] = H.prolong[l] = nullptr;
            continue;
        }
        blob_to_dev(ts, H.smooth[l], st, err);
        blob_to_dev(tr, H.restr[l], st, err);
        blob_to_dev(tp, H.prolong[l], st, err);
        if (H.fused) {
            H.g_fpre[l] = fa.start[fa.n];
            H.g_fpost[l] = fb.start[fb.n];
            blob_to_dev(fa, H.fpre[l], st, err);
            blob_to_dev(fb, H.fpost[l], st, err);
        }
    }
    H.g_rhs.assign(nl, 0);
    H.g_interp.assign(nl, 0);
    if (P.shared.fmg) {
        // full-multigrid start: b restricted from l to l + 1 for every level pair
        // of a problem, and u_l = P u_(l+1) for the levels the level kernels
        // solve -- on the black cells only when a Gauss-Seidel red half-sweep
        // follows (it overwrites the red ones without reading them)
        H.interp_black = pre > 0 && P.shared.omega == 1.0;
        for (int l = 0; l < nl; ++l) {
            LaunchTab<T> trh{}, tin{};
            for (int p = 0; p < P.n; ++p) {
                const ProblemPlan &q = P.pr[p];
                const std::vector<LevelDev<T>> &v = views(q);
                if (l < q.L - 1) {
                    trh.f[trh.n] = v[l];
                    trh.c[trh.n] = v[l + 1];
                    trh.start[trh.n + 1] =
                        trh.start[trh.n] + mg_blocks((size_t)v[l + 1].nz * v[l + 1].nr * v[l].nm);
                    ++trh.n;
                }
                if (l < q.smoothed()) {
                    tin.f[tin.n] = v[l];
                    tin.c[tin.n] = v[l + 1];
                    tin.start[tin.n + 1] =
                        tin.start[tin.n] +
                        mg_blocks((size_t)v[l].nz * (H.interp_black ? v[l].nr / 2 : v[l].nr) * v[l].nm);
                    ++tin.n;
                }
            }
            H.g_rhs[l] = trh.start[trh.n];
            H.g_interp[l] = tin.start[tin.n];
            if (trh.n) blob_to_dev(trh, H.rhs[l], st, err);
            if (tin.n) blob_to_dev(tin, H.interp[l], st, err);
        }
    }
    CoarseTab<T> tc{};
    DenseTab<T> td{};
    BottomTab<T> tb{};
    tc.done = td.done = tb.done = ctrl_done(P);
    size_t smem_b = 0;
    for (int p = 0; p < P.n; ++p) {
        const ProblemPlan &q = P.pr[p];
        const CoarseDev<T> &cd = coarse(q);
        if (q.bottom) {
            const LevelDev<T> &U = views(q)[q.L - 2];
            BottomProb<T> bp{};
            bp.U = U;
            bp.D = cd;
            bp.pre = pre;
            bp.post = post;
            bp.red_only = pre > 0 && P.shared.omega == 1.0;
            bp.black_only = post > 0 && P.shared.omega == 1.0;
            tb.pid[tb.n] = p;
            tb.p[tb.n] = bp;
            tb.start[tb.n + 1] = tb.start[tb.n] + 2u * (unsigned)q.nm;   // (mode, real / imaginary part)
            smem_b = std::max(smem_b, bottom_smem_bytes<T>(U.nr, U.nz, U.ncls, cd.nr, cd.nz));
            ++tb.n;
            continue;
        }
        if (cd.nact > 0) {   // dense coarsest solve: two GEMMs over all modes
            td.pid[td.n] = p;
            td.f[td.n] = views(q)[q.L - 1];
            td.c[td.n] = cd;
            td.start[td.n + 1] = td.start[td.n] + 2u * (unsigned)q.nm;
            td.gstart[td.n + 1] = td.gstart[td.n] + dense_gemm_blocks(cd.nact, q.nm);
            ++td.n;
            continue;
        }
        tc.pid[tc.n] = p;
        tc.f[tc.n] = views(q)[q.L - 1];
        tc.c[tc.n] = cd;
        tc.start[tc.n + 1] = tc.start[tc.n] + 2u * (unsigned)q.nm;   // (mode, real / imaginary part)
        const size_t sm = ((size_t)cd.nr * cd.nz + 3 * (size_t)(cd.nr + 1) * cd.nz +
                           (size_t)(cd.nz - cd.nz / 2) * cd.nz + (size_t)cd.nr) * sizeof(T);
        tc.smem = std::max(tc.smem, sm);
        ++tc.n;
    }
    H.g_coarse = tc.start[tc.n];
    H.smem_coarse = tc.smem;
    blob_to_dev(tc, H.coarse, st, err);
    H.g_dense_prep = td.start[td.n];
    H.g_dense_gemm = td.gstart[td.n];
    if (td.n) blob_to_dev(td, H.dense, st, err);
    H.g_bottom = tb.start[tb.n];
    H.smem_bottom = smem_b;
    if (tb.n) blob_to_dev(tb, H.bottom, st, err);
}

int upload(pic_poisson_plan_s &P) {
    cudaError_t err = cudaSuccess;
    const cudaStream_t st = P.stream;
    const bool mixed = P.shared.precision == PIC_POISSON_MIXED;
    for (int p = 0; p < P.n; ++p) {
        ProblemPlan &q = P.pr[p];
        for (size_t l = 0; l < q.dl.size(); ++l) upload_level(q.lv[l], q.dl[l], st, err);
        for (size_t l = 0; l < q.fl.size(); ++l) upload_level(q.lv[l], q.fl[l], st, err);
        std::vector<double> V, e, piv, cpr;
        if (q.nact > 0) {   // composite domain: dense coarsest solve
            std::vector<int> aidx, amap;
            std::vector<double> Q, QT, lam, isq, lamm;
            const int rc = dense_factors(q, aidx, amap, Q, QT, lam, isq, lamm);
            if (rc) return rc;
            auto put = [&](auto &cd) {
                ints_to_dev(aidx, cd.aidx, st, err);
                ints_to_dev(amap, cd.amap, st, err);
                to_dev(Q, cd.Q, st, err);
                to_dev(QT, cd.QT, st, err);
                to_dev(lam, cd.lam, st, err);
                to_dev(isq, cd.isq, st, err);
                to_dev(lamm, cd.lamm, st, err);
            };
            if (!mixed) put(q.cd);
            else put(q.cf);
        } else {
            coarse_factors(q, V, e, piv, cpr);
            auto put = [&](auto &cd) {
                to_dev(V, cd.V, st, err);
                to_dev(e, cd.e, st, err);
                to_dev(piv, cd.piv, st, err);
                to_dev(cpr, cd.cpr, st, err);
            };
            if (!mixed) put(q.cd);
            else put(q.cf);
        }
        const int nt = q.d.ntheta, M = nt / 2;
        std::vector<double> tw(2 * std::max(M / 2, 1), 0.0), tw2(2 * (M + 1), 0.0);
        auto scale_ratio = [](double *out, int t, int n) {   // e^{-2 pi i t / n} as (a, b), see tw_rot
            const double th = 2.0 * kPi * t / n - (tw_rot(t, n) ? 0.5 * kPi : 0.0);
            out[0] = std::cos(th);
            out[1] = -std::tan(th);
        };
        for (int t = 0; t < M / 2; ++t) scale_ratio(&tw[2 * t], t, M);
        if (M / 2 == 0) tw[0] = 1.0;
        for (int m = 0; m <= M; ++m) scale_ratio(&tw2[2 * m], m, nt);
        to_dev(tw, q.tw, st, err);
        to_dev(tw2, q.tw2, st, err);
        // double-float copies: each binary64 entry as hi = its binary32 rounding, lo = the rest rounded
        auto split = [](const std::vector<double> &v) {   // binary32 values, held exactly in binary64
            std::vector<double> f(2 * v.size());
            for (size_t e = 0; e < v.size(); ++e) {
                f[2 * e] = (double)(float)v[e];
                f[2 * e + 1] = (double)(float)(v[e] - f[2 * e]);
            }
            return f;
        };
        to_dev(split(tw), (float *)q.twf, st, err);
        to_dev(split(tw2), (float *)q.tw2f, st, err);
        // level-0 right-hand-side factors: s_i (Eq. mode_rhs) and b^D (Eq. boundary_rhs_appendix)
        const LevelHost &h = q.lv[0];
        std::vector<double> s(h.nr), bD((size_t)h.nr * h.nz, 0.0);
        for (int i = 0; i < h.nr; ++i) s[i] = h.rc[i] * h.drc[i] * h.dz / q.d.eps0;
        if (h.act.empty()) {
            for (int k = 0; k < h.nz; ++k)
                for (int i = 0; i < h.nr; ++i) {
                    double v = 0.0;
                    const double rm = h.rf[i], rp = h.rf[i + 1];
                    if (i == 0) v += rm * h.dz / (h.rc[i] - rm) * wall_rin(q.d, k);
                    if (i == h.nr - 1) v += rp * h.dz / (rp - h.rc[i]) * wall_rout(q.d, k);
                    if (k == 0) v += 2.0 * h.cz[i] * q.d.phi_z0;
                    if (k == h.nz - 1) v += 2.0 * h.cz[i] * q.d.phi_z1;
                    bD[(size_t)k * h.nr + i] = v;
                }
        } else {
            // composite domain: s per cell (zero outside the patches, so their charge is ignored);
            // a Dirichlet face takes its wall's potential on the grid boundary, phi_exposed inside
            std::vector<double> s2((size_t)h.nr * h.nz, 0.0);
            for (int k = 0; k < h.nz; ++k)
                for (int i = 0; i < h.nr; ++i) {
                    if (!h.act[(size_t)k * h.nr + i]) continue;
                    s2[(size_t)k * h.nr + i] = s_eps0_cell(h, i, k) / q.d.eps0;
                    double g[4];
                    int dir[4];
                    cell_faces(h, i, k, g, dir);
                    const double pe = q.d.phi_exposed;
                    double v = 0.0;
                    if (dir[0]) v += g[0] * (i == 0 ? wall_rin(q.d, k) : pe);
                    if (dir[1]) v += g[1] * (i == h.nr - 1 ? wall_rout(q.d, k) : pe);
                    if (dir[2]) v += g[2] * (k == 0 ? q.d.phi_z0 : pe);
                    if (dir[3]) v += g[3] * (k == h.nz - 1 ? q.d.phi_z1 : pe);
                    bD[(size_t)k * h.nr + i] = v;
                }
            s.swap(s2);
            to_dev(std::vector<double>(h.act.begin(), h.act.end()), q.mask0, st, err);
        }
        to_dev(s, q.s0, st, err);
        to_dev(bD, q.bD0, st, err);
        // face-field reconstruction: wall potentials and the azimuthal arcs
        std::vector<double> win(h.nz), wout(h.nz), inv_rda(h.nr);
        for (int k = 0; k < h.nz; ++k) {
            win[k] = wall_rin(q.d, k);
            wout[k] = wall_rout(q.d, k);
        }
        const double da = q.d.theta_span / q.d.ntheta;
        for (int i = 0; i < h.nr; ++i) inv_rda[i] = 1.0 / (h.rc[i] * da);
        std::vector<double> inv_rd(h.nr + 1);   // 1 / the distances of the radial faces' differences
        for (int a = 0; a <= h.nr; ++a)
            inv_rd[a] = 1.0 / (a == 0 ? h.rc[0] - h.rf[0] : (a == h.nr ? h.rf[a] - h.rc[a - 1] : h.rc[a] - h.rc[a - 1]));
        to_dev(inv_rd, q.finv_rd, st, err);
        to_dev(win, q.fwin, st, err);
        to_dev(wout, q.fwout, st, err);
        to_dev(inv_rda, q.finv_rda, st, err);
        // CIC deposit and projection: node control volumes (centre to centre,
        // cut at the walls; exact r dr integral) and the cells' radial octant shares
        std::vector<double> ivr(h.nr + 1), ivz(h.nz + 1), flo(h.nr), fhi(h.nr);
        auto rface = [&](int a) { return h.rf[a]; };
        auto rcen = [&](int i) { return h.rc[i]; };
        for (int a = 0; a <= h.nr; ++a) {
            const double lo = a == 0 ? rface(0) : rcen(a - 1), hi = a == h.nr ? rface(h.nr) : rcen(a);
            ivr[a] = 1.0 / ((hi - lo) * (hi + lo) / 2);   // 1 / integral of r dr, factored
        }
        for (int c = 0; c <= h.nz; ++c) ivz[c] = 1.0 / (da * ((c == 0 || c == h.nz) ? 0.5 * h.dz : h.dz));
        for (int i = 0; i < h.nr; ++i) {
            const double r0 = rface(i), r1 = rface(i + 1), rc = rcen(i), all = (r1 - r0) * (r1 + r0);
            flo[i] = (rc - r0) * (rc + r0) / all;
            fhi[i] = (r1 - rc) * (r1 + rc) / all;
        }
        to_dev(ivr, q.dep_inv_vr, st, err);
        to_dev(ivz, q.dep_inv_vz, st, err);
        to_dev(flo, q.dep_flo, st, err);
        to_dev(fhi, q.dep_fhi, st, err);
        // the same steps on non-uniform axial faces and composite domains: axial
        // face distances, centre-to-face distances, the active flags, the node
        // volumes of active octants, and the cell lookups of the deposit
        const std::vector<double> zf = level_zfaces(q, 0);
        std::vector<double> zc(h.nz);
        for (int k = 0; k < h.nz; ++k) zc[k] = 0.5 * (zf[k] + zf[k + 1]);
        std::vector<double> inv_zd(h.nz + 1);
        for (int c = 0; c <= h.nz; ++c)
            inv_zd[c] = 1.0 / (c == 0 ? zc[0] - zf[0] : (c == h.nz ? zf[c] - zc[c - 1] : zc[c] - zc[c - 1]));
        std::vector<double> half(2 * (size_t)h.nr + 2 * (size_t)h.nz);
        for (int i = 0; i < h.nr; ++i) {
            half[i] = 1.0 / (h.rc[i] - h.rf[i]);
            half[h.nr + i] = 1.0 / (h.rf[i + 1] - h.rc[i]);
        }
        for (int k = 0; k < h.nz; ++k) {
            half[2 * h.nr + k] = 1.0 / (zc[k] - zf[k]);
            half[2 * h.nr + h.nz + k] = 1.0 / (zf[k + 1] - zc[k]);
        }
        to_dev(inv_zd, q.finv_zd, st, err);
        to_dev(half, q.finv_half, st, err);
        // axial node intervals from centre to centre (cut at the walls) on the given faces
        for (int c = 0; c <= h.nz; ++c) {
            const double lo = c == 0 ? zf[0] : zc[c - 1], hi = c == h.nz ? zf[h.nz] : zc[c];
            ivz[c] = 1.0 / (da * (hi - lo));
        }
        if (!h.zf.empty()) to_dev(ivz, q.dep_inv_vz, st, err);
        if (q.act0) {
            if (err == cudaSuccess)
                err = cudaMemcpyAsync(q.act0, h.act.data(), h.act.size(), cudaMemcpyHostToDevice, st);
            if (err == cudaSuccess) err = cudaStreamSynchronize(st);
            // node volumes: the sum over the node's active neighbour cells of
            // the octant in each (r: the exact r dr integral of the half cell)
            std::vector<double> v2((size_t)(h.nr + 1) * (h.nz + 1), 0.0);
            for (int k = 0; k < h.nz; ++k)
                for (int i = 0; i < h.nr; ++i) {
                    if (!h.act[(size_t)k * h.nr + i]) continue;
                    const double r0 = h.rf[i], r1 = h.rf[i + 1], rc = h.rc[i], hz = 0.5 * (zf[k + 1] - zf[k]);
                    const double vlo = (rc - r0) * (rc + r0) / 2, vhi = (r1 - rc) * (r1 + rc) / 2;
                    for (int c = k; c <= k + 1; ++c) {
                        v2[(size_t)c * (h.nr + 1) + i] += da * hz * vlo;
                        v2[(size_t)c * (h.nr + 1) + i + 1] += da * hz * vhi;
                    }
                }
            for (double &v : v2) v = v > 0.0 ? 1.0 / v : 0.0;
            to_dev(v2, q.dep_inv_v2, st, err);
        }
        std::vector<double> iwr(h.nr), iwz(h.nz);
        for (int i = 0; i < h.nr; ++i) iwr[i] = 1.0 / (h.rf[i + 1] - h.rf[i]);
        for (int k = 0; k < h.nz; ++k) iwz[k] = 1.0 / (zf[k + 1] - zf[k]);
        to_dev(h.rf, q.dep_rf, st, err);
        to_dev(zf, q.dep_zf, st, err);
        to_dev(iwr, q.dep_inv_wr, st, err);
        to_dev(iwz, q.dep_inv_wz, st, err);
        ints_to_dev(lookup_table(h.rf, q.dep_nrbin), q.dep_rbin, st, err);
        ints_to_dev(lookup_table(zf, q.dep_nzbin), q.dep_zbin, st, err);
        q.dep_inv_rbw = (float)(q.dep_nrbin / (h.rf[h.nr] - h.rf[0]));
        q.dep_inv_zbw = (float)(q.dep_nzbin / (zf[h.nz] - zf[0]));
    }

    // transforms
    FFTTab &F = P.h_fwd, &G = P.h_guess, &I = P.h_inv;
    F = FFTTab{};
    G = FFTTab{};
    I = FFTTab{};
    size_t smem = 0;
    for (int p = 0; p < P.n; ++p) {
        const ProblemPlan &q = P.pr[p];
        const LevelDev<double> &d0 = q.dl[0];
        FFTProb fp{};
        fp.nr = d0.nr;
        fp.nt = q.d.ntheta;
        fp.nz = d0.nz;
        fp.nm = q.nm;
        fp.ncls = d0.ncls;
        int lg = 0;
        while ((1 << lg) < q.d.ntheta / 2) ++lg;
        fp.log2M = lg;
        fp.tw = q.tw;
        fp.tw2 = q.tw2;
        fp.twf = q.twf;
        fp.tw2f = q.tw2f;
        fp.half_inv_n = 0.5 / q.d.ntheta;
        FFTProb f = fp, g = fp, iv = fp;
        f.s = q.s0;
        f.s_rows = q.lv[0].act.empty() ? 0 : 1;
        f.rcls = d0.rcls;
        f.bD = q.bD0;
        f.invd = mixed ? nullptr : d0.invd;
        f.b = d0.b;
        f.bh = mixed ? nullptr : d0.bh;
        g.b = d0.u;                         // initial guess: plain 1/N transform of phi into u
        if (q.mask0) {                      // (composite domain: held at 0 outside the patches)
            g.s = q.mask0;
            g.s_rows = 1;
        }
        iv.uhat = d0.u;
        const unsigned blocks = (unsigned)(d0.nz * ((d0.nr + FFT_TI - 1) / FFT_TI));
        F.p[p] = f;
        G.p[p] = g;
        I.p[p] = iv;
        F.start[p + 1] = G.start[p + 1] = I.start[p + 1] = F.start[p] + blocks;
        smem = std::max(smem, fft_smem_bytes(q.d.ntheta));
    }
    F.n = G.n = I.n = P.n;
    F.smem = G.smem = I.smem = smem;
    P.g_fft = F.start[P.n];
    P.smem_fft = smem;
    blob_to_dev(F, P.fwd, st, err);
    blob_to_dev(G, P.guess, st, err);
    blob_to_dev(I, P.inv, st, err);

    // hierarchy tables
    if (mixed) {
        build_hier<float>(P, P.h32, [](const ProblemPlan &q) -> const std::vector<LevelDev<float>> & { return q.fl; },
                          [](const ProblemPlan &q) -> const CoarseDev<float> & { return q.cf; }, st, err);
    } else {
        build_hier<double>(P, P.h64, [](const ProblemPlan &q) -> const std::vector<LevelDev<double>> & { return q.dl; },
                           [](const ProblemPlan &q) -> const CoarseDev<double> & { return q.cd; }, st, err);
    }

    // single-level problems' residual norms; defect table; stage-call table
    LaunchTab<double> rs{};
    DefectTab dt{};
    rs.done = dt.done = ctrl_done(P);
    for (int p = 0; p < P.n; ++p) {
        const ProblemPlan &q = P.pr[p];
        const size_t n0 = (size_t)q.lv[0].nr * q.lv[0].nz * q.nm;
        if (q.L == 1) {
            rs.pid[rs.n] = p;
            rs.f[rs.n] = q.dl[0];
            rs.start[rs.n + 1] = rs.start[rs.n] + mg_blocks(n0);
            ++rs.n;
        }
        if (mixed) {
            dt.pid[dt.n] = p;
            dt.d[dt.n] = q.dl[0];
            dt.s[dt.n] = q.fl[0];
            dt.init_red[dt.n] = (q.L > 1 && P.shared.pre_sweeps > 0) ? 1 : 0;
            dt.start[dt.n + 1] = dt.start[dt.n] + mg_blocks(n0);
            ++dt.n;
        }
    }
    P.g_res_single = rs.start[rs.n];
    P.g_defect = dt.start[dt.n];
    blob_to_dev(rs, P.res_single, st, err);
    blob_to_dev(dt, P.defect, st, err);
    P.h_api_res = LaunchTab<double>{};
    P.h_api_res.n = 1;
    P.h_api_res.f[0] = P.pr[0].dl[0];
    P.g_api_res = mg_blocks((size_t)P.pr[0].lv[0].nr * P.pr[0].lv[0].nz * P.pr[0].nm);
    P.h_api_res.start[1] = P.g_api_res;

    // per-problem ranges of the residual-norm partials and control state
    Ctrl &C = P.hctrl;
    C = Ctrl{};
    C.n = P.n;
    C.scaled = mixed ? 1 : 0;
    C.inc = mixed ? P.shared.inner_cycles : 1;
    C.inc_first = mixed ? P.shared.inner_first : 1;
    const unsigned g_restr0 = (!mixed && P.Lmax > 1) ? P.h64.g_restr[0] : 0;
    P.res_single_offset = g_restr0;
    unsigned b0 = 0;
    int is = 0;
    for (int p = 0; p < P.n; ++p) {
        const ProblemPlan &q = P.pr[p];
        C.count[p] = (double)q.lv[0].nr * q.lv[0].nz * q.d.ntheta;
        if (mixed) {
            C.rbegin[p] = dt.start[p];
            C.rend[p] = dt.start[p + 1];
        } else if (q.L > 1) {
            // the level-0 restriction table lists the multi-level problems in order
            const unsigned nb = mg_blocks((size_t)q.lv[1].nr * q.lv[1].nz * q.nm);
            C.rbegin[p] = b0;
            C.rend[p] = b0 + nb;
            b0 += nb;
        } else {
            C.rbegin[p] = g_restr0 + rs.start[is];
            C.rend[p] = g_restr0 + rs.start[is + 1];
            ++is;
        }
    }
    // two-stage norm reduction: k_psum sums chunks of each problem's partials,
    // the convergence test reads the chunk sums
    PsumTab ps{};
    ps.n = P.n;
    for (int p = 0; p < P.n; ++p) {
        const unsigned len = C.rend[p] - C.rbegin[p];
        const unsigned chunks = std::max(1u, (len + PSUM_CHUNK - 1) / PSUM_CHUNK);
        ps.in_begin[p] = C.rbegin[p];
        ps.in_end[p] = C.rend[p];
        ps.start[p + 1] = ps.start[p] + chunks;
        C.rbegin[p] = ps.start[p];
        C.rend[p] = ps.start[p + 1];
    }
    P.g_psum = ps.start[P.n];
    blob_to_dev(ps, P.psum, st, err);
    if (err != cudaSuccess) {
        set_error("uploading plan tables failed: %s", cudaGetErrorString(err));
        return PIC_POISSON_ECUDA;
    }
    return PIC_POISSON_OK;
}

int same_settings(const pic_poisson_desc &a, const pic_poisson_desc &b) {
    return a.precision == b.precision && a.max_cycles == b.max_cycles && a.pre_sweeps == b.pre_sweeps &&
           a.post_sweeps == b.post_sweeps && a.inner_cycles == b.inner_cycles && a.flags == b.flags &&
           a.smooth_threads == b.smooth_threads && a.smooth_strip == b.smooth_strip && a.omega == b.omega &&
           a.smooth_fused == b.smooth_fused && a.local_bottom == b.local_bottom && a.fmg == b.fmg &&
           a.inner_first == b.inner_first;
}

int setup_plan(pic_poisson_plan_s &P, const pic_poisson_desc *descs, int n) {
    if (n < 1 || n > kMaxBatch) {
        set_error("batch size %d outside [1, %d]", n, kMaxBatch);
        return PIC_POISSON_EINVAL;
    }
    P.n = n;
    P.pr.resize(n);
    for (int p = 0; p < n; ++p) {
        pic_poisson_desc d;
        int rc = resolve(&descs[p], &d);
        if (rc) return rc;
        if (p == 0) P.shared = d;
        else if (!same_settings(P.shared, d)) {
            set_error("problem %d: precision, max_cycles, sweeps, inner_cycles, inner_first, smooth_threads, smooth_strip, omega, "
                      "smooth_fused and flags must match "
                      "problem 0", p);
            return PIC_POISSON_EINVAL;
        }
        rc = setup_problem(P.pr[p], d);
        if (rc) return rc;
        P.Lmax = std::max(P.Lmax, P.pr[p].L);
    }
    if (P.shared.smooth_fused) {
        const pic_poisson_desc &s = P.shared;
        bool ok = s.precision == PIC_POISSON_MIXED && s.omega == 1.0 && s.pre_sweeps >= 1 && s.pre_sweeps <= 2 &&
                  s.post_sweeps >= 1 && s.post_sweeps <= 2;
        for (const ProblemPlan &q : P.pr)
            for (int l = 0; l + 1 < q.L; ++l) ok = ok && q.lv[l].nr % 2 == 0;
        if (!ok) {
            set_error("smooth_fused needs mixed precision, omega = 1, 1 or 2 pre- and post-sweeps and even nr on "
                      "every smoothed level");
            return PIC_POISSON_EINVAL;
        }
        P.h32.fused = true;
    }
    P.masked = false;
    for (const ProblemPlan &q : P.pr) P.masked = P.masked || q.nact > 0;
    // mode-local bottom where the two coarsest levels fit in one block's shared memory
    for (ProblemPlan &q : P.pr) {
        q.bottom = false;
        if (P.shared.local_bottom != 0 || P.shared.omega != 1.0 || q.L < 3 || q.nact > 0) continue;
        const LevelHost &U = q.lv[q.L - 2], &C = q.lv[q.L - 1];
        if (U.nr % 2) continue;
        const size_t smem = P.shared.precision == PIC_POISSON_MIXED
                                ? bottom_smem_bytes<float>(U.nr, U.nz, U.ncls, C.nr, C.nz)
                                : bottom_smem_bytes<double>(U.nr, U.nz, U.ncls, C.nr, C.nz);
        q.bottom = smem <= BOTTOM_MAX_SMEM;
    }
    return PIC_POISSON_OK;
}

}  // namespace

int plan_enter(pic_poisson_plan_s *P) {
    clear_error();
    if (!P) {
        set_error("plan is NULL");
        return PIC_POISSON_EINVAL;
    }
    PP_CUDA(cudaSetDevice(P->device));
    return PIC_POISSON_OK;
}

}  // namespace pp

using namespace pp;

extern "C" {

const char *pic_poisson_last_error(void) { return pp::last_error_text(); }

int pic_poisson_query(const pic_poisson_desc *desc, pic_poisson_layout *out) {
    clear_error();
    pic_poisson_plan_s P;
    int rc = setup_plan(P, desc, 1);
    if (rc) return rc;
    if (out) {
        memset(out, 0, sizeof *out);
        out->levels = P.pr[0].L;
        for (int l = 0; l < P.pr[0].L; ++l) {
            out->nr[l] = P.pr[0].lv[l].nr;
            out->nz[l] = P.pr[0].lv[l].nz;
        }
        out->n_modes = P.pr[0].nm;
        Carver c;
        carve(P, c);
        out->workspace_bytes = c.off;
    }
    return PIC_POISSON_OK;
}

int pic_poisson_cell_coeffs(const pic_poisson_desc *desc, int i, int k, double *out) {
    clear_error();
    pic_poisson_desc d;
    int rc = resolve(desc, &d);
    if (rc) return rc;
    if (!out || i < 0 || i >= d.nr || k < 0 || k >= d.nz) {
        set_error("cell (%d, %d) outside the %d x %d grid or out is NULL", i, k, d.nr, d.nz);
        return PIC_POISSON_EINVAL;
    }
    LevelHost h;
    build_level(d, d.r_faces ? std::vector<double>(d.r_faces, d.r_faces + d.nr + 1) : uniform_faces(d, d.nr), d.nz, 1,
                h);
    if (d.n_patches > 0 || d.z_faces) {   // composite domain (exposed faces are Dirichlet faces at
                                          // phi_exposed) or non-uniform axial faces
        h.act = patch_mask(d);
        if (d.z_faces) {
            h.zf.assign(d.z_faces, d.z_faces + d.nz + 1);
            for (int a = 0; a < d.nz; ++a) {
                h.zc.push_back(0.5 * (h.zf[a] + h.zf[a + 1]));
                h.dzc.push_back(h.zf[a + 1] - h.zf[a]);
            }
        }
        for (int a = 0; a < 12; ++a) out[a] = 0.0;
        if (!h.act.empty() && !h.act[(size_t)k * d.nr + i]) return PIC_POISSON_OK;   // not an unknown
        double g[4];
        int dir[4];
        cell_faces(h, i, k, g, dir);
        const double wall[4] = {i == 0 ? (d.phi_r_in_z ? d.phi_r_in_z[k] : d.phi_r_in) : d.phi_exposed,
                                i == d.nr - 1 ? (d.phi_r_out_z ? d.phi_r_out_z[k] : d.phi_r_out) : d.phi_exposed,
                                k == 0 ? d.phi_z0 : d.phi_exposed, k == d.nz - 1 ? d.phi_z1 : d.phi_exposed};
        for (int f = 0; f < 4; ++f) {
            out[f] = g[f];
            out[4 + f] = dir[f];
            out[10] += g[f];
            if (dir[f]) out[11] += g[f] * wall[f];
        }
        out[8] = mu_cell(h, i, k);
        out[9] = s_eps0_cell(h, i, k) / d.eps0;
        return PIC_POISSON_OK;
    }
    const bool dw = i == 0, de = i == d.nr - 1, ds = k == 0, dn = k == d.nz - 1;
    const double rm = h.rf[i], rp = h.rf[i + 1];
    out[0] = dw ? rm * h.dz / (h.rc[i] - rm) : h.cw[i];
    out[1] = de ? rp * h.dz / (rp - h.rc[i]) : h.ce[i];
    out[2] = ds ? 2.0 * h.cz[i] : h.cz[i];
    out[3] = dn ? 2.0 * h.cz[i] : h.cz[i];
    out[4] = dw;
    out[5] = de;
    out[6] = ds;
    out[7] = dn;
    out[8] = h.mu[i];
    out[9] = h.rc[i] * h.drc[i] * h.dz / d.eps0;
    const int tzc = d.nz == 1 ? 4 : ((k == 0 || k == d.nz - 1) ? 3 : 2);
    out[10] = h.d0r[i] + tzc * h.cz[i];
    double bd = 0.0;
    if (dw) bd += out[0] * (d.phi_r_in_z ? d.phi_r_in_z[k] : d.phi_r_in);
    if (de) bd += out[1] * (d.phi_r_out_z ? d.phi_r_out_z[k] : d.phi_r_out);
    if (ds) bd += out[2] * d.phi_z0;
    if (dn) bd += out[3] * d.phi_z1;
    out[11] = bd;
    return PIC_POISSON_OK;
}

int pic_poisson_plan_batch(const pic_poisson_desc *descs, int n, void *stream, pic_poisson_plan_t *out) {
    clear_error();
    if (!out || !descs) {
        set_error("descs and out must be non-NULL");
        return PIC_POISSON_EINVAL;
    }
    *out = nullptr;
    pic_poisson_plan_s *P = new (std::nothrow) pic_poisson_plan_s;
    if (!P) {
        set_error("host allocation failed");
        return PIC_POISSON_ENOMEM;
    }
    int rc = setup_plan(*P, descs, n);
    if (rc) {
        delete P;
        return rc;
    }
    P->stream = (cudaStream_t)stream;
    cudaError_t err = cudaGetDevice(&P->device);
    if (err != cudaSuccess) {
        set_error("cudaGetDevice: %s", cudaGetErrorString(err));
        delete P;
        return PIC_POISSON_ECUDA;
    }
    Carver c;
    carve(*P, c);
    P->arena_bytes = c.off;
    err = cudaMalloc(&P->arena, P->arena_bytes);
    if (err != cudaSuccess) {
        set_error("cudaMalloc(%zu) failed: %s", P->arena_bytes, cudaGetErrorString(err));
        cudaGetLastError();
        delete P;
        return PIC_POISSON_ENOMEM;
    }
    c = Carver{(char *)P->arena, 0};
    carve(*P, c);
    err = cudaMallocHost(&P->hctrl_out, sizeof(Ctrl));
    if (err == cudaSuccess) err = cudaMallocHost(&P->hsum, 8 * sizeof(double));
    if (err != cudaSuccess) {
        set_error("cudaMallocHost failed: %s", cudaGetErrorString(err));
        pic_poisson_destroy(P);
        return PIC_POISSON_ENOMEM;
    }
    rc = upload(*P);
    if (rc) {
        pic_poisson_destroy(P);
        return rc;
    }
    *out = P;
    return PIC_POISSON_OK;
}

int pic_poisson_plan(const pic_poisson_desc *desc, void *stream, pic_poisson_plan_t *out) {
    return pic_poisson_plan_batch(desc, 1, stream, out);
}

int pic_poisson_set_stream(pic_poisson_plan_t plan, void *stream) {
    int rc = plan_enter(plan);
    if (rc) return rc;
    plan->stream = (cudaStream_t)stream;
    return PIC_POISSON_OK;
}

int pic_poisson_destroy(pic_poisson_plan_t plan) {
    if (!plan) return PIC_POISSON_OK;
    cudaSetDevice(plan->device);
    if (plan->stream) cudaStreamSynchronize(plan->stream);
    else cudaDeviceSynchronize();
    for (int v = 0; v < 2; ++v) {
        if (plan->gexec[v]) cudaGraphExecDestroy(plan->gexec[v]);
        if (plan->graph[v]) cudaGraphDestroy(plan->graph[v]);
    }
    if (plan->cap0) cudaStreamDestroy(plan->cap0);
    if (plan->cap1) cudaStreamDestroy(plan->cap1);
    for (cudaEvent_t e : plan->evs) cudaEventDestroy(e);
    if (plan->arena) cudaFree(plan->arena);
    if (plan->hctrl_out) cudaFreeHost(plan->hctrl_out);
    if (plan->hsum) cudaFreeHost(plan->hsum);
    if (plan->stage_rho) cudaFree(plan->stage_rho);
    if (plan->stage_phi) cudaFree(plan->stage_phi);
    delete plan;
    return PIC_POISSON_OK;
}

}  // extern "C"
