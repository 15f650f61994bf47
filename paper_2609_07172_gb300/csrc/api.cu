// C-ABI entry points, plan construction and the V-cycle driver.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <limits>
#include <new>

#include "internal.h"

namespace pp {

static thread_local char g_err[512];

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
}
void clear_error() { g_err[0] = 0; }

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr double kEps0 = 8.8541878128e-12;   // F/m, CODATA 2018
constexpr int kMaxNtheta = 256;
constexpr int kMaxCoarseCells = 4096;
constexpr int kMaxCoarseNz = 64;

// ---------------------------------------------------------------- descriptor
int resolve(const pic_poisson_desc *in, pic_poisson_desc *d) {
    if (!in) {
        set_error("desc is NULL");
        return PIC_POISSON_EINVAL;
    }
    *d = *in;
    if (d->theta_span <= 0) d->theta_span = 2.0 * kPi;
    if (d->eps0 <= 0) d->eps0 = kEps0;
    if (d->max_cycles <= 0) d->max_cycles = 200;
    if (d->pre_sweeps < 0) d->pre_sweeps = 2;
    if (d->post_sweeps < 0) d->post_sweeps = 2;
    if (d->inner_cycles <= 0) d->inner_cycles = 2;
    if (d->nr < 1 || d->nz < 1) {
        set_error("nr and nz must be >= 1 (got %d, %d)", d->nr, d->nz);
        return PIC_POISSON_EINVAL;
    }
    if (d->ntheta < 2 || d->ntheta > kMaxNtheta || (d->ntheta & (d->ntheta - 1))) {
        set_error("ntheta must be a power of two in [2, %d] (got %d)", kMaxNtheta, d->ntheta);
        return PIC_POISSON_EINVAL;
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
    if (d->pre_sweeps + d->post_sweeps == 0) {
        set_error("pre_sweeps + post_sweeps must be positive");
        return PIC_POISSON_EINVAL;
    }
    const double n = (double)d->nr * d->nz * (d->ntheta / 2 + 1);
    if (n > 2.0e9) {
        set_error("too many mode entries (nr*nz*(ntheta/2+1) = %.0f > 2e9)", n);
        return PIC_POISSON_EINVAL;
    }
    return PIC_POISSON_OK;
}

// 2:1 coarsening while both counts are even and at least 8.
int hierarchy(const pic_poisson_desc &d, int *nr, int *nz, int *levels) {
    int L = 1, r = d.nr, z = d.nz;
    nr[0] = r;
    nz[0] = z;
    while (L < PIC_POISSON_MAX_LEVELS && r % 2 == 0 && z % 2 == 0 && r >= 8 && z >= 8) {
        r /= 2;
        z /= 2;
        nr[L] = r;
        nz[L] = z;
        ++L;
    }
    *levels = L;
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
// dirichlet_face_conductances, mode_mass_coefficient).
void build_level(const pic_poisson_desc &d, int nr, int nz, int nm, LevelHost &h) {
    h.nr = nr;
    h.nz = nz;
    h.r0 = d.r_in;
    h.z0 = d.z0;
    h.dr = (d.r_out - d.r_in) / nr;
    h.dz = (d.z1 - d.z0) / nz;
    const double dr = h.dr, dz = h.dz;
    h.cw.assign(nr, 0.0);
    h.ce.assign(nr, 0.0);
    h.cz.assign(nr, 0.0);
    h.d0r.assign(nr, 0.0);
    h.mu.assign(nr, 0.0);
    for (int i = 0; i < nr; ++i) {
        const double rm = d.r_in + i * dr, rp = d.r_in + (i + 1) * dr, rc = d.r_in + (i + 0.5) * dr;
        const double gw = (i > 0) ? rm * dz / dr : rm * dz / (0.5 * dr);
        const double ge = (i < nr - 1) ? rp * dz / dr : rp * dz / (0.5 * dr);
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
                h.diag[t] = dg;
                h.invd[t] = 1.0 / dg;
                h.hw[t] = h.cw[i] / dg;
                h.he[t] = h.ce[i] / dg;
                h.hz[t] = h.cz[i] / dg;
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

}  // namespace
}  // namespace pp

using namespace pp;

struct pic_poisson_plan_s {
    pic_poisson_desc d{};
    std::vector<double> rin_z, rout_z;
    int device = 0;
    cudaStream_t stream = nullptr;
    int nm = 0, L = 0;
    std::vector<LevelHost> lv;
    void *arena = nullptr;
    size_t arena_bytes = 0;
    std::vector<LevelDev<double>> dl;   // FP64 levels (all levels for FP64; level 0 for mixed)
    std::vector<LevelDev<float>> fl;    // FP32 levels (mixed precision)
    CoarseDev<double> cd{};
    CoarseDev<float> cf{};
    FFTDev fft{};
    double *s0 = nullptr, *bD0 = nullptr;
    double *partials = nullptr;
    int npartials = 0;
    double *dnorm = nullptr;
    double *hnorm = nullptr;            // pinned, 8 doubles
    double *stage_rho = nullptr, *stage_phi = nullptr;
    std::vector<cudaEvent_t> evs;
};

namespace pp {
namespace {

// Lay out (or size) the plan's device workspace.
void carve(pic_poisson_plan_s &P, Carver &c) {
    const int nm = P.nm, L = P.L;
    const bool mixed = P.d.precision == PIC_POISSON_MIXED;
    P.dl.assign(mixed ? 1 : L, LevelDev<double>{});
    P.fl.assign(mixed ? L : 0, LevelDev<float>{});
    for (int l = 0; l < (int)P.dl.size(); ++l) {
        const LevelHost &h = P.lv[l];
        LevelDev<double> &v = P.dl[l];
        v.nr = h.nr; v.nz = h.nz; v.nm = nm; v.ncls = h.ncls;
        const size_t n = (size_t)h.nr * h.nz * nm;
        const size_t nt = (size_t)h.ncls * h.nr * nm;
        v.u = c.take<double2>(n);
        v.b = c.take<double2>(n);
        v.bh = c.take<double2>(n);
        v.cw = c.take<double>(h.nr); v.ce = c.take<double>(h.nr); v.cz = c.take<double>(h.nr);
        v.invd = c.take<double>(nt);
        v.diag = c.take<double>(nt);
        v.hw = c.take<double>(nt); v.he = c.take<double>(nt); v.hz = c.take<double>(nt);
    }
    for (int l = 0; l < (int)P.fl.size(); ++l) {
        const LevelHost &h = P.lv[l];
        LevelDev<float> &v = P.fl[l];
        v.nr = h.nr; v.nz = h.nz; v.nm = nm; v.ncls = h.ncls;
        const size_t n = (size_t)h.nr * h.nz * nm;
        const size_t nt = (size_t)h.ncls * h.nr * nm;
        v.u = c.take<float2>(n);
        v.b = c.take<float2>(n);
        v.bh = c.take<float2>(n);
        v.cw = c.take<float>(h.nr); v.ce = c.take<float>(h.nr); v.cz = c.take<float>(h.nr);
        v.invd = c.take<float>(nt);
        v.diag = c.take<float>(nt);
        v.hw = c.take<float>(nt); v.he = c.take<float>(nt); v.hz = c.take<float>(nt);
    }
    const LevelHost &hc = P.lv[L - 1];
    const size_t nf = (size_t)nm * hc.nz * hc.nr;
    if (!mixed) {
        P.cd.nr = hc.nr; P.cd.nz = hc.nz; P.cd.nm = nm;
        P.cd.V = c.take<double>((size_t)hc.nz * hc.nz);
        P.cd.e = c.take<double>(hc.nr);
        P.cd.piv = c.take<double>(nf);
        P.cd.cpr = c.take<double>(nf);
    } else {
        P.cf.nr = hc.nr; P.cf.nz = hc.nz; P.cf.nm = nm;
        P.cf.V = c.take<float>((size_t)hc.nz * hc.nz);
        P.cf.e = c.take<float>(hc.nr);
        P.cf.piv = c.take<float>(nf);
        P.cf.cpr = c.take<float>(nf);
    }
    const int M = P.d.ntheta / 2;
    P.fft.nt = P.d.ntheta;
    P.fft.tw = (const double *)c.take<double2>(std::max(M / 2, 1));
    P.fft.tw2 = (const double *)c.take<double2>(M + 1);
    P.s0 = c.take<double>(P.lv[0].nr);
    P.bD0 = c.take<double>((size_t)P.lv[0].nr * P.lv[0].nz);
    // partial sums: the largest grid of any reducing launch, twice (residual + rhs norms)
    const LevelHost &h0 = P.lv[0];
    const long fwd_blocks = (long)h0.nz * ((h0.nr + 31) / 32);
    const long res_blocks = ((long)h0.nr * h0.nz * nm + 255) / 256;
    P.npartials = (int)(2 * std::max(fwd_blocks, res_blocks) + 64);
    P.partials = c.take<double>(P.npartials);
    P.dnorm = c.take<double>(8);
}

template <class T> void to_dev(const std::vector<double> &src, const T *dst, std::vector<char> &tmp,
                               cudaStream_t st, cudaError_t &err) {
    if (err != cudaSuccess || src.empty()) return;
    std::vector<T> conv(src.begin(), src.end());
    err = cudaMemcpyAsync((void *)dst, conv.data(), conv.size() * sizeof(T), cudaMemcpyHostToDevice, st);
    if (err == cudaSuccess) err = cudaStreamSynchronize(st);
    (void)tmp;
}

// Coarsest-level factors: axial eigenbasis (closed form for the uniform
// cell-centred Dirichlet operator: V_kj ~ sin(pi (j+1)(k+1/2)/nz), eigenvalue
// 4 sin^2(pi (j+1) / (2 nz))) and the Thomas factorisation of the radial
// tridiagonal system of every (mode, axial eigenvector).
void coarse_factors(const pic_poisson_plan_s &P, std::vector<double> &V, std::vector<double> &e,
                    std::vector<double> &piv, std::vector<double> &cpr) {
    const LevelHost &h = P.lv[P.L - 1];
    const int nr = h.nr, nz = h.nz, nm = P.nm;
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
        const double lm = lambda_m(P.d, m);
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

int upload(pic_poisson_plan_s &P) {
    cudaError_t err = cudaSuccess;
    std::vector<char> tmp;
    const cudaStream_t st = P.stream;
    for (size_t l = 0; l < P.dl.size(); ++l) {
        const LevelHost &h = P.lv[l];
        to_dev(h.cw, P.dl[l].cw, tmp, st, err);
        to_dev(h.ce, P.dl[l].ce, tmp, st, err);
        to_dev(h.cz, P.dl[l].cz, tmp, st, err);
        to_dev(h.invd, P.dl[l].invd, tmp, st, err);
        to_dev(h.diag, P.dl[l].diag, tmp, st, err);
        to_dev(h.hw, P.dl[l].hw, tmp, st, err);
        to_dev(h.he, P.dl[l].he, tmp, st, err);
        to_dev(h.hz, P.dl[l].hz, tmp, st, err);
    }
    for (size_t l = 0; l < P.fl.size(); ++l) {
        const LevelHost &h = P.lv[l];
        to_dev(h.cw, P.fl[l].cw, tmp, st, err);
        to_dev(h.ce, P.fl[l].ce, tmp, st, err);
        to_dev(h.cz, P.fl[l].cz, tmp, st, err);
        to_dev(h.invd, P.fl[l].invd, tmp, st, err);
        to_dev(h.diag, P.fl[l].diag, tmp, st, err);
        to_dev(h.hw, P.fl[l].hw, tmp, st, err);
        to_dev(h.he, P.fl[l].he, tmp, st, err);
        to_dev(h.hz, P.fl[l].hz, tmp, st, err);
    }
    std::vector<double> V, e, piv, cpr;
    coarse_factors(P, V, e, piv, cpr);
    if (P.d.precision == PIC_POISSON_FP64) {
        to_dev(V, P.cd.V, tmp, st, err);
        to_dev(e, P.cd.e, tmp, st, err);
        to_dev(piv, P.cd.piv, tmp, st, err);
        to_dev(cpr, P.cd.cpr, tmp, st, err);
    } else {
        to_dev(V, P.cf.V, tmp, st, err);
        to_dev(e, P.cf.e, tmp, st, err);
        to_dev(piv, P.cf.piv, tmp, st, err);
        to_dev(cpr, P.cf.cpr, tmp, st, err);
    }
    // FFT twiddles
    const int nt = P.d.ntheta, M = nt / 2;
    std::vector<double> tw(2 * std::max(M / 2, 1), 0.0), tw2(2 * (M + 1), 0.0);
    for (int t = 0; t < M / 2; ++t) {
        tw[2 * t] = std::cos(2.0 * kPi * t / M);
        tw[2 * t + 1] = -std::sin(2.0 * kPi * t / M);
    }
    if (M / 2 == 0) tw[0] = 1.0;
    for (int m = 0; m <= M; ++m) {
        tw2[2 * m] = std::cos(2.0 * kPi * m / nt);
        tw2[2 * m + 1] = -std::sin(2.0 * kPi * m / nt);
    }
    to_dev(tw, P.fft.tw, tmp, st, err);
    to_dev(tw2, P.fft.tw2, tmp, st, err);
    // level-0 right-hand-side factors: s_i (Eq. mode_rhs) and b^D (Eq. boundary_rhs_appendix)
    const LevelHost &h = P.lv[0];
    std::vector<double> s(h.nr), bD((size_t)h.nr * h.nz, 0.0);
    for (int i = 0; i < h.nr; ++i) {
        const double rc = P.d.r_in + (i + 0.5) * h.dr;
        s[i] = rc * h.dr * h.dz / P.d.eps0;
    }
    for (int k = 0; k < h.nz; ++k)
        for (int i = 0; i < h.nr; ++i) {
            double v = 0.0;
            const double rm = P.d.r_in + i * h.dr, rp = P.d.r_in + (i + 1) * h.dr;
            if (i == 0) v += rm * h.dz / (0.5 * h.dr) * wall_rin(P.d, k);
            if (i == h.nr - 1) v += rp * h.dz / (0.5 * h.dr) * wall_rout(P.d, k);
            if (k == 0) v += 2.0 * h.cz[i] * P.d.phi_z0;
            if (k == h.nz - 1) v += 2.0 * h.cz[i] * P.d.phi_z1;
            bD[(size_t)k * h.nr + i] = v;
        }
    to_dev(s, P.s0, tmp, st, err);
    to_dev(bD, P.bD0, tmp, st, err);
    if (err != cudaSuccess) {
        set_error("uploading plan tables failed: %s", cudaGetErrorString(err));
        return PIC_POISSON_ECUDA;
    }
    return PIC_POISSON_OK;
}

int setup_plan(pic_poisson_plan_s &P, const pic_poisson_desc &d) {
    P.d = d;
    if (d.phi_r_in_z) {
        P.rin_z.assign(d.phi_r_in_z, d.phi_r_in_z + d.nz);
        P.d.phi_r_in_z = P.rin_z.data();
    }
    if (d.phi_r_out_z) {
        P.rout_z.assign(d.phi_r_out_z, d.phi_r_out_z + d.nz);
        P.d.phi_r_out_z = P.rout_z.data();
    }
    int nr[PIC_POISSON_MAX_LEVELS], nz[PIC_POISSON_MAX_LEVELS];
    int rc = hierarchy(P.d, nr, nz, &P.L);
    if (rc) return rc;
    P.nm = d.ntheta / 2 + 1;
    P.lv.resize(P.L);
    for (int l = 0; l < P.L; ++l) build_level(P.d, nr[l], nz[l], P.nm, P.lv[l]);
    return PIC_POISSON_OK;
}

// ---------------------------------------------------------------- launch bookkeeping
struct Runner {
    pic_poisson_plan_s &P;
    pic_poisson_info *info;
    bool prof;
    int nev = 0;
    std::vector<int> phase;
    int launches[PIC_POISSON_NPHASE] = {0};

    Runner(pic_poisson_plan_s &p, pic_poisson_info *i) : P(p), info(i), prof(p.d.flags & PIC_POISSON_PROFILE) {}

    cudaError_t pre() {
        if (!prof) return cudaSuccess;
        while ((int)P.evs.size() < 2 * (nev + 1)) {
            cudaEvent_t e;
            cudaError_t err = cudaEventCreate(&e);
            if (err != cudaSuccess) return err;
            P.evs.push_back(e);
        }
        return cudaEventRecord(P.evs[2 * nev], P.stream);
    }
    cudaError_t post(int ph) {
        launches[ph]++;
        if (!prof) return cudaSuccess;
        phase.push_back(ph);
        return cudaEventRecord(P.evs[2 * nev++ + 1], P.stream);
    }
    double bytes[PIC_POISSON_NPHASE] = {0}, flops[PIC_POISSON_NPHASE] = {0};
    // algorithmic traffic and arithmetic of the launch just made
    void account(int ph, double b, double f) {
        bytes[ph] += b;
        flops[ph] += f;
    }
    int finish() {
        if (!info) return PIC_POISSON_OK;
        int tot = 0;
        for (int p = 0; p < PIC_POISSON_NPHASE; ++p) {
            info->launches_phase[p] += launches[p];
            info->bytes_phase[p] += bytes[p];
            info->flops_phase[p] += flops[p];
            tot += launches[p];
        }
        info->launches += tot;
        if (!prof) return PIC_POISSON_OK;
        PP_CUDA(cudaStreamSynchronize(P.stream));
        for (int e = 0; e < nev; ++e) {
            float ms = 0.f;
            PP_CUDA(cudaEventElapsedTime(&ms, P.evs[2 * e], P.evs[2 * e + 1]));
            info->ms_phase[phase[e]] += ms;
        }
        return PIC_POISSON_OK;
    }
};

#define RUN(R, PH, EXPR)                                                                      \
    do {                                                                                      \
        cudaError_t e0_ = (R).pre();                                                          \
        cudaError_t e1_ = (e0_ == cudaSuccess) ? (cudaError_t)(EXPR) : e0_;                   \
        cudaError_t e2_ = (e1_ == cudaSuccess) ? (R).post(PH) : e1_;                          \
        if (e2_ != cudaSuccess) {                                                             \
            set_error("%s failed: %s", #EXPR, cudaGetErrorString(e2_));                       \
            return PIC_POISSON_ECUDA;                                                         \
        }                                                                                     \
    } while (0)

int read_norms(pic_poisson_plan_s &P, int count, double *out) {
    PP_CUDA(cudaMemcpyAsync(P.hnorm, P.dnorm, count * sizeof(double), cudaMemcpyDeviceToHost, P.stream));
    PP_CUDA(cudaStreamSynchronize(P.stream));
    for (int i = 0; i < count; ++i) out[i] = P.hnorm[i];
    return PIC_POISSON_OK;
}

// `sweeps` red-black sweeps on one level.  skip_first_red: the first sweep
// starts at its black half, because the kernel that initialised the level
// already performed the red half-sweep from a zero iterate.
// Per-entry models: a complex entry of a level is
// sizeof(V2<T>) bytes; FMA = 2 flops.
template <class T> double vbytes(const LevelDev<T> &L) { return (double)L.nr * L.nz * L.nm * sizeof(V2<T>); }
template <class T> double ventries(const LevelDev<T> &L) { return (double)L.nr * L.nz * L.nm; }

// Half-sweep: read the other colour of u and this colour of b_hat, write this
// colour of u (1.5 V); 4 operations (7 flops) per real component.
template <class T>
int smooth_level(Runner &R, const LevelDev<T> &L, int sweeps, bool skip_first_red, int phase) {
    for (int s = 0; s < sweeps; ++s) {
        for (int color = (s == 0 && skip_first_red) ? 1 : 0; color < 2; ++color) {
            RUN(R, phase, launch_smooth(L, color, R.P.stream));
            R.account(phase, 1.5 * vbytes(L), 14.0 * 0.5 * ventries(L));
        }
    }
    return PIC_POISSON_OK;
}

// Residual + restriction from fine level F into C: reads u (V_F) and b of the
// evaluated cells, writes coarse b (and b_hat, u when init > 0); 18 flops per
// evaluated complex entry (+4 with norms), 2-4 per coarse entry.
template <class T>
void account_restrict(Runner &R, const LevelDev<T> &F, bool red_only, int init, bool norms) {
    const double frac = red_only ? 0.5 : 1.0;
    const double b = vbytes(F) * (1.0 + frac) + 0.25 * vbytes(F) * (init > 0 ? 3.0 : 1.0);
    const double f = frac * ventries(F) * (18.0 + (norms ? 4.0 : 0.0)) + 0.25 * ventries(F) * (init > 0 ? 4.0 : 2.0);
    R.account(PIC_POISSON_PHASE_RESTRICT, b, f);
}

// Prolongation + correction: reads the coarse correction (V_F / 4), reads and
// writes u of the corrected cells; 16 flops per corrected complex entry.
template <class T>
void account_prolong(Runner &R, const LevelDev<T> &F, bool black_only) {
    const double frac = black_only ? 0.5 : 1.0;
    R.account(PIC_POISSON_PHASE_PROLONG, 0.25 * vbytes(F) + 2.0 * frac * vbytes(F), 16.0 * frac * ventries(F));
}

// Separable coarsest solve: reads b, writes u, reads the Thomas factors;
// 2 dense axial transforms (4 nz flops per real component each) + Thomas.
template <class T>
void account_coarse(Runner &R, const LevelDev<T> &L) {
    const double fac = 2.0 * L.nm * L.nz * L.nr * sizeof(T);
    R.account(PIC_POISSON_PHASE_COARSE, 2.0 * vbytes(L) + fac, ventries(L) * (16.0 * L.nz + 20.0));
}

// Batched real FFT of one length-nt column: ~5 (M/2) log2 M * 2 flops for the
// complex length-M transform plus ~14 per unpacked mode (M = nt / 2).
double fft_flops(int nt) {
    const double M = nt / 2;
    return 5.0 * M * std::log2(std::max(M, 1.0)) + 14.0 * (M + 1);
}

// What the restriction from level l writes into level l+1 of an L-level
// hierarchy: only b into the coarsest level (solved directly); otherwise b_hat
// and the iterate, which is the first red half-sweep from zero when the
// coarse level is pre-smoothed.
int restrict_init(int l, int L, int pre) { return (l + 1 == L - 1) ? 0 : (pre > 0 ? 2 : 1); }

// Coarse-grid correction below level `top`: level top+1 holds the restricted
// residual and its initialised iterate; returns with the correction
// prolongated into level `top` and post-smoothed there.
template <class T>
int descend_ascend(Runner &R, std::vector<LevelDev<T>> &lv, const CoarseDev<T> &cd, int top) {
    pic_poisson_plan_s &P = R.P;
    const int L = (int)lv.size(), pre = P.d.pre_sweeps, post = P.d.post_sweeps;
    for (int l = top + 1; l < L - 1; ++l) {
        int rc = smooth_level(R, lv[l], pre, pre > 0, PIC_POISSON_PHASE_SMOOTH_COARSE);
        if (rc) return rc;
        RUN(R, PIC_POISSON_PHASE_RESTRICT,
            launch_residual_restrict(lv[l], lv[l + 1], P.d.ntheta, pre > 0, restrict_init(l, L, pre),
                                     (double *)nullptr, (int *)nullptr, P.stream));
        account_restrict(R, lv[l], pre > 0, restrict_init(l, L, pre), false);
    }
    RUN(R, PIC_POISSON_PHASE_COARSE, launch_coarse(lv[L - 1], cd, P.stream));
    account_coarse(R, lv[L - 1]);
    for (int l = L - 2; l >= top; --l) {
        RUN(R, PIC_POISSON_PHASE_PROLONG, launch_prolong(lv[l], lv[l + 1], post > 0, P.stream));
        account_prolong(R, lv[l], post > 0);
        int rc = smooth_level(R, lv[l], post, false,
                              l == 0 ? PIC_POISSON_PHASE_SMOOTH : PIC_POISSON_PHASE_SMOOTH_COARSE);
        if (rc) return rc;
    }
    return PIC_POISSON_OK;
}

struct StopRule {
    double tol, best = std::numeric_limits<double>::infinity();
    int stall = 0;
    // returns 1 when converged (tol met, or floor reached when tol <= 0)
    int done(double rel) {
        if (tol > 0) return rel <= tol;
        if (rel < 0.5 * best) {
            best = rel;
            stall = 0;
            return 0;
        }
        best = std::min(best, rel);
        return ++stall >= 2;
    }
};

// FP64 V-cycles.  The convergence test reads the residual that the fused
// residual/restriction kernel produces after pre-smoothing, i.e. of the
// current iterate; a converged iterate is returned as is.
int mg_fp64(Runner &R, double tol, double bnorm2, pic_poisson_info *info, int *status) {
    pic_poisson_plan_s &P = R.P;
    LevelDev<double> &F = P.dl[0];
    const int pre = P.d.pre_sweeps;
    StopRule stop{tol};
    double rel = 1.0;
    int cycles = 0, nb = 0;
    if (P.L == 1) {
        RUN(R, PIC_POISSON_PHASE_COARSE, launch_coarse(F, P.cd, P.stream));
        account_coarse(R, F);
        RUN(R, PIC_POISSON_PHASE_RESTRICT, launch_residual(F, (double2 *)nullptr, P.d.ntheta, P.partials, &nb, P.stream));
        R.account(PIC_POISSON_PHASE_RESTRICT, 2.0 * vbytes(F), 22.0 * ventries(F));
        RUN(R, PIC_POISSON_PHASE_NORM, launch_sum(P.partials, nb, P.dnorm + 1, P.stream));
        double nn[2];
        int rc = read_norms(P, 2, nn);
        if (rc) return rc;
        rel = std::sqrt(nn[1] / bnorm2);
        cycles = 1;
        *status = !std::isfinite(rel) ? PIC_POISSON_ENONFINITE
                                       : ((tol > 0 && rel > tol) ? PIC_POISSON_ENOTCONVERGED : PIC_POISSON_OK);
    } else {
        for (;;) {
            int rc = smooth_level(R, F, pre, false, PIC_POISSON_PHASE_SMOOTH);
            if (rc) return rc;
            RUN(R, PIC_POISSON_PHASE_RESTRICT,
                launch_residual_restrict(F, P.dl[1], P.d.ntheta, pre > 0, restrict_init(0, P.L, pre), P.partials,
                                         &nb, P.stream));
            account_restrict(R, F, pre > 0, restrict_init(0, P.L, pre), true);
            RUN(R, PIC_POISSON_PHASE_NORM, launch_sum(P.partials, nb, P.dnorm + 1, P.stream));
            double nn[2];
            rc = read_norms(P, 2, nn);
            if (rc) return rc;
            rel = std::sqrt(nn[1] / bnorm2);
            if (!std::isfinite(rel)) {
                *status = PIC_POISSON_ENONFINITE;
                break;
            }
            if (stop.done(rel)) {
                *status = PIC_POISSON_OK;
                break;
            }
            if (cycles >= P.d.max_cycles) {
                *status = PIC_POISSON_ENOTCONVERGED;
                break;
            }
            rc = descend_ascend(R, P.dl, P.cd, 0);
            if (rc) return rc;
            ++cycles;
        }
    }
    if (info) {
        info->cycles = cycles;
        info->rel_res = rel;
    }
    return PIC_POISSON_OK;
}

// Power of two closest to 1 / sqrt(mean square): scales the FP32 correction
// problem to O(1) values exactly (no rounding from the scale itself).
double pow2_scale(double sumsq, double count) {
    const double rms = std::sqrt(sumsq / std::max(count, 1.0));
    if (!(rms > 0) || !std::isfinite(rms)) return 1.0;
    int ex = 0;
    std::frexp(rms, &ex);
    return std::ldexp(1.0, -ex);
}

// Mixed precision: FP64 defect correction x <- x + A^{-1}_FP32 (b - A x).
// Each outer step forms the FP64 residual of the current iterate (the
// convergence test), solves the correction equation approximately with
// inner_cycles FP32 V-cycles on the FP32 hierarchy, and adds it in FP64.
int mg_mixed(Runner &R, double tol, double bnorm2, pic_poisson_info *info, int *status) {
    pic_poisson_plan_s &P = R.P;
    LevelDev<double> &D = P.dl[0];
    std::vector<LevelDev<float>> &S = P.fl;
    const int pre = P.d.pre_sweeps, L = P.L;
    const double count = (double)D.nr * D.nz * P.d.ntheta;
    StopRule stop{tol};
    double rel = 1.0, sigma = pow2_scale(bnorm2, count);
    int cycles = 0, outer = 0, nb = 0;
    for (;;) {
        RUN(R, PIC_POISSON_PHASE_DEFECT,
            launch_defect(D, S[0], sigma, P.d.ntheta, L > 1 && pre > 0, P.partials, &nb, P.stream));
        R.account(PIC_POISSON_PHASE_DEFECT, 2.0 * vbytes(D) + 3.0 * vbytes(S[0]), 26.0 * ventries(D));
        RUN(R, PIC_POISSON_PHASE_NORM, launch_sum(P.partials, nb, P.dnorm + 1, P.stream));
        double nn[2];
        int rc = read_norms(P, 2, nn);
        if (rc) return rc;
        rel = std::sqrt(nn[1] / bnorm2);
        if (!std::isfinite(rel)) {
            *status = PIC_POISSON_ENONFINITE;
            break;
        }
        if (stop.done(rel)) {
            *status = PIC_POISSON_OK;
            break;
        }
        if (cycles >= P.d.max_cycles) {
            *status = PIC_POISSON_ENOTCONVERGED;
            break;
        }
        if (L == 1) {
            RUN(R, PIC_POISSON_PHASE_COARSE, launch_coarse(S[0], P.cf, P.stream));
            account_coarse(R, S[0]);
            ++cycles;
        } else {
            for (int c = 0; c < P.d.inner_cycles; ++c) {
                rc = smooth_level(R, S[0], pre, c == 0 && pre > 0, PIC_POISSON_PHASE_SMOOTH);
                if (rc) return rc;
                RUN(R, PIC_POISSON_PHASE_RESTRICT,
                    launch_residual_restrict(S[0], S[1], P.d.ntheta, pre > 0, restrict_init(0, L, pre),
                                             (double *)nullptr, (int *)nullptr, P.stream));
                account_restrict(R, S[0], pre > 0, restrict_init(0, L, pre), false);
                rc = descend_ascend(R, S, P.cf, 0);
                if (rc) return rc;
                ++cycles;
            }
        }
        RUN(R, PIC_POISSON_PHASE_DEFECT, launch_update(D, S[0], 1.0 / sigma, P.stream));
        R.account(PIC_POISSON_PHASE_DEFECT, 2.0 * vbytes(D) + vbytes(S[0]), 4.0 * ventries(D));
        ++outer;
        sigma = pow2_scale(nn[1] / 2.0, count);
    }
    if (info) {
        info->cycles = cycles;
        info->outer_iterations = outer;
        info->rel_res = rel;
    }
    return PIC_POISSON_OK;
}

int solve_dev(pic_poisson_plan_s &P, const double *rho, double *phi, double tol, pic_poisson_info *info) {
    Runner R(P, info);
    const pic_poisson_desc &d = P.d;
    const LevelHost &h0 = P.lv[0];
    LevelDev<double> &F = P.dl[0];
    const bool mixed = d.precision == PIC_POISSON_MIXED;
    const size_t n0 = (size_t)h0.nr * h0.nz * P.nm;
    int nb = 0;
    RUN(R, PIC_POISSON_PHASE_FORWARD,
        launch_forward(rho, F.b, h0.nr, d.ntheta, h0.nz, P.fft, P.s0, P.bD0, P.partials, &nb,
                       mixed ? (double2 *)nullptr : F.bh, F.invd, F.ncls, P.stream));
    const double X = (double)h0.nr * h0.nz * d.ntheta * sizeof(double);
    const double columns = (double)h0.nr * h0.nz;
    R.account(PIC_POISSON_PHASE_FORWARD, X + (mixed ? 1.0 : 2.0) * vbytes(F), columns * fft_flops(d.ntheta));
    RUN(R, PIC_POISSON_PHASE_NORM, launch_sum(P.partials, nb, P.dnorm, P.stream));
    const bool guess = d.flags & PIC_POISSON_USE_INITIAL_GUESS;
    if (guess) {
        RUN(R, PIC_POISSON_PHASE_FORWARD,
            launch_forward(phi, F.u, h0.nr, d.ntheta, h0.nz, P.fft, (const double *)nullptr,
                           (const double *)nullptr, (double *)nullptr, (int *)nullptr, (double2 *)nullptr,
                           (const double *)nullptr, 0, P.stream));
        R.account(PIC_POISSON_PHASE_FORWARD, X + vbytes(F), columns * fft_flops(d.ntheta));
    } else {
        PP_CUDA(cudaMemsetAsync(F.u, 0, n0 * sizeof(double2), P.stream));
    }
    double nn[1];
    int rc = read_norms(P, 1, nn);
    if (rc) return rc;
    const double bnorm2 = nn[0];
    int status = PIC_POISSON_OK;
    if (info) info->rel_res0 = 1.0;
    if (!std::isfinite(bnorm2)) {
        status = PIC_POISSON_ENONFINITE;
        if (info) info->rel_res = std::numeric_limits<double>::quiet_NaN();
    } else if (bnorm2 == 0.0) {
        PP_CUDA(cudaMemsetAsync(F.u, 0, n0 * sizeof(double2), P.stream));
        if (info) info->rel_res = 0.0;
    } else {
        if (guess) {
            RUN(R, PIC_POISSON_PHASE_RESTRICT,
                launch_residual(F, (double2 *)nullptr, d.ntheta, P.partials, &nb, P.stream));
            R.account(PIC_POISSON_PHASE_RESTRICT, 2.0 * vbytes(F), 22.0 * ventries(F));
            RUN(R, PIC_POISSON_PHASE_NORM, launch_sum(P.partials, nb, P.dnorm + 1, P.stream));
            double r2[2];
            rc = read_norms(P, 2, r2);
            if (rc) return rc;
            if (info) info->rel_res0 = std::sqrt(r2[1] / bnorm2);
        }
        rc = mixed ? mg_mixed(R, tol, bnorm2, info, &status) : mg_fp64(R, tol, bnorm2, info, &status);
        if (rc) return rc;
    }
    if (status != PIC_POISSON_ENONFINITE)
    {
        RUN(R, PIC_POISSON_PHASE_INVERSE, launch_inverse(F.u, phi, h0.nr, d.ntheta, h0.nz, P.fft, P.stream));
        R.account(PIC_POISSON_PHASE_INVERSE, X + vbytes(F), columns * fft_flops(d.ntheta));
    }
    rc = R.finish();
    if (rc) return rc;
    if (status == PIC_POISSON_ENONFINITE) set_error("non-finite right-hand side or residual");
    if (status == PIC_POISSON_ENOTCONVERGED) set_error("tolerance not reached in max_cycles");
    return status;
}

int enter(pic_poisson_plan_s *P) {
    clear_error();
    if (!P) {
        set_error("plan is NULL");
        return PIC_POISSON_EINVAL;
    }
    PP_CUDA(cudaSetDevice(P->device));
    return PIC_POISSON_OK;
}

}  // namespace
}  // namespace pp

// ====================================================================== C ABI
extern "C" {

const char *pic_poisson_last_error(void) { return pp::g_err; }

int pic_poisson_query(const pic_poisson_desc *desc, pic_poisson_layout *out) {
    clear_error();
    pic_poisson_desc d;
    int rc = resolve(desc, &d);
    if (rc) return rc;
    pic_poisson_plan_s P;
    rc = setup_plan(P, d);
    if (rc) return rc;
    if (out) {
        memset(out, 0, sizeof *out);
        out->levels = P.L;
        for (int l = 0; l < P.L; ++l) {
            out->nr[l] = P.lv[l].nr;
            out->nz[l] = P.lv[l].nz;
        }
        out->n_modes = P.nm;
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
    build_level(d, d.nr, d.nz, 1, h);
    const bool dw = i == 0, de = i == d.nr - 1, ds = k == 0, dn = k == d.nz - 1;
    const double rm = d.r_in + i * h.dr, rp = d.r_in + (i + 1) * h.dr;
    out[0] = dw ? rm * h.dz / (0.5 * h.dr) : h.cw[i];
    out[1] = de ? rp * h.dz / (0.5 * h.dr) : h.ce[i];
    out[2] = ds ? 2.0 * h.cz[i] : h.cz[i];
    out[3] = dn ? 2.0 * h.cz[i] : h.cz[i];
    out[4] = dw; out[5] = de; out[6] = ds; out[7] = dn;
    out[8] = h.mu[i];
    const double rc_ = d.r_in + (i + 0.5) * h.dr;
    out[9] = rc_ * h.dr * h.dz / d.eps0;
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

int pic_poisson_plan(const pic_poisson_desc *desc, void *stream, pic_poisson_plan_t *out) {
    clear_error();
    if (!out) {
        set_error("out is NULL");
        return PIC_POISSON_EINVAL;
    }
    *out = nullptr;
    pic_poisson_desc d;
    int rc = resolve(desc, &d);
    if (rc) return rc;
    pic_poisson_plan_s *P = new (std::nothrow) pic_poisson_plan_s;
    if (!P) {
        set_error("host allocation failed");
        return PIC_POISSON_ENOMEM;
    }
    rc = setup_plan(*P, d);
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
    err = cudaMallocHost(&P->hnorm, 8 * sizeof(double));
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

int pic_poisson_set_stream(pic_poisson_plan_t plan, void *stream) {
    int rc = enter(plan);
    if (rc) return rc;
    plan->stream = (cudaStream_t)stream;
    return PIC_POISSON_OK;
}

int pic_poisson_solve(pic_poisson_plan_t plan, const double *rho_dev, double *phi_dev, double tol,
                      pic_poisson_info *info) {
    int rc = enter(plan);
    if (rc) return rc;
    if (!rho_dev || !phi_dev || (const void *)rho_dev == (const void *)phi_dev) {
        set_error("rho_dev and phi_dev must be distinct non-NULL device pointers");
        return PIC_POISSON_EINVAL;
    }
    if (std::isnan(tol)) {
        set_error("tol is NaN");
        return PIC_POISSON_EINVAL;
    }
    if (info) memset(info, 0, sizeof *info);
    rc = solve_dev(*plan, rho_dev, phi_dev, tol, info);
    if (info) info->status = rc;
    return rc;
}

int pic_poisson_solve_host(pic_poisson_plan_t plan, const double *rho_host, double *phi_host, double tol,
                           pic_poisson_info *info) {
    int rc = enter(plan);
    if (rc) return rc;
    if (!rho_host || !phi_host) {
        set_error("rho_host and phi_host must be non-NULL");
        return PIC_POISSON_EINVAL;
    }
    pic_poisson_plan_s &P = *plan;
    const size_t bytes = (size_t)P.d.nr * P.d.ntheta * P.d.nz * sizeof(double);
    if (!P.stage_rho) {
        cudaError_t err = cudaMalloc(&P.stage_rho, bytes);
        if (err == cudaSuccess) err = cudaMalloc(&P.stage_phi, bytes);
        if (err != cudaSuccess) {
            cudaGetLastError();
            set_error("staging allocation failed: %s", cudaGetErrorString(err));
            return PIC_POISSON_ENOMEM;
        }
    }
    PP_CUDA(cudaMemcpyAsync(P.stage_rho, rho_host, bytes, cudaMemcpyHostToDevice, P.stream));
    if (P.d.flags & PIC_POISSON_USE_INITIAL_GUESS)
        PP_CUDA(cudaMemcpyAsync(P.stage_phi, phi_host, bytes, cudaMemcpyHostToDevice, P.stream));
    if (info) memset(info, 0, sizeof *info);
    rc = solve_dev(P, P.stage_rho, P.stage_phi, tol, info);
    if (info) info->status = rc;
    if (rc == PIC_POISSON_OK || rc == PIC_POISSON_ENOTCONVERGED) {
        PP_CUDA(cudaMemcpyAsync(phi_host, P.stage_phi, bytes, cudaMemcpyDeviceToHost, P.stream));
        PP_CUDA(cudaStreamSynchronize(P.stream));
    }
    return rc;
}

int pic_poisson_forward(pic_poisson_plan_t plan, const double *rho_dev, double *bhat_dev) {
    int rc = enter(plan);
    if (rc) return rc;
    if (!rho_dev || !bhat_dev) {
        set_error("NULL pointer");
        return PIC_POISSON_EINVAL;
    }
    const pic_poisson_plan_s &P = *plan;
    cudaError_t err = launch_forward(rho_dev, (double2 *)bhat_dev, P.d.nr, P.d.ntheta, P.d.nz, P.fft, P.s0,
                                     P.bD0, nullptr, nullptr, nullptr, nullptr, 0, P.stream);
    if (err != cudaSuccess) {
        set_error("forward transform launch failed: %s", cudaGetErrorString(err));
        return PIC_POISSON_ECUDA;
    }
    return PIC_POISSON_OK;
}

int pic_poisson_inverse(pic_poisson_plan_t plan, const double *phihat_dev, double *phi_dev) {
    int rc = enter(plan);
    if (rc) return rc;
    if (!phihat_dev || !phi_dev) {
        set_error("NULL pointer");
        return PIC_POISSON_EINVAL;
    }
    const pic_poisson_plan_s &P = *plan;
    cudaError_t err = launch_inverse((const double2 *)phihat_dev, phi_dev, P.d.nr, P.d.ntheta, P.d.nz, P.fft,
                                     P.stream);
    if (err != cudaSuccess) {
        set_error("inverse transform launch failed: %s", cudaGetErrorString(err));
        return PIC_POISSON_ECUDA;
    }
    return PIC_POISSON_OK;
}

int pic_poisson_mode_residual(pic_poisson_plan_t plan, const double *uhat_dev, const double *bhat_dev,
                              double *rhat_dev, double *rel_res) {
    int rc = enter(plan);
    if (rc) return rc;
    if (!uhat_dev || !bhat_dev) {
        set_error("NULL pointer");
        return PIC_POISSON_EINVAL;
    }
    pic_poisson_plan_s &P = *plan;
    LevelDev<double> L = P.dl.empty() ? LevelDev<double>{} : P.dl[0];
    L.u = (double2 *)uhat_dev;
    L.b = (double2 *)bhat_dev;
    int nb = 0;
    cudaError_t err = launch_residual(L, (double2 *)rhat_dev, P.d.ntheta, rel_res ? P.partials : nullptr, &nb,
                                      P.stream);
    if (err == cudaSuccess && rel_res) err = launch_sum(P.partials, nb, P.dnorm + 2, P.stream);
    if (err == cudaSuccess && rel_res) err = launch_sum(P.partials + nb, nb, P.dnorm + 3, P.stream);
    if (err != cudaSuccess) {
        set_error("residual launch failed: %s", cudaGetErrorString(err));
        return PIC_POISSON_ECUDA;
    }
    if (rel_res) {
        double nn[4];
        rc = read_norms(P, 4, nn);
        if (rc) return rc;
        *rel_res = nn[3] > 0 ? std::sqrt(nn[2] / nn[3]) : std::sqrt(nn[2]);
    }
    return PIC_POISSON_OK;
}

int pic_poisson_destroy(pic_poisson_plan_t plan) {
    if (!plan) return PIC_POISSON_OK;
    cudaSetDevice(plan->device);
    if (plan->stream) cudaStreamSynchronize(plan->stream);
    else cudaDeviceSynchronize();
    for (cudaEvent_t e : plan->evs) cudaEventDestroy(e);
    if (plan->arena) cudaFree(plan->arena);
    if (plan->hnorm) cudaFreeHost(plan->hnorm);
    if (plan->stage_rho) cudaFree(plan->stage_rho);
    if (plan->stage_phi) cudaFree(plan->stage_phi);
    delete plan;
    return PIC_POISSON_OK;
}

int pic_poisson_measure_fma_peaks(void *stream, double *fp64_gflops, double *fp32_gflops) {
    clear_error();
    if (!fp64_gflops || !fp32_gflops) {
        set_error("NULL output pointer");
        return PIC_POISSON_EINVAL;
    }
    cudaError_t err = measure_fma((cudaStream_t)stream, fp64_gflops, fp32_gflops);
    if (err != cudaSuccess) {
        set_error("FMA probe failed: %s", cudaGetErrorString(err));
        return PIC_POISSON_ECUDA;
    }
    return PIC_POISSON_OK;
}

}  // extern "C"
