// The solve: launch sequences of one solve (prologue, convergence-loop body,
// epilogue), driven either by a host loop that reads the device-side
// convergence flag after each test or by one CUDA graph whose while-node
// repeats the body until the check kernel clears its condition.  Also the
// stage entry points (forward / inverse transform, mode residual).
#include <algorithm>
#include <cstddef>
#include <cmath>
#include <cstring>
#include <functional>

#include "plan.h"

namespace pp {
namespace {

// ---------------------------------------------------------------- launch bookkeeping
struct Runner {
    pic_poisson_plan_s &P;
    cudaStream_t st;
    bool prof;
    bool use_handle;
    Tally &tally;
    int nev = 0;
    std::vector<int> phase;

    Runner(pic_poisson_plan_s &p, cudaStream_t s, bool pr, bool uh, Tally &t)
        : P(p), st(s), prof(pr), use_handle(uh), tally(t) {}

    cudaError_t pre() {
        if (!prof) return cudaSuccess;
        while ((int)P.evs.size() < 2 * (nev + 1)) {
            cudaEvent_t e;
            cudaError_t err = cudaEventCreate(&e);
            if (err != cudaSuccess) return err;
            P.evs.push_back(e);
        }
        return cudaEventRecord(P.evs[2 * nev], st);
    }
    cudaError_t post(int ph) {
        tally.launches[ph]++;
        if (!prof) return cudaSuccess;
        phase.push_back(ph);
        return cudaEventRecord(P.evs[2 * nev++ + 1], st);
    }
    void account(int ph, double b, double f) {
        tally.bytes[ph] += b;
        tally.flops[ph] += f;
    }
    int event_times(double *ms) {
        if (!prof) return PIC_POISSON_OK;
        PP_CUDA(cudaStreamSynchronize(st));
        for (int e = 0; e < nev; ++e) {
            float t = 0.f;
            PP_CUDA(cudaEventElapsedTime(&t, P.evs[2 * e], P.evs[2 * e + 1]));
            ms[phase[e]] += t;
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

// ---------------------------------------------------------------- work models
// Per-entry models of algorithmic bytes and flops.  A complex entry is sizeof(V2<T>)
// bytes; FMA = 2 flops.  Sums run over the problems a table covers.
template <class T> const std::vector<LevelDev<T>> &views(const ProblemPlan &q);
template <> const std::vector<LevelDev<double>> &views<double>(const ProblemPlan &q) { return q.dl; }
template <> const std::vector<LevelDev<float>> &views<float>(const ProblemPlan &q) { return q.fl; }

template <class T> double level_entries(const pic_poisson_plan_s &P, int l) {
    double n = 0;
    for (const ProblemPlan &q : P.pr)
        if (l < q.smoothed()) n += (double)q.lv[l].nr * q.lv[l].nz * q.nm;
    return n;
}
double coarse_entries(const pic_poisson_plan_s &P, double *flops_per) {
    double n = 0, f = 0;
    for (const ProblemPlan &q : P.pr) {
        if (q.bottom || q.nact > 0) continue;
        const LevelHost &h = q.lv[q.L - 1];
        const double e = (double)h.nr * h.nz * q.nm;
        n += e;
        f += e * (4.0 * h.nz + 12.0);   // folded axial transforms (2 nz FMA) + Thomas, two parts
    }
    *flops_per = f;
    return n;
}
// Dense coarsest solves: the level's complex entries, the eigenvector
// matrices (read by the two GEMMs) and the FP32 multiply-adds.
double dense_work(const pic_poisson_plan_s &P, double *qbytes, double *flops) {
    double n = 0, qb = 0, f = 0;
    for (const ProblemPlan &q : P.pr) {
        if (q.bottom || q.nact == 0) continue;
        const LevelHost &h = q.lv[q.L - 1];
        const double na = q.nact;
        n += (double)h.nr * h.nz * q.nm;
        qb += 2.0 * na * na * sizeof(float);
        f += 2.0 * 2.0 * na * na * 2.0 * q.nm;   // two n x n by n x 2 nm products
    }
    *qbytes = qb;
    *flops = f;
    return n;
}
double level0_entries(const pic_poisson_plan_s &P, int which /*0 all, 1 single-level only*/) {
    double n = 0;
    for (const ProblemPlan &q : P.pr)
        if (which == 0 || q.L == 1) n += (double)q.lv[0].nr * q.lv[0].nz * q.nm;
    return n;
}
double fft_flops_all(const pic_poisson_plan_s &P, double *bytes3d) {
    double f = 0, x = 0;
    for (const ProblemPlan &q : P.pr) {
        const double M = q.d.ntheta / 2;
        const double cols = (double)q.lv[0].nr * q.lv[0].nz;
        f += cols * (5.0 * M * std::log2(std::max(M, 1.0)) + 14.0 * (M + 1));
        x += cols * q.d.ntheta * sizeof(double);
    }
    *bytes3d = x;
    return f;
}

// `sweeps` red-black sweeps on level l of every problem that is smoothed
// there.  skip_first_red: the first sweep starts at its black half, because
// the kernel that initialised the level already performed the red half-sweep
// from a zero iterate.  Half-sweep: 1.5 V, 14 flops per updated complex entry
// (over-relaxed: 2 V, 18 flops -- the cell's own value is read and weighted).
// With the fused FP32 smoother (H.fused) the sweeps of a pre- or
// post-smoothing are one launch (pre: u -> u2, post: u2 -> u), starting red:
// after a fused first red half-sweep from zero, repeating it gives the same
// values, so skip_first_red needs no special case.  2 * sweeps half-sweeps
// move 3 V (the iterate and b_hat read once, the iterate written once).
template <class T>
int smooth_level(Runner &R, const Hier<T> &H, int l, int sweeps, bool skip_first_red, bool post) {
    if (!H.smooth[l]) return PIC_POISSON_OK;
    const int ph = l == 0 ? PIC_POISSON_PHASE_SMOOTH : PIC_POISSON_PHASE_SMOOTH_COARSE;
    const double n = level_entries<T>(R.P, l);
    if (H.fused) {
        if (sweeps == 0) return PIC_POISSON_OK;
        const bool res = !post && H.fres[l];
        RUN(R, ph, launch_smooth_fused(post ? H.fpost[l] : H.fpre[l], post ? H.g_fpost[l] : H.g_fpre[l],
                                       2 * sweeps, res, R.st, R.P.masked));
        R.account(ph, 3.0 * n * sizeof(V2<T>), 14.0 * sweeps * n);
        if (res)   // the fused restriction: b of the red cells, the coarse b, b_hat, u -- booked
                   // with the launch that moves them, so a phase's bytes and time match
            R.account(ph, n * sizeof(V2<T>) * (0.5 + 0.75), 9.0 * n);
        return PIC_POISSON_OK;
    }
    for (int s = 0; s < sweeps; ++s) {
        for (int color = (s == 0 && skip_first_red) ? 1 : 0; color < 2; ++color) {
            const bool sor = R.P.shared.omega != 1.0;
            RUN(R, ph, launch_smooth(H.smooth[l], H.g_smooth[l], color, R.P.shared.smooth_threads, H.strip[l], sor,
                                     R.st, R.P.masked));
            R.account(ph, (sor ? 2.0 : 1.5) * n * sizeof(V2<T>), (sor ? 18.0 : 14.0) * 0.5 * n);
        }
    }
    return PIC_POISSON_OK;
}

// Residual + restriction from level l: reads u (V) and b of the evaluated
// cells, writes coarse b (and b_hat, u when initialising); 18 flops per
// evaluated complex entry (+4 with norms), 2-4 per coarse entry.
template <class T>
int restrict_level(Runner &R, const Hier<T> &H, int l, double *partials) {
    if (!H.restr[l]) return PIC_POISSON_OK;
    if (H.fused && H.fres[l] && !partials) return PIC_POISSON_OK;   // done by the fused pre-smoothing
    // after a Gauss-Seidel black half-sweep the black residuals vanish; an
    // over-relaxed one leaves them nonzero, so then every cell is evaluated
    const bool red_only = R.P.shared.pre_sweeps > 0 && R.P.shared.omega == 1.0;
    RUN(R, PIC_POISSON_PHASE_RESTRICT, launch_residual_restrict(H.restr[l], H.g_restr[l], red_only, partials, R.st, R.P.masked));
    const double n = level_entries<T>(R.P, l), frac = red_only ? 0.5 : 1.0;
    R.account(PIC_POISSON_PHASE_RESTRICT, n * sizeof(V2<T>) * (1.0 + frac + 0.75),
              frac * n * (partials ? 22.0 : 18.0) + n);
    return PIC_POISSON_OK;
}

// The coarsest levels: the separable solve (k_coarse) for the problems that
// end there, the mode-local bottom (k_bottom) for the others.
template <class T>
int coarse_and_bottom(Runner &R, const Hier<T> &H) {
    pic_poisson_plan_s &P = R.P;
    double cf = 0;
    const double cn = coarse_entries(P, &cf);
    if (H.g_coarse) {
        RUN(R, PIC_POISSON_PHASE_COARSE, launch_coarse(H.coarse, H.g_coarse, H.smem_coarse, R.st));
        R.account(PIC_POISSON_PHASE_COARSE, 2.0 * cn * sizeof(V2<T>) + cn * 2 * sizeof(T), cf);
    }
    if (H.g_dense_prep) {
        double qb = 0, df = 0;
        const double dn = dense_work(P, &qb, &df);
        // y: b in, y out; each GEMM: Q, one FP32 column block in, one out
        RUN(R, PIC_POISSON_PHASE_COARSE, launch_dense(H.dense, 0, H.g_dense_prep, H.g_dense_gemm, R.st));
        R.account(PIC_POISSON_PHASE_COARSE, dn * (sizeof(V2<T>) + sizeof(float2)), 0.0);
        for (int stage = 1; stage <= 2; ++stage) {
            RUN(R, PIC_POISSON_PHASE_COARSE, launch_dense(H.dense, stage, H.g_dense_prep, H.g_dense_gemm, R.st));
            R.account(PIC_POISSON_PHASE_COARSE, 0.5 * qb + dn * (stage == 1 ? 2 * sizeof(float2) : sizeof(float2) + sizeof(V2<T>)),
                      0.5 * df);
        }
    }
    if (H.g_bottom) {
        // per mode and part: b, b_hat in, u out of the level above the coarsest
        double nb = 0, fb = 0;
        for (const ProblemPlan &q : P.pr) {
            if (!q.bottom) continue;
            const LevelHost &u = q.lv[q.L - 2], &c = q.lv[q.L - 1];
            const double e = (double)u.nr * u.nz * q.nm, ec = (double)c.nr * c.nz * q.nm;
            nb += e;
            fb += e * 7.0 * (P.shared.pre_sweeps + P.shared.post_sweeps) + e * 13.0 + ec * (4.0 * c.nz + 12.0);
        }
        RUN(R, PIC_POISSON_PHASE_COARSE, launch_bottom(H.bottom, H.g_bottom, H.smem_bottom, R.st));
        R.account(PIC_POISSON_PHASE_COARSE, 3.0 * nb * sizeof(V2<T>), fb);
    }
    return PIC_POISSON_OK;
}

// Coarse-grid correction below level lend: level lend + 1 holds the
// restricted residual and its initialised iterate; returns with the
// correction prolongated into level lend and post-smoothed there (lend = 0:
// the V-cycle's coarse-grid correction of the finest level).
template <class T>
int descend_ascend(Runner &R, const Hier<T> &H, int lend = 0) {
    pic_poisson_plan_s &P = R.P;
    const int nl = P.Lmax - 1, pre = P.shared.pre_sweeps, post = P.shared.post_sweeps;
    for (int l = lend + 1; l < nl; ++l) {
        int rc = smooth_level(R, H, l, pre, pre > 0, false);
        if (rc) return rc;
        rc = restrict_level(R, H, l, nullptr);
        if (rc) return rc;
    }
    int rc0 = coarse_and_bottom(R, H);
    if (rc0) return rc0;
    for (int l = nl - 1; l >= lend; --l) {
        if (!H.prolong[l]) continue;
        // the red half-sweep that follows overwrites the red cells unread
        // (Gauss-Seidel only: an over-relaxed update reads the old value)
        const bool black_only = post > 0 && P.shared.omega == 1.0;
        RUN(R, PIC_POISSON_PHASE_PROLONG, launch_prolong(H.prolong[l], H.g_prolong[l], black_only, R.st, R.P.masked));
        const double n = level_entries<T>(P, l), frac = black_only ? 0.5 : 1.0;
        R.account(PIC_POISSON_PHASE_PROLONG, n * sizeof(V2<T>) * (0.25 + 2.0 * frac), 16.0 * frac * n);
        int rc = smooth_level(R, H, l, post, false, true);
        if (rc) return rc;
    }
    return PIC_POISSON_OK;
}

// Level-0 residual norms of the FP64 path and the convergence test.
int fp64_residual_and_check(Runner &R, int counting) {
    pic_poisson_plan_s &P = R.P;
    if (P.Lmax > 1) {
        int rc = restrict_level(R, P.h64, 0, P.partials);
        if (rc) return rc;
    }
    if (P.g_res_single) {
        RUN(R, PIC_POISSON_PHASE_RESTRICT,
            launch_residual(P.res_single, P.g_res_single, false, P.partials + P.res_single_offset, 0u, R.st, P.masked));
        const double n = level0_entries(P, 1);
        R.account(PIC_POISSON_PHASE_RESTRICT, 2.0 * n * sizeof(double2), 22.0 * n);
    }
    RUN(R, PIC_POISSON_PHASE_NORM, launch_psum(P.psum, P.g_psum, P.partials, P.partials2, R.st));
    RUN(R, PIC_POISSON_PHASE_NORM,
        launch_check(P.ctrl, P.partials2, counting, P.handle, P.handle_first, R.use_handle ? 1 : 0, R.st));
    return PIC_POISSON_OK;
}

// The mixed form's first correction runs more FP32 V-cycles than the others.
bool larger_first(const pic_poisson_plan_s &P) {
    return P.shared.precision == PIC_POISSON_MIXED && P.shared.inner_first > P.shared.inner_cycles;
}

int mixed_defect_and_check(Runner &R, int counting, bool zero_x = false) {
    pic_poisson_plan_s &P = R.P;
    RUN(R, PIC_POISSON_PHASE_DEFECT, launch_defect(P.defect, P.g_defect, P.ctrl, P.partials, zero_x, R.st, P.masked));
    const double n = level0_entries(P, 0);
    R.account(PIC_POISSON_PHASE_DEFECT, n * (2.0 * sizeof(double2) + 3.0 * sizeof(float2)), (zero_x ? 6.0 : 26.0) * n);
    RUN(R, PIC_POISSON_PHASE_NORM, launch_psum(P.psum, P.g_psum, P.partials, P.partials2, R.st));
    // the first test also decides the if node of a larger first pass
    const int which = R.use_handle ? (counting == 0 && larger_first(P) ? 3 : 1) : 0;
    RUN(R, PIC_POISSON_PHASE_NORM,
        launch_check(P.ctrl, P.partials2, counting, P.handle, P.handle_first, which, R.st));
    return PIC_POISSON_OK;
}

// Full-multigrid start of a solve from a zero iterate (FP64 levels): the
// right-hand side restricted to every level, the coarsest levels solved (the
// separable solve, or the mode-local bottom), then from the coarsest level up
// the iterate prolongated to the next finer level as its initial value and one
// V-cycle there -- up to level 0, whose prolongated iterate starts the main
// iteration.  The restriction of b is the residuals' (a finite-volume sum), so
// each level's problem is the discretisation of the same field on its cells.
int fmg_start(Runner &R) {
    pic_poisson_plan_s &P = R.P;
    const Hier<double> &H = P.h64;
    const int nl = P.Lmax - 1, pre = P.shared.pre_sweeps;
    for (int l = 0; l < nl; ++l) {
        if (!H.g_rhs[l]) continue;
        RUN(R, PIC_POISSON_PHASE_RESTRICT, launch_rhs_restrict(H.rhs[l], H.g_rhs[l], R.st, R.P.masked));
        const double n = level_entries<double>(P, l);
        R.account(PIC_POISSON_PHASE_RESTRICT, n * sizeof(double2) * (1.0 + 0.75), 0.5 * n);
    }
    int rc = coarse_and_bottom(R, H);
    if (rc) return rc;
    for (int l = nl - 1; l >= 0; --l) {
        if (!H.g_interp[l]) continue;
        RUN(R, PIC_POISSON_PHASE_PROLONG,
            launch_interp(H.interp[l], H.g_interp[l], R.st, R.P.masked, H.interp_black));
        const double n = level_entries<double>(P, l), frac = H.interp_black ? 0.5 : 1.0;
        R.account(PIC_POISSON_PHASE_PROLONG, n * sizeof(double2) * (0.25 + frac), 16.0 * frac * n);
        if (l == 0) break;   // the main iteration takes over on level 0
        rc = smooth_level(R, H, l, pre, false, false);
        if (rc) return rc;
        rc = restrict_level(R, H, l, nullptr);
        if (rc) return rc;
        rc = descend_ascend(R, H, l);
        if (rc) return rc;
    }
    return PIC_POISSON_OK;
}

// Full-multigrid start from a given level-0 iterate (FP64 levels): the same
// nested iteration on the correction equation.  The residual of the given
// iterate is evaluated on every level-0 cell and restricted to level 1; that
// right-hand side is restricted on to every coarser level, the coarsest
// levels are solved, and from there up each level gets the prolongated
// coarser correction and one V-cycle, up to level 1, whose correction is
// prolongated into level 0.  The level-0 pre-smoothing of the solve follows
// (its first red half-sweep overwrites the red cells, so the prolongation
// corrects the black ones only).  A given iterate then keeps the
// full-multigrid start that a zero iterate gets, for about the same work.
int fmg_correction(Runner &R) {
    pic_poisson_plan_s &P = R.P;
    const Hier<double> &H = P.h64;
    const int nl = P.Lmax - 1, pre = P.shared.pre_sweeps;
    if (H.restr[0]) {   // r = b - A u on every cell (the given iterate is not smoothed)
        RUN(R, PIC_POISSON_PHASE_RESTRICT,
            launch_residual_restrict(H.restr[0], H.g_restr[0], false, nullptr, R.st, R.P.masked));
        const double n = level_entries<double>(P, 0);
        R.account(PIC_POISSON_PHASE_RESTRICT, n * sizeof(double2) * 2.75, 19.0 * n);
    }
    for (int l = 1; l < nl; ++l) {
        if (!H.g_rhs[l]) continue;
        RUN(R, PIC_POISSON_PHASE_RESTRICT, launch_rhs_restrict(H.rhs[l], H.g_rhs[l], R.st, R.P.masked));
        const double n = level_entries<double>(P, l);
        R.account(PIC_POISSON_PHASE_RESTRICT, n * sizeof(double2) * (1.0 + 0.75), 0.5 * n);
    }
    int rc = coarse_and_bottom(R, H);
    if (rc) return rc;
    for (int l = nl - 1; l >= 1; --l) {
        if (!H.g_interp[l]) continue;
        RUN(R, PIC_POISSON_PHASE_PROLONG,
            launch_interp(H.interp[l], H.g_interp[l], R.st, R.P.masked, H.interp_black));
        const double n = level_entries<double>(P, l), frac = H.interp_black ? 0.5 : 1.0;
        R.account(PIC_POISSON_PHASE_PROLONG, n * sizeof(double2) * (0.25 + frac), 16.0 * frac * n);
        rc = smooth_level(R, H, l, pre, false, false);
        if (rc) return rc;
        rc = restrict_level(R, H, l, nullptr);
        if (rc) return rc;
        rc = descend_ascend(R, H, l);
        if (rc) return rc;
    }
    if (H.prolong[0]) {   // level 1's correction into the level-0 iterate
        const bool black_only = pre > 0 && P.shared.omega == 1.0;
        RUN(R, PIC_POISSON_PHASE_PROLONG, launch_prolong(H.prolong[0], H.g_prolong[0], black_only, R.st, R.P.masked));
        const double n = level_entries<double>(P, 0), frac = black_only ? 0.5 : 1.0;
        R.account(PIC_POISSON_PHASE_PROLONG, n * sizeof(double2) * (0.25 + 2.0 * frac), 16.0 * frac * n);
    }
    return PIC_POISSON_OK;
}

// Forward transform + right-hand side, ||b||, initial iterate, first
// evaluation of the residual and the first convergence test.
// guess: 0 = zero initial iterate, 1 = transform of phi, 2 = mode-layout iterate.
int enqueue_prologue(Runner &R, int guess) {
    pic_poisson_plan_s &P = R.P;
    const bool mixed = P.shared.precision == PIC_POISSON_MIXED;
    double x3 = 0;
    const double ff = fft_flops_all(P, &x3), n0 = level0_entries(P, 0);
    // the mixed form's forward transform in double-float arithmetic (fft_df.cu)
    auto forward = mixed ? launch_forward_df : launch_forward;
    RUN(R, PIC_POISSON_PHASE_FORWARD, forward(P.fwd, P.g_fft, P.smem_fft, P.partials_fwd, R.st));
    R.account(PIC_POISSON_PHASE_FORWARD, x3 + (mixed ? 1.0 : 2.0) * n0 * sizeof(double2), ff);
    RUN(R, PIC_POISSON_PHASE_NORM, launch_bnorm(P.ctrl, P.fwd, P.partials_fwd, R.st));
    if (guess == 1) {
        RUN(R, PIC_POISSON_PHASE_FORWARD, forward(P.guess, P.g_fft, P.smem_fft, nullptr, R.st));
        R.account(PIC_POISSON_PHASE_FORWARD, x3 + n0 * sizeof(double2), ff);
    } else if (guess == 2) {
        RUN(R, PIC_POISSON_PHASE_FORWARD, launch_copy_guess(P.guess, P.g_fft, R.st));
        R.account(PIC_POISSON_PHASE_FORWARD, 2.0 * n0 * sizeof(double2), 0.0);
    }
    if (guess != 0) {
        if (!mixed && P.shared.fmg && P.Lmax > 1) {
            int rc = fmg_correction(R);   // full-multigrid start on the given iterate's correction
            if (rc) return rc;
        }
    } else if (!mixed && P.shared.fmg && P.Lmax > 1) {
        int rc = fmg_start(R);   // with the red half-sweep below, writes every level-0 iterate
        if (rc) return rc;
    } else if (!mixed) {   // (the mixed form's first defect writes the zero iterate itself)
        for (const ProblemPlan &q : P.pr) {
            const size_t n = (size_t)q.lv[0].nr * q.lv[0].nz * q.nm;
            PP_CUDA(cudaMemsetAsync(q.dl[0].u, 0, n * sizeof(double2), R.st));
        }
    }
    if (mixed) return mixed_defect_and_check(R, 0, guess == 0);
    if (P.Lmax > 1) {
        int rc = smooth_level(R, P.h64, 0, P.shared.pre_sweeps, false, false);
        if (rc) return rc;
    }
    return fp64_residual_and_check(R, 0);
}

// One pass of the convergence loop: FP64, one V-cycle (coarse-grid correction
// and post-smoothing of the current cycle, pre-smoothing and residual of the
// next); mixed, inner_cycles FP32 V-cycles on the correction equation (first:
// inner_first, the solve's first pass), the FP64 update and the next FP64
// defect.
int enqueue_body(Runner &R, bool first = false) {
    pic_poisson_plan_s &P = R.P;
    const int pre = P.shared.pre_sweeps;
    if (P.shared.precision == PIC_POISSON_FP64) {
        int rc = descend_ascend(R, P.h64);
        if (rc) return rc;
        if (P.Lmax > 1) {
            rc = smooth_level(R, P.h64, 0, pre, false, false);
            if (rc) return rc;
        }
        return fp64_residual_and_check(R, 1);
    }
    const int inner = first ? P.shared.inner_first : P.shared.inner_cycles;
    for (int c = 0; c < inner; ++c) {
        if (P.Lmax > 1) {
            int rc = smooth_level(R, P.h32, 0, pre, c == 0 && pre > 0, false);
            if (rc) return rc;
            rc = restrict_level(R, P.h32, 0, nullptr);
            if (rc) return rc;
        }
        int rc = descend_ascend(R, P.h32);
        if (rc) return rc;
    }
    RUN(R, PIC_POISSON_PHASE_DEFECT, launch_update(P.defect, P.g_defect, P.ctrl, R.st));
    const double n = level0_entries(P, 0);
    R.account(PIC_POISSON_PHASE_DEFECT, n * (2.0 * sizeof(double2) + sizeof(float2)), 4.0 * n);
    return mixed_defect_and_check(R, first ? 2 : 1);
}

int enqueue_epilogue(Runner &R) {
    pic_poisson_plan_s &P = R.P;
    double x3 = 0;
    const double ff = fft_flops_all(P, &x3), n0 = level0_entries(P, 0);
    // binary64 in both forms: an error in phi reaches the residual amplified by
    // the operator (up to ~N^2 for its high frequencies), an error in b does not
    RUN(R, PIC_POISSON_PHASE_INVERSE, launch_inverse(P.inv, P.g_fft, P.smem_fft, R.st));
    R.account(PIC_POISSON_PHASE_INVERSE, x3 + n0 * sizeof(double2), ff);
    return PIC_POISSON_OK;
}

// ---------------------------------------------------------------- per-solve inputs
int set_io(pic_poisson_plan_s &P, const double *const *rho, double *const *phi, const double *const *guess,
           double tol) {
    bool changed = !P.io_valid;
    for (int p = 0; p < P.n; ++p)
        changed = changed || P.last_rho[p] != rho[p] || P.last_phi[p] != phi[p] ||
                  P.last_guess[p] != (guess ? guess[p] : nullptr);
    if (changed) {
        for (int p = 0; p < P.n; ++p) {
            P.h_fwd.p[p].rho = rho[p];
            P.h_guess.p[p].rho = phi[p];
            P.h_guess.p[p].guess = (const double2 *)(guess ? guess[p] : nullptr);
            P.h_inv.p[p].phi = phi[p];
            P.last_rho[p] = rho[p];
            P.last_phi[p] = phi[p];
            P.last_guess[p] = guess ? guess[p] : nullptr;
        }
        PP_CUDA(cudaMemcpyAsync(P.fwd, &P.h_fwd, sizeof(FFTTab), cudaMemcpyHostToDevice, P.stream));
        PP_CUDA(cudaMemcpyAsync(P.guess, &P.h_guess, sizeof(FFTTab), cudaMemcpyHostToDevice, P.stream));
        PP_CUDA(cudaMemcpyAsync(P.inv, &P.h_inv, sizeof(FFTTab), cudaMemcpyHostToDevice, P.stream));
        P.io_valid = true;
    }
    Ctrl &C = P.hctrl;
    C.tol = tol;
    C.max_cycles = P.shared.max_cycles;
    C.cycles = 0;
    C.cont = 1;
    for (int p = 0; p < P.n; ++p) {
        C.rel[p] = 1.0;
        C.rel_first[p] = 1.0;
        C.best[p] = INFINITY;
        C.stall[p] = 0;
        C.status[p] = PIC_POISSON_OK;
        C.done[p] = 0;
        C.done_cycles[p] = 0;
        C.sigma_used[p] = C.inv_sigma_used[p] = C.sigma_next[p] = 1.0;
    }
    PP_CUDA(cudaMemcpyAsync(P.ctrl, &C, sizeof(Ctrl), cudaMemcpyHostToDevice, P.stream));
    return PIC_POISSON_OK;
}

int read_cont(pic_poisson_plan_s &P, int *cont) {
    // the leading scalars of Ctrl hold the loop flag
    PP_CUDA(cudaMemcpyAsync(P.hctrl_out, P.ctrl, offsetof(Ctrl, cont) + sizeof(int), cudaMemcpyDeviceToHost,
                            P.stream));
    PP_CUDA(cudaStreamSynchronize(P.stream));
    *cont = P.hctrl_out->cont;
    return PIC_POISSON_OK;
}

// ---------------------------------------------------------------- drivers
int run_host_loop(pic_poisson_plan_s &P, int guess, Tally &tally, double *ms) {
    const bool prof = P.shared.flags & PIC_POISSON_PROFILE;
    Runner R(P, P.stream, prof, false, tally);
    int rc = enqueue_prologue(R, guess);
    if (rc) return rc;
    int cont = 0;
    rc = read_cont(P, &cont);
    if (rc) return rc;
    if (cont && larger_first(P)) {
        rc = enqueue_body(R, true);
        if (rc) return rc;
        rc = read_cont(P, &cont);
        if (rc) return rc;
    }
    while (cont) {
        rc = enqueue_body(R);
        if (rc) return rc;
        rc = read_cont(P, &cont);
        if (rc) return rc;
    }
    rc = enqueue_epilogue(R);
    if (rc) return rc;
    return R.event_times(ms);
}

int capture_graph(pic_poisson_plan_s &P, int guess) {
    const int v = guess == 2 ? 1 : 0;
    if (!P.cap0) PP_CUDA(cudaStreamCreateWithFlags(&P.cap0, cudaStreamNonBlocking));
    if (!P.cap1) PP_CUDA(cudaStreamCreateWithFlags(&P.cap1, cudaStreamNonBlocking));
    for (Tally &t : P.seg[v]) t = Tally{};
    const cudaStreamCaptureMode mode = cudaStreamCaptureModeThreadLocal;
    cudaGraph_t graph = nullptr;
    bool body_open = false;
    auto fail = [&](int rc) {
        if (body_open) {
            cudaGraph_t tmp = nullptr;
            cudaStreamEndCapture(P.cap1, &tmp);
        }
        cudaGraph_t tmp = nullptr;
        cudaStreamEndCapture(P.cap0, &tmp);
        if (tmp) cudaGraphDestroy(tmp);
        cudaGetLastError();
        return rc;
    };
    PP_CUDA(cudaStreamBeginCapture(P.cap0, mode));
    cudaStreamCaptureStatus status;
    if (cudaStreamGetCaptureInfo(P.cap0, &status, nullptr, &graph, nullptr, nullptr, nullptr) != cudaSuccess ||
        cudaGraphConditionalHandleCreate(&P.handle, graph, 0, 0) != cudaSuccess) {
        set_error("graph conditional handle creation failed");
        return fail(PIC_POISSON_ECUDA);
    }
    const bool first = larger_first(P);
    if (first && cudaGraphConditionalHandleCreate(&P.handle_first, graph, 0, 0) != cudaSuccess) {
        set_error("graph conditional handle creation failed");
        return fail(PIC_POISSON_ECUDA);
    }
    Runner R0(P, P.cap0, false, true, P.seg[v][0]);
    int rc = enqueue_prologue(R0, guess);
    if (rc) return fail(rc);
    const cudaGraphNode_t *deps = nullptr;
    size_t ndeps = 0;
    if (cudaStreamGetCaptureInfo(P.cap0, &status, nullptr, &graph, &deps, nullptr, &ndeps) != cudaSuccess) {
        set_error("cudaStreamGetCaptureInfo failed");
        return fail(PIC_POISSON_ECUDA);
    }
    if (first) {
        // the larger first pass: an if node on the first convergence test,
        // ahead of the while node (whose condition that pass's test sets)
        cudaGraphNodeParams ip{};
        ip.type = cudaGraphNodeTypeConditional;
        ip.conditional.handle = P.handle_first;
        ip.conditional.type = cudaGraphCondTypeIf;
        ip.conditional.size = 1;
        cudaGraphNode_t inode;
        if (cudaGraphAddNode(&inode, graph, deps, nullptr, ndeps, &ip) != cudaSuccess ||
            cudaStreamUpdateCaptureDependencies(P.cap0, &inode, nullptr, 1, cudaStreamSetCaptureDependencies) !=
                cudaSuccess) {
            set_error("adding the if node failed");
            return fail(PIC_POISSON_ECUDA);
        }
        cudaGraph_t fbody = ip.conditional.phGraph_out[0];
        if (cudaStreamBeginCaptureToGraph(P.cap1, fbody, nullptr, nullptr, 0, mode) != cudaSuccess) {
            set_error("capturing the first pass failed to start");
            return fail(PIC_POISSON_ECUDA);
        }
        body_open = true;
        Runner RF(P, P.cap1, false, true, P.seg[v][3]);
        rc = enqueue_body(RF, true);
        if (rc) return fail(rc);
        body_open = false;
        if (cudaStreamEndCapture(P.cap1, &fbody) != cudaSuccess) {
            set_error("capturing the first pass failed");
            return fail(PIC_POISSON_ECUDA);
        }
        if (cudaStreamGetCaptureInfo(P.cap0, &status, nullptr, &graph, &deps, nullptr, &ndeps) != cudaSuccess) {
            set_error("cudaStreamGetCaptureInfo failed");
            return fail(PIC_POISSON_ECUDA);
        }
    }
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = P.handle;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cnode;
    if (cudaGraphAddNode(&cnode, graph, deps, nullptr, ndeps, &cp) != cudaSuccess ||
        cudaStreamUpdateCaptureDependencies(P.cap0, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies) !=
            cudaSuccess) {
        set_error("adding the while node failed");
        return fail(PIC_POISSON_ECUDA);
    }
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    if (cudaStreamBeginCaptureToGraph(P.cap1, body, nullptr, nullptr, 0, mode) != cudaSuccess) {
        set_error("capturing the loop body failed to start");
        return fail(PIC_POISSON_ECUDA);
    }
    body_open = true;
    Runner R1(P, P.cap1, false, true, P.seg[v][1]);
    rc = enqueue_body(R1);
    if (rc) return fail(rc);
    body_open = false;
    if (cudaStreamEndCapture(P.cap1, &body) != cudaSuccess) {
        set_error("capturing the loop body failed");
        return fail(PIC_POISSON_ECUDA);
    }
    Runner R2(P, P.cap0, false, false, P.seg[v][2]);
    rc = enqueue_epilogue(R2);
    if (rc) return fail(rc);
    cudaError_t err = cudaStreamEndCapture(P.cap0, &graph);
    if (err != cudaSuccess) {
        set_error("graph capture failed: %s", cudaGetErrorString(err));
        cudaGetLastError();
        return PIC_POISSON_ECUDA;
    }
    P.graph[v] = graph;
    err = cudaGraphInstantiate(&P.gexec[v], P.graph[v], 0);
    if (err != cudaSuccess) {
        set_error("cudaGraphInstantiate failed: %s", cudaGetErrorString(err));
        cudaGetLastError();
        cudaGraphDestroy(P.graph[v]);
        P.graph[v] = nullptr;
        P.gexec[v] = nullptr;
        return PIC_POISSON_ECUDA;
    }
    return PIC_POISSON_OK;
}

int solve_batch(pic_poisson_plan_s &P, const double *const *rho, double *const *phi, double tol,
                pic_poisson_info *infos, const double *const *guess_modes = nullptr) {
    int rc = set_io(P, rho, phi, guess_modes, tol);
    if (rc) return rc;
    Tally tally;
    double ms[PIC_POISSON_NPHASE] = {0};
    const int guess = guess_modes ? 2 : ((P.shared.flags & PIC_POISSON_USE_INITIAL_GUESS) ? 1 : 0);
    const int v = guess == 2 ? 1 : 0;
    const bool graph = (P.shared.flags & PIC_POISSON_GRAPH) && !(P.shared.flags & PIC_POISSON_PROFILE);
    if (graph) {
        if (!P.gexec[v]) {
            rc = capture_graph(P, guess);
            if (rc) return rc;
        }
        PP_CUDA(cudaGraphLaunch(P.gexec[v], P.stream));
    } else {
        rc = run_host_loop(P, guess, tally, ms);
        if (rc) return rc;
    }
    PP_CUDA(cudaMemcpyAsync(P.hctrl_out, P.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, P.stream));
    PP_CUDA(cudaStreamSynchronize(P.stream));
    const Ctrl &C = *P.hctrl_out;
    const int inc = std::max(P.hctrl.inc, 1), inc_first = std::max(P.hctrl.inc_first, 1);
    const bool first = larger_first(P);
    // passes of the loop body behind a cycle count (after the larger first pass, if any)
    auto body_passes = [&](int cycles) { return first ? (cycles >= inc_first ? (cycles - inc_first) / inc : 0)
                                                       : cycles / inc; };
    if (graph) {
        const int passes = body_passes(C.cycles), fp = first && C.cycles >= inc_first ? 1 : 0;
        for (int ph = 0; ph < PIC_POISSON_NPHASE; ++ph) {
            const Tally *sg = P.seg[v];
            tally.bytes[ph] = sg[0].bytes[ph] + passes * sg[1].bytes[ph] + sg[2].bytes[ph] + fp * sg[3].bytes[ph];
            tally.flops[ph] = sg[0].flops[ph] + passes * sg[1].flops[ph] + sg[2].flops[ph] + fp * sg[3].flops[ph];
            tally.launches[ph] =
                sg[0].launches[ph] + passes * sg[1].launches[ph] + sg[2].launches[ph] + fp * sg[3].launches[ph];
        }
    }
    int worst = PIC_POISSON_OK;
    for (int p = 0; p < P.n; ++p) {
        const int s = C.status[p];
        if (s == PIC_POISSON_ENONFINITE || (s == PIC_POISSON_ENOTCONVERGED && worst == PIC_POISSON_OK)) worst = s;
        if (!infos) continue;
        pic_poisson_info &I = infos[p];
        memset(&I, 0, sizeof I);
        I.status = s;
        I.cycles = C.done_cycles[p];   // a problem of a batch stops being iterated when it converges
        const int dc = C.done_cycles[p];
        I.outer_iterations = P.shared.precision != PIC_POISSON_MIXED ? 0
                             : first ? (dc >= inc_first ? 1 + body_passes(dc) : 0) : dc / inc;
        I.rel_res = C.rel[p];
        I.rel_res0 = C.rel_first[p];
        for (int ph = 0; ph < PIC_POISSON_NPHASE; ++ph) {
            I.ms_phase[ph] = ms[ph];
            I.launches_phase[ph] = tally.launches[ph];
            I.bytes_phase[ph] = tally.bytes[ph];
            I.flops_phase[ph] = tally.flops[ph];
            I.launches += tally.launches[ph];
        }
    }
    if (worst == PIC_POISSON_ENONFINITE) set_error("non-finite right-hand side or residual");
    if (worst == PIC_POISSON_ENOTCONVERGED) set_error("tolerance not reached in max_cycles");
    return worst;
}

int single_only(const pic_poisson_plan_s &P, const char *what) {
    if (P.n != 1) {
        set_error("%s needs a single-problem plan (this plan holds %d problems)", what, P.n);
        return PIC_POISSON_EINVAL;
    }
    return PIC_POISSON_OK;
}

// Device address of page-locked host memory mapped into the device's address
// space, or null (pageable or unregistered memory: the caller stages).
void *mapped_host(const void *p) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

}  // namespace
}  // namespace pp

using namespace pp;

extern "C" {

int pic_poisson_solve(pic_poisson_plan_t plan, const double *rho_dev, double *phi_dev, double tol,
                      pic_poisson_info *info) {
    int rc = plan_enter(plan);
    if (rc) return rc;
    rc = single_only(*plan, "pic_poisson_solve");
    if (rc) return rc;
    if (!rho_dev || !phi_dev || (const void *)rho_dev == (const void *)phi_dev) {
        set_error("rho_dev and phi_dev must be distinct non-NULL device pointers");
        return PIC_POISSON_EINVAL;
    }
    if (std::isnan(tol)) {
        set_error("tol is NaN");
        return PIC_POISSON_EINVAL;
    }
    return solve_batch(*plan, &rho_dev, &phi_dev, tol, info);
}

int pic_poisson_solve_batch(pic_poisson_plan_t plan, const double *const *rho_dev, double *const *phi_dev,
                            double tol, pic_poisson_info *infos) {
    int rc = plan_enter(plan);
    if (rc) return rc;
    if (!rho_dev || !phi_dev || std::isnan(tol)) {
        set_error("rho_dev and phi_dev arrays must be non-NULL and tol a number");
        return PIC_POISSON_EINVAL;
    }
    for (int p = 0; p < plan->n; ++p) {
        if (!rho_dev[p] || !phi_dev[p] || (const void *)rho_dev[p] == (const void *)phi_dev[p]) {
            set_error("problem %d: rho and phi must be distinct non-NULL device pointers", p);
            return PIC_POISSON_EINVAL;
        }
    }
    return solve_batch(*plan, rho_dev, phi_dev, tol, infos);
}

int pic_poisson_solve_host(pic_poisson_plan_t plan, const double *rho_host, double *phi_host, double tol,
                           pic_poisson_info *info) {
    int rc = plan_enter(plan);
    if (rc) return rc;
    rc = single_only(*plan, "pic_poisson_solve_host");
    if (rc) return rc;
    if (!rho_host || !phi_host) {
        set_error("rho_host and phi_host must be non-NULL");
        return PIC_POISSON_EINVAL;
    }
    pic_poisson_plan_s &P = *plan;
    const pic_poisson_desc &d = P.pr[0].d;
    const size_t bytes = (size_t)d.nr * d.ntheta * d.nz * sizeof(double);
    if (!(P.shared.flags & PIC_POISSON_HOST_STAGED)) {
        const double *r = static_cast<const double *>(mapped_host(rho_host));
        double *f = static_cast<double *>(mapped_host(phi_host));
        if (r && f) return solve_batch(P, &r, &f, tol, info);   // synchronises before it returns
    }
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
    if (P.shared.flags & PIC_POISSON_USE_INITIAL_GUESS)
        PP_CUDA(cudaMemcpyAsync(P.stage_phi, phi_host, bytes, cudaMemcpyHostToDevice, P.stream));
    const double *r = P.stage_rho;
    double *f = P.stage_phi;
    rc = solve_batch(P, &r, &f, tol, info);
    if (rc == PIC_POISSON_OK || rc == PIC_POISSON_ENOTCONVERGED) {
        PP_CUDA(cudaMemcpyAsync(phi_host, P.stage_phi, bytes, cudaMemcpyDeviceToHost, P.stream));
        PP_CUDA(cudaStreamSynchronize(P.stream));
    }
    return rc;
}

int pic_poisson_forward(pic_poisson_plan_t plan, const double *rho_dev, double *bhat_dev) {
    int rc = plan_enter(plan);
    if (rc) return rc;
    rc = single_only(*plan, "pic_poisson_forward");
    if (rc) return rc;
    if (!rho_dev || !bhat_dev) {
        set_error("NULL pointer");
        return PIC_POISSON_EINVAL;
    }
    pic_poisson_plan_s &P = *plan;
    FFTTab t = P.h_fwd;
    t.p[0].rho = rho_dev;
    t.p[0].b = (double2 *)bhat_dev;
    t.p[0].bh = nullptr;
    t.p[0].invd = nullptr;
    PP_CUDA(cudaMemcpyAsync(P.api_fft, &t, sizeof t, cudaMemcpyHostToDevice, P.stream));
    PP_CUDA(launch_forward(P.api_fft, P.g_fft, P.smem_fft, nullptr, P.stream));
    return PIC_POISSON_OK;
}

int pic_poisson_inverse(pic_poisson_plan_t plan, const double *phihat_dev, double *phi_dev) {
    int rc = plan_enter(plan);
    if (rc) return rc;
    rc = single_only(*plan, "pic_poisson_inverse");
    if (rc) return rc;
    if (!phihat_dev || !phi_dev) {
        set_error("NULL pointer");
        return PIC_POISSON_EINVAL;
    }
    pic_poisson_plan_s &P = *plan;
    FFTTab t = P.h_inv;
    t.p[0].uhat = (const double2 *)phihat_dev;
    t.p[0].phi = phi_dev;
    PP_CUDA(cudaMemcpyAsync(P.api_fft, &t, sizeof t, cudaMemcpyHostToDevice, P.stream));
    PP_CUDA(launch_inverse(P.api_fft, P.g_fft, P.smem_fft, P.stream));
    return PIC_POISSON_OK;
}

int pic_poisson_mode_residual(pic_poisson_plan_t plan, const double *uhat_dev, const double *bhat_dev,
                              double *rhat_dev, double *rel_res) {
    int rc = plan_enter(plan);
    if (rc) return rc;
    rc = single_only(*plan, "pic_poisson_mode_residual");
    if (rc) return rc;
    if (!uhat_dev || !bhat_dev) {
        set_error("NULL pointer");
        return PIC_POISSON_EINVAL;
    }
    pic_poisson_plan_s &P = *plan;
    LaunchTab<double> t = P.h_api_res;
    t.f[0].u = (double2 *)uhat_dev;
    t.f[0].b = (double2 *)bhat_dev;
    t.c[0].u = (double2 *)rhat_dev;
    PP_CUDA(cudaMemcpyAsync(P.api_res, &t, sizeof t, cudaMemcpyHostToDevice, P.stream));
    const unsigned g = P.g_api_res;
    PP_CUDA(launch_residual(P.api_res, g, rhat_dev != nullptr, rel_res ? P.partials : nullptr, g, P.stream, P.masked));
    if (rel_res) {
        PP_CUDA(launch_sum(P.partials, (int)g, P.dsum, P.stream));
        PP_CUDA(launch_sum(P.partials + g, (int)g, P.dsum + 1, P.stream));
        PP_CUDA(cudaMemcpyAsync(P.hsum, P.dsum, 2 * sizeof(double), cudaMemcpyDeviceToHost, P.stream));
        PP_CUDA(cudaStreamSynchronize(P.stream));
        *rel_res = P.hsum[1] > 0 ? std::sqrt(P.hsum[0] / P.hsum[1]) : std::sqrt(P.hsum[0]);
    }
    return PIC_POISSON_OK;
}

int pic_poisson_solve_modes(pic_poisson_plan_t plan, const double *rho_dev, const double *uhat_guess_dev,
                            double *phi_dev, double tol, pic_poisson_info *info) {
    int rc = plan_enter(plan);
    if (rc) return rc;
    rc = single_only(*plan, "pic_poisson_solve_modes");
    if (rc) return rc;
    if (!rho_dev || !phi_dev || !uhat_guess_dev || (const void *)rho_dev == (const void *)phi_dev || std::isnan(tol)) {
        set_error("rho_dev, uhat_guess_dev and phi_dev must be non-NULL (rho != phi) and tol a number");
        return PIC_POISSON_EINVAL;
    }
    return solve_batch(*plan, &rho_dev, &phi_dev, tol, info, &uhat_guess_dev);
}

int pic_poisson_analyze(pic_poisson_plan_t plan, const double *phi_dev, double *uhat_dev) {
    int rc = plan_enter(plan);
    if (rc) return rc;
    rc = single_only(*plan, "pic_poisson_analyze");
    if (rc) return rc;
    if (!phi_dev || !uhat_dev) {
        set_error("NULL pointer");
        return PIC_POISSON_EINVAL;
    }
    pic_poisson_plan_s &P = *plan;
    FFTTab t = P.h_guess;
    t.p[0].rho = phi_dev;
    t.p[0].b = (double2 *)uhat_dev;
    PP_CUDA(cudaMemcpyAsync(P.api_fft, &t, sizeof t, cudaMemcpyHostToDevice, P.stream));
    PP_CUDA(launch_forward(P.api_fft, P.g_fft, P.smem_fft, nullptr, P.stream));
    return PIC_POISSON_OK;
}

int pic_poisson_get_modes(pic_poisson_plan_t plan, double *uhat_dev) {
    int rc = plan_enter(plan);
    if (rc) return rc;
    rc = single_only(*plan, "pic_poisson_get_modes");
    if (rc) return rc;
    if (!uhat_dev) {
        set_error("NULL pointer");
        return PIC_POISSON_EINVAL;
    }
    const ProblemPlan &q = plan->pr[0];
    const size_t n = (size_t)q.lv[0].nr * q.lv[0].nz * q.nm;
    PP_CUDA(cudaMemcpyAsync(uhat_dev, q.dl[0].u, n * sizeof(double2), cudaMemcpyDeviceToDevice, plan->stream));
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
