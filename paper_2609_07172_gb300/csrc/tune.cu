// Autotuner: picks the smoothing schedule (pre / post sweeps), the number of
// FP32 V-cycles per FP64 defect correction (mixed precision) and the smoother's
// block size and strip by timing complete solves of the caller's own problems.
//
// Stage 1 times every schedule (and inner-cycle count) at the default block
// size and one entry per thread; stage 2 times the other block sizes for the
// best schedule, stage 3 strips of 2 and 4 rows at the best block size, stage 4
// over-relaxation factors with the short schedules, stage 5 (mixed precision)
// the fused FP32 smoother with the short schedules and 1 to 6 inner cycles
// (FP64: the full-multigrid start with three schedules), stage 6 (mixed) a
// larger first correction (inner_first) for the best setting.  Each
// candidate gets its own plan, one untimed solve (which also captures the
// graph when PIC_POISSON_GRAPH is set) and `repeats` timed solves; its score
// is the median wall time of a solve call, which includes every host-side
// cost a caller pays.  Candidates that do not reach the tolerance are skipped.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <vector>

#include "internal.h"

namespace pp {
namespace {

struct Cand {
    int pre, post, inner, threads, strip;
    double omega;
    int fused, fmg;
    double ms;
    int first = 0;   // FP32 V-cycles of the first correction (0: inner)
};

int time_candidate(const pic_poisson_desc *descs, int n, const double *const *rho, double *const *phi, double tol,
                   void *stream, int repeats, Cand &c) {
    std::vector<pic_poisson_desc> d(descs, descs + n);
    for (auto &x : d) {
        x.pre_sweeps = c.pre;
        x.post_sweeps = c.post;
        x.inner_cycles = c.inner;
        x.smooth_threads = c.threads;
        x.smooth_strip = c.strip;
        x.omega = c.omega;
        x.smooth_fused = c.fused;
        x.fmg = c.fmg;
        x.inner_first = c.first;
        x.flags &= ~PIC_POISSON_PROFILE;
    }
    pic_poisson_plan_t plan = nullptr;
    int rc = pic_poisson_plan_batch(d.data(), n, stream, &plan);
    if (rc) return rc;
    rc = pic_poisson_solve_batch(plan, rho, phi, tol, nullptr);
    std::vector<double> t;
    for (int r = 0; rc == PIC_POISSON_OK && r < repeats; ++r) {
        const auto t0 = std::chrono::steady_clock::now();
        rc = pic_poisson_solve_batch(plan, rho, phi, tol, nullptr);
        const auto t1 = std::chrono::steady_clock::now();
        t.push_back(std::chrono::duration<double, std::milli>(t1 - t0).count());
    }
    pic_poisson_destroy(plan);
    if (rc) return rc;
    std::sort(t.begin(), t.end());
    c.ms = t[t.size() / 2];
    return PIC_POISSON_OK;
}

}  // namespace
}  // namespace pp

using namespace pp;

extern "C" int pic_poisson_autotune(const pic_poisson_desc *descs, int n, const double *const *rho_dev,
                                    double *const *phi_dev, double tol, void *stream, int repeats,
                                    pic_poisson_tuning *out) {
    clear_error();
    if (!descs || n < 1 || n > PIC_POISSON_MAX_BATCH || !rho_dev || !phi_dev || !out || !(tol > 0)) {
        set_error("autotune needs descs, 1 <= n <= %d, rho/phi arrays, tol > 0 and out", PIC_POISSON_MAX_BATCH);
        return PIC_POISSON_EINVAL;
    }
    repeats = std::max(1, std::min(repeats, 16));
    memset(out, 0, sizeof *out);
    const bool mixed = descs[0].precision == PIC_POISSON_MIXED;
    bool composite = false;   // the fused smoother does not take non-uniform axial meshes
    for (int p = 0; p < n; ++p) composite = composite || descs[p].z_faces;
    static const int sched[][2] = {{1, 1}, {2, 1}, {1, 2}, {2, 2}, {3, 2}, {2, 3}, {3, 3}};
    std::vector<Cand> cands;
    for (const auto &s : sched) {
        if (mixed) {
            for (int inner = 1; inner <= 4; ++inner) cands.push_back({s[0], s[1], inner, 256, 0, 1.0, 0, 0, 0.0});
        } else {
            cands.push_back({s[0], s[1], 2, 256, 0, 1.0, 0, 0, 0.0});
        }
    }
    Cand best{0, 0, 0, 0, 0, 1.0, 0, 0, 1e300};
    int last_err = PIC_POISSON_OK;
    auto record = [&](Cand &c) {
        const int rc = time_candidate(descs, n, rho_dev, phi_dev, tol, stream, repeats, c);
        if (rc == PIC_POISSON_ENOMEM || rc == PIC_POISSON_ECUDA || rc == PIC_POISSON_EINVAL) last_err = rc;
        if (rc != PIC_POISSON_OK) return rc;
        if (out->tried < PIC_POISSON_MAX_TUNE) {
            const int k = out->tried++;
            out->ms_tried[k] = c.ms;
            out->pre_tried[k] = c.pre;
            out->post_tried[k] = c.post;
            out->inner_tried[k] = c.inner;
            out->threads_tried[k] = c.threads;
            out->strip_tried[k] = c.strip;
            out->omega_tried[k] = c.omega;
            out->fused_tried[k] = c.fused;
            out->fmg_tried[k] = c.fmg;
            out->first_tried[k] = c.first;
        }
        if (c.ms < best.ms) best = c;
        return rc;
    };
    for (Cand &c : cands) {
        const int rc = record(c);
        if (rc == PIC_POISSON_ENOMEM || rc == PIC_POISSON_ECUDA || rc == PIC_POISSON_EINVAL) return rc;
    }
    if (best.pre == 0 && best.post == 0) {
        set_error("no candidate schedule reached tol %g", tol);
        return last_err ? last_err : PIC_POISSON_ENOTCONVERGED;
    }
    for (int threads : {64, 128, 512}) {
        Cand c{best.pre, best.post, best.inner, threads, 0, 1.0, 0, 0, 0.0};
        const int rc = record(c);
        if (rc == PIC_POISSON_ENOMEM || rc == PIC_POISSON_ECUDA || rc == PIC_POISSON_EINVAL) return rc;
    }
    for (int strip : {2, 4}) {
        Cand c{best.pre, best.post, best.inner, best.threads, strip, 1.0, 0, 0, 0.0};
        const int rc = record(c);
        if (rc == PIC_POISSON_ENOMEM || rc == PIC_POISSON_ECUDA || rc == PIC_POISSON_EINVAL) return rc;
    }
    static const int sor_sched[][2] = {{1, 1}, {1, 2}, {2, 1}, {2, 2}};
    const Cand base = best;
    for (double omega : {1.1, 1.2, 1.3})
        for (const auto &s : sor_sched) {
            Cand c{s[0], s[1], base.inner, base.threads, base.strip, omega, 0, 0, 0.0};
            const int rc = record(c);
            if (rc == PIC_POISSON_ENOMEM || rc == PIC_POISSON_ECUDA || rc == PIC_POISSON_EINVAL) return rc;
        }
    if (mixed && !composite)
        for (const auto &s : sor_sched)
            for (int inner = 1; inner <= 6; ++inner) {
                Cand c{s[0], s[1], inner, base.threads, base.strip, 1.0, 1, 0, 0.0};
                const int rc = record(c);
                if (rc == PIC_POISSON_ENOMEM || rc == PIC_POISSON_ECUDA || rc == PIC_POISSON_EINVAL) return rc;
            }
    static const int fmg_sched[][2] = {{1, 2}, {2, 1}, {2, 2}};
    if (!mixed)
        for (const auto &s : fmg_sched) {
            Cand c{s[0], s[1], base.inner, base.threads, base.strip, 1.0, 0, 1, 0.0};
            const int rc = record(c);
            if (rc == PIC_POISSON_ENOMEM || rc == PIC_POISSON_ECUDA || rc == PIC_POISSON_EINVAL) return rc;
        }
    // a larger first correction: two outer iterations may then reach tol
    // where three were needed (one FP64 defect, update and test fewer)
    if (mixed) {
        const Cand top = best;
        for (int inner : {top.inner, top.inner - 1})
            for (int extra = 1; inner >= 1 && extra <= 3; ++extra) {
                Cand c = top;
                c.inner = inner;
                c.first = inner + extra;
                const int rc = record(c);
                if (rc == PIC_POISSON_ENOMEM || rc == PIC_POISSON_ECUDA || rc == PIC_POISSON_EINVAL) return rc;
            }
    }
    out->pre_sweeps = best.pre;
    out->post_sweeps = best.post;
    out->inner_cycles = best.inner;
    out->inner_first = best.first > best.inner ? best.first : best.inner;
    out->smooth_threads = best.threads;
    out->smooth_strip = best.strip;
    out->omega = best.omega;
    out->smooth_fused = best.fused;
    out->fmg = best.fmg;
    out->ms = best.ms;
    return PIC_POISSON_OK;
}
