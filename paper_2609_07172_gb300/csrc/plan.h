// The plan: host-side description of a batch of problems, its device
// workspace, the launch tables of every kernel, and the captured graph.
#pragma once

#include "internal.h"

namespace pp {

struct ProblemPlan {
    pic_poisson_desc d{};                       // resolved descriptor (wall arrays point below)
    std::vector<double> rin_z, rout_z;
    std::vector<double> rf0;                    // level-0 radial faces (given or uniform)
    std::vector<int> patches;                   // composite domain: 4 ints per patch (empty: the annulus)
    std::vector<double> zf0;                    // level-0 axial faces when given (empty: uniform)
    int nact = 0;                               // composite domain: active cells of the coarsest level
    bool uniform_r = true;
    int L = 0, nm = 0;
    std::vector<LevelHost> lv;
    std::vector<LevelDev<double>> dl;           // FP64 levels (all for FP64 plans, level 0 for mixed)
    std::vector<LevelDev<float>> fl;            // FP32 levels (mixed)
    std::vector<float2 *> u2;                   // FP32 levels: second iterate buffer of the fused smoother
    CoarseDev<double> cd{};
    CoarseDev<float> cf{};
    const double *tw = nullptr, *tw2 = nullptr; // FFT twiddles
    const float4 *twf = nullptr, *tw2f = nullptr; // the same in double-float (mixed form)
    bool bottom = false;                        // levels L-2 and L-1 solved by k_bottom
    int smoothed() const { return L - 1 - (bottom ? 1 : 0); }   // levels 0 .. smoothed()-1 use the level kernels
    double *s0 = nullptr, *bD0 = nullptr;       // level-0 right-hand-side factors
    double *mask0 = nullptr;                    // composite domain: 1 on active cells, 0 elsewhere [nz][nr]
    double *fwin = nullptr, *fwout = nullptr;   // face-field reconstruction: r-wall potentials [nz]
    double *finv_rda = nullptr;                 // and 1 / (r_i dalpha) [nr]
    double *finv_rd = nullptr;                  // and 1 / radial face distances [nr + 1]
    double *dep_inv_vr = nullptr, *dep_inv_vz = nullptr;   // CIC deposit: 1 / node-volume factors [nr+1], [nz+1]
    double *dep_flo = nullptr, *dep_fhi = nullptr;         // projection: radial octant shares [nr]
    // level-0 geometry of the steps around the solve on non-uniform meshes and
    // composite domains (field.cu, deposit.cu)
    double *finv_zd = nullptr;                  // face field: 1 / axial face distances [nz + 1]
    double *finv_half = nullptr;                // 1 / centre-to-face distances: r lower, r upper [nr] each,
                                                // z lower, z upper [nz] each
    unsigned char *act0 = nullptr;              // composite domain: active flags [nz][nr] (null otherwise)
    double *dep_inv_v2 = nullptr;               // composite: 1 / node volumes of active octants [nz+1][nr+1]
    double *dep_rf = nullptr, *dep_zf = nullptr;         // faces [nr + 1], [nz + 1]
    double *dep_inv_wr = nullptr, *dep_inv_wz = nullptr; // 1 / cell widths [nr], [nz]
    int *dep_rbin = nullptr, *dep_zbin = nullptr;        // cell at the lower end of each lookup bin
    int dep_nrbin = 0, dep_nzbin = 0;                    // lookup bins per axis
    float dep_inv_rbw = 0.f, dep_inv_zbw = 0.f;          // 1 / bin widths (a guess only; binary32)
};

// Launch tables of one precision's hierarchy, per level l = 0 .. Lmax-2
// (problems that have a level below l), plus the coarsest-level solve.
template <class T> struct Hier {
    std::vector<LaunchTab<T> *> smooth, restr, prolong;   // device tables (null when no problem takes part)
    std::vector<unsigned> g_smooth, g_restr, g_prolong;   // grids
    std::vector<int> strip;                               // smoother strip per level
    bool fused = false;                                   // FP32 fused smoother (pre: u -> u2, post: u2 -> u)
    std::vector<FusedTab *> fpre, fpost;
    std::vector<unsigned> g_fpre, g_fpost;
    std::vector<char> fres;                               // per level: pre-smoothing also restricts
    CoarseTab<T> *coarse = nullptr;           // problems solved by k_coarse (separable coarsest level)
    DenseTab<T> *dense = nullptr;             // problems with a dense coarsest solve (csrc/dense.cu)
    unsigned g_dense_prep = 0, g_dense_gemm = 0;
    unsigned g_coarse = 0;
    size_t smem_coarse = 0;
    std::vector<LaunchTab<T> *> rhs, interp;  // full-multigrid start: b restricted to l + 1, u_l = P u_(l+1)
    bool interp_black = false;                // u_l = P u_(l+1) on the black cells only (the red half-sweep
                                              // that follows overwrites the red ones unread)
    std::vector<unsigned> g_rhs, g_interp;
    BottomTab<T> *bottom = nullptr;           // problems with a mode-local bottom
    unsigned g_bottom = 0;
    size_t smem_bottom = 0;
};

// Algorithmic traffic / arithmetic / launches recorded per kernel class.
struct Tally {
    double bytes[PIC_POISSON_NPHASE] = {0}, flops[PIC_POISSON_NPHASE] = {0};
    int launches[PIC_POISSON_NPHASE] = {0};
};

}  // namespace pp

struct pic_poisson_plan_s {
    int n = 0;
    std::vector<pp::ProblemPlan> pr;
    pic_poisson_desc shared{};                  // settings common to the batch (descs[0])
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t cap0 = nullptr, cap1 = nullptr;// capture streams (graph construction)
    int Lmax = 0;
    void *arena = nullptr;
    size_t arena_bytes = 0;

    // launch tables (device) and their grids
    pp::FFTTab *fwd = nullptr, *guess = nullptr, *inv = nullptr, *api_fft = nullptr;
    unsigned g_fft = 0;
    size_t smem_fft = 0;
    pp::FFTTab h_fwd{}, h_guess{}, h_inv{};     // host copies (rho / phi pointers patched per solve)
    pp::Hier<double> h64;
    pp::Hier<float> h32;
    pp::LaunchTab<double> *res_single = nullptr;// FP64 residual norms of single-level problems
    unsigned g_res_single = 0;
    unsigned res_single_offset = 0;             // their place in the partials buffer
    pp::LaunchTab<double> *api_res = nullptr;   // mode-residual stage call (problem 0)
    pp::LaunchTab<double> h_api_res{};
    unsigned g_api_res = 0;
    pp::DefectTab *defect = nullptr;
    unsigned g_defect = 0;

    pp::Ctrl *ctrl = nullptr;                   // device
    pp::Ctrl hctrl{};                           // per-solve initial state
    pp::Ctrl *hctrl_out = nullptr;              // pinned, results
    double *partials = nullptr, *partials_fwd = nullptr;
    size_t npartials = 0, npartials_fwd = 0;
    double *partials2 = nullptr;                // first-stage sums of the residual partials (PsumTab)
    pp::PsumTab *psum = nullptr;                // device, its table
    unsigned g_psum = 0;                        // its blocks
    double *dsum = nullptr, *hsum = nullptr;    // small device / pinned scratch for stage calls

    // graphs of the whole solve (PIC_POISSON_GRAPH); [0]: initial iterate per
    // the plan's flags, [1]: mode-layout initial iterate
    cudaGraph_t graph[2] = {nullptr, nullptr};
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    cudaGraphConditionalHandle handle{};        // the convergence loop's while node
    cudaGraphConditionalHandle handle_first{};  // if node of a larger first pass (mixed, inner_first)
    pp::Tally seg[2][4];                        // prologue, loop body, epilogue, first pass (at capture)
    const double *last_guess[pp::kMaxBatch] = {};

    std::vector<cudaEvent_t> evs;               // PROFILE events
    double *stage_rho = nullptr, *stage_phi = nullptr;   // pic_poisson_solve_host staging
    const double *last_rho[pp::kMaxBatch] = {};
    double *last_phi[pp::kMaxBatch] = {};
    bool io_valid = false;
    bool masked = false;                        // some problem has per-row tables (composite domain or
                                                // non-uniform axial mesh): the masked kernel variants
};

namespace pp {
int plan_enter(pic_poisson_plan_s *P);
}
