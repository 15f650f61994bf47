// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "fastdiv.h"
#include "pic_poisson.h"

namespace pp {

// ------------------------------------------------------------------ errors
void set_error(const char *fmt, ...);
void clear_error();

#define PP_CUDA(call)                                                                   \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess) {                                                        \
            ::pp::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),     \
                            __FILE__, __LINE__);                                        \
            return PIC_POISSON_ECUDA;                                                   \
        }                                                                               \
    } while (0)

// ------------------------------------------------------------------ complex vector types
template <class T> struct V2t;
template <> struct V2t<double> { using type = double2; };
template <> struct V2t<float> { using type = float2; };
template <class T> using V2 = typename V2t<T>::type;

constexpr int kMaxBatch = PIC_POISSON_MAX_BATCH;

// ------------------------------------------------------------------ one multigrid level
// Coefficients of A_m on a uniform level (appendix Eqs. interior_face_conductances,
// dirichlet_face_conductances), separated by direction:
//   (A_m u)_(i,k) = (D0r_i + tz_k cz_i + lambda_m mu_i) u_(i,k)
//                   - cw_i u_(i-1,k) - ce_i u_(i+1,k) - cz_i (u_(i,k-1) + u_(i,k+1))
// with cw_0 = ce_(nr-1) = 0 (Dirichlet r faces fold into D0r) and the axial
// neighbour terms dropped on the wall rows, whose tz is 3 (one interior face plus
// a half-distance Dirichlet face of conductance 2 cz) instead of 2.
struct LevelHost {
    int nr = 0, nz = 0;
    double dr = 0, dz = 0;        // dr: the mean radial width (the spacing itself on a uniform mesh)
    std::vector<double> rf;       // [nr + 1] radial faces
    std::vector<double> rc, drc;  // [nr] cell centres (face midpoints) and widths
    int ncls = 0;                 // distinct axial row classes: min(nz, 3)
    std::vector<double> cw, ce, cz, d0r, mu;   // per radial index
    std::vector<double> tz;       // per class
    std::vector<double> invd, diag;             // [ncls][nr][nm]
    std::vector<double> hw, he, hz;             // [ncls][nr][nm]: cw, ce, cz divided by diag
    // composite domain (empty otherwise): active flags [nz][nr], the coefficient
    // class of every row [nz] (rows with the same active pattern in themselves
    // and both neighbours share one), and each class's sum of face conductances
    // D0 [ncls][nr] (zero for inactive cells)
    std::vector<unsigned char> act;
    std::vector<int> rcls;
    std::vector<double> d0c;
    // non-uniform axial mesh (empty otherwise): faces [nz+1], centres and widths [nz]
    std::vector<double> zf, zc, dzc;
    // per-row tables (composite domain or non-uniform axial mesh): north
    // coupling hn [ncls][nr][nm] (hz then holds the south one) and the four
    // face conductances toward active neighbours [ncls][nr] (0 across a
    // Dirichlet face) for the residual
    std::vector<double> hn, ccw, cce, ccs, ccn;
};

// One level of one problem, as the kernels see it.
template <class T> struct LevelDev {
    int nr, nz, nm, ncls;
    unsigned rnm, rnr, rhr;       // floor((2^32 - 1) / d) for d = nm, nr, nr / 2 (fdiv, fastdiv.h)
    int nt;                       // azimuthal cells (Parseval weights of the norms)
    int init;                     // what a restriction into the next level writes (see launch_residual_restrict)
    int strip;                    // smoother: rows of one parity updated per thread (1, 2 or 4; 0: one entry)
    T relax;                      // 1 - omega (over-relaxed smoother; the h tables and invd carry omega)
    const T *cw, *ce, *cz;        // [nr]
    const T *invd, *diag;         // [ncls][nr][nm]: omega / diag, diag
    const T *hw, *he, *hz;        // [ncls][nr][nm] omega * off-diagonal conductances / diag
    const int *rcls;              // per-row tables (composite domain or non-uniform axial mesh): coefficient
                                  // class of each row [nz]; null: rows 0 and nz-1 are classes 0 and
                                  // ncls-1, the others class 1.  An inactive cell has zero diag, invd and
                                  // h entries, holds u = 0 and has no residual
    int holes;                    // the level has cells outside a composite domain's patches
    const T *hn;                  // per-row tables: omega * north conductance / diag (hz: the south one)
    const T *ccw, *cce, *ccs, *ccn;   // per-row tables: face conductances [ncls][nr] for the residual
    V2<T> *u;                     // iterate / correction, [nz][nr][nm]
    V2<T> *b;                     // right-hand side, [nz][nr][nm]
    V2<T> *bh;                    // right-hand side / diag, [nz][nr][nm]
};

// Coarsest level: separable direct solve (z eigenbasis, tridiagonal in r).
template <class T> struct CoarseDev {
    int nr, nz, nm;
    const T *V;                   // [nz][nz] orthonormal eigenvectors of the axial operator, V[k*nz+j]
    const T *e;                   // [nr] off-diagonal -ce_i of the radial operator
    const T *piv;                 // [nm][nz][nr] inverse pivots of the Thomas factorisation
    const T *cpr;                 // [nm][nz][nr] upper multipliers of the Thomas factorisation
    // composite domain (nact > 0): dense solve over the nact active cells,
    // A_m = A_0 + lambda_m diag(mu) = M^(-1/2) Q (Lambda + lambda_m) Q^T M^(-1/2) with M = diag(mu)
    int nact;
    const int *aidx;              // [nact] cell index k nr + i of each active cell
    const int *amap;              // [nz][nr] active index of a cell, -1 when inactive
    // (applied in FP32 for both precisions: a coarse-grid correction)
    const float *Q;               // [nact][nact] eigenvectors, Q[a nact + j]
    const float *QT;              // [nact][nact] the transpose
    const float *lam;             // [nact] eigenvalues of M^(-1/2) A_0 M^(-1/2)
    const float *isq;             // [nact] 1 / sqrt(mu) of each active cell
    const float *lamm;            // [nm] lambda_m
    float *Y, *Z;                 // [2 nm][nact] scratch of the dense solve: y = M^(-1/2) b scaled, then
                                  // z = (Lambda + lambda_m)^(-1) Q^T y, one column per (mode, part)
    double *up;                   // [2 nm] the power of two each column was scaled down by
};

// Work of one launch over a batch of problems: problem p owns the blocks
// [start[p], start[p+1]) of the grid; f / c are its fine / coarse level views.
// done: the convergence loop's per-problem stop flags (Ctrl::done) or null;
// blocks of a problem that has stopped return at once, so its iterate stays
// the one whose residual was reported while other problems of the batch go on.
template <class T> struct LaunchTab {
    int n;
    const int *done;
    int pid[kMaxBatch];           // problem index of each entry (entries list only the problems that take part)
    unsigned start[kMaxBatch + 1];
    LevelDev<T> f[kMaxBatch];
    LevelDev<T> c[kMaxBatch];
};

template <class T> struct CoarseTab {
    int n;
    const int *done;
    int pid[kMaxBatch];           // problem index of each entry (entries list only the problems that take part)
    unsigned start[kMaxBatch + 1];
    LevelDev<T> f[kMaxBatch];
    CoarseDev<T> c[kMaxBatch];
    size_t smem;                  // dynamic shared memory of the largest problem
};

// The dense coarsest solves of a batch (csrc/dense.cu): problem p owns the
// blocks [start[p], start[p+1]) of the preparation launch (one per mode and
// part) and [gstart[p], gstart[p+1]) of each GEMM launch (one per tile).
template <class T> struct DenseTab {
    int n;
    const int *done;
    int pid[kMaxBatch];
    unsigned start[kMaxBatch + 1];
    unsigned gstart[kMaxBatch + 1];
    LevelDev<T> f[kMaxBatch];     // the coarsest level (b in, u out)
    CoarseDev<T> c[kMaxBatch];
};

struct DefectTab {                // mixed precision: FP64 level 0 and FP32 level 0 of each problem
    int n;
    const int *done;
    int pid[kMaxBatch];           // problem index of each entry (entries list only the problems that take part)
    unsigned start[kMaxBatch + 1];
    LevelDev<double> d[kMaxBatch];
    LevelDev<float> s[kMaxBatch];
    int init_red[kMaxBatch];
};

// Azimuthal transforms of one problem's finest level.
struct FFTProb {
    int nr, nt, nz, nm, ncls, log2M;
    const double *tw;             // [max(M/2,1)] e^{-2 pi i t / M}, M = nt / 2, as (scale, ratio) pairs
    const double *tw2;            // [M+1] e^{-2 pi i m / nt}, same form (see tw_rot)
    const float4 *twf, *tw2f;     // the same tables in double-float, (a_hi, a_lo, b_hi, b_lo)
    double half_inv_n;            // 1 / (2 nt)
    const double *s;              // [nr] s_i (Eq. mode_rhs), [nz][nr] when s_rows; null: plain 1/N transform
    int s_rows;                   // composite domain: s per cell, 0 outside the patches
    const int *rcls;              // composite domain: level-0 coefficient class per row (b_hat)
    const double *bD;             // [nz][nr] Dirichlet right-hand side; may be null
    const double *invd;           // level-0 inverse diagonal [ncls][nr][nm]; null: no b_hat
    double2 *b;                   // mode-layout output of the forward transform
    double2 *bh;                  // b / diag (may be null)
    const double2 *uhat;          // mode-layout input of the inverse transform
    const double *rho;            // (nz, nt, nr) input of the forward transform
    double *phi;                  // (nz, nt, nr) output of the inverse transform
    const double2 *guess;         // mode-layout initial iterate copied into b (mode-space guesses)
};

struct FFTTab {
    int n;
    unsigned start[kMaxBatch + 1];
    FFTProb p[kMaxBatch];
    size_t smem;
};

// Device-side state of the convergence loop (one per plan).
// tol <= 0 (solve to the rounding floor): the loop stops once the relative
// residual has not fallen below half of its last reference value (the value
// at the last halving) in this many consecutive convergence tests.  Six
// tolerates a contraction of up to 0.89 per test, as on strongly stretched
// meshes where the point smoother loses much of its effect.
constexpr int kFloorWindow = 6;

struct Ctrl {
    double tol;                   // per solve
    int max_cycles;               // per solve
    int inc;                      // cycles added by one pass of the loop body
    int inc_first;                // cycles added by the first pass (mixed: inner_first)
    int cycles;                   // V-cycles applied so far
    int cont;                     // 1 while some problem is still iterating
    int n;                        // problems
    int scaled;                   // residual partials are of the sigma-scaled residual (mixed)
    double bnorm2[kMaxBatch];     // Parseval-weighted ||b||^2
    double rel[kMaxBatch];        // latest relative residual
    double best[kMaxBatch];       // reference relative residual: the value at the last halving (floor detection)
    double sigma_used[kMaxBatch]; // mixed: scale of the correction problem being solved
    double inv_sigma_used[kMaxBatch];
    double sigma_next[kMaxBatch]; // mixed: scale for the next defect
    double count[kMaxBatch];      // cells of the 3-D grid (scale normalisation)
    double rel_first[kMaxBatch];  // relative residual at the first convergence test
    int stall[kMaxBatch];
    int status[kMaxBatch];
    int done[kMaxBatch];
    int done_cycles[kMaxBatch];
    unsigned rbegin[kMaxBatch];   // residual-norm partials of problem p: [rbegin, rend)
    unsigned rend[kMaxBatch];
};

// First stage of the residual-norm reduction: each block sums PSUM_CHUNK
// consecutive block partials of one problem, so the convergence test (one
// block) adds a few dozen numbers instead of tens of thousands -- on one SM
// the FP64 additions alone took longer than the rest of the test.
constexpr int PSUM_CHUNK = 2048;
struct PsumTab {
    int n;
    unsigned start[kMaxBatch + 1];    // blocks (chunks) of problem p: [start[p], start[p+1])
    unsigned in_begin[kMaxBatch];     // its first-level partials
    unsigned in_end[kMaxBatch];
};

// ------------------------------------------------------------------ launchers
// All launchers enqueue on `st` and return cudaGetLastError().  `grid` is the
// table's total block count (start[n]); tables live in device memory.
cudaError_t launch_forward(const FFTTab *tab, unsigned grid, size_t smem, double *partials, cudaStream_t st);
cudaError_t launch_inverse(const FFTTab *tab, unsigned grid, size_t smem, cudaStream_t st);
// The forward transform in double-float arithmetic (fft_df.cu), for the mixed form.
cudaError_t launch_forward_df(const FFTTab *tab, unsigned grid, size_t smem, double *partials, cudaStream_t st);
// b = guess for every problem of the table (mode-layout initial iterates).
cudaError_t launch_copy_guess(const FFTTab *tab, unsigned grid, cudaStream_t st);

// threads: block size of the smoother (64, 128, 256 or 512; the table's block
// ranges must have been computed with the same size).
// strip: see pic_poisson_desc.smooth_strip; sor: over-relaxed update (omega != 1).
template <class T>
cudaError_t launch_smooth(const LaunchTab<T> *tab, unsigned grid, int color, int threads, int strip, bool sor,
                          cudaStream_t st, bool rowwise = false);
// red_only: residual of the red fine cells only (valid right after a black half-sweep).
// Per problem, f.init selects what is written into the coarse level c: 0 = b only
// (coarsest, solved directly); 1 = also b_hat and u = 0; 2 = also b_hat and
// u = (red ? b_hat : 0), the first red half-sweep from zero.
// masked: the plan holds per-row tables -- a composite domain or a
// non-uniform axial mesh (class tables per row, no residual or correction
// outside the patches); false runs the plain kernels.
template <class T>
cudaError_t launch_residual_restrict(const LaunchTab<T> *tab, unsigned grid, bool red_only, double *partials,
                                     cudaStream_t st, bool masked = false);
// r = b - A_m u on level f of every problem (r_out: optional per-problem output
// in c[p].u), Parseval-weighted norms of r and b into partials[block] and
// partials[partial_stride + block].
template <class T>
cudaError_t launch_residual(const LaunchTab<T> *tab, unsigned grid, bool write_r, double *partials,
                            unsigned partial_stride, cudaStream_t st, bool masked = false);
template <class T>
cudaError_t launch_prolong(const LaunchTab<T> *tab, unsigned grid, bool black_only, cudaStream_t st,
                           bool masked = false);
template <class T>
cudaError_t launch_coarse(const CoarseTab<T> *tab, unsigned grid, size_t smem, cudaStream_t st);
// Dense coarsest solves, in stage order: 0 preparation (g_prep blocks), 1 and 2 the two GEMMs (g_gemm blocks).
template <class T>
cudaError_t launch_dense(const DenseTab<T> *tab, int stage, unsigned g_prep, unsigned g_gemm, cudaStream_t st);
unsigned dense_gemm_blocks(int nact, int nm);   // GEMM blocks of one problem
// Full-multigrid start: u_f = P u_c on every fine cell (black_only: on the
// black ones, for a red Gauss-Seidel half-sweep to follow); coarse b =
// restricted fine b.
template <class T>
cudaError_t launch_interp(const LaunchTab<T> *tab, unsigned grid, cudaStream_t st, bool masked = false,
                          bool black_only = false);
template <class T>
cudaError_t launch_rhs_restrict(const LaunchTab<T> *tab, unsigned grid, cudaStream_t st, bool masked = false);

// zero_x: the FP64 iterate is zero (r = b; the kernel also writes x = 0).
cudaError_t launch_defect(const DefectTab *tab, unsigned grid, const Ctrl *ctrl, double *partials, bool zero_x,
                          cudaStream_t st, bool masked = false);
cudaError_t launch_update(const DefectTab *tab, unsigned grid, const Ctrl *ctrl, cudaStream_t st);

// Sums of the forward transform's partials per problem -> ctrl->bnorm2; initial
// scale of the mixed correction problem.
cudaError_t launch_bnorm(Ctrl *ctrl, const FFTTab *fft, const double *partials, cudaStream_t st);
// Convergence test: per-problem residual norms from partials, stop rule,
// cycle count (+inc when counting == 1, +inc_first when 2), graph
// conditionals (use_handle bit 0: handle, bit 1: handle2).
// out[start[p] + c] = sum of chunk c of problem p's partials (fixed order).
cudaError_t launch_psum(const PsumTab *tab, unsigned grid, const double *partials, double *out, cudaStream_t st);
cudaError_t launch_check(Ctrl *ctrl, const double *partials, int counting, cudaGraphConditionalHandle handle,
                         cudaGraphConditionalHandle handle2, int use_handle, cudaStream_t st);
// Plain sum of n partials into *out (single problem helpers).
cudaError_t launch_sum(const double *partials, int n, double *out, cudaStream_t st);

cudaError_t measure_fma(cudaStream_t st, double *fp64_gflops, double *fp32_gflops);

// Threads per block of the multigrid kernels and the block count a launch
// over `entries` work items of one problem needs.
constexpr int MG_THREADS = 256;
inline unsigned mg_blocks(size_t entries, int threads = MG_THREADS) {
    return (unsigned)((entries + threads - 1) / threads);
}
// Blocks of one smoother launch over a level (see k_smooth): rows of each
// parity in strips of `strip`, and per strip the (nr/2) * nm entries of one
// colour of a row.
inline unsigned smooth_blocks(int nr, int nz, int nm, int strip, int threads) {
    const size_t w = (size_t)(nr / 2) * nm;
    const unsigned bx = (unsigned)((w + threads - 1) / threads);
    const unsigned s0 = (unsigned)(((nz + 1) / 2 + strip - 1) / strip), s1 = (unsigned)((nz / 2 + strip - 1) / strip);
    return (s0 + s1) * bx;
}
// Fused multi-sweep smoother of one FP32 level of one problem (fused.cu).
struct FusedProb {
    LevelDev<float> L;            // the level (coefficient tables, b_hat; L.u is not used)
    LevelDev<float> C;            // the next coarser level (restriction fused into pre-smoothing)
    int init;                     // what the fused restriction writes into C (as LevelDev::init)
    const float2 *in;             // iterate before the half-sweeps
    float2 *out;                  // iterate after them (another buffer)
    int G, ngroups;               // modes per block, mode groups
    int P, ntiles;                // column pairs per block (halo included), column tiles
    int R, nkr;                   // output rows per block, row ranges
};
struct FusedTab {
    int n;
    const int *done;
    int pid[kMaxBatch];           // problem index of each entry (entries list only the problems that take part)
    unsigned start[kMaxBatch + 1];
    FusedProb p[kMaxBatch];
};
constexpr int FUSED_THREADS = 256;
// nh = 2 or 4 half-sweeps, red first; res: also the red-cell residual and
// its restriction into FusedProb::C (levels coarsened 2:1 in r and z).
// rw: per-row coefficient classes (composite domains; plain problems of the
// batch keep the three-class path).
cudaError_t launch_smooth_fused(const FusedTab *tab, unsigned grid, int nh, bool res, cudaStream_t st, bool rw);
// Block shape and count for an nr x nz level with nm modes (about target_blocks blocks).
void fused_shape(int nr, int nz, int nm, int nh, bool res, int target_blocks, FusedProb &f, unsigned &blocks);

// Mode-local bottom of the V-cycle (bottom.cu): the level above the coarsest
// (U) and the coarsest level's solve, one block per (problem, mode, part).
template <class T> struct BottomProb {
    LevelDev<T> U;
    CoarseDev<T> D;
    int pre, post;                // sweeps
    int red_only, black_only;     // restriction of the red cells, prolongation to the black cells
};
template <class T> struct BottomTab {
    int n;
    const int *done;
    int pid[kMaxBatch];           // problem index of each entry (entries list only the problems that take part)
    unsigned start[kMaxBatch + 1];
    BottomProb<T> p[kMaxBatch];
};
constexpr int BOTTOM_THREADS = 1024;
constexpr size_t BOTTOM_MAX_SMEM = 200 * 1024;
template <class T> size_t bottom_smem_bytes(int nr, int nz, int ncls, int ncr, int ncz);
template <class T> cudaError_t launch_bottom(const BottomTab<T> *tab, unsigned grid, size_t smem, cudaStream_t st);

// Pieces of the separable coarsest-level solve shared by k_coarse (mg.cu) and
// k_bottom (bottom.cu).
//
// One element copied from global to shared memory by cp.async (4 or 8
// bytes, no register round trip): a block issues every load of its problem
// before it waits once, instead of one L2 round trip per loop step.
template <class T> __device__ __forceinline__ void cp_async_elem(T *smem, const T *gmem) {
    static_assert(sizeof(T) == 4 || sizeof(T) == 8, "4- or 8-byte elements");
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(sa), "l"(gmem), "n"((int)sizeof(T)) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
// Close the thread's current group of copies; wait until at most N groups are in flight.
__device__ __forceinline__ void cp_async_group_close() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_group_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// The radial tridiagonal solves of the separable coarsest solve, one per
// axial eigenvector j < nz, in place on the rows ws[j][0 .. nr) (row stride
// lw): forward y_i = (w_i - e_(i-1) y_(i-1)) piv_i, back x_i = y_i - cpr_i x_(i+1),
// with the factorisation piv, cpr ([nz][lw]) and e ([nr - 1]) staged in shared
// memory, so that a step of the recurrence waits on shared memory rather than
// on L2.  The nz recurrences are spread over the block's first four warps
// (one per SM sub-partition; the block has at least 128 threads).
template <class T>
__device__ __forceinline__ void thomas_rows(T *ws, const T *ps, const T *cs, const T *es, int nz, int nr, int lw) {
    const int w = (int)(threadIdx.x >> 5), lane = (int)(threadIdx.x & 31), per = (nz + 3) >> 2;
    if (w >= 4) return;
    for (int l = lane; l < per; l += 32) {
        const int j = w * per + l;
        if (j >= nz) break;
        const T *piv = ps + (size_t)j * lw, *cpr = cs + (size_t)j * lw;
        T *row = ws + (size_t)j * lw;
        T y = row[0] * piv[0];
        row[0] = y;
        for (int i = 1; i < nr; ++i) {
            y = (row[i] - es[i - 1] * y) * piv[i];
            row[i] = y;
        }
        T x = y;
        for (int i = nr - 2; i >= 0; --i) {
            x = row[i] - cpr[i] * x;
            row[i] = x;
        }
    }
}

constexpr int FFT_TI = 32;        // radial columns per transform CTA
constexpr int FFT_THREADS = 256;
size_t fft_smem_bytes(int nt);

// Twiddle tables of the transforms hold w = e^{-i theta}, theta = 2 pi t / n,
// as a scale and a ratio: w = rho a (1 + i b) with a = cos theta', b =
// -tan theta', theta' = theta - rot pi/2 and rho = (-i)^rot, where rot = 1
// for theta in (pi/4, 3 pi/4) keeps |b| <= 1.  A complex product w z then
// costs two multiply-adds, u = z + i b z, plus the scale a, which folds into
// the butterfly's own multiply-adds; the factor rho is a swap of the parts
// of u and a sign, done with integer instructions.
__host__ __device__ inline bool tw_rot(int t, int n) { return !(8 * t <= n || 8 * t >= 3 * n); }

// 3x3 convolution on the tcgen05 tensor cores (conv_tc.cu): 0 on success, 1
// when the shape or alignment is not taken (run the mma.sync kernel), else a
// PIC_POISSON_* error.
int launch_conv3x3_tc(const void *in, int cin, const void *w, const float *bias, void *out, float *out32, int cout,
                      int n, int h, int wd, int relu, cudaStream_t st);

}  // namespace pp
