// Mode-batched matrix-free multigrid kernels (steps a-3 .. a-7), the FP64
// defect / update kernels of the mixed-precision form, and the device-side
// convergence test.
//
// Every kernel works on the cell-major, mode-fast layout of Eq. mode_fast_layout
// (entry (k, i, m) at (k*nr + i)*nm + m, unpadded): consecutive threads take
// consecutive modes of one cell and then move to the next cell, so every load
// and store of a warp is contiguous.  Only the diagonal shift lambda_m mu of
// A_m depends on the mode (Eq. shifted_operator_family); it enters through
// per-level tables indexed (row class, i, m).
//
// One launch serves a batch of independent problems of different sizes (and
// different azimuthal mode counts): problem p owns a contiguous range of
// blocks, found by a binary search over the launch table; every block belongs
// to one problem, so per-block norm partials never mix problems.
//
// On GB300 FP64 runs at 1/64 of the FP32 rate, so the FP64 kernels are bound
// by FP64 instructions, and every kernel here is arranged to issue as few as
// the iteration allows (all rewrites below are exact in exact arithmetic):
//  * the smoother uses coefficients pre-divided by the diagonal and a
//    right-hand side b_hat = b / diag, so one Gauss-Seidel update is
//    u = b_hat + h_z (u_S + u_N) + h_w u_W + h_e u_E (4 FP64 ops per component);
//  * after a black half-sweep the black cells satisfy their equations, so the
//    residual (and the restricted right-hand side) only needs the red cells;
//  * the red half-sweep that follows a prolongation overwrites the red cells
//    without reading them, so only black cells receive the correction;
//  * on coarse levels the first red half-sweep from a zero iterate is just
//    u_red = b_hat_red, written by the restriction kernel.
#include "internal.h"

namespace pp {
namespace {

template <class T> __device__ __forceinline__ V2<T> mk(T x, T y);
template <> __device__ __forceinline__ double2 mk<double>(double x, double y) { return make_double2(x, y); }
template <> __device__ __forceinline__ float2 mk<float>(float x, float y) { return make_float2(x, y); }

__device__ __forceinline__ int row_class(int k, int nz, int ncls) {
    return k == 0 ? 0 : (k == nz - 1 ? ncls - 1 : 1);
}

// Coefficient class of row k of a level: its own per-row table in a composite
// domain, else first / interior / last row.
template <class T> __device__ __forceinline__ int lclass(const LevelDev<T> &L, int k) {
    return L.rcls ? L.rcls[k] : row_class(k, L.nz, L.ncls);
}

template <class T> __device__ __forceinline__ V2<T> fma2(T a, V2<T> x, V2<T> y) {
    return mk<T>(fma(a, x.x, y.x), fma(a, x.y, y.y));
}

// Parseval weight of mode m for a real signal of length nt: 1 for m = 0 and
// m = nt/2, 2 otherwise (the conjugate partner of m carries the same energy).
__device__ __forceinline__ double parseval_w(int m, int nt) { return (m == 0 || 2 * m == nt) ? 1.0 : 2.0; }

// Sum of v over the block, valid in thread 0; sh holds blockDim doubles.  The
// values go through shared memory and one warp adds them, so the reduction
// issues about blockDim/32 + 5 FP64 additions per block instead of 5 per
// thread.
__device__ __forceinline__ double block_sum(double v, double *sh) {
    __syncthreads();   // a previous reduction may still be reading sh
    sh[threadIdx.x] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x < 32) {
        for (int j = threadIdx.x; j < (int)blockDim.x; j += 32) s += sh[j];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    return s;
}

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Problem owning block `blk`: the last p with start[p] <= blk.
__device__ __forceinline__ int find_problem(const unsigned *__restrict__ start, int n, unsigned blk) {
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (start[mid] <= blk) lo = mid;
        else hi = mid;
    }
    return lo;
}

// b - A_m u at entry (k, i, m), Eq. matrix_free_mode_operator.
template <class T, bool MASK>
__device__ __forceinline__ V2<T> residual_at(const LevelDev<T> &L, int k, int i, int m, size_t idx) {
    const size_t rowstride = (size_t)L.nr * L.nm;
    if (MASK && L.rcls) {
        // per-row tables (composite domain or non-uniform axial mesh; in a batch
        // the plain problems take the path below): the row class's face
        // conductances, zero across a Dirichlet face, south and north apart
        const size_t ci = (size_t)L.rcls[k] * L.nr + i;
        const T d = L.diag[ci * L.nm + m];
        // a cell outside a composite domain's patches (zero diagonal) has no
        // residual: nothing else is loaded for it
        if (d == T(0)) return mk<T>(0, 0);
        V2<T> acc = L.b[idx];
        if (k > 0) acc = fma2<T>(L.ccs[ci], L.u[idx - rowstride], acc);
        if (k < L.nz - 1) acc = fma2<T>(L.ccn[ci], L.u[idx + rowstride], acc);
        if (i > 0) acc = fma2<T>(L.ccw[ci], L.u[idx - L.nm], acc);
        if (i < L.nr - 1) acc = fma2<T>(L.cce[ci], L.u[idx + L.nm], acc);
        return fma2<T>(-d, L.u[idx], acc);
    }
    V2<T> s = mk<T>(0, 0);
    if (k > 0) s = L.u[idx - rowstride];
    if (k < L.nz - 1) {
        const V2<T> n = L.u[idx + rowstride];
        s = (k > 0) ? mk<T>(s.x + n.x, s.y + n.y) : n;
    }
    V2<T> acc = fma2<T>(L.cz[i], s, L.b[idx]);
    if (i > 0) acc = fma2<T>(L.cw[i], L.u[idx - L.nm], acc);
    if (i < L.nr - 1) acc = fma2<T>(L.ce[i], L.u[idx + L.nm], acc);
    const T d = L.diag[((size_t)row_class(k, L.nz, L.ncls) * L.nr + i) * L.nm + m];
    return fma2<T>(-d, L.u[idx], acc);
}

// One red-black Gauss-Seidel half-sweep over the cells of one colour:
//   u_q <- (b_q + sum_q' G_qq' u_q') / (D0_q + lambda_m mu_q)
// written as u = b_hat + h_z (u_S + u_N) + h_w u_W + h_e u_E with h = G / diag.
// Cells of one colour in rows of one parity share their radial index, so a
// thread owns one (radial cell, mode) and updates a strip of S rows of that
// parity (k, k+2, ...): the north neighbour of row k is the south neighbour
// of row k+2, the interior rows share one set of coefficients, and the index
// arithmetic is done once per strip.  All loads of the strip are issued before
// its first store -- the launch reads only the other colour and b_hat, which
// it does not write -- so they are in flight together.  Consecutive threads
// take consecutive modes of a cell: every load and store of a warp is
// contiguous.  Blocks: per parity, strips of rows; per strip,
// ceil((nr/2) nm / NT) blocks (smooth_blocks).
// S = 0: one entry per thread, consecutive threads over the cells of one
// colour in cell-major, mode-fast order (blocks: mg_blocks of the entries).
// SOR: over-relaxation u <- (1 - omega) u + omega u_GS, the tables carrying
// omega (one more load and multiply-add per component); otherwise omega = 1.
// RW: the plan holds per-row tables (composite domain or non-uniform axial
// mesh); the plain variant keeps the three-class rule and no such branch.
template <class T, int NT, int S, bool SOR, bool RW>
__global__ void __launch_bounds__(NT, S == 0 ? 2048 / NT : 1) k_smooth(const LaunchTab<T> *__restrict__ tab, int color) {
    const int p = find_problem(tab->start, tab->n, blockIdx.x);
    if (tab->done && tab->done[tab->pid[p]]) return;   // stopped problem of a batch
    const LevelDev<T> L = tab->f[p];
    const unsigned nm = L.nm;
    if constexpr (S == 0) {
        const unsigned e = (blockIdx.x - tab->start[p]) * NT + threadIdx.x;
        if (e >= (unsigned)L.nz * (unsigned)(L.nr >> 1) * nm) return;
        // (plain divisions: this kernel is capped at 32 registers for full
        // occupancy, and the multiply-high form needs more)
        const unsigned c = e / nm;
        const int m = (int)(e - c * nm);
        const unsigned hr = (unsigned)L.nr >> 1;
        const int k = (int)(c / hr);
        const int i = 2 * (int)(c - (unsigned)k * hr) + ((k + color) & 1);
        const size_t idx = ((size_t)k * L.nr + i) * nm + m;
        const size_t tb = ((size_t)(RW ? lclass(L, k) : row_class(k, L.nz, L.ncls)) * L.nr + i) * nm + m;
        const size_t rowstride = (size_t)L.nr * nm;
        V2<T> acc;
        if (RW && L.holes && L.invd[tb] == T(0)) return;   // outside a composite domain: u stays 0
        if (RW && L.rcls && sizeof(T) == sizeof(double)) {   // per-row tables, FP64: south (hz) and
                                                             // north (hn) couplings apart
            acc = L.bh[idx];
            if (k > 0) acc = fma2<T>(L.hz[tb], L.u[idx - rowstride], acc);
            if (k < L.nz - 1) acc = fma2<T>(L.hn[tb], L.u[idx + rowstride], acc);
        } else if (RW && L.rcls) {
            // per-row tables, FP32: u = invd (b + sum G u) from the row class's
            // face conductances (small, cached) and one per-entry table rather
            // than four per-entry h tables (on a non-uniform axial mesh every
            // row is a class, so those are as large as u).  Two more
            // multiplies: worth it on the FP32 pipe, not on the FP64 one
            // (measured both ways)
            const size_t ci = (size_t)L.rcls[k] * L.nr + i;
            acc = L.b[idx];
            if (k > 0) acc = fma2<T>(L.ccs[ci], L.u[idx - rowstride], acc);
            if (k < L.nz - 1) acc = fma2<T>(L.ccn[ci], L.u[idx + rowstride], acc);
            if (i > 0) acc = fma2<T>(L.ccw[ci], L.u[idx - nm], acc);
            if (i < L.nr - 1) acc = fma2<T>(L.cce[ci], L.u[idx + nm], acc);
            const T inv = L.invd[tb];
            acc = mk<T>(acc.x * inv, acc.y * inv);
            if (SOR) acc = fma2<T>(L.relax, L.u[idx], acc);
            L.u[idx] = acc;
            return;
        } else {
            V2<T> s = mk<T>(0, 0);
            if (k > 0) s = L.u[idx - rowstride];
            if (k < L.nz - 1) {
                const V2<T> n = L.u[idx + rowstride];
                s = (k > 0) ? mk<T>(s.x + n.x, s.y + n.y) : n;
            }
            acc = fma2<T>(L.hz[tb], s, L.bh[idx]);
        }
        if (i > 0) acc = fma2<T>(L.hw[tb], L.u[idx - nm], acc);
        if (i < L.nr - 1) acc = fma2<T>(L.he[tb], L.u[idx + nm], acc);
        if (SOR) acc = fma2<T>(L.relax, L.u[idx], acc);
        L.u[idx] = acc;
    } else {
        const unsigned w = (unsigned)(L.nr >> 1) * nm;
        const unsigned bx = (w + NT - 1) / NT;
        const unsigned lb = blockIdx.x - tab->start[p];
        const unsigned g = lb / bx;
        const unsigned x = (lb - g * bx) * NT + threadIdx.x;
        if (x >= w) return;
        const unsigned s0 = ((unsigned)(L.nz + 1) / 2 + S - 1) / S;
        const int par = g < s0 ? 0 : 1;
        const int k0 = par + 2 * (int)(g < s0 ? g : g - s0) * S;
        const unsigned j = x / nm;
        const int m = (int)(x - j * nm);
        const int i = 2 * (int)j + ((par + color) & 1);
        const size_t rs = (size_t)L.nr * nm;                 // one row of cells, all modes
        const size_t tcol = (size_t)i * nm + m;              // (i, m) within a row / a coefficient class
        const size_t t1 = (L.ncls > 1 ? rs : 0) + tcol;      // interior coefficient class
        const T hz1 = __ldg(L.hz + t1), hw1 = __ldg(L.hw + t1), he1 = __ldg(L.he + t1);
        const V2<T> zero = mk<T>(0, 0);
        const size_t idx0 = (size_t)k0 * rs + tcol;
        V2<T> south = k0 > 0 ? __ldg(L.u + idx0 - rs) : zero;
        V2<T> vn[S], vw[S], ve[S], vb[S], vo[S];
#pragma unroll
        for (int t = 0; t < S; ++t) {
            const int k = k0 + 2 * t;
            const size_t idx = idx0 + (size_t)(2 * t) * rs;
            vn[t] = vw[t] = ve[t] = vb[t] = vo[t] = zero;
            if (k < L.nz) {
                if (k < L.nz - 1) vn[t] = __ldg(L.u + idx + rs);
                if (i > 0) vw[t] = __ldg(L.u + idx - nm);
                if (i < L.nr - 1) ve[t] = __ldg(L.u + idx + nm);
                // per-row tables in FP32: b (the update multiplies by invd), else b_hat
                vb[t] = __ldg(((RW && L.rcls && sizeof(T) == sizeof(float)) ? L.b : L.bh) + idx);
                if (SOR) vo[t] = L.u[idx];   // this colour: written below, so not through the read-only path
            }
        }
#pragma unroll
        for (int t = 0; t < S; ++t) {
            const int k = k0 + 2 * t;
            if (k >= L.nz) break;
            if (RW && L.rcls && L.holes && L.invd[(size_t)L.rcls[k] * rs + tcol] == T(0)) {   // outside the patches
                south = vn[t];
                continue;
            }
            T hz = hz1, hw = hw1, he = he1;
            V2<T> acc;
            if (RW && L.rcls && sizeof(T) == sizeof(double)) {   // per-row tables, FP64
                const size_t tb = (size_t)L.rcls[k] * rs + tcol;
                hw = L.hw[tb];
                he = L.he[tb];
                acc = fma2<T>(L.hz[tb], south, vb[t]);   // absent neighbours are zero
                acc = fma2<T>(L.hn[tb], vn[t], acc);
            } else if (RW && L.rcls) {   // per-row tables, FP32: u = invd (b + sum G u), as in the S = 0 path
                const size_t ci = (size_t)L.rcls[k] * L.nr + i;
                const size_t idx = idx0 + (size_t)(2 * t) * rs;
                acc = fma2<T>(L.ccs[ci], south, vb[t]);   // absent neighbours are zero
                acc = fma2<T>(L.ccn[ci], vn[t], acc);
                if (i > 0) acc = fma2<T>(L.ccw[ci], vw[t], acc);
                if (i < L.nr - 1) acc = fma2<T>(L.cce[ci], ve[t], acc);
                const T inv = L.invd[(size_t)L.rcls[k] * rs + tcol];
                acc = mk<T>(acc.x * inv, acc.y * inv);
                if (SOR) acc = fma2<T>(L.relax, vo[t], acc);
                L.u[idx] = acc;
                south = vn[t];
                continue;
            } else {
                if (k == 0 || k == L.nz - 1) {   // boundary rows have their own coefficient class
                    const size_t tb = (size_t)row_class(k, L.nz, L.ncls) * rs + tcol;
                    hz = L.hz[tb];
                    hw = L.hw[tb];
                    he = L.he[tb];
                }
                const V2<T> s = mk<T>(south.x + vn[t].x, south.y + vn[t].y);   // absent neighbours are zero
                acc = fma2<T>(hz, s, vb[t]);
            }
            if (i > 0) acc = fma2<T>(hw, vw[t], acc);
            if (i < L.nr - 1) acc = fma2<T>(he, ve[t], acc);
            if (SOR) acc = fma2<T>(L.relax, vo[t], acc);
            L.u[idx0 + (size_t)(2 * t) * rs] = acc;
            south = vn[t];
        }
    }
}

// Residual of the fine cells of each coarse cell, summed into the coarse
// right-hand side (finite-volume restriction: a residual is a cell integral),
// with optional Parseval-weighted squared-norm partials.  RED_ONLY: only the
// two red fine cells (after a black half-sweep the black residuals vanish).
// F.init selects what else the coarse level receives (see internal.h).
template <class T, bool RED_ONLY, bool MASK>
__global__ void __launch_bounds__(MG_THREADS)
k_residual_restrict(const LaunchTab<T> *__restrict__ tab, double *__restrict__ partials) {
    __shared__ double red[MG_THREADS];
    const int p = find_problem(tab->start, tab->n, blockIdx.x);
    if (tab->done && tab->done[tab->pid[p]]) return;   // stopped problem of a batch
    const LevelDev<T> F = tab->f[p];
    const LevelDev<T> C = tab->c[p];
    const unsigned e = (blockIdx.x - tab->start[p]) * blockDim.x + threadIdx.x;
    double acc = 0.0;
    if (e < (unsigned)C.nz * (unsigned)C.nr * (unsigned)C.nm) {
        const unsigned nm = C.nm;
        // multiply-high divisions on the FP32 pipe's kernel only: with them
        // the FP64 kernel ran 6 % slower (measured)
        const unsigned cc = sizeof(T) == sizeof(float) ? fdiv(e, nm, C.rnm) : e / nm;
        const int m = (int)(e - cc * nm);
        const int K = (int)(sizeof(T) == sizeof(float) ? fdiv(cc, (unsigned)C.nr, C.rnr) : cc / (unsigned)C.nr);
        const int I = (int)(cc - (unsigned)K * C.nr);
        // coarsening factors of this level pair (semi-coarsening keeps one direction)
        const int fz = F.nz == C.nz ? 1 : 2, fr = F.nr == C.nr ? 1 : 2;
        // fine cells that carry a residual, c < nc: RED_ONLY keeps the red ones
        // (k + i even) -- the (0,0) and (1,1) corners of a 2x2 block, one cell
        // of a 2x1 pair -- otherwise all fz * fr cells
        const int nc = RED_ONLY ? (fz == 2 && fr == 2 ? 2 : 1) : fz * fr;
        auto cell = [&](int c, int &k, int &i) {
            if (RED_ONLY) {
                k = fz * K + (fz == 2 ? (fr == 2 ? c : (I & 1)) : 0);
                i = fr * I + (fr == 2 ? (fz == 2 ? c : (K & 1)) : 0);
            } else {
                k = fz * K + (fr == 2 ? (c >> 1) : c);
                i = fr * I + (fr == 2 ? (c & 1) : 0);
            }
        };
        int k, i;
        cell(0, k, i);
        V2<T> sum = residual_at<T, MASK>(F, k, i, m, ((size_t)k * F.nr + i) * nm + m);
        if (partials) acc = fma((double)sum.y, (double)sum.y, (double)sum.x * (double)sum.x);
        auto more = [&](int c) {
            cell(c, k, i);
            const V2<T> r = residual_at<T, MASK>(F, k, i, m, ((size_t)k * F.nr + i) * nm + m);
            sum = mk<T>(sum.x + r.x, sum.y + r.y);
            if (partials) acc = fma((double)r.y, (double)r.y, fma((double)r.x, (double)r.x, acc));
        };
        if constexpr (sizeof(T) == sizeof(double)) {
            // a loop, not a predicated unroll: FP64 work only for the cells that exist
#pragma unroll 1
            for (int c = 1; c < nc; ++c) more(c);
        } else {
            // FP32 is bound by load latency: unrolled, all loads in flight together
#pragma unroll
            for (int c = 1; c < 4; ++c)
                if (c < nc) more(c);
        }
        C.b[e] = sum;
        if (F.init > 0) {
            const T inv = C.invd[((size_t)(MASK ? lclass(C, K) : row_class(K, C.nz, C.ncls)) * C.nr + I) * nm + m];
            const V2<T> bh = mk<T>(sum.x * inv, sum.y * inv);
            C.bh[e] = bh;
            C.u[e] = (F.init == 2 && ((K + I) & 1) == 0) ? bh : mk<T>(0, 0);
        }
        if (partials) acc *= parseval_w(m, F.nt);
    }
    if (partials) {
        const double tot = block_sum(acc, red);
        if (threadIdx.x == 0) partials[blockIdx.x] = tot;
    }
}

// r = b - A_m u on level f (r written to c.u when write_r), Parseval-weighted
// squared norms of r into partials[block] and, when stride > 0, of b into
// partials[stride + block].
template <class T, bool MASK>
__global__ void __launch_bounds__(MG_THREADS)
k_residual(const LaunchTab<T> *__restrict__ tab, int write_r, double *__restrict__ partials, unsigned stride) {
    __shared__ double red[MG_THREADS];
    const int p = find_problem(tab->start, tab->n, blockIdx.x);
    if (tab->done && tab->done[tab->pid[p]]) return;   // stopped problem of a batch
    const LevelDev<T> L = tab->f[p];
    const unsigned e = (blockIdx.x - tab->start[p]) * blockDim.x + threadIdx.x;
    double ar = 0.0, ab = 0.0;
    if (e < (unsigned)L.nz * (unsigned)L.nr * (unsigned)L.nm) {
        const unsigned nm = L.nm;
        const unsigned c = fdiv(e, nm, L.rnm);
        const int m = (int)(e - c * nm);
        const int k = (int)fdiv(c, (unsigned)L.nr, L.rnr);
        const int i = (int)(c - (unsigned)k * L.nr);
        const V2<T> r = residual_at<T, MASK>(L, k, i, m, e);
        if (write_r) tab->c[p].u[e] = r;
        const V2<T> b = L.b[e];
        const double w = parseval_w(m, L.nt);
        ar = w * ((double)r.x * r.x + (double)r.y * r.y);
        ab = w * ((double)b.x * b.x + (double)b.y * b.y);
    }
    if (partials) {
        const double tr = block_sum(ar, red);
        if (threadIdx.x == 0) partials[blockIdx.x] = tr;
        if (stride) {
            const double tb = block_sum(ab, red);
            if (threadIdx.x == 0) partials[stride + blockIdx.x] = tb;
        }
    }
}

// Cell-centred prolongation of the coarse correction and update u += P e:
// bilinear (weights 9/16, 3/16, 3/16, 1/16 from the four nearest coarse
// centres) after 2:1 coarsening in both directions, linear (3/4, 1/4) along
// the coarsened direction after semi-coarsening.  Beyond a wall the coarse
// value is reflected with a sign change (the correction vanishes on the
// Dirichlet face).  BLACK_ONLY: only black fine cells (the red half-sweep that
// follows overwrites the red ones).
template <class T, bool BLACK_ONLY, bool ASSIGN, bool MASK>
__global__ void __launch_bounds__(MG_THREADS) k_prolong(const LaunchTab<T> *__restrict__ tab) {
    const int p = find_problem(tab->start, tab->n, blockIdx.x);
    if (tab->done && tab->done[tab->pid[p]]) return;   // stopped problem of a batch
    const LevelDev<T> F = tab->f[p];
    const LevelDev<T> C = tab->c[p];
    const unsigned e = (blockIdx.x - tab->start[p]) * blockDim.x + threadIdx.x;
    const unsigned nm = F.nm;
    const unsigned total = (unsigned)F.nz * (unsigned)(BLACK_ONLY ? (F.nr >> 1) : F.nr) * nm;
    if (e >= total) return;
    // 32-bit offsets (a plan rejects levels of 2^31 entries or more) and
    // divisions by multiply-high (fastdiv.h): the FP32 kernel is bound by
    // instruction issue, and the two 32-bit divisions and 64-bit offsets were
    // a large part of what it issued per entry
    const unsigned c = fdiv(e, nm, F.rnm);
    const int m = (int)(e - c * nm);
    int k, i;
    if (BLACK_ONLY) {
        const unsigned hr = (unsigned)F.nr >> 1;
        k = (int)fdiv(c, hr, F.rhr);
        i = 2 * (int)(c - (unsigned)k * hr) + ((k + 1) & 1);
    } else {
        k = (int)fdiv(c, (unsigned)F.nr, F.rnr);
        i = (int)(c - (unsigned)k * F.nr);
    }
    const unsigned idx = ((unsigned)k * F.nr + i) * nm + m;
    // composite domain: a cell outside the patches keeps u = 0 (in a batch the
    // masked variant also runs the plain problems, whose rcls is null; a level
    // without inactive cells -- a non-uniform axial mesh -- reads no diag)
    if (MASK && F.rcls && F.holes && F.diag[((size_t)F.rcls[k] * F.nr + i) * nm + m] == T(0)) {
        if (ASSIGN) F.u[idx] = mk<T>(0, 0);
        return;
    }
    const bool cz2 = F.nz != C.nz, cr2 = F.nr != C.nr;
    const int K = cz2 ? (k >> 1) : k, I = cr2 ? (i >> 1) : i;
    const int K2 = K + ((k & 1) ? 1 : -1);
    const int I2 = I + ((i & 1) ? 1 : -1);
    bool kin = K2 >= 0 && K2 < C.nz;
    bool iin = I2 >= 0 && I2 < C.nr;
    if (MASK && C.rcls && C.holes) {   // an exposed face reflects like a wall: the correction vanishes on it
        if (iin) iin = C.diag[((size_t)C.rcls[K] * C.nr + I2) * nm + m] != T(0);
        if (kin) kin = C.diag[((size_t)C.rcls[K2] * C.nr + I) * nm + m] != T(0);
    }
    const int Kx = kin ? K2 : K, Ix = iin ? I2 : I;
    const unsigned crow = (unsigned)C.nr * nm;   // coarse row stride
    const V2<T> *cu = C.u + m;
    const V2<T> c0 = cu[(unsigned)K * crow + (unsigned)I * nm];
    V2<T> u = ASSIGN ? mk<T>(0, 0) : F.u[idx];   // ASSIGN: u = P c (full-multigrid interpolation)
    if (cz2 && cr2) {
        const V2<T> c1 = cu[(unsigned)K * crow + (unsigned)Ix * nm];
        const V2<T> c2 = cu[(unsigned)Kx * crow + (unsigned)I * nm];
        const V2<T> c3 = cu[(unsigned)Kx * crow + (unsigned)Ix * nm];
        // signed weights by selection (no FP64 multiply), four multiply-adds per part
        const T w1 = iin ? T(0.1875) : T(-0.1875), w2 = kin ? T(0.1875) : T(-0.1875);
        const T w3 = iin == kin ? T(0.0625) : T(-0.0625);
        u.x = fma(w3, c3.x, fma(w2, c2.x, fma(w1, c1.x, fma(T(0.5625), c0.x, u.x))));
        u.y = fma(w3, c3.y, fma(w2, c2.y, fma(w1, c1.y, fma(T(0.5625), c0.y, u.y))));
    } else {
        // linear along the coarsened direction
        const V2<T> c1 = cz2 ? cu[(unsigned)Kx * crow + (unsigned)I * nm] : cu[(unsigned)K * crow + (unsigned)Ix * nm];
        const T w1 = (cz2 ? kin : iin) ? T(0.25) : T(-0.25);
        u.x = fma(w1, c1.x, fma(T(0.75), c0.x, u.x));
        u.y = fma(w1, c1.y, fma(T(0.75), c0.y, u.y));
    }
    F.u[idx] = u;
}

// Full-multigrid start: the right-hand side restricted to the next coarser
// level (the finite-volume sum of b over the fine cells of each coarse cell,
// the restriction the residuals get), b_hat = b / diag, and a zero iterate.
template <class T, bool MASK>
__global__ void __launch_bounds__(MG_THREADS) k_rhs_restrict(const LaunchTab<T> *__restrict__ tab) {
    // (MASK: the class tables of a composite domain's rows)
    const int p = find_problem(tab->start, tab->n, blockIdx.x);
    if (tab->done && tab->done[tab->pid[p]]) return;   // stopped problem of a batch
    const LevelDev<T> F = tab->f[p];
    const LevelDev<T> C = tab->c[p];
    const unsigned e = (blockIdx.x - tab->start[p]) * blockDim.x + threadIdx.x;
    if (e >= (unsigned)C.nz * (unsigned)C.nr * (unsigned)C.nm) return;
    const unsigned nm = C.nm;
    const unsigned cc = fdiv(e, nm, C.rnm);
    const int m = (int)(e - cc * nm);
    const int K = (int)fdiv(cc, (unsigned)C.nr, C.rnr);
    const int I = (int)(cc - (unsigned)K * C.nr);
    const int fz = F.nz == C.nz ? 1 : 2, fr = F.nr == C.nr ? 1 : 2;
    V2<T> sum = F.b[((size_t)(fz * K) * F.nr + fr * I) * nm + m];
    for (int c = 1; c < fz * fr; ++c) {
        const int k = fz * K + (fr == 2 ? (c >> 1) : c), i = fr * I + (fr == 2 ? (c & 1) : 0);
        const V2<T> b = F.b[((size_t)k * F.nr + i) * nm + m];
        sum = mk<T>(sum.x + b.x, sum.y + b.y);
    }
    C.b[e] = sum;
    const T inv = C.invd[((size_t)(MASK ? lclass(C, K) : row_class(K, C.nz, C.ncls)) * C.nr + I) * nm + m];
    C.bh[e] = mk<T>(sum.x * inv, sum.y * inv);
    C.u[e] = mk<T>(0, 0);
}

// Conversions between binary64 and binary32 with a power-of-two scale 2^s,
// done on the IEEE-754 bit patterns with integer instructions: on this GPU the
// FP64 unit's conversions cost several FP64 instruction slots each, and the
// FP64 unit is what bounds the defect and update kernels.
//   to binary32: the 52-bit mantissa is cut to 23 bits and rounded to nearest
//   (ties away from zero; a carry moves into the exponent, up to infinity);
//   results below the binary32 normal range become signed zero, above it
//   infinity; infinities stay infinite and NaN stays NaN.
//   to binary64: exact for normal binary32 values; binary32 subnormals become
//   signed zero.
__device__ __forceinline__ float f64_to_f32_pow2(double x, int s) {
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const unsigned sign = hi & 0x80000000u;
    const int e = (int)((hi >> 20) & 0x7ffu);
    const unsigned m = hi & 0xfffffu;
    if (e == 0x7ff) return __uint_as_float(sign | 0x7f800000u | ((m | lo) ? 0x400000u : 0u));
    const int ef = e - 1023 + 127 + s;
    if (e == 0 || ef <= 0) return __uint_as_float(sign);
    if (ef >= 255) return __uint_as_float(sign | 0x7f800000u);
    const unsigned bits = (((unsigned)ef << 23) | (m << 3) | (lo >> 29)) + ((lo >> 28) & 1u);
    return __uint_as_float(sign | bits);
}
__device__ __forceinline__ double f32_to_f64_pow2(float f, int s) {
    const unsigned b = __float_as_uint(f);
    const unsigned sign = b & 0x80000000u;
    const int e = (int)((b >> 23) & 0xffu);
    const unsigned m = b & 0x7fffffu;
    if (e == 0) return __hiloint2double((int)sign, 0);
    if (e == 0xff) return __hiloint2double((int)(sign | 0x7ff00000u | (m ? 0x80000u : 0u)), 0);
    const int ed = e - 127 + 1023 + s;
    if (ed <= 0) return __hiloint2double((int)sign, 0);
    if (ed >= 0x7ff) return __hiloint2double((int)(sign | 0x7ff00000u), 0);
    return __hiloint2double((int)(sign | ((unsigned)ed << 20) | (m >> 3)), (int)(m << 29));
}
// Exponent s of a positive power of two 2^s held in a double.
__device__ __forceinline__ int pow2_exponent(double v) { return ((__double2hiint(v) >> 20) & 0x7ff) - 1023; }

// Mixed precision, FP64 defect: r = b - A_m x on the FP64 level 0 (all cells)
// and the FP32 level-0 right-hand side of the correction equation, scaled by
// sigma (a power of two, exact): b32 = r sigma, b_hat32 = b32 / diag and
// u32 = (red ? b_hat32 : 0) -- the first red half-sweep of the FP32 V-cycle
// from a zero correction -- or u32 = 0.  The squared norm of the scaled
// residual is accumulated in FP32 per entry (it only decides convergence).
// ZERO_X: the iterate is zero (first defect of a solve from a zero initial
// guess), so r = b and the kernel also writes x = 0 -- a memory pass, no FP64
// stencil.
template <bool ZERO_X, bool MASK>
__global__ void __launch_bounds__(MG_THREADS, 6)   // 48 warps per SM for the FP64 pipe (measured best)
k_defect(const DefectTab *__restrict__ tab, const Ctrl *__restrict__ ctrl, double *__restrict__ partials) {
    __shared__ double red[MG_THREADS];
    const int p = find_problem(tab->start, tab->n, blockIdx.x);
    if (tab->done && tab->done[tab->pid[p]]) return;   // stopped problem of a batch
    const LevelDev<double> D = tab->d[p];
    const LevelDev<float> S = tab->s[p];
    const int init_red = tab->init_red[p];
    const int ls = pow2_exponent(ctrl->sigma_next[p]);
    const unsigned e = (blockIdx.x - tab->start[p]) * blockDim.x + threadIdx.x;
    double acc = 0.0;
    if (e < (unsigned)D.nz * (unsigned)D.nr * (unsigned)D.nm) {
        const unsigned nm = D.nm;
        const unsigned c = fdiv(e, nm, D.rnm);
        const int m = (int)(e - c * nm);
        const int k = (int)fdiv(c, (unsigned)D.nr, D.rnr);
        const int i = (int)(c - (unsigned)k * D.nr);
        double2 r;
        if (ZERO_X) {
            r = D.b[e];
            D.u[e] = make_double2(0.0, 0.0);
        } else {
            r = residual_at<double, MASK>(D, k, i, m, e);
        }
        const float2 b32 = make_float2(f64_to_f32_pow2(r.x, ls), f64_to_f32_pow2(r.y, ls));
        const float w = (m == 0 || 2 * m == D.nt) ? 1.f : 2.f;
        acc = f32_to_f64_pow2(w * fmaf(b32.x, b32.x, b32.y * b32.y), 0);
        const float inv = S.invd[((size_t)(MASK ? lclass(S, k) : row_class(k, S.nz, S.ncls)) * S.nr + i) * nm + m];
        const float2 bh = make_float2(b32.x * inv, b32.y * inv);
        S.b[e] = b32;
        S.bh[e] = bh;
        S.u[e] = (init_red && ((k + i) & 1) == 0) ? bh : make_float2(0.f, 0.f);
    }
    const double tot = block_sum(acc, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = tot;
}

// Mixed precision, FP64 update: x += e32 / sigma (the scale of the correction
// problem just solved; 1/sigma is an exact power of two).
__global__ void __launch_bounds__(MG_THREADS) k_update(const DefectTab *__restrict__ tab, const Ctrl *__restrict__ ctrl) {
    const int p = find_problem(tab->start, tab->n, blockIdx.x);
    if (tab->done && tab->done[tab->pid[p]]) return;   // stopped problem of a batch
    const LevelDev<double> D = tab->d[p];
    const LevelDev<float> S = tab->s[p];
    const int ls = pow2_exponent(ctrl->inv_sigma_used[p]);
    const unsigned e = (blockIdx.x - tab->start[p]) * blockDim.x + threadIdx.x;
    if (e >= (unsigned)D.nz * (unsigned)D.nr * (unsigned)D.nm) return;
    const float2 c = S.u[e];
    double2 x = D.u[e];
    x.x += f32_to_f64_pow2(c.x, ls);
    x.y += f32_to_f64_pow2(c.y, ls);
    D.u[e] = x;
}

// Coarsest level, exact separable solve, one CTA per (problem, mode, real or
// imaginary part).  On a uniform level A_m = I_z (x) K_m + T_z (x) diag(cz)
// with K_m the radial tridiagonal operator (diagonal D0r + lambda_m mu) and
// T_z = tridiag(-1, 2, -1) with 3 in both corners (Dirichlet faces at half a
// cell).  T_z = V Lambda V^T with the DST-II basis V[k][j] = c_j
// sin(pi (j+1)(k+1/2)/nz), so for each axial eigenvector j the system is
// tridiagonal in r: (K_m + Lambda_j diag(cz)) w_j = (V^T b)_j, factorised at
// plan time (Thomas: inverse pivots piv, multipliers cpr), and u = V w.
// The basis is mirror-symmetric, V[nz-1-k][j] = (-1)^j V[k][j], so both
// transforms fold the axial index: with P_k = b_k + b_(nz-1-k) and
// Q_k = b_k - b_(nz-1-k), (V^T b)_j sums V[k][j] P_k (even j) or V[k][j] Q_k
// (odd j) over the first half only, and u_k, u_(nz-1-k) = E_k +- O_k with E, O
// the sums over even and odd j -- half the FP64 multiply-adds of the plain
// products.  Only rows k < ceil(nz/2) of V are read.
template <class T>
__global__ void __launch_bounds__(MG_THREADS) k_coarse(const CoarseTab<T> *__restrict__ tab) {
    extern __shared__ unsigned char smraw[];
    const int p = find_problem(tab->start, tab->n, blockIdx.x);
    if (tab->done && tab->done[tab->pid[p]]) return;   // stopped problem of a batch
    const LevelDev<T> L = tab->f[p];
    const CoarseDev<T> D = tab->c[p];
    const int nr = D.nr, nz = D.nz, nm = D.nm;
    const int lb = (int)(blockIdx.x - tab->start[p]);
    const int m = lb >> 1, comp = lb & 1;
    // (a composite domain or non-uniform axial mesh takes the dense solve of csrc/dense.cu)
    const int h = nz >> 1, hz = nz - h;      // mirror pairs, rows with k <= nz-1-k
    T *bs = (T *)smraw;                      // [nz][nr]: b, then P (rows < hz) and Q (row nz-1-k)
    const int lw = nr + 1;                   // padded rows: the Thomas threads walk rows
    T *ws = bs + (size_t)nz * nr;            // [nz][lw]
    T *Vs = ws + (size_t)nz * lw;            // [hz][nz]
    T *ps = Vs + (size_t)hz * nz;            // [nz][lw] this mode's inverse pivots
    T *cs = ps + (size_t)nz * lw;            // [nz][lw] and upper multipliers
    T *es = cs + (size_t)nz * lw;            // [nr] off-diagonal
    // every load of the block is in flight before the one wait (cp.async)
    const T *bg = (const T *)L.b + comp;
    for (int f = threadIdx.x; f < nz * nr; f += blockDim.x) cp_async_elem(bs + f, bg + 2 * ((size_t)f * nm + m));
    for (int f = threadIdx.x; f < hz * nz; f += blockDim.x) cp_async_elem(Vs + f, D.V + f);
    {
        const T *gp = D.piv + (size_t)m * nz * nr, *gc = D.cpr + (size_t)m * nz * nr;
        for (int f = threadIdx.x; f < nz * nr; f += blockDim.x) {
            const int j = f / nr, i = f - j * nr;
            cp_async_elem(ps + j * lw + i, gp + f);
            cp_async_elem(cs + j * lw + i, gc + f);
        }
        for (int i = threadIdx.x; i + 1 < nr; i += blockDim.x) cp_async_elem(es + i, D.e + i);
    }
    cp_async_wait_all();
    __syncthreads();
    for (int f = threadIdx.x; f < h * nr; f += blockDim.x) {
        const int k = f / nr, i = f - k * nr;
        const T lo = bs[k * nr + i], hi = bs[(nz - 1 - k) * nr + i];
        bs[k * nr + i] = lo + hi;
        bs[(nz - 1 - k) * nr + i] = lo - hi;
    }
    __syncthreads();
    // w[j][i] = sum_k V[k][j] b[k][i], folded
    for (int f = threadIdx.x; f < nz * nr; f += blockDim.x) {
        const int j = f / nr, i = f - j * nr;
        T a = 0;
        if ((j & 1) == 0) {
            for (int k = 0; k < hz; ++k) a = fma(Vs[k * nz + j], bs[k * nr + i], a);
        } else {
            for (int k = 0; k < h; ++k) a = fma(Vs[k * nz + j], bs[(nz - 1 - k) * nr + i], a);
        }
        ws[j * lw + i] = a;
    }
    __syncthreads();
    // tridiagonal solves along r, one per axial eigenvector j
    thomas_rows(ws, ps, cs, es, nz, nr, lw);
    __syncthreads();
    // u[k][i] = sum_j V[k][j] w[j][i] = E +- O for the mirror pair (k, nz-1-k)
    T *ug = (T *)L.u + comp;
    for (int f = threadIdx.x; f < hz * nr; f += blockDim.x) {
        const int k = f / nr, i = f - k * nr;
        T e = 0, o = 0;
        for (int j = 0; j + 1 < nz; j += 2) {
            e = fma(Vs[k * nz + j], ws[j * lw + i], e);
            o = fma(Vs[k * nz + j + 1], ws[(j + 1) * lw + i], o);
        }
        if (nz & 1) e = fma(Vs[k * nz + nz - 1], ws[(nz - 1) * lw + i], e);
        ug[2 * ((size_t)(k * nr + i) * nm + m)] = e + o;
        if (nz - 1 - k != k) ug[2 * ((size_t)((nz - 1 - k) * nr + i) * nm + m)] = e - o;
    }
}

// Power of two closest to 1 / sqrt(mean square): scales an FP32 correction
// problem to O(1) values without any rounding from the scale itself.
__device__ double pow2_scale(double sumsq, double count) {
    const double rms = sqrt(sumsq / fmax(count, 1.0));
    if (!(rms > 0.0) || isinf(rms) || isnan(rms)) return 1.0;
    int ex = 0;
    frexp(rms, &ex);
    return ldexp(1.0, -ex);
}

// Deterministic sums of per-problem ranges of block partials by one CTA:
// with n problems and W warps, problem p is summed by the warps w = p, p + n,
// ... (each lane a fixed strided subset, then a fixed shuffle tree), and the
// group's warp sums are added in warp order.  Result in out[p].
__device__ void range_sums(const double *__restrict__ partials, const unsigned *__restrict__ begin,
                           const unsigned *__restrict__ end, int n, double *out, double *wsum) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, W = blockDim.x >> 5;
    for (int base = 0; base < n; base += W) {
        const int cnt = min(n - base, W);
        const int p = base + warp % cnt, g = W / cnt, rank = warp / cnt;
        double s = 0.0;
        if (rank < g) {
            const unsigned b0 = begin[p], b1 = end[p];
            for (unsigned b = b0 + rank * 32 + lane; b < b1; b += 32u * g) s += partials[b];
        }
        s = warp_sum(s);
        if (lane == 0) wsum[warp] = (rank < g) ? s : 0.0;
        __syncthreads();
        if (threadIdx.x < cnt) {
            double t = 0.0;
            for (int r = 0; r < g; ++r) t += wsum[r * cnt + threadIdx.x];
            out[base + threadIdx.x] = t;
        }
        __syncthreads();
    }
}

// First-stage sums of the residual-norm partials (PsumTab): block c of
// problem p adds partials in_begin[p] + c PSUM_CHUNK .. (+ PSUM_CHUNK, at most
// in_end[p]), each thread a strided subset in order, then the block tree.
__global__ void __launch_bounds__(256) k_psum(const PsumTab *__restrict__ tab, const double *__restrict__ partials,
                                              double *__restrict__ out) {
    __shared__ double red[256];
    const int p = find_problem(tab->start, tab->n, blockIdx.x);
    const unsigned c = blockIdx.x - tab->start[p];
    const unsigned b0 = tab->in_begin[p] + c * (unsigned)PSUM_CHUNK;
    const unsigned b1 = min(tab->in_end[p], b0 + (unsigned)PSUM_CHUNK);
    double s = 0.0;
    for (unsigned b = b0 + threadIdx.x; b < b1; b += blockDim.x) s += partials[b];
    const double tot = block_sum(s, red);
    if (threadIdx.x == 0) out[blockIdx.x] = tot;
}

// ||b||^2 per problem from the forward transform's block partials, and the
// first correction scale.
__global__ void __launch_bounds__(1024) k_bnorm(Ctrl *__restrict__ ctrl, const FFTTab *__restrict__ fft,
                                                const double *__restrict__ partials) {
    __shared__ double wsum[32];
    __shared__ double sums[kMaxBatch];
    range_sums(partials, fft->start, fft->start + 1, fft->n, sums, wsum);
    for (int p = threadIdx.x; p < fft->n; p += blockDim.x) {
        ctrl->bnorm2[p] = sums[p];
        ctrl->sigma_next[p] = pow2_scale(sums[p], ctrl->count[p]);
    }
}

// Device-side convergence test after a residual evaluation.  Per problem: the
// Parseval-weighted ||r||^2 from its block partials (mixed precision: of the
// residual scaled by sigma), rel = ||r|| / ||b||, and the stop rule: tol > 0
// stops at rel <= tol; tol <= 0 stops once rel has not halved for two
// evaluations (the rounding floor); non-finite stops with ENONFINITE; the
// cycle cap with ENOTCONVERGED.  A problem that stopped is left alone: the
// kernels skip its blocks (launch tables' done flags) and its rel stays the
// residual of its returned iterate while the others go on.
// counting: 1 adds ctrl->inc to the cycle count first (evaluations after a
// pass of the loop body), 2 adds ctrl->inc_first (after the first pass of a
// solve whose first correction is larger).  use_handle bit 0 / bit 1 set the
// graph conditionals `handle` / `handle2` to "some problem goes on".
__global__ void __launch_bounds__(1024) k_check(Ctrl *__restrict__ ctrl, const double *__restrict__ partials,
                                                int counting, cudaGraphConditionalHandle handle,
                                                cudaGraphConditionalHandle handle2, int use_handle) {
    __shared__ double wsum[32];
    __shared__ double sums[kMaxBatch];
    __shared__ int s_any;
    const int cycles = ctrl->cycles + (counting == 2 ? ctrl->inc_first : counting ? ctrl->inc : 0);
    if (threadIdx.x == 0) s_any = 0;
    range_sums(partials, ctrl->rbegin, ctrl->rend, ctrl->n, sums, wsum);
    const double tol = ctrl->tol;
    for (int p = threadIdx.x; p < ctrl->n; p += blockDim.x) {
        if (ctrl->done[p]) continue;   // stopped: its kernels no longer run, rel stays the reported one
        double rr2 = sums[p];
        if (ctrl->scaled) {
            const double su = ctrl->sigma_next[p];
            ctrl->sigma_used[p] = su;
            ctrl->inv_sigma_used[p] = 1.0 / su;
            rr2 = rr2 / (su * su);
            ctrl->sigma_next[p] = pow2_scale(rr2, ctrl->count[p]);
        }
        const double bb = ctrl->bnorm2[p];
        const double rel = bb > 0.0 ? sqrt(rr2 / bb) : sqrt(rr2);
        ctrl->rel[p] = rel;
        if (!counting) ctrl->rel_first[p] = rel;
        {
            int stop = 0, status = PIC_POISSON_OK;
            if (isnan(rel) || isinf(rel)) {
                stop = 1;
                status = PIC_POISSON_ENONFINITE;
            } else if (tol > 0.0) {
                stop = rel <= tol;
            } else if (rel < 0.5 * ctrl->best[p]) {   // halved since the last reference point
                ctrl->best[p] = rel;
                ctrl->stall[p] = 0;
            } else {   // rounding floor: no halving within kFloorWindow tests in a row
                stop = ++ctrl->stall[p] >= kFloorWindow;
            }
            if (!stop && cycles >= ctrl->max_cycles) {
                stop = 1;
                status = PIC_POISSON_ENOTCONVERGED;
            }
            if (stop) {
                ctrl->done[p] = 1;
                ctrl->status[p] = status;
                ctrl->done_cycles[p] = cycles;
            } else {
                atomicOr(&s_any, 1);
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        ctrl->cycles = cycles;
        ctrl->cont = s_any;
        if (use_handle & 1) cudaGraphSetConditional(handle, s_any ? 1u : 0u);
        if (use_handle & 2) cudaGraphSetConditional(handle2, s_any ? 1u : 0u);
    }
}

// Deterministic single-CTA sum of n partials (fixed order per thread, fixed tree).
__global__ void __launch_bounds__(1024) k_sum(const double *__restrict__ p, int n, double *__restrict__ out) {
    __shared__ double red[1024];
    double s = 0.0;
    for (int f = threadIdx.x; f < n; f += blockDim.x) s += p[f];
    const double t = block_sum(s, red);
    if (threadIdx.x == 0) *out = t;
}

}  // namespace

template <class T, int S, bool SOR, bool RW>
void launch_smooth_s(const LaunchTab<T> *tab, unsigned grid, int color, int threads, cudaStream_t st) {
    switch (threads) {
    case 64: k_smooth<T, 64, S, SOR, RW><<<grid, 64, 0, st>>>(tab, color); break;
    case 128: k_smooth<T, 128, S, SOR, RW><<<grid, 128, 0, st>>>(tab, color); break;
    case 512: k_smooth<T, 512, S, SOR, RW><<<grid, 512, 0, st>>>(tab, color); break;
    default: k_smooth<T, 256, S, SOR, RW><<<grid, 256, 0, st>>>(tab, color); break;
    }
}

template <class T, bool SOR, bool RW>
cudaError_t launch_smooth_r(const LaunchTab<T> *tab, unsigned grid, int color, int threads, int strip,
                            cudaStream_t st) {
    switch (strip) {
    case 0: launch_smooth_s<T, 0, SOR, RW>(tab, grid, color, threads, st); break;
    case 1: launch_smooth_s<T, 1, SOR, RW>(tab, grid, color, threads, st); break;
    case 2: launch_smooth_s<T, 2, SOR, RW>(tab, grid, color, threads, st); break;
    case 4: launch_smooth_s<T, 4, SOR, RW>(tab, grid, color, threads, st); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_smooth(const LaunchTab<T> *tab, unsigned grid, int color, int threads, int strip, bool sor,
                          cudaStream_t st, bool rowwise) {
    if (rowwise)
        return sor ? launch_smooth_r<T, true, true>(tab, grid, color, threads, strip, st)
                   : launch_smooth_r<T, false, true>(tab, grid, color, threads, strip, st);
    return sor ? launch_smooth_r<T, true, false>(tab, grid, color, threads, strip, st)
               : launch_smooth_r<T, false, false>(tab, grid, color, threads, strip, st);
}

template <class T>
cudaError_t launch_residual_restrict(const LaunchTab<T> *tab, unsigned grid, bool red_only, double *partials,
                                     cudaStream_t st, bool masked) {
    if (masked) {
        if (red_only) k_residual_restrict<T, true, true><<<grid, MG_THREADS, 0, st>>>(tab, partials);
        else k_residual_restrict<T, false, true><<<grid, MG_THREADS, 0, st>>>(tab, partials);
    } else {
        if (red_only) k_residual_restrict<T, true, false><<<grid, MG_THREADS, 0, st>>>(tab, partials);
        else k_residual_restrict<T, false, false><<<grid, MG_THREADS, 0, st>>>(tab, partials);
    }
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_residual(const LaunchTab<T> *tab, unsigned grid, bool write_r, double *partials,
                            unsigned partial_stride, cudaStream_t st, bool masked) {
    if (masked) k_residual<T, true><<<grid, MG_THREADS, 0, st>>>(tab, write_r ? 1 : 0, partials, partial_stride);
    else k_residual<T, false><<<grid, MG_THREADS, 0, st>>>(tab, write_r ? 1 : 0, partials, partial_stride);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_prolong(const LaunchTab<T> *tab, unsigned grid, bool black_only, cudaStream_t st, bool masked) {
    if (masked) {
        if (black_only) k_prolong<T, true, false, true><<<grid, MG_THREADS, 0, st>>>(tab);
        else k_prolong<T, false, false, true><<<grid, MG_THREADS, 0, st>>>(tab);
    } else {
        if (black_only) k_prolong<T, true, false, false><<<grid, MG_THREADS, 0, st>>>(tab);
        else k_prolong<T, false, false, false><<<grid, MG_THREADS, 0, st>>>(tab);
    }
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_interp(const LaunchTab<T> *tab, unsigned grid, cudaStream_t st, bool masked, bool black_only) {
    if (black_only) {
        if (masked) k_prolong<T, true, true, true><<<grid, MG_THREADS, 0, st>>>(tab);
        else k_prolong<T, true, true, false><<<grid, MG_THREADS, 0, st>>>(tab);
    } else {
        if (masked) k_prolong<T, false, true, true><<<grid, MG_THREADS, 0, st>>>(tab);
        else k_prolong<T, false, true, false><<<grid, MG_THREADS, 0, st>>>(tab);
    }
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_rhs_restrict(const LaunchTab<T> *tab, unsigned grid, cudaStream_t st, bool masked) {
    if (masked) k_rhs_restrict<T, true><<<grid, MG_THREADS, 0, st>>>(tab);
    else k_rhs_restrict<T, false><<<grid, MG_THREADS, 0, st>>>(tab);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_coarse(const CoarseTab<T> *tab, unsigned grid, size_t smem, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(k_coarse<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_coarse<T><<<grid, MG_THREADS, smem, st>>>(tab);
    return cudaGetLastError();
}

cudaError_t launch_defect(const DefectTab *tab, unsigned grid, const Ctrl *ctrl, double *partials, bool zero_x,
                          cudaStream_t st, bool masked) {
    if (masked) {
        if (zero_x) k_defect<true, true><<<grid, MG_THREADS, 0, st>>>(tab, ctrl, partials);
        else k_defect<false, true><<<grid, MG_THREADS, 0, st>>>(tab, ctrl, partials);
    } else {
        if (zero_x) k_defect<true, false><<<grid, MG_THREADS, 0, st>>>(tab, ctrl, partials);
        else k_defect<false, false><<<grid, MG_THREADS, 0, st>>>(tab, ctrl, partials);
    }
    return cudaGetLastError();
}

cudaError_t launch_update(const DefectTab *tab, unsigned grid, const Ctrl *ctrl, cudaStream_t st) {
    k_update<<<grid, MG_THREADS, 0, st>>>(tab, ctrl);
    return cudaGetLastError();
}

cudaError_t launch_bnorm(Ctrl *ctrl, const FFTTab *fft, const double *partials, cudaStream_t st) {
    k_bnorm<<<1, 1024, 0, st>>>(ctrl, fft, partials);
    return cudaGetLastError();
}

cudaError_t launch_psum(const PsumTab *tab, unsigned grid, const double *partials, double *out, cudaStream_t st) {
    k_psum<<<grid, 256, 0, st>>>(tab, partials, out);
    return cudaGetLastError();
}

cudaError_t launch_check(Ctrl *ctrl, const double *partials, int counting, cudaGraphConditionalHandle handle,
                         cudaGraphConditionalHandle handle2, int use_handle, cudaStream_t st) {
    k_check<<<1, 1024, 0, st>>>(ctrl, partials, counting, handle, handle2, use_handle);
    return cudaGetLastError();
}

cudaError_t launch_sum(const double *partials, int n, double *out, cudaStream_t st) {
    k_sum<<<1, 1024, 0, st>>>(partials, n, out);
    return cudaGetLastError();
}

#define PP_INST(T)                                                                                         \
    template cudaError_t launch_smooth<T>(const LaunchTab<T> *, unsigned, int, int, int, bool, cudaStream_t, \
                                          bool);                                                           \
    template cudaError_t launch_residual_restrict<T>(const LaunchTab<T> *, unsigned, bool, double *,       \
                                                     cudaStream_t, bool);                                  \
    template cudaError_t launch_residual<T>(const LaunchTab<T> *, unsigned, bool, double *, unsigned,      \
                                            cudaStream_t, bool);                                           \
    template cudaError_t launch_prolong<T>(const LaunchTab<T> *, unsigned, bool, cudaStream_t, bool);      \
    template cudaError_t launch_interp<T>(const LaunchTab<T> *, unsigned, cudaStream_t, bool, bool);       \
    template cudaError_t launch_rhs_restrict<T>(const LaunchTab<T> *, unsigned, cudaStream_t, bool);       \
    template cudaError_t launch_coarse<T>(const CoarseTab<T> *, unsigned, size_t, cudaStream_t);
PP_INST(double)
PP_INST(float)
#undef PP_INST

}  // namespace pp
