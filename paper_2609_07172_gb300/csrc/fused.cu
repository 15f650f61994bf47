// Fused red-black smoothing of an FP32 level: NH half-sweeps (NH/2 full
// sweeps, red first) in one pass over the level's data, for the
// mixed-precision form, where the FP32 smoother is bound by memory traffic
// rather than arithmetic.  Separate half-sweeps move 1.5 vectors each (the
// other colour, b_hat of this colour, this colour written), so two full sweeps
// move 6 vectors; fused, they read the iterate and b_hat once and write the
// iterate once: 3 vectors.
//
// Work decomposition.  A block owns G consecutive modes of one problem, a tile
// of P radial column pairs (2j, 2j+1) and a range of R output rows.  Thread
// (pair pl, mode gl) holds both columns of its pair for a sliding window of
// NH+2 axial rows in registers and streams the rows top to bottom as a
// wavefront: when row k enters, half-sweep s (colour s % 2, red = 0) updates
// row k-1-s, so each half-sweep sees its vertical neighbours in the state the
// previous half-sweep left them (row k-s was updated by half-sweep s-1 in this
// step, row k-2-s two steps earlier) -- exactly the order of separate
// half-sweeps.  In every row exactly one cell of a pair has the colour being
// updated, so no thread idles.  Its horizontal neighbour inside the pair is in
// the thread's registers, the other one belongs to the neighbouring pair: each
// thread publishes, in shared memory, the column its neighbours will need in
// the next step, with one barrier per step.
//
// Halos.  A half-sweep can update a cell only if its neighbours are valid, so
// every half-sweep loses one row and one column at the edges of a block's
// data: blocks read NH rows and NH columns (NH/2 pairs) beyond their output on
// each side and write only their output cells.  Reading the old iterate
// (`in`) and writing the new one (`out`, another buffer) keeps blocks that
// share halo cells independent.  Results are bitwise those of the separate
// half-sweeps (same operations, same order per cell).
//
// Latency.  Each step needs the next row from HBM; rows are fetched DEPTH
// steps ahead with cp.async into shared-memory rings (zero-filled beyond the
// level): the iterate's into a short ring read into the window registers,
// b_hat (and b) into a ring that keeps each row until its last half-sweep,
// so those values take no registers.
#include <algorithm>
#include <type_traits>

#include "internal.h"

namespace pp {
namespace {

__device__ __forceinline__ int find_problem(const unsigned *__restrict__ start, int n, unsigned blk) {
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (start[mid] <= blk) lo = mid;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ int row_class(int k, int nz, int ncls) {
    return k == 0 ? 0 : (k == nz - 1 ? ncls - 1 : 1);
}

__device__ __forceinline__ void cp_async8(float2 *smem, const float2 *gmem, bool valid) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(sa), "l"(gmem), "r"(valid ? 8 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

constexpr int PAD = 16;           // >= the largest mode group: neighbour reads of the outermost pairs stay in the array

// Sizes of a variant.  The row loop runs in groups of U = 8 steps, each
// unrolled, and every per-row resource cycles with a period dividing U: the
// register window (U rows; a step touches at most NH + 3), the iterate's ring
// (UR slots, fetched DEPTH rows ahead), the ring that keeps b_hat (and b)
// from its fetch until its last half-sweep (BR slots; the restriction reads
// b NH + 1 steps after the row entered) and the two publication buffers.  So
// in each unrolled copy the register that holds a given row, the parity of
// every row (hence the colour a half-sweep updates in a pair and the column a
// thread publishes) and every ring slot are compile-time constants: no
// register shifts, selects or slot arithmetic per step.
//
// Shared memory against L1.  The rows arrive by cp.async through L1, which
// shares each SM's 256 KB with shared memory in fixed carveouts (..., 132,
// 164, 196, 228 KB of shared memory).  Without the restriction the kernel
// needs about 80 registers, so three blocks fit an SM; with NH = 4, a 4-slot
// iterate ring (2 rows ahead) takes 67.7 KB per block and the three blocks
// the 228 KB carveout, leaving L1 28 KB -- measured 0.4 ms slower per mixed
// solve than a 2-slot ring fetched one row ahead (59.5 KB, the 196 KB
// carveout, L1 60 KB).  With the restriction (two blocks per SM) the 4-slot
// ring fits the 196 KB carveout, and there the deeper prefetch is faster
// than a shorter ring in the 164 KB carveout.
template <int NH, bool RES> struct FusedCfg {
    static constexpr bool SHORT = !RES && NH == 4;
    static constexpr int U = 8;
    static constexpr int UR = SHORT ? 2 : 4;
    static constexpr int DEPTH = SHORT ? 1 : 2;
    static constexpr int BR = 8;
    static constexpr int NB = RES ? 3 : 2;                  // b_hat col 0, b_hat col 1 (, b of the red cell)
    static constexpr int NP = NH + (RES ? 1 : 0);           // published columns per step
    static constexpr int PS = FUSED_THREADS + 2 * PAD;      // published row stride
    static constexpr size_t smem_floats2 =
        (size_t)UR * 2 * FUSED_THREADS + (size_t)BR * NB * FUSED_THREADS + PAD + (size_t)2 * NP * PS;
    static_assert(NH + 2 + (RES ? 1 : 0) <= U, "the window holds every row a step touches");
    static_assert(DEPTH < UR && DEPTH + NH + 2 <= BR, "a ring slot is refilled only after its last read");
    static_assert(U % UR == 0 && U % BR == 0 && U % 2 == 0, "static ring slots, parities and buffers");
};

// RES (pre-smoothing of a level coarsened 2:1 in both directions): after the
// last half-sweep, the kernel also evaluates the residual of the red cells
// -- the black ones vanish after a black half-sweep -- and sums the two red
// cells of each 2x2 block into the coarse right-hand side, exactly as
// k_residual_restrict<float, RED_ONLY> (same operations in the same order).
// The residual of row r needs the final values of rows r +- 1 and of the
// neighbouring columns, so the halo grows by one row and one column pair.
template <int NH, bool RES, bool RW>
__global__ void __launch_bounds__(FUSED_THREADS, RES ? 2 : 3) k_smooth_fused(const FusedTab *__restrict__ tab) {
    using Cfg = FusedCfg<NH, RES>;
    constexpr int U = Cfg::U, UR = Cfg::UR, DEPTH = Cfg::DEPTH, BR = Cfg::BR, NB = Cfg::NB, NP = Cfg::NP;
    constexpr int PS = Cfg::PS;
    constexpr int HP = NH / 2 + (RES ? 1 : 0);  // halo pairs on each side
    constexpr int NT = FUSED_THREADS;
    extern __shared__ float2 dsm[];
    float2 *uring = dsm;                            // [UR][2][NT]
    float2 *bring = uring + UR * 2 * NT;            // [BR][NB][NT]
    float2 *pubs = bring + BR * NB * NT + PAD;      // [2][NP][PS], PAD entries before each row
    const int p = find_problem(tab->start, tab->n, blockIdx.x);
    if (tab->done && tab->done[tab->pid[p]]) return;   // stopped problem of a batch
    const FusedProb &F = tab->p[p];
    const LevelDev<float> &L = F.L;
    const int nr = L.nr, nz = L.nz, nm = L.nm, ncls = L.ncls;
    // per-row coefficient classes (a composite domain): every row's class from
    // its table, south and north couplings apart (plain problems of a mixed
    // batch keep the three-class path)
    const bool rw = RW && L.rcls != nullptr;
    const int G = F.G, P = F.P;
    const unsigned lb = blockIdx.x - tab->start[p];
    const int g = (int)(lb % (unsigned)F.ngroups);
    const unsigned rest = lb / (unsigned)F.ngroups;
    const int kr = (int)(rest % (unsigned)F.nkr);
    const int tile = (int)(rest / (unsigned)F.nkr);

    const int t = threadIdx.x;
    const int gl = t % G, pl = t / G;
    const bool active = pl < P;
    const int m = g * G + gl;
    const bool mvalid = active && m < nm;
    const int j = tile * (P - 2 * HP) - HP + pl;   // global column pair
    const int i0 = 2 * j, i1 = 2 * j + 1;
    const bool v0 = mvalid && i0 >= 0 && i0 < nr, v1 = mvalid && i1 >= 0 && i1 < nr;
    const bool outpair = pl >= HP && pl < P - HP;
    const int hr = NH + (RES ? 1 : 0);                       // halo rows
    const int k0 = kr * F.R, k1 = min(nz, k0 + F.R);
    // rows read: [ks, ke); ks is even (one more halo row when k0 - hr is odd),
    // so row k of unrolled copy c has the parity of c
    const int ks = max(0, (k0 - hr) & ~1), ke = min(nz, k1 + hr);
    const int klast = k1 - 1 + hr;                           // last step

    // element offsets fit 32 bits: a plan rejects levels of 2^31 entries or more
    const unsigned rs = (unsigned)nr * nm;
    const unsigned c0 = (unsigned)(v0 ? i0 : 0) * nm + (mvalid ? m : 0);
    const unsigned c1 = (unsigned)(v1 ? i1 : 0) * nm + (mvalid ? m : 0);
    const unsigned cls1 = ncls > 1 ? rs : 0;
    // Cells outside the level or the mode range get zero coefficients (and a
    // zero b_hat from the zero-filled copies), so they stay exactly zero
    // without a predicate on every update: a valid neighbour reads 0, as
    // when it is left out.
    const float hz0 = v0 ? L.hz[cls1 + c0] : 0.f, hw0 = v0 ? L.hw[cls1 + c0] : 0.f,
                he0 = v0 ? L.he[cls1 + c0] : 0.f;
    const float hz1 = v1 ? L.hz[cls1 + c1] : 0.f, hw1 = v1 ? L.hw[cls1 + c1] : 0.f,
                he1 = v1 ? L.he[cls1 + c1] : 0.f;

    // Fetch row `row` into the ring slots of unrolled copy cs (ring slots and
    // the row's parity follow from cs: ks is even and a group has U steps);
    // zeros for rows at or beyond ke and for invalid cells.  FAST: the row is
    // known to lie below ke.
    const float2 *gin0 = F.in + c0, *gin1 = F.in + c1, *gb0 = L.bh + c0, *gb1 = L.bh + c1;
    const float2 *gr0 = L.b + c0, *gr1 = L.b + c1;
    auto fetch = [&](int row, const int cs, auto fast_tag) {
        constexpr bool FAST = decltype(fast_tag)::value;
        const bool ok = FAST || row < ke;
        const unsigned o = (unsigned)(ok ? row : ks) * rs;
        float2 *ru = uring + (cs % UR) * 2 * NT + t;
        float2 *rb = bring + (cs % BR) * NB * NT + t;
        cp_async8(ru, gin0 + o, ok && v0);
        cp_async8(ru + NT, gin1 + o, ok && v1);
        cp_async8(rb, gb0 + o, ok && v0);
        cp_async8(rb + NT, gb1 + o, ok && v1);
        if (RES) {   // b of the row's red cell: column parity = row parity
            if ((cs & 1) == 0) cp_async8(rb + 2 * NT, gr0 + o, ok && v0);
            else cp_async8(rb + 2 * NT, gr1 + o, ok && v1);
        }
        cp_async_commit();
    };
    // zero padding around the published rows: the outermost pairs read it
    for (int e = t; e < 2 * NP * 2 * PAD; e += NT) {
        const int row = e / (2 * PAD), x = e % (2 * PAD);
        pubs[row * PS + (x < PAD ? x - PAD : NT + x - PAD)] = make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int d = 0; d < DEPTH; ++d) fetch(ks + d, d, std::false_type{});

    // residual coefficients of the pair's columns (RES)
    float cz0 = 0.f, cw0 = 0.f, ce0 = 0.f, dg0 = 0.f, cz1 = 0.f, cw1 = 0.f, ce1 = 0.f, dg1 = 0.f;
    if (RES) {
        const int ii0 = v0 ? i0 : 0, ii1 = v1 ? i1 : 0;
        cz0 = L.cz[ii0];
        cw0 = L.cw[ii0];
        ce0 = L.ce[ii0];
        dg0 = L.diag[cls1 + c0];
        cz1 = L.cz[ii1];
        cw1 = L.cw[ii1];
        ce1 = L.ce[ii1];
        dg1 = L.diag[cls1 + c1];
    }
    float2 rsum = make_float2(0.f, 0.f);   // residual of the even row of a coarse cell (RES)
    // the coarse level's outputs, in registers (the stores below must not make
    // the compiler reload them from the launch table)
    float2 *const cb = F.C.b, *const cbh = F.C.bh, *const cu = F.C.u;
    const float *const cinvd = F.C.invd;
    const int cnr = F.C.nr, cnz = F.C.nz, cncls = F.C.ncls, finit = F.init;
    const int *const crcls = RW ? F.C.rcls : nullptr;   // the coarse level's row classes (per-row tables)
    const bool cwrite = RES && outpair && v0 && j < cnr;
    const unsigned ccol = (unsigned)(cwrite ? j : 0) * nm + (mvalid ? m : 0);
    const float cinv1 = RES && cwrite ? cinvd[(cncls > 1 ? (unsigned)cnr * nm : 0) + ccol] : 0.f;
    float2 *const gout = F.out;

    const float2 zero = make_float2(0.f, 0.f);
    // window: row k - d lives in register (c - d) mod U at unrolled copy c
    float2 u0[U], u1[U];
#pragma unroll
    for (int w = 0; w < U; ++w) u0[w] = u1[w] = zero;
#define IX(d) ((((c) - (d)) % U + U) % U)
#define SLOT(d, N) ((((c) - (d)) % (N) + (N)) % (N))
    // One step: row k enters at unrolled copy c.  FAST (decided per step,
    // uniformly): every row the step updates, evaluates or writes lies inside
    // the block's rows and off the level's first and last rows, row k + DEPTH
    // lies below ke, and the level has the plain coefficient classes -- the
    // interior of the sweep, where no range, edge or class test remains.
    auto step = [&](const int c, const int k, auto fast_tag) {
        constexpr bool FAST = decltype(fast_tag)::value;
        const int buf = c & 1;   // publication buffer written at this step
        // (a) row k into the window; fetch row k + DEPTH
        cp_async_wait<DEPTH - 1>();
        u0[IX(0)] = uring[(c % UR) * 2 * NT + t];
        u1[IX(0)] = uring[(c % UR) * 2 * NT + NT + t];
        fetch(k + DEPTH, c + DEPTH, fast_tag);
        // (b) half-sweep s on row k - 1 - s
#pragma unroll
        for (int s = 0; s < NH; ++s) {
            const int r = k - 1 - s;
            if (!FAST && (unsigned)(r - ks) >= (unsigned)(ke - ks)) continue;   // uniform: r outside [ks, ke)
            const int sl = IX(1 + s);   // row r
            const int sn = IX(s);       // row r + 1
            const int ss = IX(2 + s);   // row r - 1
            const int q = (c - 1 - s + (s & 1)) & 1;   // the pair's cell of this colour (static)
            const bool edge = !FAST && (r == 0 || r == nz - 1);
            const float2 *pr = pubs + (size_t)((buf ^ 1) * NP + s) * PS;
            const float2 *bh = bring + SLOT(1 + s, BR) * NB * NT + t;
            // Rows outside the level are zero in the window and the wall
            // columns have zero coefficients towards the wall (h_w = 0 at
            // i = 0, h_e = 0 at i = nr - 1), so every update is the same
            // four multiply-adds per part -- the neighbour that does not
            // exist contributes exactly zero, as when it is left out.
            // The pair beyond a block's outermost pair reads padding
            // (halo cells only).
            if (q == 0) {
                const float2 uw = pr[t - G];   // west: column 1 of the pair on the left
                const float2 b = bh[0];
                float hz = hz0, hw = hw0, he = he0;
                float2 acc;
                if (!FAST && rw) {   // the row's class: south and north apart
                    const unsigned tb = (unsigned)L.rcls[r] * rs + c0;
                    const float hs = v0 ? L.hz[tb] : 0.f, hn = v0 ? L.hn[tb] : 0.f;
                    hw = v0 ? L.hw[tb] : 0.f;
                    he = v0 ? L.he[tb] : 0.f;
                    acc = make_float2(fmaf(hs, u0[ss].x, b.x), fmaf(hs, u0[ss].y, b.y));
                    acc = make_float2(fmaf(hn, u0[sn].x, acc.x), fmaf(hn, u0[sn].y, acc.y));
                } else {
                    const float2 vs = make_float2(u0[ss].x + u0[sn].x, u0[ss].y + u0[sn].y);
                    if (edge) {
                        const unsigned tb = (unsigned)row_class(r, nz, ncls) * rs + c0;
                        hz = v0 ? L.hz[tb] : 0.f;
                        hw = v0 ? L.hw[tb] : 0.f;
                        he = v0 ? L.he[tb] : 0.f;
                    }
                    acc = make_float2(fmaf(hz, vs.x, b.x), fmaf(hz, vs.y, b.y));
                }
                acc = make_float2(fmaf(hw, uw.x, acc.x), fmaf(hw, uw.y, acc.y));
                acc = make_float2(fmaf(he, u1[sl].x, acc.x), fmaf(he, u1[sl].y, acc.y));
                u0[sl] = acc;
            } else {
                const float2 ue = pr[t + G];   // east: column 0 of the pair on the right
                const float2 b = bh[NT];
                float hz = hz1, hw = hw1, he = he1;
                float2 acc;
                if (!FAST && rw) {
                    const unsigned tb = (unsigned)L.rcls[r] * rs + c1;
                    const float hs = v1 ? L.hz[tb] : 0.f, hn = v1 ? L.hn[tb] : 0.f;
                    hw = v1 ? L.hw[tb] : 0.f;
                    he = v1 ? L.he[tb] : 0.f;
                    acc = make_float2(fmaf(hs, u1[ss].x, b.x), fmaf(hs, u1[ss].y, b.y));
                    acc = make_float2(fmaf(hn, u1[sn].x, acc.x), fmaf(hn, u1[sn].y, acc.y));
                } else {
                    const float2 vs = make_float2(u1[ss].x + u1[sn].x, u1[ss].y + u1[sn].y);
                    if (edge) {
                        const unsigned tb = (unsigned)row_class(r, nz, ncls) * rs + c1;
                        hz = v1 ? L.hz[tb] : 0.f;
                        hw = v1 ? L.hw[tb] : 0.f;
                        he = v1 ? L.he[tb] : 0.f;
                    }
                    acc = make_float2(fmaf(hz, vs.x, b.x), fmaf(hz, vs.y, b.y));
                }
                acc = make_float2(fmaf(hw, u0[sl].x, acc.x), fmaf(hw, u0[sl].y, acc.y));
                acc = make_float2(fmaf(he, ue.x, acc.x), fmaf(he, ue.y, acc.y));
                u1[sl] = acc;
            }
        }
        // (c) residual of the red cell of row k - NH - 1 and the coarse
        // right-hand side of its 2x2 block (RES)
        if (RES) {
            const int rr = k - NH - 1;
            if (FAST || (rr >= k0 && rr < k1)) {   // uniform
                const int sl = IX(NH + 1), sn = IX(NH), ss = IX(NH + 2);
                const float2 *pr = pubs + (size_t)((buf ^ 1) * NP + NH) * PS;
                const float2 bred = bring[SLOT(NH + 1, BR) * NB * NT + 2 * NT + t];
                const bool edge = !FAST && (rr == 0 || rr == nz - 1);
                float2 res;
                if (((c - NH - 1) & 1) == 0) {   // red cell in column 0: west from the left pair
                    const float2 uw = pr[t - G];
                    float d, cw = cw0, ce = ce0;
                    float2 a;
                    if (!FAST && rw) {   // the row's class: face conductances toward active neighbours
                        const unsigned cl = (unsigned)L.rcls[rr];
                        const unsigned ci = cl * nr + (v0 ? i0 : 0);
                        d = v0 ? L.diag[cl * rs + c0] : 0.f;
                        cw = L.ccw[ci];
                        ce = L.cce[ci];
                        a = make_float2(fmaf(L.ccs[ci], u0[ss].x, bred.x), fmaf(L.ccs[ci], u0[ss].y, bred.y));
                        a = make_float2(fmaf(L.ccn[ci], u0[sn].x, a.x), fmaf(L.ccn[ci], u0[sn].y, a.y));
                    } else {
                        d = edge ? L.diag[(unsigned)row_class(rr, nz, ncls) * rs + c0] : dg0;
                        const float2 s = make_float2(u0[ss].x + u0[sn].x, u0[ss].y + u0[sn].y);
                        a = make_float2(fmaf(cz0, s.x, bred.x), fmaf(cz0, s.y, bred.y));
                    }
                    a = make_float2(fmaf(cw, uw.x, a.x), fmaf(cw, uw.y, a.y));
                    a = make_float2(fmaf(ce, u1[sl].x, a.x), fmaf(ce, u1[sl].y, a.y));
                    res = make_float2(fmaf(-d, u0[sl].x, a.x), fmaf(-d, u0[sl].y, a.y));
                    rsum = res;
                } else {                          // red cell in column 1: east from the right pair
                    const float2 ue = pr[t + G];
                    float d, cw = cw1, ce = ce1;
                    float2 a;
                    if (!FAST && rw) {
                        const unsigned cl = (unsigned)L.rcls[rr];
                        const unsigned ci = cl * nr + (v1 ? i1 : 0);
                        d = v1 ? L.diag[cl * rs + c1] : 0.f;
                        cw = L.ccw[ci];
                        ce = L.cce[ci];
                        a = make_float2(fmaf(L.ccs[ci], u1[ss].x, bred.x), fmaf(L.ccs[ci], u1[ss].y, bred.y));
                        a = make_float2(fmaf(L.ccn[ci], u1[sn].x, a.x), fmaf(L.ccn[ci], u1[sn].y, a.y));
                    } else {
                        d = edge ? L.diag[(unsigned)row_class(rr, nz, ncls) * rs + c1] : dg1;
                        const float2 s = make_float2(u1[ss].x + u1[sn].x, u1[ss].y + u1[sn].y);
                        a = make_float2(fmaf(cz1, s.x, bred.x), fmaf(cz1, s.y, bred.y));
                    }
                    a = make_float2(fmaf(cw, u0[sl].x, a.x), fmaf(cw, u0[sl].y, a.y));
                    a = make_float2(fmaf(ce, ue.x, a.x), fmaf(ce, ue.y, a.y));
                    res = make_float2(fmaf(-d, u1[sl].x, a.x), fmaf(-d, u1[sl].y, a.y));
                    const float2 sum = make_float2(rsum.x + res.x, rsum.y + res.y);
                    if (cwrite) {
                        const int K = rr >> 1;
                        const unsigned e = (unsigned)K * cnr * nm + ccol;
                        cb[e] = sum;
                        if (finit > 0) {
                            const float inv =
                                crcls ? cinvd[(unsigned)crcls[K] * cnr * nm + ccol]
                                : (K == 0 || K == cnz - 1)
                                    ? cinvd[(unsigned)row_class(K, cnz, cncls) * cnr * nm + ccol]
                                    : cinv1;
                            const float2 bhc = make_float2(sum.x * inv, sum.y * inv);
                            cbh[e] = bhc;
                            cu[e] = (finit == 2 && ((K + j) & 1) == 0) ? bhc : zero;
                        }
                    }
                }
            }
        }
        // (d) publish for the next step: half-sweep s will update row k - s
        // and read the neighbouring pair's column of the other colour;
        // the restriction reads the final black column of row k - NH
        float2 *pw = pubs + (size_t)(buf * NP) * PS + t;
#pragma unroll
        for (int s = 0; s < NH; ++s) {
            const int qn = (c - s + (s & 1)) & 1;
            pw[(size_t)s * PS] = qn == 0 ? u1[IX(s)] : u0[IX(s)];
        }
        if (RES) pw[(size_t)NH * PS] = ((c - NH) & 1) == 0 ? u1[IX(NH)] : u0[IX(NH)];
        // (e) the output row k - NH is final
        const int ro = k - NH;
        if (outpair && (FAST || (ro >= k0 && ro < k1))) {
            const unsigned o = (unsigned)ro * rs;
            if (v0) gout[o + c0] = u0[IX(NH)];
            if (v1) gout[o + c1] = u1[IX(NH)];
        }
        __syncthreads();
    };
    // the steps that take the FAST body: kf0 <= k < kf0 + nfast (none for
    // per-row classes; an empty range when the block's rows are too few)
    const int kf0 = max(k0, 1) + NH + (RES ? 1 : 0);
    const unsigned nfast = rw ? 0u : (unsigned)max(min(ke - DEPTH - 1, k1 + NH - 1) - kf0 + 1, 0);
#pragma unroll 1
    for (int n0 = 0;; n0 += U) {
#pragma unroll
        for (int c = 0; c < U; ++c) {
            const int k = ks + n0 + c;   // the row entering at this step
            if ((unsigned)(k - kf0) < nfast) {   // uniform
                step(c, k, std::true_type{});
            } else {
                if (k > klast) goto finished;   // uniform
                step(c, k, std::false_type{});
            }
        }
    }
#undef SLOT
#undef IX
finished:
    cp_async_wait<0>();   // no copy outlives the block
}

}  // namespace

template <int NH, bool RES, bool RW> cudaError_t launch_nh(const FusedTab *tab, unsigned grid, cudaStream_t st) {
    const size_t smem = FusedCfg<NH, RES>::smem_floats2 * sizeof(float2);
    cudaError_t e =
        cudaFuncSetAttribute(k_smooth_fused<NH, RES, RW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_smooth_fused<NH, RES, RW><<<grid, FUSED_THREADS, smem, st>>>(tab);
    return cudaGetLastError();
}

cudaError_t launch_smooth_fused(const FusedTab *tab, unsigned grid, int nh, bool res, cudaStream_t st, bool rw) {
    switch (nh * 4 + (res ? 2 : 0) + (rw ? 1 : 0)) {
    case 8: return launch_nh<2, false, false>(tab, grid, st);
    case 9: return launch_nh<2, false, true>(tab, grid, st);
    case 10: return launch_nh<2, true, false>(tab, grid, st);
    case 11: return launch_nh<2, true, true>(tab, grid, st);
    case 16: return launch_nh<4, false, false>(tab, grid, st);
    case 17: return launch_nh<4, false, true>(tab, grid, st);
    case 18: return launch_nh<4, true, false>(tab, grid, st);
    case 19: return launch_nh<4, true, true>(tab, grid, st);
    default: return cudaErrorInvalidValue;
    }
}

void fused_shape(int nr, int nz, int nm, int nh, bool res, int target_blocks, FusedProb &f, unsigned &blocks) {
    f.ngroups = (nm + 15) / 16;
    f.G = (nm + f.ngroups - 1) / f.ngroups;
    const int hp = nh / 2 + (res ? 1 : 0), pairs = nr / 2;
    f.P = std::min(FUSED_THREADS / f.G, pairs + 2 * hp);
    if (f.P < 2 * hp + 1) f.P = 2 * hp + 1;
    f.ntiles = (pairs + (f.P - 2 * hp) - 1) / (f.P - 2 * hp);
    const int per = f.ngroups * f.ntiles;
    int nkr = std::max(1, target_blocks / per);   // at most target_blocks: no partial last wave
    f.R = std::max(8, (nz + nkr - 1) / nkr);
    f.R += f.R & 1;   // even: the two rows of a coarse cell belong to one block
    f.nkr = (nz + f.R - 1) / f.R;
    blocks = (unsigned)(per * f.nkr);
}

}  // namespace pp
