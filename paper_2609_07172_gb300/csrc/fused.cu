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
// steps ahead with cp.async into a shared-memory ring (zero-filled beyond
// the level), so a thread's window registers are filled from shared memory
// and DEPTH rows of loads stay in flight.
#include <algorithm>

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

constexpr int DEPTH = 8;          // rows in flight ahead of the window
constexpr int RING = DEPTH + 1;   // ring slots (the slot being refilled is never the one just read)
constexpr int PAD = 16;           // >= the largest mode group: neighbour reads of the outermost pairs stay in the array

template <int NH>
__global__ void __launch_bounds__(FUSED_THREADS, 2) k_smooth_fused(const FusedTab *__restrict__ tab) {
    constexpr int W = NH + 2;      // window rows: k-NH-1 .. k
    constexpr int HP = NH / 2;     // halo pairs on each side
    constexpr int NT = FUSED_THREADS;
    extern __shared__ float2 dsm[];
    float2 *ring = dsm;                   // [RING][4][NT]: u col 0, u col 1, b_hat col 0, b_hat col 1
    float2 *pubs = dsm + RING * 4 * NT + PAD;   // [2][NH][NT + 2 PAD], PAD entries before each row
    const int p = find_problem(tab->start, tab->n, blockIdx.x);
    const FusedProb &F = tab->p[p];
    const LevelDev<float> &L = F.L;
    const int nr = L.nr, nz = L.nz, nm = L.nm, ncls = L.ncls;
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
    const int k0 = kr * F.R, k1 = min(nz, k0 + F.R);
    const int ks = max(0, k0 - NH), ke = min(nz, k1 + NH);   // rows read: [ks, ke)
    const int klast = k1 - 1 + NH;                           // last step (its output row is k1 - 1)

    const size_t rs = (size_t)nr * nm;
    const size_t c0 = (size_t)(v0 ? i0 : 0) * nm + (mvalid ? m : 0);
    const size_t c1 = (size_t)(v1 ? i1 : 0) * nm + (mvalid ? m : 0);
    const size_t cls1 = ncls > 1 ? rs : 0;
    const float hz0 = L.hz[cls1 + c0], hw0 = L.hw[cls1 + c0], he0 = L.he[cls1 + c0];
    const float hz1 = L.hz[cls1 + c1], hw1 = L.hw[cls1 + c1], he1 = L.he[cls1 + c1];

    // fetch row `row` into ring slot `slot` (zeros for rows outside [ks, ke) and invalid cells)
    const float2 *gin0 = F.in + c0, *gin1 = F.in + c1, *gb0 = L.bh + c0, *gb1 = L.bh + c1;
    auto fetch = [&](int row, int slot) {
        const bool ok = row < ke;
        const size_t o = (size_t)(ok ? row : ks) * rs;
        float2 *r = ring + slot * 4 * NT + t;
        cp_async8(r, gin0 + o, ok && v0);
        cp_async8(r + NT, gin1 + o, ok && v1);
        cp_async8(r + 2 * NT, gb0 + o, ok && v0);
        cp_async8(r + 3 * NT, gb1 + o, ok && v1);
        cp_async_commit();
    };
#pragma unroll
    for (int d = 0; d < DEPTH; ++d) fetch(ks + d, d);

    const float2 zero = make_float2(0.f, 0.f);
    float2 u0[W], u1[W], b0[W], b1[W];
#pragma unroll
    for (int w = 0; w < W; ++w) u0[w] = u1[w] = b0[w] = b1[w] = zero;
    int buf = 0;
    int rslot = 0;   // ring slot of the row entering now
    for (int kb = ks; kb <= klast; kb += W) {
#pragma unroll
        for (int ph = 0; ph < W; ++ph) {
            const int k = kb + ph;   // the row entering at this step
            if (k > klast) break;    // uniform over the block
            // (a) row k from the ring into window slot ph; fetch row k + DEPTH
            cp_async_wait<DEPTH - 1>();
            {
                const float2 *r = ring + rslot * 4 * NT + t;
                u0[ph] = r[0];
                u1[ph] = r[NT];
                b0[ph] = r[2 * NT];
                b1[ph] = r[3 * NT];
            }
            {
                int fs = rslot + DEPTH;
                if (fs >= RING) fs -= RING;
                fetch(k + DEPTH, fs);
            }
            rslot = rslot + 1 == RING ? 0 : rslot + 1;
            // (b) half-sweep s on row k - 1 - s
#pragma unroll
            for (int s = 0; s < NH; ++s) {
                const int r = k - 1 - s;
                if (r < ks || r >= ke) continue;           // uniform
                const int sl = (ph - 1 - s + 2 * W) % W;   // row r
                const int sn = (ph - s + 2 * W) % W;       // row r + 1
                const int ss = (ph - 2 - s + 2 * W) % W;   // row r - 1
                const int q = (r + (s & 1)) & 1;           // the pair's cell of this colour (uniform)
                const bool edge = r == 0 || r == nz - 1;
                const float2 *pr = pubs + (size_t)((buf ^ 1) * NH + s) * (NT + 2 * PAD);
                // Rows outside the level are zero in the window and the wall
                // columns have zero coefficients towards the wall (h_w = 0 at
                // i = 0, h_e = 0 at i = nr - 1), so every update is the same
                // four multiply-adds per part -- the neighbour that does not
                // exist contributes exactly zero, as when it is left out.
                // The pair beyond a block's outermost pair reads padding
                // (halo cells only).
                if (q == 0) {
                    const float2 vs = make_float2(u0[ss].x + u0[sn].x, u0[ss].y + u0[sn].y);
                    float hz = hz0, hw = hw0, he = he0;
                    if (edge) {
                        const size_t tb = (size_t)row_class(r, nz, ncls) * rs + c0;
                        hz = L.hz[tb];
                        hw = L.hw[tb];
                        he = L.he[tb];
                    }
                    const float2 uw = pr[t - G];   // west: column 1 of the pair on the left
                    float2 acc = make_float2(fmaf(hz, vs.x, b0[sl].x), fmaf(hz, vs.y, b0[sl].y));
                    acc = make_float2(fmaf(hw, uw.x, acc.x), fmaf(hw, uw.y, acc.y));
                    acc = make_float2(fmaf(he, u1[sl].x, acc.x), fmaf(he, u1[sl].y, acc.y));
                    if (v0) u0[sl] = acc;
                } else {
                    const float2 vs = make_float2(u1[ss].x + u1[sn].x, u1[ss].y + u1[sn].y);
                    float hz = hz1, hw = hw1, he = he1;
                    if (edge) {
                        const size_t tb = (size_t)row_class(r, nz, ncls) * rs + c1;
                        hz = L.hz[tb];
                        hw = L.hw[tb];
                        he = L.he[tb];
                    }
                    const float2 ue = pr[t + G];   // east: column 0 of the pair on the right
                    float2 acc = make_float2(fmaf(hz, vs.x, b1[sl].x), fmaf(hz, vs.y, b1[sl].y));
                    acc = make_float2(fmaf(hw, u0[sl].x, acc.x), fmaf(hw, u0[sl].y, acc.y));
                    acc = make_float2(fmaf(he, ue.x, acc.x), fmaf(he, ue.y, acc.y));
                    if (v1) u1[sl] = acc;
                }
            }
            // (c) publish for the next step: half-sweep s will update row k - s
            // and read the neighbouring pair's column of the other colour
            float2 *pw = pubs + (size_t)(buf * NH) * (NT + 2 * PAD) + t;
#pragma unroll
            for (int s = 0; s < NH; ++s) {
                const int sl = (ph - s + 2 * W) % W;
                const int qn = (k - s + (s & 1)) & 1;
                pw[(size_t)s * (NT + 2 * PAD)] = qn == 0 ? u1[sl] : u0[sl];
            }
            // (d) the output row k - NH is final
            const int ro = k - NH;
            if (outpair && ro >= k0 && ro < k1) {
                const int so = (ph + 2) % W;   // (ph - NH) mod W
                const size_t o = (size_t)ro * rs;
                if (v0) F.out[o + c0] = u0[so];
                if (v1) F.out[o + c1] = u1[so];
            }
            __syncthreads();
            buf ^= 1;
        }
    }
    cp_async_wait<0>();   // no copy outlives the block
}

}  // namespace

template <int NH> cudaError_t launch_nh(const FusedTab *tab, unsigned grid, cudaStream_t st) {
    const size_t smem = ((size_t)RING * 4 * FUSED_THREADS + PAD + (size_t)2 * NH * (FUSED_THREADS + 2 * PAD)) *
                        sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(k_smooth_fused<NH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_smooth_fused<NH><<<grid, FUSED_THREADS, smem, st>>>(tab);
    return cudaGetLastError();
}

cudaError_t launch_smooth_fused(const FusedTab *tab, unsigned grid, int nh, cudaStream_t st) {
    switch (nh) {
    case 2: return launch_nh<2>(tab, grid, st);
    case 4: return launch_nh<4>(tab, grid, st);
    default: return cudaErrorInvalidValue;
    }
}

void fused_shape(int nr, int nz, int nm, int nh, int target_blocks, FusedProb &f, unsigned &blocks) {
    f.ngroups = (nm + 15) / 16;
    f.G = (nm + f.ngroups - 1) / f.ngroups;
    const int hp = nh / 2, pairs = nr / 2;
    f.P = std::min(FUSED_THREADS / f.G, pairs + 2 * hp);
    if (f.P < 2 * hp + 1) f.P = 2 * hp + 1;
    f.ntiles = (pairs + (f.P - 2 * hp) - 1) / (f.P - 2 * hp);
    const int per = f.ngroups * f.ntiles;
    int nkr = std::max(1, target_blocks / per);   // at most target_blocks: no partial last wave
    f.R = std::max(8, (nz + nkr - 1) / nkr);
    f.nkr = (nz + f.R - 1) / f.R;
    blocks = (unsigned)(per * f.nkr);
}

}  // namespace pp
