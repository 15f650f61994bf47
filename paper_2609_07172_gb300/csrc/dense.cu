// Dense coarsest-level solve (step a-6 on a composite domain or a
// non-uniform axial mesh, where the coarsest operator does not separate):
//   u = M^(-1/2) Q (Lambda + lambda_m)^(-1) Q^T M^(-1/2) b
// over the level's active cells, with Q Lambda Q^T = M^(-1/2) A_0 M^(-1/2)
// factored at plan time and M = diag(mu) (the lambda_m term of
// Eq. shifted_operator_family is lambda_m M).  Q and Lambda are shared by all
// modes, so the N_theta + 2 right-hand sides of a problem (mode m, real and
// imaginary part) are solved together as two GEMMs of n x n by n x 2 N_m
// (n active cells): three launches instead of one block per right-hand side
// that each streamed Q twice.
//
//   k_dense_prep  one block per right-hand side: scale b by the power of two
//                 that brings its largest value to O(1) (exact; FP32 then
//                 spans any FP64 range), y = M^(-1/2) b in FP32, u = 0 on the
//                 inactive cells;
//   k_dense_gemm<1>  z_col = (Lambda + lambda_m)^(-1) Q^T y_col;
//   k_dense_gemm<2>  u = M^(-1/2) Q z_col, scaled back, into the level's
//                 complex layout.
//
// FP32 for both hierarchies: a coarse-grid correction needs no FP64
// accuracy, and the FP32 pipe runs at 64 times the FP64 rate.  Each dot
// product accumulates its n terms in index order with one fused multiply-add
// per term, the order of the per-block loops it replaces, so the result is
// bitwise the same.
#include "internal.h"

namespace pp {
namespace {

constexpr int TR = 32;   // output rows (cells or eigenvectors) per block
constexpr int TC = 32;   // right-hand sides per block
constexpr int TK = 32;   // contraction chunk staged in shared memory
constexpr int DENSE_THREADS = 256;

__device__ __forceinline__ int find_problem(const unsigned *__restrict__ start, int n, unsigned blk) {
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (start[mid] <= blk) lo = mid;
        else hi = mid;
    }
    return lo;
}

template <class T>
__global__ void __launch_bounds__(DENSE_THREADS) k_dense_prep(const DenseTab<T> *__restrict__ tab) {
    __shared__ int s_emax;
    const int p = find_problem(tab->start, tab->n, blockIdx.x);
    if (tab->done && tab->done[tab->pid[p]]) return;   // stopped problem of a batch
    const LevelDev<T> &L = tab->f[p];
    const CoarseDev<T> &D = tab->c[p];
    const int col = (int)(blockIdx.x - tab->start[p]);
    const int m = col >> 1, comp = col & 1, nm = D.nm, n = D.nact;
    const T *bg = (const T *)L.b + comp;
    if (threadIdx.x == 0) s_emax = -1100;
    __syncthreads();
    // b of this thread's cells a = t, t + 256, ... (n <= PIC_POISSON_MAX_DENSE
    // = 4 * 256), read once and kept for the scaled write
    constexpr int PER = (PIC_POISSON_MAX_DENSE + DENSE_THREADS - 1) / DENSE_THREADS;
    double v[PER];
    int em = -1100;
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int a = threadIdx.x + i * DENSE_THREADS;
        v[i] = a < n ? (double)bg[2 * ((size_t)D.aidx[a] * nm + m)] : 0.0;
        int e = -1100;
        if (v[i] != 0.0) frexp(v[i], &e);
        em = max(em, e);
    }
    atomicMax(&s_emax, em);
    __syncthreads();
    const int E = s_emax > -1100 ? s_emax : 0;
    const double down = ldexp(1.0, -E);
    if (threadIdx.x == 0) D.up[col] = ldexp(1.0, E);
    float *y = D.Y + (size_t)col * n;
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int a = threadIdx.x + i * DENSE_THREADS;
        if (a < n) y[a] = (float)(v[i] * down) * D.isq[a];
    }
    T *ug = (T *)L.u + comp;   // cells outside the domain hold u = 0
    for (int f = threadIdx.x; f < D.nr * D.nz; f += blockDim.x)
        if (D.amap[f] < 0) ug[2 * ((size_t)f * nm + m)] = T(0);
}

// C[col][r] = sum_k A[r][k] B[col][k] for a TR x TC tile, k in order.
// STAGE 1: A = Q^T (row j of Q^T is column j of Q), B = y; writes
// z[col][j] = C / (lambda_j + lambda_m).  STAGE 2: A = Q, B = z; writes
// u at cell aidx[a] of mode m, part comp: C M^(-1/2) times the scale.
template <class T, int STAGE>
__global__ void __launch_bounds__(DENSE_THREADS) k_dense_gemm(const DenseTab<T> *__restrict__ tab) {
    // A row-major (a lane's row, conflict-free); B k-major so that a thread's
    // four adjacent columns are one 16-byte broadcast load per k
    __shared__ float As[TR][TK + 1];
    __shared__ __align__(16) float Bs[TK][TC + 4];
    const int p = find_problem(tab->gstart, tab->n, blockIdx.x);
    if (tab->done && tab->done[tab->pid[p]]) return;
    const LevelDev<T> &L = tab->f[p];
    const CoarseDev<T> &D = tab->c[p];
    const int n = D.nact, ncol = 2 * D.nm;
    const int rtiles = (n + TR - 1) / TR;
    const int lb = (int)(blockIdx.x - tab->gstart[p]);
    const int r0 = (lb % rtiles) * TR, c0 = (lb / rtiles) * TC;
    const float *A = STAGE == 1 ? D.QT : D.Q;
    const float *B = STAGE == 1 ? D.Y : D.Z;
    const int t = threadIdx.x;
    const int tr = t % TR, tc = t / TR;   // row of the tile; columns 4 tc .. 4 tc + 3
    static_assert(TC == 4 * (DENSE_THREADS / TR), "four adjacent columns per thread");
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    // The next chunk's tiles are loaded into registers (read-only path, all
    // issued together) while the current one is multiplied from shared memory.
    constexpr int PER = TR * TK / DENSE_THREADS;   // values of each tile per thread
    static_assert(TR * TK == TC * TK && TR * TK % DENSE_THREADS == 0, "tile load mapping");
    float ra[PER], rb[PER];
    auto load = [&](int k0) {
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const int e = t + i * DENSE_THREADS, x = e / TK, kk = e - x * TK, gk = k0 + kk;
            const int gr = r0 + x, gc = c0 + x;
            ra[i] = (gr < n && gk < n) ? __ldg(A + (size_t)gr * n + gk) : 0.f;
            rb[i] = (gc < ncol && gk < n) ? __ldg(B + (size_t)gc * n + gk) : 0.f;
        }
    };
    load(0);
    for (int k0 = 0; k0 < n; k0 += TK) {
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const int e = t + i * DENSE_THREADS, x = e / TK, kk = e - x * TK;
            As[x][kk] = ra[i];
            Bs[kk][x] = rb[i];
        }
        __syncthreads();
        if (k0 + TK < n) load(k0 + TK);
        const int kmax = min(TK, n - k0);   // padded terms are not accumulated: the order and count match
#pragma unroll 8
        for (int kk = 0; kk < kmax; ++kk) {
            const float a = As[tr][kk];
            const float4 b = *reinterpret_cast<const float4 *>(&Bs[kk][4 * tc]);
            acc[0] = fmaf(a, b.x, acc[0]);
            acc[1] = fmaf(a, b.y, acc[1]);
            acc[2] = fmaf(a, b.z, acc[2]);
            acc[3] = fmaf(a, b.w, acc[3]);
        }
        __syncthreads();
    }
    const int r = r0 + tr;
    if (r >= n) return;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int col = c0 + 4 * tc + q;
        if (col >= ncol) continue;
        if (STAGE == 1) {
            D.Z[(size_t)col * n + r] = acc[q] / (D.lam[r] + D.lamm[col >> 1]);
        } else {
            const float x = acc[q] * D.isq[r];
            T *ug = (T *)L.u + (col & 1);
            ug[2 * ((size_t)D.aidx[r] * D.nm + (col >> 1))] = (T)((double)x * D.up[col]);
        }
    }
}

}  // namespace

unsigned dense_gemm_blocks(int nact, int nm) {
    return (unsigned)(((nact + TR - 1) / TR) * ((2 * nm + TC - 1) / TC));
}

template <class T>
cudaError_t launch_dense(const DenseTab<T> *tab, int stage, unsigned g_prep, unsigned g_gemm, cudaStream_t st) {
    switch (stage) {
    case 0: k_dense_prep<T><<<g_prep, DENSE_THREADS, 0, st>>>(tab); break;
    case 1: k_dense_gemm<T, 1><<<g_gemm, DENSE_THREADS, 0, st>>>(tab); break;
    default: k_dense_gemm<T, 2><<<g_gemm, DENSE_THREADS, 0, st>>>(tab); break;
    }
    return cudaGetLastError();
}

template cudaError_t launch_dense<double>(const DenseTab<double> *, int, unsigned, unsigned, cudaStream_t);
template cudaError_t launch_dense<float>(const DenseTab<float> *, int, unsigned, unsigned, cudaStream_t);

}  // namespace pp
