// Mode-local bottom of the V-cycle: the level above the coarsest (U) and the
// coarsest level (C) of one problem, solved per azimuthal mode and per real or
// imaginary part in one block's shared memory.
//
// Below the fine levels every kernel of the V-cycle is short (C1: a 64 x 50
// level of 65 modes is 3.3 MB) and the cost is launch latency and idle SMs:
// 6 half-sweeps, a restriction, the coarsest solve and a prolongation are 9
// dependent launches per cycle of a few microseconds of work each.  The
// modes, and the two real parts of a mode, are independent problems with the
// same real operator (Eq. shifted_operator_family), so one block per
// (problem, mode, part) can run that whole piece of the cycle with block
// barriers only: load b and b_hat of U, pre-smooth from zero, restrict the
// red-cell residual, solve C exactly (the separable solve of k_coarse), add
// the prolongated correction, post-smooth, store U's iterate for the
// prolongation to the next finer level.  Every cell is updated with the
// operations of the level kernels in mg.cu in the same order, so the result
// is bitwise that of the separate launches; only where the values live
// changes.
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

// One red-black half-sweep of colour `color` on U (one real part, shared memory).
template <class T>
__device__ void half_sweep(T *u, const T *bh, const T *hz, const T *hw, const T *he, int nr, int nz, int ncls,
                           int color) {
    const int hr = nr >> 1, ncell = nz * hr;
    for (int c = threadIdx.x; c < ncell; c += blockDim.x) {
        const int k = c / hr;
        const int i = 2 * (c - k * hr) + ((k + color) & 1);
        const int f = k * nr + i;
        const int tb = row_class(k, nz, ncls) * nr + i;
        T s = 0;
        if (k > 0) s = u[f - nr];
        if (k < nz - 1) {
            const T n = u[f + nr];
            s = (k > 0) ? s + n : n;
        }
        T acc = fma(hz[tb], s, bh[f]);
        if (i > 0) acc = fma(hw[tb], u[f - 1], acc);
        if (i < nr - 1) acc = fma(he[tb], u[f + 1], acc);
        u[f] = acc;
    }
    __syncthreads();
}

// b - A_m u at cell (k, i) of U (as residual_at in mg.cu).
template <class T>
__device__ __forceinline__ T residual(const T *u, const T *b, const T *cw, const T *ce, const T *cz, const T *dg,
                                      int k, int i, int nr, int nz, int ncls) {
    const int f = k * nr + i;
    T s = 0;
    if (k > 0) s = u[f - nr];
    if (k < nz - 1) {
        const T n = u[f + nr];
        s = (k > 0) ? s + n : n;
    }
    T acc = fma(cz[i], s, b[f]);
    if (i > 0) acc = fma(cw[i], u[f - 1], acc);
    if (i < nr - 1) acc = fma(ce[i], u[f + 1], acc);
    return fma(-dg[row_class(k, nz, ncls) * nr + i], u[f], acc);
}

template <class T>
__global__ void __launch_bounds__(BOTTOM_THREADS) k_bottom(const BottomTab<T> *__restrict__ tab) {
    extern __shared__ unsigned char smraw[];
    const int p = find_problem(tab->start, tab->n, blockIdx.x);
    if (tab->done && tab->done[tab->pid[p]]) return;   // stopped problem of a batch
    const BottomProb<T> &B = tab->p[p];
    const LevelDev<T> &U = B.U;
    const CoarseDev<T> &D = B.D;
    const int nr = U.nr, nz = U.nz, nm = U.nm, ncls = U.ncls, n = nr * nz;
    const int ncr = D.nr, ncz = D.nz, nc = ncr * ncz;
    const int lb = (int)(blockIdx.x - tab->start[p]);
    const int m = lb >> 1, part = lb & 1;
    const int fz = nz == ncz ? 1 : 2, fr = nr == ncr ? 1 : 2;

    // shared memory (element type T): U: u, b_hat, b [n]; tables [ncls][nr] x 4, [nr] x 3;
    // C: right-hand side / correction [nc]; separable solve: w [ncz][ncr + 1], V [ceil(ncz/2)][ncz],
    // this mode's Thomas factorisation piv, cpr [ncz][ncr + 1] and the off-diagonal e [ncr]
    T *u = (T *)smraw;
    T *bh = u + n;
    T *b = bh + n;
    T *hz = b + n;
    T *hw = hz + ncls * nr;
    T *he = hw + ncls * nr;
    T *dg = he + ncls * nr;
    T *cw = dg + ncls * nr;
    T *ce = cw + nr;
    T *cz = ce + nr;
    T *bc = cz + nr;
    const int lw = ncr + 1, hzc = ncz - ncz / 2, hc = ncz / 2;
    T *ws = bc + nc;
    T *Vs = ws + ncz * lw;
    T *ps = Vs + hzc * ncz;
    T *cs = ps + ncz * lw;
    T *es = cs + ncz * lw;

    // Every load of the block is issued at once (cp.async) in two groups: what
    // the pre-smoothing reads (b_hat, the smoother's tables), then what only
    // the restriction and the coarsest solve read (b -- of the red cells when
    // only those carry a residual -- the residual's tables, V and this mode's
    // factorisation), which arrives while the pre-smoothing runs.
    const T *gb = (const T *)U.b + part, *gbh = (const T *)U.bh + part;
    for (int f = threadIdx.x; f < n; f += blockDim.x) {
        cp_async_elem(bh + f, gbh + 2 * ((size_t)f * nm + m));
        u[f] = 0;
    }
    for (int f = threadIdx.x; f < ncls * nr; f += blockDim.x) {
        const size_t t = (size_t)f * nm + m;   // (class, i) -> ((class * nr + i) * nm + m)
        cp_async_elem(hz + f, U.hz + t);
        cp_async_elem(hw + f, U.hw + t);
        cp_async_elem(he + f, U.he + t);
    }
    cp_async_group_close();
    if (B.red_only) {
        const int hr = nr >> 1;
        for (int c = threadIdx.x; c < nz * hr; c += blockDim.x) {
            const int k = c / hr, f = k * nr + 2 * (c - k * hr) + (k & 1);   // (k + i) even
            cp_async_elem(b + f, gb + 2 * ((size_t)f * nm + m));
        }
    } else {
        for (int f = threadIdx.x; f < n; f += blockDim.x) cp_async_elem(b + f, gb + 2 * ((size_t)f * nm + m));
    }
    for (int f = threadIdx.x; f < ncls * nr; f += blockDim.x) cp_async_elem(dg + f, U.diag + (size_t)f * nm + m);
    for (int i = threadIdx.x; i < nr; i += blockDim.x) {
        cp_async_elem(cw + i, U.cw + i);
        cp_async_elem(ce + i, U.ce + i);
        cp_async_elem(cz + i, U.cz + i);
    }
    for (int f = threadIdx.x; f < hzc * ncz; f += blockDim.x) cp_async_elem(Vs + f, D.V + f);
    {
        const T *gp = D.piv + (size_t)m * ncz * ncr, *gc = D.cpr + (size_t)m * ncz * ncr;
        for (int f = threadIdx.x; f < ncz * ncr; f += blockDim.x) {
            const int j = f / ncr, i = f - j * ncr;
            cp_async_elem(ps + j * lw + i, gp + f);
            cp_async_elem(cs + j * lw + i, gc + f);
        }
        for (int i = threadIdx.x; i + 1 < ncr; i += blockDim.x) cp_async_elem(es + i, D.e + i);
    }
    cp_async_group_close();
    cp_async_group_wait<1>();
    __syncthreads();

    // pre-smoothing from zero (the restriction's fused first red half-sweep
    // gives the same values as the red half-sweep done here)
    for (int s = 0; s < B.pre; ++s) {
        half_sweep(u, bh, hz, hw, he, nr, nz, ncls, 0);
        half_sweep(u, bh, hz, hw, he, nr, nz, ncls, 1);
    }
    cp_async_group_wait<0>();
    __syncthreads();
    // residual of the fine cells of each coarse cell, summed (red cells only
    // after a black half-sweep), as k_residual_restrict
    for (int e = threadIdx.x; e < nc; e += blockDim.x) {
        const int K = e / ncr, I = e - K * ncr;
        const int ncells = B.red_only ? (fz == 2 && fr == 2 ? 2 : 1) : fz * fr;
        T sum = 0;
        for (int c = 0; c < ncells; ++c) {
            int k, i;
            if (B.red_only) {
                k = fz * K + (fz == 2 ? (fr == 2 ? c : (I & 1)) : 0);
                i = fr * I + (fr == 2 ? (fz == 2 ? c : (K & 1)) : 0);
            } else {
                k = fz * K + (fr == 2 ? (c >> 1) : c);
                i = fr * I + (fr == 2 ? (c & 1) : 0);
            }
            const T r = residual(u, b, cw, ce, cz, dg, k, i, nr, nz, ncls);
            sum = c == 0 ? r : sum + r;
        }
        bc[e] = sum;
    }
    __syncthreads();

    // exact solve on C (the separable, mirror-folded solve of k_coarse)
    for (int f = threadIdx.x; f < hc * ncr; f += blockDim.x) {
        const int k = f / ncr, i = f - k * ncr;
        const T lo = bc[k * ncr + i], hi = bc[(ncz - 1 - k) * ncr + i];
        bc[k * ncr + i] = lo + hi;
        bc[(ncz - 1 - k) * ncr + i] = lo - hi;
    }
    __syncthreads();
    for (int f = threadIdx.x; f < nc; f += blockDim.x) {
        const int j = f / ncr, i = f - j * ncr;
        T a = 0;
        if ((j & 1) == 0) {
            for (int k = 0; k < hzc; ++k) a = fma(Vs[k * ncz + j], bc[k * ncr + i], a);
        } else {
            for (int k = 0; k < hc; ++k) a = fma(Vs[k * ncz + j], bc[(ncz - 1 - k) * ncr + i], a);
        }
        ws[j * lw + i] = a;
    }
    __syncthreads();
    thomas_rows(ws, ps, cs, es, ncz, ncr, lw);
    __syncthreads();
    for (int f = threadIdx.x; f < hzc * ncr; f += blockDim.x) {   // correction into bc
        const int k = f / ncr, i = f - k * ncr;
        T e = 0, o = 0;
        for (int j = 0; j + 1 < ncz; j += 2) {
            e = fma(Vs[k * ncz + j], ws[j * lw + i], e);
            o = fma(Vs[k * ncz + j + 1], ws[(j + 1) * lw + i], o);
        }
        if (ncz & 1) e = fma(Vs[k * ncz + ncz - 1], ws[(ncz - 1) * lw + i], e);
        bc[k * ncr + i] = e + o;
        if (ncz - 1 - k != k) bc[(ncz - 1 - k) * ncr + i] = e - o;
    }
    __syncthreads();

    // prolongation of the correction (as k_prolong; black cells only when the
    // red half-sweep that follows overwrites the red ones)
    {
        const bool cz2 = fz == 2, cr2 = fr == 2;
        const int ncell = B.black_only ? nz * (nr >> 1) : n;
        for (int c = threadIdx.x; c < ncell; c += blockDim.x) {
            int k, i;
            if (B.black_only) {
                const int hr = nr >> 1;
                k = c / hr;
                i = 2 * (c - k * hr) + ((k + 1) & 1);
            } else {
                k = c / nr;
                i = c - k * nr;
            }
            const int K = cz2 ? (k >> 1) : k, I = cr2 ? (i >> 1) : i;
            const int K2 = K + ((k & 1) ? 1 : -1);
            const int I2 = I + ((i & 1) ? 1 : -1);
            const bool kin = K2 >= 0 && K2 < ncz;
            const bool iin = I2 >= 0 && I2 < ncr;
            const int Kx = kin ? K2 : K, Ix = iin ? I2 : I;
            const T c0 = bc[K * ncr + I];
            T v = u[k * nr + i];
            if (cz2 && cr2) {
                const T c1 = bc[K * ncr + Ix], c2 = bc[Kx * ncr + I], c3 = bc[Kx * ncr + Ix];
                const T w1 = iin ? T(0.1875) : T(-0.1875), w2 = kin ? T(0.1875) : T(-0.1875);
                const T w3 = iin == kin ? T(0.0625) : T(-0.0625);
                v = fma(w3, c3, fma(w2, c2, fma(w1, c1, fma(T(0.5625), c0, v))));
            } else {
                const T c1 = cz2 ? bc[Kx * ncr + I] : bc[K * ncr + Ix];
                const T w1 = (cz2 ? kin : iin) ? T(0.25) : T(-0.25);
                v = fma(w1, c1, fma(T(0.75), c0, v));
            }
            u[k * nr + i] = v;
        }
    }
    __syncthreads();
    for (int s = 0; s < B.post; ++s) {
        half_sweep(u, bh, hz, hw, he, nr, nz, ncls, 0);
        half_sweep(u, bh, hz, hw, he, nr, nz, ncls, 1);
    }
    T *gu = (T *)U.u + part;
    for (int f = threadIdx.x; f < n; f += blockDim.x) gu[2 * ((size_t)f * nm + m)] = u[f];
}

}  // namespace

template <class T> size_t bottom_smem_bytes(int nr, int nz, int ncls, int ncr, int ncz) {
    const size_t n = (size_t)nr * nz, nc = (size_t)ncr * ncz;
    return (3 * n + 4 * (size_t)ncls * nr + 3 * (size_t)nr + nc + 3 * (size_t)ncz * (ncr + 1) +
            (size_t)(ncz - ncz / 2) * ncz + (size_t)ncr) * sizeof(T);
}

template <class T> cudaError_t launch_bottom(const BottomTab<T> *tab, unsigned grid, size_t smem, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(k_bottom<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_bottom<T><<<grid, BOTTOM_THREADS, smem, st>>>(tab);
    return cudaGetLastError();
}

template size_t bottom_smem_bytes<double>(int, int, int, int, int);
template size_t bottom_smem_bytes<float>(int, int, int, int, int);
template cudaError_t launch_bottom<double>(const BottomTab<double> *, unsigned, size_t, cudaStream_t);
template cudaError_t launch_bottom<float>(const BottomTab<float> *, unsigned, size_t, cudaStream_t);

}  // namespace pp
