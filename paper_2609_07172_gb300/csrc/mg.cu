// Mode-batched matrix-free multigrid kernels (steps a-3 .. a-7) and the
// FP64 defect / update kernels of the mixed-precision form.
//
// Every kernel works on the cell-major, mode-fast layout of Eq. mode_fast_layout
// (entry (k, i, m) at (k*nr + i)*nm + m, unpadded): consecutive threads take
// consecutive modes of one cell and then move to the next cell, so every load
// and store of a warp is contiguous.  Only the diagonal shift lambda_m mu of
// A_m depends on the mode (Eq. shifted_operator_family); it enters through
// per-level tables indexed (row class, i, m).
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

constexpr int MG_THREADS = 256;

template <class T> __device__ __forceinline__ V2<T> mk(T x, T y);
template <> __device__ __forceinline__ double2 mk<double>(double x, double y) { return make_double2(x, y); }
template <> __device__ __forceinline__ float2 mk<float>(float x, float y) { return make_float2(x, y); }

__device__ __forceinline__ int row_class(int k, int nz, int ncls) {
    return k == 0 ? 0 : (k == nz - 1 ? ncls - 1 : 1);
}

template <class T> __device__ __forceinline__ V2<T> fma2(T a, V2<T> x, V2<T> y) {
    return mk<T>(fma(a, x.x, y.x), fma(a, x.y, y.y));
}

// Parseval weight of mode m for a real signal of length nt: 1 for m = 0 and
// m = nt/2, 2 otherwise (the conjugate partner of m carries the same energy).
__device__ __forceinline__ double parseval_w(int m, int nt) { return (m == 0 || 2 * m == nt) ? 1.0 : 2.0; }

__device__ __forceinline__ double block_sum(double v, double *red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    return s;
}

// (k, i) of the c-th cell of colour `color` ((i + k) % 2 == color) on a level
// with an even number of radial cells.
__device__ __forceinline__ void colour_cell(unsigned c, int nr, int color, int &k, int &i) {
    const unsigned hr = (unsigned)nr >> 1;
    k = (int)(c / hr);
    i = 2 * (int)(c - (unsigned)k * hr) + ((k + color) & 1);
}

// b - A_m u at entry (k, i, m), Eq. matrix_free_mode_operator.
template <class T>
__device__ __forceinline__ V2<T> residual_at(const LevelDev<T> &L, int k, int i, int m, size_t idx) {
    const size_t rowstride = (size_t)L.nr * L.nm;
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
template <class T>
__global__ void __launch_bounds__(MG_THREADS) k_smooth(const LevelDev<T> L, int color, unsigned total) {
    const unsigned e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total) return;
    const unsigned nm = L.nm;
    const unsigned c = e / nm;
    const int m = (int)(e - c * nm);
    int k, i;
    colour_cell(c, L.nr, color, k, i);
    const size_t idx = ((size_t)k * L.nr + i) * nm + m;
    const size_t tab = ((size_t)row_class(k, L.nz, L.ncls) * L.nr + i) * nm + m;
    const size_t rowstride = (size_t)L.nr * nm;
    V2<T> s = mk<T>(0, 0);
    if (k > 0) s = L.u[idx - rowstride];
    if (k < L.nz - 1) {
        const V2<T> n = L.u[idx + rowstride];
        s = (k > 0) ? mk<T>(s.x + n.x, s.y + n.y) : n;
    }
    V2<T> acc = fma2<T>(L.hz[tab], s, L.bh[idx]);
    if (i > 0) acc = fma2<T>(L.hw[tab], L.u[idx - nm], acc);
    if (i < L.nr - 1) acc = fma2<T>(L.he[tab], L.u[idx + nm], acc);
    L.u[idx] = acc;
}

// Residual of the fine cells of each coarse cell, summed into the coarse
// right-hand side (finite-volume restriction: a residual is a cell integral),
// with optional Parseval-weighted squared-norm partials.
//  RED_ONLY: only the two red fine cells (after a black half-sweep the black
//            residuals vanish); otherwise all four.
//  INIT: 0 = write coarse b only (coarsest level, solved directly);
//        1 = also b_hat = b / diag and u = 0;
//        2 = also b_hat and u = (red ? b_hat : 0), i.e. the first red
//            half-sweep from a zero iterate.
template <class T, bool RED_ONLY, int INIT>
__global__ void __launch_bounds__(MG_THREADS)
k_residual_restrict(const LevelDev<T> F, const LevelDev<T> C, int nt, double *__restrict__ partials, unsigned total) {
    __shared__ double red[MG_THREADS / 32];
    const unsigned e = blockIdx.x * blockDim.x + threadIdx.x;
    double acc = 0.0;
    if (e < total) {
        const unsigned nm = C.nm;
        const unsigned cc = e / nm;
        const int m = (int)(e - cc * nm);
        const int K = (int)(cc / (unsigned)C.nr);
        const int I = (int)(cc - (unsigned)K * C.nr);
        V2<T> sum = mk<T>(0, 0);
#pragma unroll
        for (int a = 0; a < 2; ++a) {
#pragma unroll
            for (int bb = 0; bb < 2; ++bb) {
                if (RED_ONLY && a != bb) continue;
                const int k = 2 * K + a, i = 2 * I + bb;
                const size_t idx = ((size_t)k * F.nr + i) * nm + m;
                const V2<T> r = residual_at(F, k, i, m, idx);
                sum.x += r.x;
                sum.y += r.y;
                if (partials) acc += (double)r.x * r.x + (double)r.y * r.y;
            }
        }
        C.b[e] = sum;
        if (INIT > 0) {
            const T inv = C.invd[((size_t)row_class(K, C.nz, C.ncls) * C.nr + I) * nm + m];
            const V2<T> bh = mk<T>(sum.x * inv, sum.y * inv);
            C.bh[e] = bh;
            C.u[e] = (INIT == 2 && ((K + I) & 1) == 0) ? bh : mk<T>(0, 0);
        }
        if (partials) acc *= parseval_w(m, nt);
    }
    if (partials) {
        const double tot = block_sum(acc, red);
        if (threadIdx.x == 0) partials[blockIdx.x] = tot;
    }
}

// r = b - A_m u on one level (r may be null), with Parseval-weighted squared
// norms of r and b in partials[0..nblocks) and partials[nblocks..2 nblocks).
template <class T>
__global__ void __launch_bounds__(MG_THREADS)
k_residual(const LevelDev<T> L, V2<T> *__restrict__ r_out, int nt, double *__restrict__ partials, unsigned total) {
    __shared__ double red[MG_THREADS / 32];
    const unsigned e = blockIdx.x * blockDim.x + threadIdx.x;
    double ar = 0.0, ab = 0.0;
    if (e < total) {
        const unsigned nm = L.nm;
        const unsigned c = e / nm;
        const int m = (int)(e - c * nm);
        const int k = (int)(c / (unsigned)L.nr);
        const int i = (int)(c - (unsigned)k * L.nr);
        const V2<T> r = residual_at(L, k, i, m, e);
        if (r_out) r_out[e] = r;
        const V2<T> b = L.b[e];
        const double w = parseval_w(m, nt);
        ar = w * ((double)r.x * r.x + (double)r.y * r.y);
        ab = w * ((double)b.x * b.x + (double)b.y * b.y);
    }
    if (partials) {
        const double tr = block_sum(ar, red);
        if (threadIdx.x == 0) partials[blockIdx.x] = tr;
        const double tb = block_sum(ab, red);
        if (threadIdx.x == 0) partials[gridDim.x + blockIdx.x] = tb;
    }
}

// Bilinear cell-centred prolongation of the coarse correction and update
// u += P e.  Weights 9/16, 3/16, 3/16, 1/16 from the four nearest coarse
// centres; beyond a wall the coarse value is reflected with a sign change
// (the correction vanishes on the Dirichlet face).  BLACK_ONLY: only black
// fine cells (the red half-sweep that follows overwrites the red ones).
template <class T, bool BLACK_ONLY>
__global__ void __launch_bounds__(MG_THREADS) k_prolong(const LevelDev<T> F, const LevelDev<T> C, unsigned total) {
    const unsigned e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total) return;
    const unsigned nm = F.nm;
    const unsigned c = e / nm;
    const int m = (int)(e - c * nm);
    int k, i;
    if (BLACK_ONLY) {
        colour_cell(c, F.nr, 1, k, i);
    } else {
        k = (int)(c / (unsigned)F.nr);
        i = (int)(c - (unsigned)k * F.nr);
    }
    const size_t idx = ((size_t)k * F.nr + i) * nm + m;
    const int K = k >> 1, I = i >> 1;
    const int K2 = K + ((k & 1) ? 1 : -1);
    const int I2 = I + ((i & 1) ? 1 : -1);
    const bool kin = K2 >= 0 && K2 < C.nz;
    const bool iin = I2 >= 0 && I2 < C.nr;
    const int Kx = kin ? K2 : K, Ix = iin ? I2 : I;
    const T sk = kin ? T(1) : T(-1), si = iin ? T(1) : T(-1);
    const V2<T> c0 = C.u[((size_t)K * C.nr + I) * nm + m];
    const V2<T> c1 = C.u[((size_t)K * C.nr + Ix) * nm + m];
    const V2<T> c2 = C.u[((size_t)Kx * C.nr + I) * nm + m];
    const V2<T> c3 = C.u[((size_t)Kx * C.nr + Ix) * nm + m];
    const T w1 = T(0.1875) * si, w2 = T(0.1875) * sk, w3 = T(0.0625) * si * sk;
    V2<T> u = F.u[idx];
    u.x += fma(w3, c3.x, fma(w2, c2.x, fma(w1, c1.x, T(0.5625) * c0.x)));
    u.y += fma(w3, c3.y, fma(w2, c2.y, fma(w1, c1.y, T(0.5625) * c0.y)));
    F.u[idx] = u;
}

// Mixed precision, FP64 defect: r = b - A_m x on the FP64 level-0 view D
// (all cells), Parseval-weighted ||r||^2 partials, and the FP32 level-0
// right-hand side of the correction equation, scaled by sigma (a power of two,
// exact): b32 = r * sigma, b_hat32 = b32 / diag, u32 = (red ? b_hat32 : 0) --
// the first red half-sweep of the FP32 V-cycle from a zero correction
// (INIT_RED) -- or u32 = 0.
template <bool INIT_RED>
__global__ void __launch_bounds__(MG_THREADS)
k_defect(const LevelDev<double> D, const LevelDev<float> S, double sigma, int nt, double *__restrict__ partials,
         unsigned total) {
    __shared__ double red[MG_THREADS / 32];
    const unsigned e = blockIdx.x * blockDim.x + threadIdx.x;
    double acc = 0.0;
    if (e < total) {
        const unsigned nm = D.nm;
        const unsigned c = e / nm;
        const int m = (int)(e - c * nm);
        const int k = (int)(c / (unsigned)D.nr);
        const int i = (int)(c - (unsigned)k * D.nr);
        const double2 r = residual_at(D, k, i, m, e);
        acc = parseval_w(m, nt) * (r.x * r.x + r.y * r.y);
        const float2 b32 = make_float2((float)(r.x * sigma), (float)(r.y * sigma));
        const float inv = S.invd[((size_t)row_class(k, S.nz, S.ncls) * S.nr + i) * nm + m];
        const float2 bh = make_float2(b32.x * inv, b32.y * inv);
        S.b[e] = b32;
        S.bh[e] = bh;
        S.u[e] = (INIT_RED && ((k + i) & 1) == 0) ? bh : make_float2(0.f, 0.f);
    }
    const double tot = block_sum(acc, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = tot;
}

// Mixed precision, FP64 update: x += e32 / sigma.
__global__ void __launch_bounds__(MG_THREADS)
k_update(const LevelDev<double> D, const LevelDev<float> S, double inv_sigma, unsigned total) {
    const unsigned e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total) return;
    const float2 c = S.u[e];
    double2 x = D.u[e];
    x.x = fma((double)c.x, inv_sigma, x.x);
    x.y = fma((double)c.y, inv_sigma, x.y);
    D.u[e] = x;
}

// Coarsest level, exact separable solve, one CTA per mode.  On a uniform
// level A_m = I_z (x) K_m + T_z (x) diag(cz) with K_m the radial tridiagonal
// operator (diagonal D0r + lambda_m mu) and T_z = tridiag(-1, tz_k, -1).
// T_z = V Lambda V^T (V given), so for each axial eigenvector j the system is
// tridiagonal in r: (K_m + Lambda_j diag(cz)) w_j = (V^T b)_j, factorised at
// plan time (Thomas: inverse pivots piv, multipliers cpr).  u = V w.
template <class T>
__global__ void __launch_bounds__(MG_THREADS) k_coarse(const LevelDev<T> L, const CoarseDev<T> D) {
    extern __shared__ unsigned char smraw[];
    const int nr = D.nr, nz = D.nz, nm = D.nm;
    const int m = blockIdx.x;
    V2<T> *bs = (V2<T> *)smraw;              // [nz][nr]
    V2<T> *ws = bs + (size_t)nz * nr;        // [nz][nr]
    T *Vs = (T *)(ws + (size_t)nz * nr);     // [nz][nz]
    const int n = nr * nz;
    for (int f = threadIdx.x; f < n; f += blockDim.x) bs[f] = L.b[(size_t)f * nm + m];
    for (int f = threadIdx.x; f < nz * nz; f += blockDim.x) Vs[f] = D.V[f];
    __syncthreads();
    // w[j][i] = sum_k V[k][j] b[k][i]
    for (int f = threadIdx.x; f < n; f += blockDim.x) {
        const int j = f / nr, i = f - j * nr;
        T ax = 0, ay = 0;
        for (int k = 0; k < nz; ++k) {
            const T v = Vs[k * nz + j];
            const V2<T> b = bs[k * nr + i];
            ax = fma(v, b.x, ax);
            ay = fma(v, b.y, ay);
        }
        ws[f] = mk<T>(ax, ay);
    }
    __syncthreads();
    // tridiagonal solves along r, one thread per (j, component)
    for (int t = threadIdx.x; t < 2 * nz; t += blockDim.x) {
        const int j = t >> 1, comp = t & 1;
        const T *piv = D.piv + ((size_t)m * nz + j) * nr;
        const T *cpr = D.cpr + ((size_t)m * nz + j) * nr;
        T *row = ((T *)(ws + (size_t)j * nr)) + comp;   // stride 2
        T y = row[0] * piv[0];
        row[0] = y;
        for (int i = 1; i < nr; ++i) {
            y = (row[2 * i] - D.e[i - 1] * y) * piv[i];
            row[2 * i] = y;
        }
        T x = y;
        for (int i = nr - 2; i >= 0; --i) {
            x = row[2 * i] - cpr[i] * x;
            row[2 * i] = x;
        }
    }
    __syncthreads();
    // u[k][i] = sum_j V[k][j] w[j][i]
    for (int f = threadIdx.x; f < n; f += blockDim.x) {
        const int k = f / nr, i = f - k * nr;
        T ax = 0, ay = 0;
        for (int j = 0; j < nz; ++j) {
            const T v = Vs[k * nz + j];
            const V2<T> w = ws[j * nr + i];
            ax = fma(v, w.x, ax);
            ay = fma(v, w.y, ay);
        }
        L.u[(size_t)f * nm + m] = mk<T>(ax, ay);
    }
}

// Deterministic single-CTA sum of n partials (fixed order per thread, fixed tree).
__global__ void __launch_bounds__(1024) k_sum(const double *__restrict__ p, int n, double *__restrict__ out) {
    __shared__ double red[32];
    double s = 0.0;
    for (int f = threadIdx.x; f < n; f += blockDim.x) s += p[f];
    const double t = block_sum(s, red);
    if (threadIdx.x == 0) *out = t;
}

inline unsigned nblk(unsigned total) { return (total + MG_THREADS - 1) / MG_THREADS; }

}  // namespace

template <class T>
cudaError_t launch_smooth(const LevelDev<T> &L, int color, cudaStream_t st) {
    const unsigned total = (unsigned)L.nz * (unsigned)(L.nr / 2) * (unsigned)L.nm;
    k_smooth<T><<<nblk(total), MG_THREADS, 0, st>>>(L, color, total);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_residual_restrict(const LevelDev<T> &L, const LevelDev<T> &C, int nt, bool red_only, int init,
                                     double *partials, int *nblocks, cudaStream_t st) {
    const unsigned total = (unsigned)C.nz * (unsigned)C.nr * (unsigned)C.nm;
    const unsigned nb = nblk(total);
    if (red_only) {
        if (init == 0) k_residual_restrict<T, true, 0><<<nb, MG_THREADS, 0, st>>>(L, C, nt, partials, total);
        else if (init == 1) k_residual_restrict<T, true, 1><<<nb, MG_THREADS, 0, st>>>(L, C, nt, partials, total);
        else k_residual_restrict<T, true, 2><<<nb, MG_THREADS, 0, st>>>(L, C, nt, partials, total);
    } else {
        if (init == 0) k_residual_restrict<T, false, 0><<<nb, MG_THREADS, 0, st>>>(L, C, nt, partials, total);
        else if (init == 1) k_residual_restrict<T, false, 1><<<nb, MG_THREADS, 0, st>>>(L, C, nt, partials, total);
        else k_residual_restrict<T, false, 2><<<nb, MG_THREADS, 0, st>>>(L, C, nt, partials, total);
    }
    if (nblocks) *nblocks = (int)nb;
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_residual(const LevelDev<T> &L, V2<T> *r, int nt, double *partials, int *nblocks,
                            cudaStream_t st) {
    const unsigned total = (unsigned)L.nz * (unsigned)L.nr * (unsigned)L.nm;
    k_residual<T><<<nblk(total), MG_THREADS, 0, st>>>(L, r, nt, partials, total);
    if (nblocks) *nblocks = (int)nblk(total);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_prolong(const LevelDev<T> &L, const LevelDev<T> &C, bool black_only, cudaStream_t st) {
    if (black_only) {
        const unsigned total = (unsigned)L.nz * (unsigned)(L.nr / 2) * (unsigned)L.nm;
        k_prolong<T, true><<<nblk(total), MG_THREADS, 0, st>>>(L, C, total);
    } else {
        const unsigned total = (unsigned)L.nz * (unsigned)L.nr * (unsigned)L.nm;
        k_prolong<T, false><<<nblk(total), MG_THREADS, 0, st>>>(L, C, total);
    }
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_coarse(const LevelDev<T> &L, const CoarseDev<T> &C, cudaStream_t st) {
    const size_t smem = (size_t)2 * C.nr * C.nz * sizeof(V2<T>) + (size_t)C.nz * C.nz * sizeof(T);
    cudaFuncSetAttribute(k_coarse<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_coarse<T><<<C.nm, MG_THREADS, smem, st>>>(L, C);
    return cudaGetLastError();
}

cudaError_t launch_defect(const LevelDev<double> &D, const LevelDev<float> &S, double sigma, int nt, bool init_red,
                          double *partials, int *nblocks, cudaStream_t st) {
    const unsigned total = (unsigned)D.nz * (unsigned)D.nr * (unsigned)D.nm;
    if (init_red) k_defect<true><<<nblk(total), MG_THREADS, 0, st>>>(D, S, sigma, nt, partials, total);
    else k_defect<false><<<nblk(total), MG_THREADS, 0, st>>>(D, S, sigma, nt, partials, total);
    if (nblocks) *nblocks = (int)nblk(total);
    return cudaGetLastError();
}

cudaError_t launch_update(const LevelDev<double> &D, const LevelDev<float> &S, double inv_sigma, cudaStream_t st) {
    const unsigned total = (unsigned)D.nz * (unsigned)D.nr * (unsigned)D.nm;
    k_update<<<nblk(total), MG_THREADS, 0, st>>>(D, S, inv_sigma, total);
    return cudaGetLastError();
}

cudaError_t launch_sum(const double *partials, int n, double *out, cudaStream_t st) {
    k_sum<<<1, 1024, 0, st>>>(partials, n, out);
    return cudaGetLastError();
}

#define PP_INST(T)                                                                                          \
    template cudaError_t launch_smooth<T>(const LevelDev<T> &, int, cudaStream_t);                          \
    template cudaError_t launch_residual_restrict<T>(const LevelDev<T> &, const LevelDev<T> &, int, bool, int, \
                                                     double *, int *, cudaStream_t);                        \
    template cudaError_t launch_residual<T>(const LevelDev<T> &, V2<T> *, int, double *, int *, cudaStream_t); \
    template cudaError_t launch_prolong<T>(const LevelDev<T> &, const LevelDev<T> &, bool, cudaStream_t);   \
    template cudaError_t launch_coarse<T>(const LevelDev<T> &, const CoarseDev<T> &, cudaStream_t);
PP_INST(double)
PP_INST(float)
#undef PP_INST

}  // namespace pp
