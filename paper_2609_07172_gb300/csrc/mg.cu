// Mode-batched matrix-free multigrid kernels (steps a-3 .. a-7).
//
// Every kernel works on the cell-major, mode-fast layout of Eq. mode_fast_layout
// (entry (k, i, m) at (k*nr + i)*nm + m, unpadded): consecutive threads take
// consecutive modes of one cell and then move to the next cell, so every load
// and store of a warp is contiguous, and the cell's coefficients are the same
// for all of its modes (Eq. shifted_operator_family: only the diagonal shift
// lambda_m mu_q depends on the mode, and it lives in the per-level inverse-
// diagonal table).  All modes of all cells are processed by one launch.
#include "internal.h"

namespace pp {
namespace {

constexpr int MG_THREADS = 256;

template <class T> __device__ __forceinline__ V2<T> mk(T x, T y);
template <> __device__ __forceinline__ double2 mk<double>(double x, double y) { return make_double2(x, y); }
template <> __device__ __forceinline__ float2 mk<float>(float x, float y) { return make_float2(x, y); }

template <class T> __device__ __forceinline__ V2<T> ld(const V2<T> *p) { return *p; }

__device__ __forceinline__ int row_class(int k, int nz, int ncls) {
    return k == 0 ? 0 : (k == nz - 1 ? ncls - 1 : 1);
}

template <class T> struct Acc {
    __device__ __forceinline__ static V2<T> fma2(T a, V2<T> x, V2<T> y) {
        return mk<T>(fma(a, x.x, y.x), fma(a, x.y, y.y));
    }
};

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
    V2<T> acc = Acc<T>::fma2(L.cz[i], s, L.b[idx]);
    if (i > 0) acc = Acc<T>::fma2(L.cw[i], L.u[idx - L.nm], acc);
    if (i < L.nr - 1) acc = Acc<T>::fma2(L.ce[i], L.u[idx + L.nm], acc);
    const T d = L.diag[((size_t)row_class(k, L.nz, L.ncls) * L.nr + i) * L.nm + m];
    const V2<T> uc = L.u[idx];
    return Acc<T>::fma2(-d, uc, acc);
}

// One red-black Gauss-Seidel half-sweep (colour (i + k) % 2 == color):
//   u_q <- (b_q + sum_q' G_qq' u_q') / (D0_q + lambda_m mu_q)
// the same real coefficients act on the real and imaginary parts.
template <class T>
__global__ void __launch_bounds__(MG_THREADS) k_smooth(const LevelDev<T> L, int color, unsigned total) {
    const unsigned e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total) return;
    const unsigned nm = L.nm, hr = L.nr >> 1;
    const unsigned c = e / nm;
    const int m = (int)(e - c * nm);
    const int k = (int)(c / hr);
    const int i = 2 * (int)(c - (unsigned)k * hr) + ((k + color) & 1);
    const size_t idx = ((size_t)k * L.nr + i) * nm + m;
    const size_t rowstride = (size_t)L.nr * nm;
    V2<T> s = mk<T>(0, 0);
    if (k > 0) s = L.u[idx - rowstride];
    if (k < L.nz - 1) {
        const V2<T> n = L.u[idx + rowstride];
        s = (k > 0) ? mk<T>(s.x + n.x, s.y + n.y) : n;
    }
    V2<T> acc = Acc<T>::fma2(L.cz[i], s, L.b[idx]);
    if (i > 0) acc = Acc<T>::fma2(L.cw[i], L.u[idx - nm], acc);
    if (i < L.nr - 1) acc = Acc<T>::fma2(L.ce[i], L.u[idx + nm], acc);
    const T inv = L.invd[((size_t)row_class(k, L.nz, L.ncls) * L.nr + i) * nm + m];
    L.u[idx] = mk<T>(acc.x * inv, acc.y * inv);
}

// Residual of the four fine cells of each coarse cell, summed into the coarse
// right-hand side (finite-volume restriction: the residual is a cell integral),
// coarse iterate zeroed, and (if partials) the Parseval-weighted squared norm.
template <class T>
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
                const int k = 2 * K + a, i = 2 * I + bb;
                const size_t idx = ((size_t)k * F.nr + i) * nm + m;
                const V2<T> r = residual_at(F, k, i, m, idx);
                sum.x += r.x;
                sum.y += r.y;
                if (partials) acc += (double)r.x * r.x + (double)r.y * r.y;
            }
        }
        C.b[e] = sum;
        C.u[e] = mk<T>(0, 0);
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
// (the correction vanishes on the Dirichlet face).
template <class T>
__global__ void __launch_bounds__(MG_THREADS) k_prolong(const LevelDev<T> F, const LevelDev<T> C, unsigned total) {
    const unsigned e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total) return;
    const unsigned nm = F.nm;
    const unsigned c = e / nm;
    const int m = (int)(e - c * nm);
    const int k = (int)(c / (unsigned)F.nr);
    const int i = (int)(c - (unsigned)k * F.nr);
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
    V2<T> u = F.u[e];
    u.x += fma(w3, c3.x, fma(w2, c2.x, fma(w1, c1.x, T(0.5625) * c0.x)));
    u.y += fma(w3, c3.y, fma(w2, c2.y, fma(w1, c1.y, T(0.5625) * c0.y)));
    F.u[e] = u;
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
cudaError_t launch_residual_restrict(const LevelDev<T> &L, const LevelDev<T> &C, int nt, double *partials,
                                     int *nblocks, cudaStream_t st) {
    const unsigned total = (unsigned)C.nz * (unsigned)C.nr * (unsigned)C.nm;
    k_residual_restrict<T><<<nblk(total), MG_THREADS, 0, st>>>(L, C, nt, partials, total);
    if (nblocks) *nblocks = (int)nblk(total);
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
cudaError_t launch_prolong(const LevelDev<T> &L, const LevelDev<T> &C, cudaStream_t st) {
    const unsigned total = (unsigned)L.nz * (unsigned)L.nr * (unsigned)L.nm;
    k_prolong<T><<<nblk(total), MG_THREADS, 0, st>>>(L, C, total);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_coarse(const LevelDev<T> &L, const CoarseDev<T> &C, cudaStream_t st) {
    const size_t smem = (size_t)2 * C.nr * C.nz * sizeof(V2<T>) + (size_t)C.nz * C.nz * sizeof(T);
    cudaFuncSetAttribute(k_coarse<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_coarse<T><<<C.nm, MG_THREADS, smem, st>>>(L, C);
    return cudaGetLastError();
}

cudaError_t launch_sum(const double *partials, int n, double *out, cudaStream_t st) {
    k_sum<<<1, 1024, 0, st>>>(partials, n, out);
    return cudaGetLastError();
}

#define PP_INST(T)                                                                                          \
    template cudaError_t launch_smooth<T>(const LevelDev<T> &, int, cudaStream_t);                          \
    template cudaError_t launch_residual_restrict<T>(const LevelDev<T> &, const LevelDev<T> &, int, double *, \
                                                     int *, cudaStream_t);                                  \
    template cudaError_t launch_residual<T>(const LevelDev<T> &, V2<T> *, int, double *, int *, cudaStream_t); \
    template cudaError_t launch_prolong<T>(const LevelDev<T> &, const LevelDev<T> &, cudaStream_t);         \
    template cudaError_t launch_coarse<T>(const LevelDev<T> &, const CoarseDev<T> &, cudaStream_t);
PP_INST(double)
PP_INST(float)
#undef PP_INST

}  // namespace pp
