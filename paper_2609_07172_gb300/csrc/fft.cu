// Batched azimuthal real DFT (step a-1, fused with the right-hand side build)
// and its inverse (step a-8).
//
// Forward, Eq. azimuthal_dft with the 1/N_theta scale, then Eq. mode_rhs:
//   b_(i,k),m = s_i * (1/N) sum_j rho_(i,j,k) e^{-2 pi i m j / N} + b^D_(i,k) delta_m0
// Inverse (Sec. 3.1, inverse transform, no scale), with conjugate symmetry:
//   phi_j = sum_{m=0}^{N-1} phihat_m e^{2 pi i m j / N}
//
// Each CTA owns one axial plane k of one problem and TI = 32 consecutive radial
// columns; lane l of every warp works on column i0 + l, so global loads of rho
// (r fastest) and shared-memory accesses are contiguous across a warp.  A real
// sequence of length N is packed as z_n = x_2n + i x_2n+1 (n < M = N/2),
// transformed by an in-place radix-2 decimation-in-time FFT of length M in
// shared memory (bit-reversed load), and unpacked into the N/2+1 half-spectrum.
// The CTA's output is the contiguous mode-layout block of cells
// (k, i0 .. i0+TI-1), staged in shared memory and stored with coalesced writes.
// Problems of a batch may differ in size and N_theta; the dynamic shared
// memory is sized for the largest.
#include "internal.h"

namespace pp {
namespace {

constexpr int TI = FFT_TI;
constexpr int LD = TI + 1;   // padded row of the transform buffer (conflict-free 16-byte lanes)

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {   // conj(a) * b
    return make_double2(fma(a.x, b.x, a.y * b.y), fma(a.x, b.y, -a.y * b.x));
}

__device__ __forceinline__ int bitrev(int n, int log2M) {
    return log2M == 0 ? 0 : (int)(__brev((unsigned)n) >> (32 - log2M));
}

__device__ __forceinline__ int find_problem(const unsigned *__restrict__ start, int n, unsigned blk) {
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (start[mid] <= blk) lo = mid;
        else hi = mid;
    }
    return lo;
}

// In-place radix-2 DIT FFT of length M on buf[M][LD] (bit-reversed input).
// INVERSE: conjugated twiddles (e^{+2 pi i t / M}).  Twiddles w = 1 (pos = 0)
// and w = -i / +i (pos = h/2) need no multiplication.
template <bool INVERSE>
__device__ __forceinline__ void fft_stages(double2 *buf, const double2 *__restrict__ tw, int M, int lane, int warp,
                                           int nw) {
    const int half = M >> 1;
    int log2h = 0;
    for (int h = 1; h < M; h <<= 1, ++log2h) {
        const int stride = half >> log2h;           // twiddle index step: M / (2h)
        for (int bi = warp; bi < half; bi += nw) {
            const int pos = bi & (h - 1);
            const int top = ((bi >> log2h) << (log2h + 1)) + pos;
            const int bot = top + h;
            const double2 zt = buf[top * LD + lane];
            const double2 zb = buf[bot * LD + lane];
            double2 t;
            if (pos == 0) {
                t = zb;
            } else if (2 * pos == h) {
                t = INVERSE ? make_double2(-zb.y, zb.x) : make_double2(zb.y, -zb.x);
            } else {
                const double2 w = tw[pos * stride];
                t = INVERSE ? cmulc(w, zb) : cmul(w, zb);
            }
            buf[top * LD + lane] = make_double2(zt.x + t.x, zt.y + t.y);
            buf[bot * LD + lane] = make_double2(zt.x - t.x, zt.y - t.y);
        }
        __syncthreads();
    }
}

__device__ __forceinline__ double block_sum(double v, double *red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0) {
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    }
    return s;
}

__global__ void __launch_bounds__(FFT_THREADS) k_forward(const FFTTab *__restrict__ tab, double *__restrict__ partials) {
    extern __shared__ double2 sm[];
    __shared__ double red[FFT_THREADS / 32];
    const int pr = find_problem(tab->start, tab->n, blockIdx.x);
    const FFTProb P = tab->p[pr];
    const int nr = P.nr, nt = P.nt, nz = P.nz;
    const int M = nt >> 1, nm = M + 1;
    double2 *buf = sm;              // [M][LD]
    double2 *outb = sm + M * LD;    // [TI][nm]

    const int tiles = (nr + TI - 1) / TI;
    const int lb = (int)(blockIdx.x - tab->start[pr]);
    const int k = lb / tiles;
    const int i0 = (lb - k * tiles) * TI;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int i = i0 + lane;
    const bool valid = i < nr;

    const double *src = P.rho + (size_t)k * nt * nr + i;
    for (int n = warp; n < M; n += nw) {
        double a = 0.0, b = 0.0;
        if (valid) {
            a = src[(size_t)(2 * n) * nr];
            b = src[(size_t)(2 * n + 1) * nr];
        }
        buf[bitrev(n, P.log2M) * LD + lane] = make_double2(a, b);
    }
    __syncthreads();
    fft_stages<false>(buf, (const double2 *)P.tw, M, lane, warp, nw);

    // Unpack: X_m = 1/2 [ (Z_m + conj Z_{M-m}) - i W^m (Z_m - conj Z_{M-m}) ], W = e^{-2 pi i / N}
    const double2 *tw2 = (const double2 *)P.tw2;
    const double scale = (P.s ? P.s[valid ? i : 0] : 1.0) * (0.5 / (double)nt);
    double acc = 0.0;
    for (int m = warp; m <= M; m += nw) {
        const double2 A = buf[(m == M ? 0 : m) * LD + lane];
        const double2 Bc = buf[(m == 0 ? 0 : M - m) * LD + lane];
        double2 x;
        if (m == 0 || m == M) {
            // Z_0 carries X_0 = Re + Im and X_M = Re - Im; both exactly real
            x = make_double2((m == 0 ? (A.x + A.y) : (A.x - A.y)) * (2.0 * scale), 0.0);
        } else {
            const double2 S = make_double2(A.x + Bc.x, A.y - Bc.y);        // Z_m + conj Z_{M-m}
            const double2 D = make_double2(A.x - Bc.x, A.y + Bc.y);        // Z_m - conj Z_{M-m}
            const double2 mid = make_double2(D.y, -D.x);                    // -i D
            const double2 t = cmul(tw2[m], mid);
            x = make_double2((S.x + t.x) * scale, (S.y + t.y) * scale);
        }
        if (m == 0 && P.bD && valid) x.x += P.bD[(size_t)k * nr + i];
        if (valid && partials) {
            const double w = (m == 0 || m == M) ? 1.0 : 2.0;
            acc += w * (x.x * x.x + x.y * x.y);
        }
        outb[lane * nm + m] = x;
    }
    __syncthreads();
    const int ncols = min(TI, nr - i0);
    double2 *dst = P.b + ((size_t)k * nr + i0) * nm;
    for (int f = threadIdx.x; f < ncols * nm; f += blockDim.x) dst[f] = outb[f];
    if (P.bh && P.invd) {
        // b_hat = b / diag for the smoother (row class of plane k, cells i0.., all modes)
        const int cls = k == 0 ? 0 : (k == nz - 1 ? P.ncls - 1 : 1);
        const double *inv = P.invd + ((size_t)cls * nr + i0) * nm;
        double2 *dh = P.bh + ((size_t)k * nr + i0) * nm;
        for (int f = threadIdx.x; f < ncols * nm; f += blockDim.x) {
            const double2 x = outb[f];
            const double v = inv[f];
            dh[f] = make_double2(x.x * v, x.y * v);
        }
    }
    if (partials) {
        const double tot = block_sum(acc, red);
        if (threadIdx.x == 0) partials[blockIdx.x] = tot;
    }
}

__global__ void __launch_bounds__(FFT_THREADS) k_inverse(const FFTTab *__restrict__ tab) {
    extern __shared__ double2 sm[];
    const int pr = find_problem(tab->start, tab->n, blockIdx.x);
    const FFTProb P = tab->p[pr];
    const int nr = P.nr, nt = P.nt;
    const int M = nt >> 1, nm = M + 1;
    double2 *buf = sm;              // [M][LD]
    double2 *inb = sm + M * LD;     // [TI][nm]

    const int tiles = (nr + TI - 1) / TI;
    const int lb = (int)(blockIdx.x - tab->start[pr]);
    const int k = lb / tiles;
    const int i0 = (lb - k * tiles) * TI;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int i = i0 + lane;
    const bool valid = i < nr;
    const int ncols = min(TI, nr - i0);

    const double2 *src = P.uhat + ((size_t)k * nr + i0) * nm;
    for (int f = threadIdx.x; f < TI * nm; f += blockDim.x)
        inb[f] = f < ncols * nm ? src[f] : make_double2(0.0, 0.0);
    __syncthreads();

    // Pack: Z_m = (X_m + conj X_{M-m}) + i w^m (X_m - conj X_{M-m}), w = e^{+2 pi i / N};
    // X_0 and X_M enter through their real parts only.
    const double2 *tw2 = (const double2 *)P.tw2;
    for (int m = warp; m < M; m += nw) {
        double2 A = inb[lane * nm + m];
        double2 B = inb[lane * nm + (M - m)];
        if (m == 0) {
            A.y = 0.0;
            B.y = 0.0;
        }
        const double2 S = make_double2(A.x + B.x, A.y - B.y);   // X_m + conj X_{M-m}
        const double2 D = make_double2(A.x - B.x, A.y + B.y);   // X_m - conj X_{M-m}
        const double2 t = cmulc(tw2[m], D);                     // w^m D
        buf[bitrev(m, P.log2M) * LD + lane] = make_double2(S.x - t.y, S.y + t.x);   // S + i t
    }
    __syncthreads();
    fft_stages<true>(buf, (const double2 *)P.tw, M, lane, warp, nw);

    if (valid) {
        double *dst = P.phi + (size_t)k * nt * nr + i;
        for (int n = warp; n < M; n += nw) {
            const double2 z = buf[n * LD + lane];
            dst[(size_t)(2 * n) * nr] = z.x;
            dst[(size_t)(2 * n + 1) * nr] = z.y;
        }
    }
}

// Mode-layout initial iterate: b = guess, each CTA copying the cells of its
// plane k and radial tile (the same block ranges as the transforms).
__global__ void __launch_bounds__(FFT_THREADS) k_copy_guess(const FFTTab *__restrict__ tab) {
    const int pr = find_problem(tab->start, tab->n, blockIdx.x);
    const FFTProb P = tab->p[pr];
    const int nm = P.nt / 2 + 1;
    const int tiles = (P.nr + TI - 1) / TI;
    const int lb = (int)(blockIdx.x - tab->start[pr]);
    const int k = lb / tiles;
    const int i0 = (lb - k * tiles) * TI;
    const int ncols = min(TI, P.nr - i0);
    const size_t off = ((size_t)k * P.nr + i0) * nm;
    for (int f = threadIdx.x; f < ncols * nm; f += blockDim.x) P.b[off + f] = P.guess[off + f];
}

}  // namespace

cudaError_t launch_copy_guess(const FFTTab *tab, unsigned grid, cudaStream_t st) {
    k_copy_guess<<<grid, FFT_THREADS, 0, st>>>(tab);
    return cudaGetLastError();
}

size_t fft_smem_bytes(int nt) {
    const int M = nt / 2, nm = M + 1;
    return (size_t)(M * LD + TI * nm) * sizeof(double2);
}

cudaError_t launch_forward(const FFTTab *tab, unsigned grid, size_t smem, double *partials, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(k_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_forward<<<grid, FFT_THREADS, smem, st>>>(tab, partials);
    return cudaGetLastError();
}

cudaError_t launch_inverse(const FFTTab *tab, unsigned grid, size_t smem, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(k_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_inverse<<<grid, FFT_THREADS, smem, st>>>(tab);
    return cudaGetLastError();
}

}  // namespace pp
