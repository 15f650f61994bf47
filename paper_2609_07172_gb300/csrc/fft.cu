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
//
// FP64 runs at 1/64 of the FP32 rate on this GPU, so the transforms are bound
// by FP64 instructions and are written to issue few of them:
//  * a butterfly top +- w bot with w = rho a (1 + i b) (see tw_rot) costs six
//    multiply-adds: u = bot + i b bot (two), top +- a rho u (four) -- instead
//    of a four-operation complex product and four additions; rho is applied
//    with integer instructions, so no FP64 instruction depends on a branch;
//  * the first stages, whose twiddles are 1 and -i (+i inverse), are
//    additions only;
//  * each thread applies two consecutive radix-2 stages to four values held
//    in registers, halving the shared-memory round trips and barriers;
//  * the unpack (pack) of the real transform treats modes m and M - m
//    together, sharing one twiddle product.
#include "internal.h"

namespace pp {
namespace {

constexpr int TI = FFT_TI;
constexpr int LD = TI + 1;   // padded row of the transform buffer (conflict-free 16-byte lanes)

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

// -x when c (sign bit flipped with an integer instruction).
__device__ __forceinline__ double flip_if(double x, bool c) {
    return __hiloint2double(__double2hiint(x) ^ (c ? (int)0x80000000 : 0), __double2loint(x));
}

// v with w z = a v for the twiddle entry ab = (a, b) of w (INVERSE: of
// conj w); rot: the entry's rotation flag (tw_rot).
template <bool INVERSE>
__device__ __forceinline__ double2 tw_v(double2 ab, bool rot, double2 z) {
    const double b = INVERSE ? -ab.y : ab.y;
    const double ux = fma(-b, z.y, z.x), uy = fma(b, z.x, z.y);   // u = z + i b z
    // rho u with rho = -i (forward) or +i (inverse) when rot, 1 otherwise
    const double vx = rot ? uy : ux, vy = rot ? ux : uy;
    return make_double2(flip_if(vx, rot && INVERSE), flip_if(vy, rot && !INVERSE));
}

// Radix-2 butterfly (top, bot) <- (top + w bot, top - w bot), w = e^{-+2 pi i t / M}.
template <bool INVERSE>
__device__ __forceinline__ void bfly(double2 &top, double2 &bot, int t, int M, const double2 *__restrict__ tw) {
    const double2 ab = tw[t];
    const double2 v = tw_v<INVERSE>(ab, tw_rot(t, M), bot);
    const double2 x = top;
    top = make_double2(fma(ab.x, v.x, x.x), fma(ab.x, v.y, x.y));
    bot = make_double2(fma(-ab.x, v.x, x.x), fma(-ab.x, v.y, x.y));
}

__device__ __forceinline__ void add_sub(double2 &a, double2 &b) {
    const double2 x = a;
    a = make_double2(x.x + b.x, x.y + b.y);
    b = make_double2(x.x - b.x, x.y - b.y);
}

// In-place radix-2 DIT FFT of length M on buf[M][LD] (bit-reversed input),
// two stages (h, 2h) per pass on four values per thread.  The first pass
// (or the first single stage when log2 M is odd) has twiddles 1 and -i only
// and is done with additions.  INVERSE: conjugated twiddles.
template <bool INVERSE>
__device__ __forceinline__ void fft_stages(double2 *buf, const double2 *__restrict__ tw, int M, int log2M, int lane,
                                           int warp, int nw) {
    int h;
    if (log2M & 1) {   // single stage h = 1
        for (int q = warp; q < (M >> 1); q += nw) {
            double2 a = buf[(2 * q) * LD + lane], b = buf[(2 * q + 1) * LD + lane];
            add_sub(a, b);
            buf[(2 * q) * LD + lane] = a;
            buf[(2 * q + 1) * LD + lane] = b;
        }
        h = 2;
    } else {           // stages 1 and 2: four-point DFTs
        for (int q = warp; q < (M >> 2); q += nw) {
            double2 *x = buf + 4 * q * LD + lane;
            double2 a0 = x[0], a1 = x[LD], a2 = x[2 * LD], a3 = x[3 * LD];
            add_sub(a0, a1);
            add_sub(a2, a3);
            add_sub(a0, a2);
            a3 = INVERSE ? make_double2(-a3.y, a3.x) : make_double2(a3.y, -a3.x);   // w = -i (+i)
            add_sub(a1, a3);
            x[0] = a0;
            x[LD] = a1;
            x[2 * LD] = a2;
            x[3 * LD] = a3;
        }
        h = 4;
    }
    __syncthreads();
    for (; 4 * h <= M; h <<= 2) {
        for (int q = warp; q < (M >> 2); q += nw) {
            const int p = q & (h - 1);
            const int g = (q - p) << 2;   // (q / h) * 4h
            double2 *x = buf + (g + p) * LD + lane;
            double2 a0 = x[0], a1 = x[h * LD], a2 = x[2 * h * LD], a3 = x[3 * h * LD];
            const int t1 = p * (M / (2 * h));          // W_{2h}^p
            bfly<INVERSE>(a0, a1, t1, M, tw);
            bfly<INVERSE>(a2, a3, t1, M, tw);
            const int t2 = p * (M / (4 * h));          // W_{4h}^p and W_{4h}^{p+h}
            bfly<INVERSE>(a0, a2, t2, M, tw);
            bfly<INVERSE>(a1, a3, t2 + (M >> 2), M, tw);
            x[0] = a0;
            x[h * LD] = a1;
            x[2 * h * LD] = a2;
            x[3 * h * LD] = a3;
        }
        __syncthreads();
    }
}

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

__global__ void __launch_bounds__(FFT_THREADS) k_forward(const FFTTab *__restrict__ tab, double *__restrict__ partials) {
    extern __shared__ double2 sm[];
    __shared__ double red[FFT_THREADS];
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
    fft_stages<false>(buf, (const double2 *)P.tw, M, P.log2M, lane, warp, nw);

    // Unpack, modes m and M - m together (W = e^{-2 pi i / N}, hs = s_i / (2N)):
    //   S = Z_m + conj Z_{M-m},  D = Z_m - conj Z_{M-m},  T = W^m D,
    //   X_m = hs (S - i T),  X_{M-m} = hs conj(S + i T);
    // X_0 = 2 hs (Re Z_0 + Im Z_0), X_M = 2 hs (Re Z_0 - Im Z_0), both exactly real.
    const double2 *tw2 = (const double2 *)P.tw2;
    // s_i, or per cell in a composite domain (zero outside its patches)
    const size_t si = valid ? (P.s_rows ? (size_t)k * nr + i : (size_t)i) : 0;
    const double hs = (P.s ? P.s[si] : 1.0) * P.half_inv_n;
    double acc_in = 0.0, acc_edge = 0.0;   // Parseval weight 2 (0 < m < M) and 1 (m = 0, M)
    double2 *ob = outb + lane * nm;
    for (int m = 1 + warp; 2 * m < M; m += nw) {
        const double2 A = buf[m * LD + lane], B = buf[(M - m) * LD + lane];
        const double2 S = make_double2(hs * (A.x + B.x), hs * (A.y - B.y));
        const double2 D = make_double2(A.x - B.x, A.y + B.y);
        const double2 ab = tw2[m];
        const double2 v = tw_v<false>(ab, tw_rot(m, nt), D);   // T = ab.x v
        const double g = hs * ab.x;
        const double2 xm = make_double2(fma(g, v.y, S.x), fma(-g, v.x, S.y));
        const double2 xp = make_double2(fma(-g, v.y, S.x), -fma(g, v.x, S.y));
        ob[m] = xm;
        ob[M - m] = xp;
        acc_in = fma(xm.x, xm.x, fma(xm.y, xm.y, acc_in));
        acc_in = fma(xp.x, xp.x, fma(xp.y, xp.y, acc_in));
    }
    if (warp == 0) {
        const double2 z = buf[lane];
        double x0 = (z.x + z.y) * (2.0 * hs);
        const double xM = (z.x - z.y) * (2.0 * hs);
        if (P.bD && valid) x0 += P.bD[(size_t)k * nr + i];
        acc_edge = fma(x0, x0, fma(xM, xM, acc_edge));
        ob[0] = make_double2(x0, 0.0);
        ob[M] = make_double2(xM, 0.0);
    }
    if (M >= 2 && warp == nw - 1) {   // m = M/2 pairs with itself: X = 2 hs conj Z
        const double2 z = buf[(M >> 1) * LD + lane];
        const double2 x = make_double2((2.0 * hs) * z.x, -(2.0 * hs) * z.y);
        ob[M >> 1] = x;
        acc_in = fma(x.x, x.x, fma(x.y, x.y, acc_in));
    }
    __syncthreads();
    const int ncols = min(TI, nr - i0);
    double2 *dst = P.b + ((size_t)k * nr + i0) * nm;
    for (int f = threadIdx.x; f < ncols * nm; f += blockDim.x) dst[f] = outb[f];
    if (P.bh && P.invd) {
        // b_hat = b / diag for the smoother (row class of plane k, cells i0.., all modes)
        const int cls = P.rcls ? P.rcls[k] : (k == 0 ? 0 : (k == nz - 1 ? P.ncls - 1 : 1));
        const double *inv = P.invd + ((size_t)cls * nr + i0) * nm;
        double2 *dh = P.bh + ((size_t)k * nr + i0) * nm;
        for (int f = threadIdx.x; f < ncols * nm; f += blockDim.x) {
            const double2 x = outb[f];
            const double v = inv[f];
            dh[f] = make_double2(x.x * v, x.y * v);
        }
    }
    if (partials) {
        const double tot = block_sum(valid ? fma(2.0, acc_in, acc_edge) : 0.0, red);
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

    // Pack, modes m and M - m together (w = e^{+2 pi i / N}):
    //   S = X_m + conj X_{M-m},  D = X_m - conj X_{M-m},  T = w^m D,
    //   Z_m = S + i T,  Z_{M-m} = conj(S - i T);
    // X_0 and X_M enter through their real parts only: Z_0 = (X_0 + X_M) + i (X_0 - X_M).
    const double2 *tw2 = (const double2 *)P.tw2;
    const double2 *ib = inb + lane * nm;
    for (int m = 1 + warp; 2 * m < M; m += nw) {
        const double2 A = ib[m], B = ib[M - m];
        const double2 S = make_double2(A.x + B.x, A.y - B.y);
        const double2 D = make_double2(A.x - B.x, A.y + B.y);
        const double2 ab = tw2[m];
        const double2 v = tw_v<true>(ab, tw_rot(m, nt), D);   // T = ab.x v
        buf[bitrev(m, P.log2M) * LD + lane] = make_double2(fma(-ab.x, v.y, S.x), fma(ab.x, v.x, S.y));
        buf[bitrev(M - m, P.log2M) * LD + lane] = make_double2(fma(ab.x, v.y, S.x), fma(ab.x, v.x, -S.y));
    }
    if (warp == 0) {
        const double a = ib[0].x, b = ib[M].x;
        buf[lane] = make_double2(a + b, a - b);
    }
    if (M >= 2 && warp == nw - 1) {   // m = M/2 pairs with itself: Z = 2 conj X
        const double2 x = ib[M >> 1];
        buf[bitrev(M >> 1, P.log2M) * LD + lane] = make_double2(x.x + x.x, -(x.y + x.y));
    }
    __syncthreads();
    fft_stages<true>(buf, (const double2 *)P.tw, M, P.log2M, lane, warp, nw);

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
