// Double-float forward azimuthal transform for the mixed-precision form: the
// same transform as k_forward in fft.cu (step a-1, Eq. azimuthal_dft with
// 1/N_theta, then Eq. mode_rhs) -- same work decomposition, packing,
// butterflies and unpacking -- with every intermediate value held as an
// unevaluated sum hi + lo of two binary32 numbers ("double-float", about 48
// significant bits) and computed on the FP32 pipe, which runs at 64 times the
// FP64 rate on this GPU.  A transform of length N in double-float arithmetic
// is accurate to a few units of 2^-46 relative to the input's norm, so b
// carries a relative error near 1e-14: the mixed form solves to 1e-10, and an
// error in b reaches the residual unamplified.  The inverse transform stays
// in binary64 (an error in phi is amplified by the operator), as does the
// plain FP64 form.
//
// Arithmetic: df.h.
//
// Range: a CTA scales its inputs by a power of two so that the largest has
// exponent 0 (integer exponent arithmetic, exact), keeping every value inside
// the binary32 range; entries below 2^-126 of the CTA's largest are dropped,
// far below its double-precision rounding.  Conversions between binary64 and
// the hi/lo pair are integer instructions plus one FP64 addition per output.
#include "df.h"
#include "internal.h"

namespace pp {
namespace {

constexpr int TI = FFT_TI;
constexpr int LD = TI + 1;   // padded row of the transform buffer

struct dfc {
    df x, y;
};
__device__ __forceinline__ float4 pack(dfc z) { return make_float4(z.x.hi, z.x.lo, z.y.hi, z.y.lo); }
__device__ __forceinline__ dfc unpack(float4 v) { return {{v.x, v.y}, {v.z, v.w}}; }

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

// Largest exponent field over the block (every thread passes its own).
__device__ __forceinline__ int block_max(int v, int *sh) {
    v = (int)__reduce_max_sync(0xffffffffu, (unsigned)v);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    int r = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = max(r, sh[w]);
    return r;
}

// v with w z = a v for the twiddle (a, b) of w; rot: the entry's rotation
// flag (tw_rot, rho = -i), as fft.cu.
__device__ __forceinline__ dfc tw_v(df b, bool rot, dfc z) {
    const df ux = df_fma(df_neg(b), z.y, z.x), uy = df_fma(b, z.x, z.y);   // u = z + i b z
    const df vx = rot ? uy : ux, vy = rot ? ux : uy;
    return {vx, df_negif(vy, rot)};
}

__device__ __forceinline__ void twiddle(const float4 *__restrict__ tw, int t, df &a, df &b) {
    const float4 v = tw[t];
    a = {v.x, v.y};
    b = {v.z, v.w};
}

__device__ __forceinline__ void bfly(dfc &top, dfc &bot, int t, int M, const float4 *__restrict__ tw) {
    df a, b;
    twiddle(tw, t, a, b);
    const dfc v = tw_v(b, tw_rot(t, M), bot);
    const dfc x = top;
    const df na = df_neg(a);
    top = {df_fma(a, v.x, x.x), df_fma(a, v.y, x.y)};
    bot = {df_fma(na, v.x, x.x), df_fma(na, v.y, x.y)};
}

__device__ __forceinline__ void add_sub(dfc &a, dfc &b) {
    const dfc x = a;
    a = {df_add(x.x, b.x), df_add(x.y, b.y)};
    b = {df_sub(x.x, b.x), df_sub(x.y, b.y)};
}

// In-place radix-2 DIT FFT of length M on buf[M][LD] (bit-reversed input),
// two stages per pass, the first pass additions only -- as fft.cu.
__device__ __forceinline__ void fft_stages(float4 *buf, const float4 *__restrict__ tw, int M, int log2M, int lane,
                                           int warp, int nw) {
    int h;
    if (log2M & 1) {
        for (int q = warp; q < (M >> 1); q += nw) {
            dfc a = unpack(buf[(2 * q) * LD + lane]), b = unpack(buf[(2 * q + 1) * LD + lane]);
            add_sub(a, b);
            buf[(2 * q) * LD + lane] = pack(a);
            buf[(2 * q + 1) * LD + lane] = pack(b);
        }
        h = 2;
    } else {
        for (int q = warp; q < (M >> 2); q += nw) {
            float4 *x = buf + 4 * q * LD + lane;
            dfc a0 = unpack(x[0]), a1 = unpack(x[LD]), a2 = unpack(x[2 * LD]), a3 = unpack(x[3 * LD]);
            add_sub(a0, a1);
            add_sub(a2, a3);
            add_sub(a0, a2);
            a3 = dfc{a3.y, df_neg(a3.x)};   // w = -i
            add_sub(a1, a3);
            x[0] = pack(a0);
            x[LD] = pack(a1);
            x[2 * LD] = pack(a2);
            x[3 * LD] = pack(a3);
        }
        h = 4;
    }
    __syncthreads();
    for (; 4 * h <= M; h <<= 2) {
        for (int q = warp; q < (M >> 2); q += nw) {
            const int p = q & (h - 1);
            const int g = (q - p) << 2;
            float4 *x = buf + (g + p) * LD + lane;
            dfc a0 = unpack(x[0]), a1 = unpack(x[h * LD]), a2 = unpack(x[2 * h * LD]), a3 = unpack(x[3 * h * LD]);
            const int t1 = p * (M / (2 * h));
            bfly(a0, a1, t1, M, tw);
            bfly(a2, a3, t1, M, tw);
            const int t2 = p * (M / (4 * h));
            bfly(a0, a2, t2, M, tw);
            bfly(a1, a3, t2 + (M >> 2), M, tw);
            x[0] = pack(a0);
            x[h * LD] = pack(a1);
            x[2 * h * LD] = pack(a2);
            x[3 * h * LD] = pack(a3);
        }
        __syncthreads();
    }
}

__device__ __forceinline__ double block_sum(double v, double *sh) {
    __syncthreads();
    sh[threadIdx.x] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x < 32) {
        for (int j = threadIdx.x; j < (int)blockDim.x; j += 32) s += sh[j];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    return s;
}

__global__ void __launch_bounds__(FFT_THREADS) k_forward_df(const FFTTab *__restrict__ tab,
                                                             double *__restrict__ partials) {
    extern __shared__ double2 sm[];
    __shared__ double red[FFT_THREADS];
    __shared__ int emx[FFT_THREADS / 32];
    const int pr = find_problem(tab->start, tab->n, blockIdx.x);
    const FFTProb P = tab->p[pr];
    const int nr = P.nr, nt = P.nt;
    const int M = nt >> 1, nm = M + 1;
    float4 *buf = reinterpret_cast<float4 *>(sm);   // [M][LD]
    double2 *outb = sm + M * LD;                    // [TI][nm]

    const int tiles = (nr + TI - 1) / TI;
    const int lb = (int)(blockIdx.x - tab->start[pr]);
    const int k = lb / tiles;
    const int i0 = (lb - k * tiles) * TI;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int i = i0 + lane;
    const bool valid = i < nr;

    // rho read once, as binary64 pairs into the transform buffer (a float4
    // slot holds a double2); the CTA's scale makes its largest input's
    // exponent 0; then each thread splits its own entries in place
    const double *src = P.rho + (size_t)k * nt * nr + i;
    double2 *raw = reinterpret_cast<double2 *>(buf);
    int em = 0;
    for (int n = warp; n < M; n += nw) {
        double a = 0.0, b = 0.0;
        if (valid) {
            a = src[(size_t)(2 * n) * nr];
            b = src[(size_t)(2 * n + 1) * nr];
        }
        em = max(em, max(exp_field(a), exp_field(b)));
        raw[bitrev(n, P.log2M) * LD + lane] = make_double2(a, b);
    }
    const int emax = max(block_max(em, emx), 1);
    const int sc = emax - 1023;   // values carry the factor 2^-sc
    for (int n = warp; n < M; n += nw) {
        const int e = bitrev(n, P.log2M) * LD + lane;
        const double2 v = raw[e];
        buf[e] = pack({split_scaled(v.x, emax), split_scaled(v.y, emax)});
    }
    __syncthreads();
    fft_stages(buf, P.twf, M, P.log2M, lane, warp, nw);

    // unpack, modes m and M - m together (as fft.cu), hs = s_i / (2N)
    // s_i, or per cell in a composite domain (zero outside its patches)
    const size_t si = valid ? (P.s_rows ? (size_t)k * nr + i : (size_t)i) : 0;
    const double hsd = (P.s ? P.s[si] : 1.0) * P.half_inv_n;
    const df hs = split_scaled(hsd, exp_field(hsd));      // hs 2^-(e - 1023): exact scaling below
    const int shs = exp_field(hsd) - 1023;
    const df two_hs = {2.f * hs.hi, 2.f * hs.lo};
    float acc_in = 0.f, acc_edge = 0.f;   // Parseval weight 2 and 1, scaled, from the high parts
    double2 *ob = outb + lane * nm;
    for (int m = 1 + warp; 2 * m < M; m += nw) {
        const dfc A = unpack(buf[m * LD + lane]), B = unpack(buf[(M - m) * LD + lane]);
        const dfc S = {df_mul(hs, df_add(A.x, B.x)), df_mul(hs, df_sub(A.y, B.y))};
        const dfc D = {df_sub(A.x, B.x), df_add(A.y, B.y)};
        df a, b;
        twiddle(P.tw2f, m, a, b);
        const dfc v = tw_v(b, tw_rot(m, nt), D);   // T = a v
        const df g = df_mul(hs, a);
        const dfc xm = {df_fma(g, v.y, S.x), df_fma(df_neg(g), v.x, S.y)};
        const dfc xp = {df_fma(df_neg(g), v.y, S.x), df_neg(df_fma(g, v.x, S.y))};
        ob[m] = make_double2(to_double(xm.x, sc + shs), to_double(xm.y, sc + shs));
        ob[M - m] = make_double2(to_double(xp.x, sc + shs), to_double(xp.y, sc + shs));
        acc_in = fmaf(xm.x.hi, xm.x.hi, fmaf(xm.y.hi, xm.y.hi, acc_in));
        acc_in = fmaf(xp.x.hi, xp.x.hi, fmaf(xp.y.hi, xp.y.hi, acc_in));
    }
    double edge_extra = 0.0;   // ||b||^2 share of the Dirichlet-shifted mode 0, in binary64
    if (warp == 0) {
        const dfc z = unpack(buf[lane]);
        double x0 = to_double(df_mul(two_hs, df_add(z.x, z.y)), sc + shs);
        const df xM = df_mul(two_hs, df_sub(z.x, z.y));
        if (P.bD && valid) x0 += P.bD[(size_t)k * nr + i];
        edge_extra = x0 * x0;
        acc_edge = fmaf(xM.hi, xM.hi, acc_edge);
        ob[0] = make_double2(x0, 0.0);
        ob[M] = make_double2(to_double(xM, sc + shs), 0.0);
    }
    if (M >= 2 && warp == nw - 1) {   // m = M/2 pairs with itself: X = 2 hs conj Z
        const dfc z = unpack(buf[(M >> 1) * LD + lane]);
        const dfc x = {df_mul(two_hs, z.x), df_neg(df_mul(two_hs, z.y))};
        ob[M >> 1] = make_double2(to_double(x.x, sc + shs), to_double(x.y, sc + shs));
        acc_in = fmaf(x.x.hi, x.x.hi, fmaf(x.y.hi, x.y.hi, acc_in));
    }
    __syncthreads();
    const int ncols = min(TI, nr - i0);
    double2 *dst = P.b + ((size_t)k * nr + i0) * nm;
    for (int f = threadIdx.x; f < ncols * nm; f += blockDim.x) dst[f] = outb[f];
    if (partials) {
        // the scaled squares times 2^(2 (sc + shs)), exactly
        const double sq = f32_times_pow2(fmaf(2.f, acc_in, acc_edge), 2 * (sc + shs));
        const double tot = block_sum(valid ? sq + edge_extra : 0.0, red);
        if (threadIdx.x == 0) partials[blockIdx.x] = tot;
    }
}

}  // namespace

cudaError_t launch_forward_df(const FFTTab *tab, unsigned grid, size_t smem, double *partials, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(k_forward_df, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_forward_df<<<grid, FFT_THREADS, smem, st>>>(tab, partials);
    return cudaGetLastError();
}

}  // namespace pp
