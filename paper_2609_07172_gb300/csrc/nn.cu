// Kernels of the learned warm start: a small U-Net that maps a mode residual
// to an approximate correction (its convolutions on BF16 tensor cores with
// FP32 accumulation), its training (weight gradients, loss, Adam), and the
// FP64 glue between the solver's mode layout and the network's tensors.
//
// Network tensors are NHWC BF16 with n = azimuthal mode (sample), y = axial
// cell k, x = radial cell i, channels contiguous.  Channel counts are
// multiples of 16 on inputs (one mma K-chunk) and of 8 on outputs (one mma
// N-tile).
#include <cuda_bf16.h>

#include "internal.h"
#include "pic_poisson_nn.h"

namespace pp {
namespace {

typedef __nv_bfloat16 bf16;

__device__ __forceinline__ unsigned ld32(const bf16 *p) { return *reinterpret_cast<const unsigned *>(p); }

__device__ __forceinline__ void mma_bf16(float (&d)[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3,
                                         unsigned b0, unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ unsigned pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<unsigned *>(&v);
}

constexpr int CONV_WARPS = 4;   // 16 output pixels per warp, 64 per CTA

// 3x3 convolution, stride 1, zero padding, as an implicit GEMM on mma.sync
// m16n8k16 (BF16 in, FP32 accumulate): rows = output pixels, columns = output
// channels, reduction = (tap, input channel).  Each warp owns 16 pixels and
// all NT*8 output channels; A fragments are gathered straight from the NHWC
// input (zero outside the image), B fragments from weights laid out
// [tap][cout][cin] so that both are 32-bit loads of channel pairs.
template <int NT>
__global__ void __launch_bounds__(CONV_WARPS * 32)
k_conv3x3(const bf16 *__restrict__ in, int cin, const bf16 *__restrict__ w, const float *__restrict__ bias,
          bf16 *__restrict__ out, float *__restrict__ out32, int n, int h, int wd, int relu) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, tig = lane & 3;
    const long P = (long)n * h * wd;
    const long p0 = ((long)blockIdx.x * CONV_WARPS + warp) * 16;
    if (p0 >= P) return;
    const int cout = NT * 8;
    long pr[2];
    int yy[2], xx[2];
    const bf16 *base[2];
    bool pv[2];
    for (int r = 0; r < 2; ++r) {
        pr[r] = p0 + g + 8 * r;
        pv[r] = pr[r] < P;
        const long q = pv[r] ? pr[r] : 0;
        xx[r] = (int)(q % wd);
        const long t = q / wd;
        yy[r] = (int)(t % h);
        base[r] = in + (t / h) * (long)h * wd * cin;
    }
    float acc[NT][4];
#pragma unroll
    for (int j = 0; j < NT; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
    for (int tap = 0; tap < 9; ++tap) {
        const int dy = tap / 3 - 1, dx = tap % 3 - 1;
        const bf16 *src[2];
        bool ok[2];
        for (int r = 0; r < 2; ++r) {
            const int sy = yy[r] + dy, sx = xx[r] + dx;
            ok[r] = pv[r] && sy >= 0 && sy < h && sx >= 0 && sx < wd;
            src[r] = base[r] + ((long)sy * wd + sx) * cin;
        }
        const bf16 *wt = w + (long)tap * cout * cin;
        for (int c = 0; c < cin; c += 16) {
            const int ca = c + 2 * tig;
            const unsigned a0 = ok[0] ? ld32(src[0] + ca) : 0u;
            const unsigned a1 = ok[1] ? ld32(src[1] + ca) : 0u;
            const unsigned a2 = ok[0] ? ld32(src[0] + ca + 8) : 0u;
            const unsigned a3 = ok[1] ? ld32(src[1] + ca + 8) : 0u;
#pragma unroll
            for (int j = 0; j < NT; ++j) {
                const bf16 *wp = wt + (long)(j * 8 + g) * cin + ca;
                mma_bf16(acc[j], a0, a1, a2, a3, ld32(wp), ld32(wp + 8));
            }
        }
    }
#pragma unroll
    for (int j = 0; j < NT; ++j) {
        const int co = j * 8 + 2 * tig;
        const float b0 = bias ? bias[co] : 0.f, b1 = bias ? bias[co + 1] : 0.f;
        for (int r = 0; r < 2; ++r) {
            if (!pv[r]) continue;
            float v0 = acc[j][2 * r] + b0, v1 = acc[j][2 * r + 1] + b1;
            if (relu) {
                v0 = fmaxf(v0, 0.f);
                v1 = fmaxf(v1, 0.f);
            }
            if (out) *reinterpret_cast<unsigned *>(out + pr[r] * cout + co) = pack_bf16(v0, v1);
            if (out32) *reinterpret_cast<float2 *>(out32 + pr[r] * cout + co) = make_float2(v0, v1);
        }
    }
}

// wt[8 - tap][ci][co] = w[tap][co][ci]: the weights of the data-gradient
// convolution (flipped taps, swapped channel roles).
__global__ void k_flip(const bf16 *__restrict__ w, bf16 *__restrict__ wt, int cout, int cin) {
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long total = 9L * cout * cin;
    if (e >= total) return;
    const int ci = (int)(e % cin);
    const long t = e / cin;
    const int co = (int)(t % cout);
    const int tap = (int)(t / cout);
    wt[((long)(8 - tap) * cin + ci) * cout + co] = w[e];
}

constexpr int WG_CHUNK = 2048;   // pixels per weight-gradient partial

// Weight and bias gradients of a 3x3 convolution, first stage: every thread
// owns one (cout, cin) pair and sums dout[p][co] * in[p shifted][ci] over the
// 9 taps for the pixels of one chunk, in FP32; partials[chunk][tap][co][ci].
__global__ void __launch_bounds__(256)
k_wgrad_partial(const bf16 *__restrict__ in, int cin, const bf16 *__restrict__ dout, int cout, int n, int h, int wd,
                float *__restrict__ part, float *__restrict__ partb) {
    const int pair = blockIdx.y * blockDim.x + threadIdx.x;
    const long P = (long)n * h * wd;
    const long c0 = (long)blockIdx.x * WG_CHUNK, c1 = min(P, c0 + WG_CHUNK);
    if (pair >= cout * cin) return;
    const int co = pair / cin, ci = pair - co * cin;
    float acc[9];
#pragma unroll
    for (int t = 0; t < 9; ++t) acc[t] = 0.f;
    float accb = 0.f;
    for (long p = c0; p < c1; ++p) {
        const float go = __bfloat162float(dout[p * cout + co]);
        if (ci == 0) accb += go;
        if (go == 0.f) continue;
        const int x = (int)(p % wd);
        const long t = p / wd;
        const int y = (int)(t % h);
        const bf16 *img = in + (t / h) * (long)h * wd * cin;
#pragma unroll
        for (int tap = 0; tap < 9; ++tap) {
            const int sy = y + tap / 3 - 1, sx = x + tap % 3 - 1;
            if (sy >= 0 && sy < h && sx >= 0 && sx < wd)
                acc[tap] = fmaf(go, __bfloat162float(img[((long)sy * wd + sx) * cin + ci]), acc[tap]);
        }
    }
    float *dst = part + (long)blockIdx.x * 9 * cout * cin;
#pragma unroll
    for (int t = 0; t < 9; ++t) dst[((long)t * cout + co) * cin + ci] = acc[t];
    if (ci == 0) partb[(long)blockIdx.x * cout + co] = accb;
}

// Second stage: sum the chunk partials in chunk order.
__global__ void k_wgrad_reduce(const float *__restrict__ part, const float *__restrict__ partb, int chunks, int cout,
                               int cin, float *__restrict__ dw, float *__restrict__ db) {
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long nw = 9L * cout * cin;
    if (e < nw) {
        float s = 0.f;
        for (int c = 0; c < chunks; ++c) s += part[(long)c * nw + e];
        dw[e] = s;
    }
    if (db && e < cout) {
        float s = 0.f;
        for (int c = 0; c < chunks; ++c) s += partb[(long)c * cout + e];
        db[e] = s;
    }
}

__global__ void k_relu_bwd(const bf16 *__restrict__ y, bf16 *__restrict__ dy, long count) {
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < count && !(__bfloat162float(y[e]) > 0.f)) dy[e] = __float2bfloat16(0.f);
}

// 2x2 average pooling (NHWC) and its adjoint.
__global__ void k_pool(const bf16 *__restrict__ in, bf16 *__restrict__ out, int n, int h, int wd, int c) {
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const int h2 = h / 2, w2 = wd / 2;
    const long total = (long)n * h2 * w2 * c;
    if (e >= total) return;
    const int ch = (int)(e % c);
    long t = e / c;
    const int x = (int)(t % w2);
    t /= w2;
    const int y = (int)(t % h2);
    const long b = t / h2;
    const bf16 *s = in + ((b * h + 2 * y) * wd + 2 * x) * c + ch;
    const float v = __bfloat162float(s[0]) + __bfloat162float(s[c]) + __bfloat162float(s[(long)wd * c]) +
                    __bfloat162float(s[(long)wd * c + c]);
    out[e] = __float2bfloat16(0.25f * v);
}

__global__ void k_pool_bwd(const bf16 *__restrict__ dout, bf16 *__restrict__ din, int n, int h, int wd, int c) {
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long total = (long)n * h * wd * c;
    if (e >= total) return;
    const int ch = (int)(e % c);
    long t = e / c;
    const int x = (int)(t % wd);
    t /= wd;
    const int y = (int)(t % h);
    const long b = t / h;
    din[e] = __float2bfloat16(0.25f * __bfloat162float(dout[((b * (h / 2) + y / 2) * (wd / 2) + x / 2) * c + ch]));
}

// Nearest-neighbour 2x upsampling of `in` (h x w, c channels) into channels
// [0, c) of `out` (2h x 2w, cstride channels), and the adjoint (sum of the
// 2x2 block) back from those channels.
__global__ void k_up(const bf16 *__restrict__ in, bf16 *__restrict__ out, int n, int h, int wd, int c, int cstride) {
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long total = (long)n * 4 * h * wd * c;
    if (e >= total) return;
    const int ch = (int)(e % c);
    long t = e / c;
    const int x = (int)(t % (2 * wd));
    t /= 2 * wd;
    const int y = (int)(t % (2 * h));
    const long b = t / (2 * h);
    out[((b * 2 * h + y) * 2 * wd + x) * cstride + ch] = in[((b * h + y / 2) * wd + x / 2) * c + ch];
}

__global__ void k_up_bwd(const bf16 *__restrict__ dout, int cstride, bf16 *__restrict__ din, int n, int h, int wd,
                         int c) {
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long total = (long)n * h * wd * c;
    if (e >= total) return;
    const int ch = (int)(e % c);
    long t = e / c;
    const int x = (int)(t % wd);
    t /= wd;
    const int y = (int)(t % h);
    const long b = t / h;
    const bf16 *s = dout + ((b * 2 * h + 2 * y) * 2 * wd + 2 * x) * cstride + ch;
    const long rs = 2L * wd * cstride;
    din[e] = __float2bfloat16(__bfloat162float(s[0]) + __bfloat162float(s[cstride]) + __bfloat162float(s[rs]) +
                              __bfloat162float(s[rs + cstride]));
}

// Copy c channels between NHWC tensors with different channel strides and offsets.
__global__ void k_copy_ch(const bf16 *__restrict__ src, int sstride, int soff, bf16 *__restrict__ dst, int dstride,
                          int doff, long pixels, int c) {
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= pixels * c) return;
    const long p = e / c;
    const int ch = (int)(e - p * c);
    dst[p * dstride + doff + ch] = src[p * sstride + soff + ch];
}

// Mean-squared error over the first `used` of `c` channels; gradient (BF16,
// channel layout of the prediction, zero on unused channels) and per-block
// loss partials.
__global__ void __launch_bounds__(256) k_mse(const float *__restrict__ pred, const float *__restrict__ target,
                                             long pixels, int c, int used, bf16 *__restrict__ dpred,
                                             float *__restrict__ part) {
    __shared__ float red[8];
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    float l = 0.f;
    if (e < pixels * c) {
        const long p = e / c;
        const int ch = (int)(e - p * c);
        float g = 0.f;
        if (ch < used) {
            const float d = pred[e] - target[p * used + ch];
            l = d * d;
            g = 2.f * d / (float)(pixels * used);
        }
        dpred[e] = __float2bfloat16(g);
    }
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = l;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.f;
        for (int w = 0; w < 8; ++w) s += red[w];
        part[blockIdx.x] = s;
    }
}

__global__ void k_sum_f(const float *__restrict__ part, int nb, long count, float *__restrict__ out) {
    __shared__ float red[32];
    float s = 0.f;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) s += part[b];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        *out = t / (float)count;
    }
}

// Adam on FP32 master weights; writes the BF16 copy the convolutions read.
__global__ void k_adam(float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m, float *__restrict__ v,
                       long count, float lr, float b1, float b2, float eps, float c1, float c2, bf16 *__restrict__ wb) {
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= count) return;
    const float gi = g[e];
    const float mi = b1 * m[e] + (1.f - b1) * gi;
    const float vi = b2 * v[e] + (1.f - b2) * gi * gi;
    m[e] = mi;
    v[e] = vi;
    const float wi = w[e] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[e] = wi;
    if (wb) wb[e] = __float2bfloat16(wi);
}

__global__ void k_add(bf16 *__restrict__ a, const bf16 *__restrict__ b, long count) {
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < count) a[e] = __float2bfloat16(__bfloat162float(a[e]) + __bfloat162float(b[e]));
}

__global__ void k_f32_to_bf16(const float *__restrict__ a, bf16 *__restrict__ b, long count) {
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < count) b[e] = __float2bfloat16(a[e]);
}

// Per-mode RMS of a complex FP64 mode-layout field over its cells, and the
// packed network input: channel 0/1 = Re/Im of the field / rms, channel 2 =
// the mode's shift ratio lambda_m mu / diag per cell, channels 3..15 = 0.
__global__ void k_mode_ss(const double2 *__restrict__ x, long cells, int nm, double *__restrict__ part) {
    // block (m-chunk of 32 modes, cell chunk); lane = mode within chunk
    const int m = blockIdx.y * 32 + (threadIdx.x & 31);
    const int row = threadIdx.x >> 5, rows = blockDim.x >> 5;
    __shared__ double red[32][33];
    double s = 0.0;
    if (m < nm) {
        for (long q = (long)blockIdx.x * rows + row; q < cells; q += (long)gridDim.x * rows) {
            const double2 v = x[q * nm + m];
            s += v.x * v.x + v.y * v.y;
        }
    }
    red[row][threadIdx.x & 31] = s;
    __syncthreads();
    if (row == 0) {
        double t = 0.0;
        for (int r = 0; r < rows; ++r) t += red[r][threadIdx.x & 31];
        if (m < nm) part[(long)blockIdx.x * nm + m] = t;
    }
}

__global__ void k_mode_rms(const double *__restrict__ part, int chunks, int nm, long cells, float *__restrict__ rms) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= nm) return;
    double s = 0.0;
    for (int c = 0; c < chunks; ++c) s += part[(long)c * nm + m];
    const double r = sqrt(s / (double)cells);
    rms[m] = r > 0.0 ? (float)r : 1.f;
}

__global__ void k_pack(const double2 *__restrict__ x, const float *__restrict__ rms, const float *__restrict__ shift,
                       int nr, int nz, int nm, bf16 *__restrict__ out) {
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;   // over (m, k, i)
    const long total = (long)nm * nz * nr;
    if (e >= total) return;
    const int i = (int)(e % nr);
    long t = e / nr;
    const int k = (int)(t % nz);
    const int m = (int)(t / nz);
    const double2 v = x[((long)k * nr + i) * nm + m];
    const float inv = 1.f / rms[m];
    bf16 *o = out + e * 16;
    uint4 z = make_uint4(0u, 0u, 0u, 0u);
    uint4 a = z;
    a.x = pack_bf16((float)v.x * inv, (float)v.y * inv);
    a.y = pack_bf16(shift ? shift[((long)k * nr + i) * nm + m] : 0.f, 0.f);
    reinterpret_cast<uint4 *>(o)[0] = a;
    reinterpret_cast<uint4 *>(o)[1] = z;
}

// Training target from a complex FP64 mode-layout field (the correction
// of a step): FP32 [nm, nz, nr, 2] = x / (rms_m / sqrt 2), rms_m the RMS of
// |x| over the mode's cells -- each real component at unit RMS.
__global__ void k_pack_target(const double2 *__restrict__ x, const float *__restrict__ rms, int nr, int nz, int nm,
                              float *__restrict__ out) {
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;   // over (m, k, i)
    const long total = (long)nm * nz * nr;
    if (e >= total) return;
    const int i = (int)(e % nr);
    const long t = e / nr;
    const int k = (int)(t % nz);
    const int m = (int)(t / nz);
    const double2 v = x[((long)k * nr + i) * nm + m];
    const double inv = 1.4142135623730951 / (double)rms[m];
    reinterpret_cast<float2 *>(out)[e] = make_float2((float)(v.x * inv), (float)(v.y * inv));
}

// A training batch: samples idx[b] of X (BF16 [n][pix][16]) and Y (FP32
// [n][pix][2]) copied into xb, yb, channels 0-1 of x and both of y multiplied
// by sign[b] (+1 or -1: the correction is odd in the residual).
__global__ void k_gather_batch(const bf16 *__restrict__ X, const float *__restrict__ Y, const long *__restrict__ idx,
                               const float *__restrict__ sign, int batch, long pix, bf16 *__restrict__ xb,
                               float *__restrict__ yb) {
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;   // over (b, pixel)
    if (e >= (long)batch * pix) return;
    const int b = (int)(e / pix);
    const long q = e - (long)b * pix;
    const long src = idx[b] * pix + q;
    const float sg = sign[b];
    const uint4 *xs = reinterpret_cast<const uint4 *>(X + src * 16);
    uint4 *xd = reinterpret_cast<uint4 *>(xb + e * 16);
    uint4 a = xs[0];
    __nv_bfloat162 c01 = *reinterpret_cast<__nv_bfloat162 *>(&a.x);
    const float2 f = __bfloat1622float2(c01);
    a.x = pack_bf16(f.x * sg, f.y * sg);   // exact: a sign change
    xd[0] = a;
    xd[1] = xs[1];
    const float2 y = reinterpret_cast<const float2 *>(Y)[src];
    reinterpret_cast<float2 *>(yb)[e] = make_float2(y.x * sg, y.y * sg);
}

// Network output (FP32 NHWC, channels 0/1 of c) back to a complex FP64 mode
// layout, scaled per mode: d = gain * rms_m * y.
__global__ void k_unpack(const float *__restrict__ y, int c, const float *__restrict__ rms, float gain, int nr, int nz,
                         int nm, double2 *__restrict__ d) {
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;   // over (k, i, m)
    const long total = (long)nm * nz * nr;
    if (e >= total) return;
    const int m = (int)(e % nm);
    const long q = e / nm;
    const int i = (int)(q % nr);
    const int k = (int)(q / nr);
    const float2 v = *reinterpret_cast<const float2 *>(y + (((long)m * nz + k) * nr + i) * c);
    const double s = (double)gain * (double)rms[m];
    d[e] = make_double2(s * v.x, s * v.y);
}

// Mode-layout 2:1 restriction (sum of the 2x2 fine cells: a finite-volume
// integral) and bilinear cell-centred prolongation with a sign-changing
// reflection at walls, between fine (nr, nz) and coarse (nr/2, nz/2).
__global__ void k_restrict2(const double2 *__restrict__ f, int nr, int nz, int nm, double2 *__restrict__ c) {
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const int nrc = nr / 2, nzc = nz / 2;
    const long total = (long)nzc * nrc * nm;
    if (e >= total) return;
    const int m = (int)(e % nm);
    const long q = e / nm;
    const int I = (int)(q % nrc), K = (int)(q / nrc);
    double2 s = make_double2(0.0, 0.0);
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            const double2 v = f[(((long)(2 * K + a)) * nr + 2 * I + b) * nm + m];
            s.x += v.x;
            s.y += v.y;
        }
    c[e] = s;
}

__global__ void k_prolong2(const double2 *__restrict__ c, int nr, int nz, int nm, double2 *__restrict__ f) {
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long total = (long)nz * nr * nm;
    if (e >= total) return;
    const int nrc = nr / 2, nzc = nz / 2;
    const int m = (int)(e % nm);
    const long q = e / nm;
    const int i = (int)(q % nr), k = (int)(q / nr);
    const int K = k >> 1, I = i >> 1;
    const int K2 = K + ((k & 1) ? 1 : -1), I2 = I + ((i & 1) ? 1 : -1);
    const bool kin = K2 >= 0 && K2 < nzc, iin = I2 >= 0 && I2 < nrc;
    const int Kx = kin ? K2 : K, Ix = iin ? I2 : I;
    const double sk = kin ? 1.0 : -1.0, si = iin ? 1.0 : -1.0;
    const double2 c0 = c[((long)K * nrc + I) * nm + m], c1 = c[((long)K * nrc + Ix) * nm + m];
    const double2 c2 = c[((long)Kx * nrc + I) * nm + m], c3 = c[((long)Kx * nrc + Ix) * nm + m];
    f[e] = make_double2(0.5625 * c0.x + 0.1875 * (si * c1.x + sk * c2.x) + 0.0625 * si * sk * c3.x,
                        0.5625 * c0.y + 0.1875 * (si * c1.y + sk * c2.y) + 0.0625 * si * sk * c3.y);
}

// Parseval-weighted inner products of mode-layout fields: partials of
// <a, b> (real part) and <b, b>.
__global__ void __launch_bounds__(256) k_dots(const double2 *__restrict__ a, const double2 *__restrict__ b, long n,
                                              int nm, int nt, double *__restrict__ part) {
    __shared__ double r1[8], r2[8];
    double s1 = 0.0, s2 = 0.0;
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
        const int m = (int)(e % nm);
        const double w = (m == 0 || 2 * m == nt) ? 1.0 : 2.0;
        const double2 x = a[e], y = b[e];
        s1 += w * (x.x * y.x + x.y * y.y);
        s2 += w * (y.x * y.x + y.y * y.y);
    }
    for (int o = 16; o > 0; o >>= 1) {
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    if ((threadIdx.x & 31) == 0) {
        r1[threadIdx.x >> 5] = s1;
        r2[threadIdx.x >> 5] = s2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t1 = 0.0, t2 = 0.0;
        for (int w = 0; w < 8; ++w) {
            t1 += r1[w];
            t2 += r2[w];
        }
        part[2 * blockIdx.x] = t1;
        part[2 * blockIdx.x + 1] = t2;
    }
}

// Sums of the dot partials (one CTA, fixed order) and the step
// alpha = sign <r, b> / <b, b> (0 when <b, b> = 0 or not finite): out[0..2].
__global__ void __launch_bounds__(512) k_dots_final(const double *__restrict__ part, int nb, double sign,
                                                    double *__restrict__ out, double *__restrict__ alpha_out) {
    __shared__ double r1[16], r2[16];
    double s1 = 0.0, s2 = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        s1 += part[2 * b];
        s2 += part[2 * b + 1];
    }
    for (int o = 16; o > 0; o >>= 1) {
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    if ((threadIdx.x & 31) == 0) {
        r1[threadIdx.x >> 5] = s1;
        r2[threadIdx.x >> 5] = s2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t1 = 0.0, t2 = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            t1 += r1[w];
            t2 += r2[w];
        }
        const double al = (t2 > 0.0 && isfinite(t1)) ? sign * t1 / t2 : 0.0;
        out[0] = t1;
        out[1] = t2;
        out[2] = al;
        if (alpha_out) *alpha_out = al;
    }
}

// out = x + alpha d with the step computed by k_dots_final.
__global__ void k_axpy_alpha(const double2 *__restrict__ x, const double2 *__restrict__ d,
                             const double *__restrict__ dots, long n, double2 *__restrict__ out) {
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const double al = dots[2];
    const double2 a = x[e], b = d[e];
    out[e] = make_double2(fma(al, b.x, a.x), fma(al, b.y, a.y));
}

inline unsigned grid1(long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

}  // namespace
}  // namespace pp

using namespace pp;

#define NN_CHECK()                                                                 \
    do {                                                                           \
        cudaError_t e_ = cudaGetLastError();                                       \
        if (e_ != cudaSuccess) {                                                   \
            set_error("nn kernel launch failed: %s", cudaGetErrorString(e_));      \
            return PIC_POISSON_ECUDA;                                              \
        }                                                                          \
    } while (0)

extern "C" {

int pic_nn_conv3x3(const void *in, int cin, const void *w, const float *bias, void *out_bf16, float *out_f32, int cout,
                   int n, int h, int wd, int relu, void *stream) {
    clear_error();
    if (in && w && (out_bf16 || out_f32) && cin > 0 && cout > 0 && n > 0 && h > 0 && wd > 0) {
        const int rc = launch_conv3x3_tc(in, cin, w, bias, out_bf16, out_f32, cout, n, h, wd, relu,
                                         (cudaStream_t)stream);
        if (rc != 1) return rc;   // done on the tcgen05 tensor cores, or an error
    }
    return pic_nn_conv3x3_mma_sync(in, cin, w, bias, out_bf16, out_f32, cout, n, h, wd, relu, stream);
}

int pic_nn_conv3x3_mma_sync(const void *in, int cin, const void *w, const float *bias, void *out_bf16, float *out_f32,
                            int cout, int n, int h, int wd, int relu, void *stream) {
    clear_error();
    if (!in || !w || (!out_bf16 && !out_f32) || cin <= 0 || cin % 16 || cout <= 0 || cout % 8 || cout > 128 ||
        n <= 0 || h <= 0 || wd <= 0) {
        set_error("conv3x3: need cin %% 16 == 0, cout %% 8 == 0 (<= 128), positive sizes, in/w/out");
        return PIC_POISSON_EINVAL;
    }
    const long P = (long)n * h * wd;
    const unsigned g = (unsigned)((P + 16 * CONV_WARPS - 1) / (16 * CONV_WARPS));
    const cudaStream_t st = (cudaStream_t)stream;
    const bf16 *I = (const bf16 *)in, *W = (const bf16 *)w;
    bf16 *O = (bf16 *)out_bf16;
    switch (cout / 8) {
#define PP_CASE(K)                                                                                   \
    case K: k_conv3x3<K><<<g, CONV_WARPS * 32, 0, st>>>(I, cin, W, bias, O, out_f32, n, h, wd, relu); break;
        PP_CASE(1) PP_CASE(2) PP_CASE(3) PP_CASE(4) PP_CASE(5) PP_CASE(6) PP_CASE(7) PP_CASE(8)
        PP_CASE(9) PP_CASE(10) PP_CASE(11) PP_CASE(12) PP_CASE(13) PP_CASE(14) PP_CASE(15) PP_CASE(16)
#undef PP_CASE
    }
    NN_CHECK();
    return PIC_POISSON_OK;
}

int pic_nn_flip_weights(const void *w, int cout, int cin, void *wt, void *stream) {
    clear_error();
    if (!w || !wt || cout <= 0 || cin <= 0) {
        set_error("flip_weights: bad arguments");
        return PIC_POISSON_EINVAL;
    }
    k_flip<<<grid1(9L * cout * cin), 256, 0, (cudaStream_t)stream>>>((const bf16 *)w, (bf16 *)wt, cout, cin);
    NN_CHECK();
    return PIC_POISSON_OK;
}

size_t pic_nn_wgrad_scratch_floats(int cin, int cout, int n, int h, int wd) {
    const long P = (long)n * h * wd;
    const long chunks = (P + WG_CHUNK - 1) / WG_CHUNK;
    return (size_t)(chunks * (9L * cout * cin + cout));
}

int pic_nn_conv3x3_wgrad(const void *in, int cin, const void *dout, int cout, int n, int h, int wd, float *dw,
                         float *dbias, float *scratch, size_t scratch_floats, void *stream) {
    clear_error();
    const long P = (long)n * h * wd;
    const int chunks = (int)((P + WG_CHUNK - 1) / WG_CHUNK);
    if (!in || !dout || !dw || !scratch || scratch_floats < pic_nn_wgrad_scratch_floats(cin, cout, n, h, wd)) {
        set_error("conv3x3_wgrad: bad arguments or scratch too small");
        return PIC_POISSON_EINVAL;
    }
    const cudaStream_t st = (cudaStream_t)stream;
    float *part = scratch, *partb = scratch + (long)chunks * 9 * cout * cin;
    dim3 grid(chunks, (cout * cin + 255) / 256);
    k_wgrad_partial<<<grid, 256, 0, st>>>((const bf16 *)in, cin, (const bf16 *)dout, cout, n, h, wd, part, partb);
    k_wgrad_reduce<<<grid1(9L * cout * cin), 256, 0, st>>>(part, partb, chunks, cout, cin, dw, dbias);
    NN_CHECK();
    return PIC_POISSON_OK;
}

int pic_nn_relu_bwd(const void *y, void *dy, long count, void *stream) {
    k_relu_bwd<<<grid1(count), 256, 0, (cudaStream_t)stream>>>((const bf16 *)y, (bf16 *)dy, count);
    NN_CHECK();
    return PIC_POISSON_OK;
}

int pic_nn_pool2(const void *in, void *out, int n, int h, int wd, int c, int backward, void *stream) {
    const cudaStream_t st = (cudaStream_t)stream;
    if (h % 2 || wd % 2) {
        set_error("pool2: h and w must be even");
        return PIC_POISSON_EINVAL;
    }
    if (!backward) k_pool<<<grid1((long)n * (h / 2) * (wd / 2) * c), 256, 0, st>>>((const bf16 *)in, (bf16 *)out, n, h, wd, c);
    else k_pool_bwd<<<grid1((long)n * h * wd * c), 256, 0, st>>>((const bf16 *)in, (bf16 *)out, n, h, wd, c);
    NN_CHECK();
    return PIC_POISSON_OK;
}

int pic_nn_up2(const void *in, void *out, int n, int h, int wd, int c, int cstride, int backward, void *stream) {
    const cudaStream_t st = (cudaStream_t)stream;
    if (!backward) k_up<<<grid1((long)n * 4 * h * wd * c), 256, 0, st>>>((const bf16 *)in, (bf16 *)out, n, h, wd, c, cstride);
    else k_up_bwd<<<grid1((long)n * h * wd * c), 256, 0, st>>>((const bf16 *)in, cstride, (bf16 *)out, n, h, wd, c);
    NN_CHECK();
    return PIC_POISSON_OK;
}

int pic_nn_copy_channels(const void *src, int sstride, int soff, void *dst, int dstride, int doff, long pixels, int c,
                         void *stream) {
    k_copy_ch<<<grid1(pixels * c), 256, 0, (cudaStream_t)stream>>>((const bf16 *)src, sstride, soff, (bf16 *)dst,
                                                                     dstride, doff, pixels, c);
    NN_CHECK();
    return PIC_POISSON_OK;
}

int pic_nn_mse(const float *pred, const float *target, long pixels, int c, int used, void *dpred, float *scratch,
               float *loss, void *stream) {
    const cudaStream_t st = (cudaStream_t)stream;
    const unsigned nb = grid1(pixels * c);
    k_mse<<<nb, 256, 0, st>>>(pred, target, pixels, c, used, (bf16 *)dpred, scratch);
    k_sum_f<<<1, 1024, 0, st>>>(scratch, (int)nb, pixels * used, loss);
    NN_CHECK();
    return PIC_POISSON_OK;
}

int pic_nn_adam(float *w, const float *g, float *m, float *v, long count, float lr, float b1, float b2, float eps,
                int step, void *w_bf16, void *stream) {
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    k_adam<<<grid1(count), 256, 0, (cudaStream_t)stream>>>(w, g, m, v, count, lr, b1, b2, eps, c1, c2,
                                                           (bf16 *)w_bf16);
    NN_CHECK();
    return PIC_POISSON_OK;
}

int pic_nn_add(void *a, const void *b, long count, void *stream) {
    k_add<<<grid1(count), 256, 0, (cudaStream_t)stream>>>((bf16 *)a, (const bf16 *)b, count);
    NN_CHECK();
    return PIC_POISSON_OK;
}

int pic_nn_to_bf16(const float *a, void *b, long count, void *stream) {
    k_f32_to_bf16<<<grid1(count), 256, 0, (cudaStream_t)stream>>>(a, (bf16 *)b, count);
    NN_CHECK();
    return PIC_POISSON_OK;
}

int pic_nn_pack_modes(const double *x, const float *shift, int nr, int nz, int nm, float *rms, double *scratch,
                      void *out, void *stream) {
    const cudaStream_t st = (cudaStream_t)stream;
    const long cells = (long)nr * nz;
    const int chunks = 256;
    dim3 g1(chunks, (nm + 31) / 32);
    k_mode_ss<<<g1, 256, 0, st>>>((const double2 *)x, cells, nm, scratch);
    k_mode_rms<<<grid1(nm), 256, 0, st>>>(scratch, chunks, nm, cells, rms);
    k_pack<<<grid1((long)nm * cells), 256, 0, st>>>((const double2 *)x, rms, shift, nr, nz, nm, (bf16 *)out);
    NN_CHECK();
    return PIC_POISSON_OK;
}

int pic_nn_pack_target(const double *x, int nr, int nz, int nm, float *rms, double *scratch, float *out,
                       void *stream) {
    clear_error();
    if (!x || !rms || !scratch || !out || nr <= 0 || nz <= 0 || nm <= 0) {
        set_error("pack_target: bad arguments");
        return PIC_POISSON_EINVAL;
    }
    const cudaStream_t st = (cudaStream_t)stream;
    const long cells = (long)nr * nz;
    const int chunks = 256;
    dim3 g1(chunks, (nm + 31) / 32);
    k_mode_ss<<<g1, 256, 0, st>>>((const double2 *)x, cells, nm, scratch);
    k_mode_rms<<<grid1(nm), 256, 0, st>>>(scratch, chunks, nm, cells, rms);
    k_pack_target<<<grid1((long)nm * cells), 256, 0, st>>>((const double2 *)x, rms, nr, nz, nm, out);
    NN_CHECK();
    return PIC_POISSON_OK;
}

int pic_nn_gather_batch(const void *X, const float *Y, const long *idx, const float *sign, int batch, long pixels,
                        void *xb, float *yb, void *stream) {
    clear_error();
    if (!X || !Y || !idx || !sign || !xb || !yb || batch <= 0 || pixels <= 0) {
        set_error("gather_batch: bad arguments");
        return PIC_POISSON_EINVAL;
    }
    k_gather_batch<<<grid1((long)batch * pixels), 256, 0, (cudaStream_t)stream>>>(
        (const bf16 *)X, Y, idx, sign, batch, pixels, (bf16 *)xb, yb);
    NN_CHECK();
    return PIC_POISSON_OK;
}

int pic_nn_unpack_modes(const float *y, int c, const float *rms, float gain, int nr, int nz, int nm, double *d,
                        void *stream) {
    k_unpack<<<grid1((long)nm * nr * nz), 256, 0, (cudaStream_t)stream>>>(y, c, rms, gain, nr, nz, nm, (double2 *)d);
    NN_CHECK();
    return PIC_POISSON_OK;
}

int pic_nn_restrict2(const double *f, int nr, int nz, int nm, double *c, void *stream) {
    if (nr % 2 || nz % 2) {
        set_error("restrict2: nr and nz must be even");
        return PIC_POISSON_EINVAL;
    }
    k_restrict2<<<grid1((long)(nr / 2) * (nz / 2) * nm), 256, 0, (cudaStream_t)stream>>>((const double2 *)f, nr, nz,
                                                                                        nm, (double2 *)c);
    NN_CHECK();
    return PIC_POISSON_OK;
}

int pic_nn_prolong2(const double *c, int nr, int nz, int nm, double *f, void *stream) {
    if (nr % 2 || nz % 2) {
        set_error("prolong2: nr and nz must be even");
        return PIC_POISSON_EINVAL;
    }
    k_prolong2<<<grid1((long)nr * nz * nm), 256, 0, (cudaStream_t)stream>>>((const double2 *)c, nr, nz, nm,
                                                                            (double2 *)f);
    NN_CHECK();
    return PIC_POISSON_OK;
}

int pic_nn_minres_step(const double *x, const double *d, const double *r, const double *b, long entries, int nm,
                       int nt, double sign, double *scratch, double *out, double *alpha, void *stream) {
    const cudaStream_t st = (cudaStream_t)stream;
    const int nb = 512;
    k_dots<<<nb, 256, 0, st>>>((const double2 *)r, (const double2 *)b, entries, nm, nt, scratch);
    k_dots_final<<<1, 512, 0, st>>>(scratch, nb, sign, scratch + 2 * nb, alpha);
    k_axpy_alpha<<<grid1(entries), 256, 0, st>>>((const double2 *)x, (const double2 *)d, scratch + 2 * nb, entries,
                                                 (double2 *)out);
    NN_CHECK();
    return PIC_POISSON_OK;
}

}  // extern "C"
