// 3x3 convolution of the learned warm start on the fifth-generation tensor
// cores: an implicit GEMM with tcgen05.mma (BF16 in, FP32 accumulated in
// tensor memory), operands staged by TMA.
//
// GEMM view: rows = output pixels (a tile of 128 consecutive pixels of one
// sample: 128 of one image row, or 128 / W whole rows when W < 128), columns =
// output channels (N = cout), reduction = (tap, input channel).  For tap
// (dy, dx) and a chunk of KC input channels the A operand of a tile is the
// input box [KC channels] x [the tile's pixels shifted by (dx, dy)]: one
// 4-D TMA load of the NHWC tensor, whose out-of-range coordinates (x = -1,
// x = W, y = -1, y = H) read zeros -- exactly the convolution's zero padding.
// The B operand is the weight slice w[tap][0:cout][c0:c0+KC] (K-major), one
// 3-D TMA load.  KC = 64, 32 or 16 channels make a 128-, 64- or 32-byte
// row, which TMA swizzles into the canonical K-major layout the MMA's shared
// memory descriptors name.
//
// Roles (192 threads): warp 4 issues the TMA loads into a ring of 4 stages (8
// for 16-channel chunks),
// warp 5 issues the MMAs (KC / 16 per stage, M = 128, N = cout, K = 16) into
// one of two TMEM accumulators, warps 0-3 drain an accumulator (tcgen05.ld,
// each warp its 32 TMEM lanes = 32 pixels), add the bias, apply ReLU and
// store BF16 and / or FP32 while the next tile accumulates into the other.
// CTAs are persistent over the tiles.  Every wait on an mbarrier is bounded;
// a wait that runs out sets an error flag (pic_nn_conv_tc_status), ends the
// CTA's loops, waits (bounded) for its own copies and MMAs, and frees its
// tensor memory.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "internal.h"

namespace pp {

__device__ int g_conv_tc_error;   // 1 + the role whose wait ran out (0: none)

namespace {

typedef __nv_bfloat16 bf16;

constexpr int TC_M = 128;                      // pixels per tile (MMA M)
constexpr int TC_MAX_STAGES = 8;                 // ring slots: 8 for 16-channel chunks (a tile's 9 loads), else 4
constexpr int TC_THREADS = 192;                // warps 0-3 epilogue, 4 TMA, 5 MMA
constexpr unsigned TC_SPIN_LIMIT = 1u << 23;   // try_wait rounds before a wait gives up

struct ConvTCArgs {
    int n, h, wd, cin, cout;
    int kc, nchunks;                 // channels per stage, cin / kc
    int bx, by;                      // tile: bx pixels along x times by rows
    int tiles_x, tiles_y, tiles;
    unsigned a_bytes, b_bytes;       // TMA bytes of one stage
    unsigned stage_bytes;            // a_bytes + b_bytes rounded up to 1024
    unsigned tmem_cols;              // columns of one accumulator (power of two >= 32)
    unsigned idesc;                  // MMA instruction descriptor
    unsigned swz, sbo;               // shared-memory descriptor: layout type, 8-row stride
    const float *bias;
    bf16 *out;
    float *out32;
    int relu;
    int stages;                      // ring slots in use (<= TC_MAX_STAGES)
    // halo variant (k_conv3x3_tc_halo): no-swizzle K-major operands
    unsigned lbo_a;                  // bytes from one 8-channel group of the halo tile to the next
    unsigned lbo_b;                  // bytes from one 8-channel group of a tap's weights to the next
    unsigned w_bytes;                // all nine taps' weights (resident)
};

// No-swizzle K-major descriptor: 8-row core matrices of 16-byte rows; LBO =
// the step to the next 8 channels (K), SBO = 128 (the next 8 rows follow
// directly), so the start may sit on any 16-byte row.
__device__ __forceinline__ uint64_t smem_desc_plain(unsigned addr, unsigned lbo) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)(128u >> 4) << 32) | ((uint64_t)1 << 46);
}

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
// Wait for the completion of the phase with parity `parity`; false if the
// limit ran out or another role gave up (*abort set).
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity, volatile int *abort) {
    for (unsigned it = 0; it < TC_SPIN_LIMIT; ++it) {
        unsigned ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
        if ((it & 1023u) == 1023u && *abort) return false;
    }
    return false;
}

__device__ __forceinline__ void tma_load_4d(unsigned dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                            unsigned bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void tma_load_3d(unsigned dst, const CUtensorMap *map, int c0, int c1, int c2,
                                            unsigned bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
        : "memory");
}

// Shared-memory matrix descriptor (tcgen05): start address >> 4 (bits 0-13),
// leading-dimension byte offset >> 4 (16-29; not used by swizzled K-major
// operands whose K extent per MMA fits one swizzle row), stride-dimension byte
// offset >> 4 (32-45: from one 8-row group to the next), the fixed version
// bit 46, base offset 0 (1024-byte aligned stages), layout type (61-63).
__device__ __forceinline__ uint64_t smem_desc(unsigned addr, unsigned sbo, unsigned swz) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)swz << 61);
}

__device__ __forceinline__ void umma_bf16(unsigned tmem_d, uint64_t a, uint64_t b, unsigned idesc, unsigned acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
// Arrive on `bar` once every MMA this thread issued before has completed.
__device__ __forceinline__ void umma_commit(unsigned bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 consecutive FP32 accumulator columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(unsigned taddr, float (&v)[16]) {
    unsigned r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int e = 0; e < 16; ++e) v[e] = __uint_as_float(r[e]);
}

__device__ __forceinline__ unsigned pack2(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<unsigned *>(&v);
}

__device__ __forceinline__ void tile_origin(const ConvTCArgs &a, int tile, int &nn, int &x0, int &y0) {
    const int tx = tile % a.tiles_x, rest = tile / a.tiles_x;
    x0 = tx * a.bx;
    y0 = (rest % a.tiles_y) * a.by;
    nn = rest / a.tiles_y;
}

__device__ __forceinline__ void give_up(volatile int *abort, int role) {
    *abort = 1;
    atomicCAS(&g_conv_tc_error, 0, 1 + role);
}

__global__ void __launch_bounds__(TC_THREADS, 1)
k_conv3x3_tc(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb, const ConvTCArgs a) {
    extern __shared__ __align__(1024) unsigned char dsm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // stages on 1024-byte boundaries (the swizzle atoms), then the barriers
    const unsigned raw = smem_u32(dsm);
    const unsigned pad = (1024u - (raw & 1023u)) & 1023u;
    const unsigned stage0 = raw + pad;
    const int S = a.stages;
    unsigned char *tail = dsm + pad + S * a.stage_bytes;
    const unsigned full0 = smem_u32(tail);                   // [S] TMA bytes landed
    const unsigned empty0 = full0 + 8 * TC_MAX_STAGES;       // [S] stage read by the MMAs
    const unsigned tfull0 = empty0 + 8 * TC_MAX_STAGES;      // [2] accumulator complete
    const unsigned tempty0 = tfull0 + 16;                    // [2] accumulator drained
    const unsigned drain = tempty0 + 16;                     // every MMA of this CTA complete
    unsigned *tmem_slot = reinterpret_cast<unsigned *>(tail + 8 * (2 * TC_MAX_STAGES + 5));
    volatile int *abort = reinterpret_cast<volatile int *>(tmem_slot + 1);
    volatile int *never = reinterpret_cast<volatile int *>(tmem_slot + 2);   // stays 0: a wait that ignores *abort
    const unsigned ncols = 2 * a.tmem_cols;
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(tfull0 + 8 * b, 1);
            mbar_init(tempty0 + 8 * b, 4 * 32);
        }
        mbar_init(drain, 1);
        *abort = 0;
        *never = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = *tmem_slot;
    const int kiters = 9 * a.nchunks;

    if (warp == 4) {
        // ---------------- TMA producer
        if (lane == 0) {
            unsigned it = 0;
            bool ok = true;
            for (int tile = blockIdx.x; ok && tile < a.tiles; tile += gridDim.x) {
                int nn, x0, y0;
                tile_origin(a, tile, nn, x0, y0);
                for (int k = 0; k < kiters; ++k, ++it) {
                    const unsigned s = it % S, u = it / S;
                    if (!mbar_wait(empty0 + 8 * s, (u & 1u) ^ 1u, abort)) {
                        give_up(abort, 0);
                        ok = false;
                        break;
                    }
                    const int tap = k / a.nchunks, c0 = (k - tap * a.nchunks) * a.kc;
                    const unsigned sa = stage0 + s * a.stage_bytes;
                    mbar_expect_tx(full0 + 8 * s, a.a_bytes + a.b_bytes);
                    tma_load_4d(sa, &ta, c0, x0 + tap % 3 - 1, y0 + tap / 3 - 1, nn, full0 + 8 * s);
                    tma_load_3d(sa + a.a_bytes, &tb, c0, 0, tap, full0 + 8 * s);
                }
            }
            // the last copies land before the CTA exits (on the normal path
            // the MMAs have consumed them already and these waits return at once)
            const unsigned first = it > (unsigned)S ? it - S : 0u;
            for (unsigned j = first; j < it; ++j)
                if (!mbar_wait(full0 + 8 * (j % S), (j / S) & 1u, never)) give_up(abort, 3);
        }
    } else if (warp == 5) {
        // ---------------- MMA issuer
        if (lane == 0) {
            unsigned it = 0, tc = 0;
            bool ok = true;
            for (int tile = blockIdx.x; ok && tile < a.tiles; tile += gridDim.x, ++tc) {
                const unsigned buf = tc & 1u, u = tc >> 1;
                if (!mbar_wait(tempty0 + 8 * buf, (u & 1u) ^ 1u, abort)) {
                    give_up(abort, 1);
                    break;
                }
                tc_fence_after();
                const unsigned d = tmem + buf * a.tmem_cols;
                for (int k = 0; k < kiters; ++k, ++it) {
                    const unsigned s = it % S, us = it / S;
                    if (!mbar_wait(full0 + 8 * s, us & 1u, abort)) {
                        give_up(abort, 1);
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const unsigned sa = stage0 + s * a.stage_bytes, sb = sa + a.a_bytes;
                    for (int kk = 0; kk < a.kc / 16; ++kk)   // K = 16 BF16 = 32 bytes per MMA
                        umma_bf16(d, smem_desc(sa + 32u * kk, a.sbo, a.swz), smem_desc(sb + 32u * kk, a.sbo, a.swz),
                                  a.idesc, (k | kk) != 0 ? 1u : 0u);
                    umma_commit(empty0 + 8 * s);   // the stage is free once these MMAs have read it
                }
                if (!ok) break;
                umma_commit(tfull0 + 8 * buf);     // the tile's accumulator is complete
            }
            umma_commit(drain);
            if (!mbar_wait(drain, 0, never)) give_up(abort, 4);
        }
    } else {
        // ---------------- epilogue: warp w drains TMEM lanes 32 w .. 32 w + 31
        const int row = threadIdx.x;   // pixel of the tile = TMEM lane
        unsigned tc = 0;
        for (int tile = blockIdx.x; tile < a.tiles; tile += gridDim.x, ++tc) {
            const unsigned buf = tc & 1u, u = tc >> 1;
            if (!mbar_wait(tfull0 + 8 * buf, u & 1u, abort)) {
                give_up(abort, 2);
                break;
            }
            tc_fence_after();
            int nn, x0, y0;
            tile_origin(a, tile, nn, x0, y0);
            const int x = x0 + row % a.bx, y = y0 + row / a.bx;
            const bool valid = y < a.h;
            const size_t p = ((size_t)nn * a.h + (valid ? y : 0)) * a.wd + x;
            const unsigned taddr = tmem + buf * a.tmem_cols + ((unsigned)(warp * 32) << 16);
            for (int c = 0; c < a.cout; c += 16) {
                float v[16];
                tmem_ld16(taddr + (unsigned)c, v);
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    float t = v[e] + (a.bias ? a.bias[c + e] : 0.f);
                    v[e] = a.relu ? fmaxf(t, 0.f) : t;
                }
                if (!valid) continue;
                if (a.out) {
                    uint4 *o = reinterpret_cast<uint4 *>(a.out + p * a.cout + c);
                    o[0] = make_uint4(pack2(v[0], v[1]), pack2(v[2], v[3]), pack2(v[4], v[5]), pack2(v[6], v[7]));
                    o[1] = make_uint4(pack2(v[8], v[9]), pack2(v[10], v[11]), pack2(v[12], v[13]),
                                      pack2(v[14], v[15]));
                }
                if (a.out32) {
                    float4 *o = reinterpret_cast<float4 *>(a.out32 + p * a.cout + c);
#pragma unroll
                    for (int q = 0; q < 4; ++q) o[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                }
            }
            tc_fence_before();
            mbar_arrive(tempty0 + 8 * buf);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
    }
}

// Halo variant for image rows of 128 pixels or more (tiles of one row) and
// small weight sets (the full- and half-resolution layers, which are bound by
// data movement): per tile and chunk of KC channels, TMA brings the three input
// rows y - 1 .. y + 1 over pixels x0 - 1 .. x0 + 128 once, as 8-channel groups
// of 390 16-byte rows (no swizzle, K-major core matrices); the nine taps are
// the same buffer seen from nine start rows, (1 + dy) * 130 + 1 + dx.  All
// nine taps' weights stay resident from the CTA's start.  A tile then moves
// 3 * 130 * cin instead of 9 * 128 * cin input values.
__global__ void __launch_bounds__(TC_THREADS, 1)
k_conv3x3_tc_halo(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb, const ConvTCArgs a) {
    extern __shared__ __align__(1024) unsigned char dsm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned raw = smem_u32(dsm);
    const unsigned pad = (1024u - (raw & 1023u)) & 1023u;
    const unsigned wbase = raw + pad;                                  // resident weights
    const unsigned stage0 = wbase + ((a.w_bytes + 1023u) & ~1023u);   // halo tiles
    const int S = a.stages;
    unsigned char *tail = dsm + pad + ((a.w_bytes + 1023u) & ~1023u) + S * a.stage_bytes;
    const unsigned full0 = smem_u32(tail);
    const unsigned empty0 = full0 + 8 * TC_MAX_STAGES;
    const unsigned tfull0 = empty0 + 8 * TC_MAX_STAGES;
    const unsigned tempty0 = tfull0 + 16;
    const unsigned drain = tempty0 + 16;
    const unsigned wbar = drain + 8;                                   // weights landed
    unsigned *tmem_slot = reinterpret_cast<unsigned *>(tail + 8 * (2 * TC_MAX_STAGES + 6));
    volatile int *abort = reinterpret_cast<volatile int *>(tmem_slot + 1);
    volatile int *never = reinterpret_cast<volatile int *>(tmem_slot + 2);
    const unsigned ncols = 2 * a.tmem_cols;
    const int groups = a.kc / 8;                 // 8-channel groups per chunk
    const int cgroups = a.cin / 8;               // per tap of the weights
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(tfull0 + 8 * b, 1);
            mbar_init(tempty0 + 8 * b, 4 * 32);
        }
        mbar_init(drain, 1);
        mbar_init(wbar, 1);
        *abort = 0;
        *never = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = *tmem_slot;

    if (warp == 4) {
        // ---------------- TMA producer: the weights once, then the halo tiles
        if (lane == 0) {
            mbar_expect_tx(wbar, a.w_bytes);
            for (int tap = 0; tap < 9; ++tap)
                for (int g = 0; g < cgroups; ++g)
                    tma_load_3d(wbase + (unsigned)(tap * cgroups + g) * a.lbo_b, &tb, 8 * g, 0, tap, wbar);
            unsigned it = 0;
            bool ok = true;
            for (int tile = blockIdx.x; ok && tile < a.tiles; tile += gridDim.x) {
                int nn, x0, y0;
                tile_origin(a, tile, nn, x0, y0);
                for (int c = 0; c < a.nchunks; ++c, ++it) {
                    const unsigned s = it % S, u = it / S;
                    if (!mbar_wait(empty0 + 8 * s, (u & 1u) ^ 1u, abort)) {
                        give_up(abort, 0);
                        ok = false;
                        break;
                    }
                    const unsigned sa = stage0 + s * a.stage_bytes;
                    mbar_expect_tx(full0 + 8 * s, a.a_bytes);
                    for (int g = 0; g < groups; ++g)
                        tma_load_4d(sa + (unsigned)g * a.lbo_a, &ta, c * a.kc + 8 * g, x0 - 1, y0 - 1, nn,
                                    full0 + 8 * s);
                }
            }
            const unsigned first = it > (unsigned)S ? it - S : 0u;
            for (unsigned j = first; j < it; ++j)
                if (!mbar_wait(full0 + 8 * (j % S), (j / S) & 1u, never)) give_up(abort, 3);
            if (!mbar_wait(wbar, 0, never)) give_up(abort, 3);
        }
    } else if (warp == 5) {
        // ---------------- MMA issuer
        if (lane == 0) {
            unsigned it = 0, tc = 0;
            bool ok = mbar_wait(wbar, 0, abort);
            if (!ok) give_up(abort, 1);
            tc_fence_after();
            for (int tile = blockIdx.x; ok && tile < a.tiles; tile += gridDim.x, ++tc) {
                const unsigned buf = tc & 1u, u = tc >> 1;
                if (!mbar_wait(tempty0 + 8 * buf, (u & 1u) ^ 1u, abort)) {
                    give_up(abort, 1);
                    break;
                }
                tc_fence_after();
                const unsigned d = tmem + buf * a.tmem_cols;
                for (int c = 0; c < a.nchunks; ++c, ++it) {
                    const unsigned s = it % S, us = it / S;
                    if (!mbar_wait(full0 + 8 * s, us & 1u, abort)) {
                        give_up(abort, 1);
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const unsigned sa = stage0 + s * a.stage_bytes;
                    for (int tap = 0; tap < 9; ++tap) {
                        const unsigned row0 = (unsigned)((tap / 3) * (a.bx + 2) + tap % 3);   // (1 + dy) W' + 1 + dx
                        for (int kk = 0; kk < a.kc / 16; ++kk) {   // K = 16: two 8-channel groups
                            const unsigned adr = sa + 2u * kk * a.lbo_a + 16u * row0;
                            const unsigned bdr = wbase + (unsigned)(tap * cgroups + c * groups + 2 * kk) * a.lbo_b;
                            umma_bf16(d, smem_desc_plain(adr, a.lbo_a), smem_desc_plain(bdr, a.lbo_b), a.idesc,
                                      (c | tap | kk) != 0 ? 1u : 0u);
                        }
                    }
                    umma_commit(empty0 + 8 * s);
                }
                if (!ok) break;
                umma_commit(tfull0 + 8 * buf);
            }
            umma_commit(drain);
            if (!mbar_wait(drain, 0, never)) give_up(abort, 4);
        }
    } else {
        // ---------------- epilogue (as in k_conv3x3_tc; tiles are one row)
        const int row = threadIdx.x;
        unsigned tc = 0;
        for (int tile = blockIdx.x; tile < a.tiles; tile += gridDim.x, ++tc) {
            const unsigned buf = tc & 1u, u = tc >> 1;
            if (!mbar_wait(tfull0 + 8 * buf, u & 1u, abort)) {
                give_up(abort, 2);
                break;
            }
            tc_fence_after();
            int nn, x0, y0;
            tile_origin(a, tile, nn, x0, y0);
            const size_t p = ((size_t)nn * a.h + y0) * a.wd + x0 + row;
            const unsigned taddr = tmem + buf * a.tmem_cols + ((unsigned)(warp * 32) << 16);
            for (int c = 0; c < a.cout; c += 16) {
                float v[16];
                tmem_ld16(taddr + (unsigned)c, v);
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    float t = v[e] + (a.bias ? a.bias[c + e] : 0.f);
                    v[e] = a.relu ? fmaxf(t, 0.f) : t;
                }
                if (a.out) {
                    uint4 *o = reinterpret_cast<uint4 *>(a.out + p * a.cout + c);
                    o[0] = make_uint4(pack2(v[0], v[1]), pack2(v[2], v[3]), pack2(v[4], v[5]), pack2(v[6], v[7]));
                    o[1] = make_uint4(pack2(v[8], v[9]), pack2(v[10], v[11]), pack2(v[12], v[13]),
                                      pack2(v[14], v[15]));
                }
                if (a.out32) {
                    float4 *o = reinterpret_cast<float4 *>(a.out32 + p * a.cout + c);
#pragma unroll
                    for (int q = 0; q < 4; ++q) o[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                }
            }
            tc_fence_before();
            mbar_arrive(tempty0 + 8 * buf);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
    }
}

}  // namespace

// ------------------------------------------------------------------ host side
namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

std::mutex g_tc_mutex;
EncodeTiledFn g_encode = nullptr;
bool g_encode_tried = false;

EncodeTiledFn encoder() {
    std::lock_guard<std::mutex> lock(g_tc_mutex);
    if (!g_encode_tried) {
        g_encode_tried = true;
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = (EncodeTiledFn)f;
        else
            cudaGetLastError();
    }
    return g_encode;
}

}  // namespace

namespace {

// Per device: SM count, shared memory per SM, and each kernel's registers per
// thread (fixed properties, queried once).
struct TCDeviceInfo {
    bool valid = false;
    int sms = 0, smem_sm = 0;
    int regs[2] = {0, 0};   // k_conv3x3_tc, k_conv3x3_tc_halo
};
TCDeviceInfo g_tc_info[64];

int conv_tc_occupancy(int which, size_t smem, unsigned tmem_cols_per_cta, int *grid_cap) {
    int dev = 0;
    PP_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) {
        set_error("device ordinal %d beyond 64", dev);
        return PIC_POISSON_EINVAL;
    }
    TCDeviceInfo info;
    {
        std::lock_guard<std::mutex> lock(g_tc_mutex);
        info = g_tc_info[dev];
    }
    if (!info.valid) {
        PP_CUDA(cudaDeviceGetAttribute(&info.sms, cudaDevAttrMultiProcessorCount, dev));
        PP_CUDA(cudaDeviceGetAttribute(&info.smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
        cudaFuncAttributes fa;
        PP_CUDA(cudaFuncGetAttributes(&fa, (const void *)k_conv3x3_tc));
        info.regs[0] = fa.numRegs;
        PP_CUDA(cudaFuncGetAttributes(&fa, (const void *)k_conv3x3_tc_halo));
        info.regs[1] = fa.numRegs;
        info.valid = true;
        std::lock_guard<std::mutex> lock(g_tc_mutex);
        g_tc_info[dev] = info;
    }
    // CTAs per SM: shared memory (1 KB reserved per CTA), registers, threads,
    // and tensor memory (512 columns per SM: no CTA waits for an allocation)
    const int regs = std::max(1, (info.regs[which] + 7) & ~7) * TC_THREADS;
    const int occ = std::min({(int)(info.smem_sm / (smem + 1024)), 65536 / regs, 2048 / TC_THREADS, 32,
                              (int)(512u / tmem_cols_per_cta)});
    *grid_cap = info.sms * std::max(1, occ);
    return PIC_POISSON_OK;
}

int set_smem(const void *kernel, size_t smem) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)   // all of the SM's unified memory as shared memory, so several CTAs fit
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) {
        set_error("conv3x3 (tcgen05): %s", cudaGetErrorString(e));
        return PIC_POISSON_ECUDA;
    }
    return PIC_POISSON_OK;
}

// The halo variant's operands: no-swizzle 4-D boxes of 8 channels x 130
// pixels x 3 rows of the input, 3-D boxes of 8 channels x cout of each tap's
// weights.
int launch_halo(ConvTCArgs a, const void *in, const void *w, EncodeTiledFn enc, cudaStream_t st) {
    a.kc = a.cin % 32 == 0 ? 32 : 16;
    a.nchunks = a.cin / a.kc;
    const unsigned groups = (unsigned)a.kc / 8, rows = 3u * (unsigned)(a.bx + 2);
    a.lbo_a = (rows * 16u + 127u) & ~127u;           // 128-byte aligned TMA destinations
    a.a_bytes = groups * rows * 16u;                  // TMA bytes of one chunk
    a.stage_bytes = (groups * a.lbo_a + 1023u) & ~1023u;
    a.lbo_b = (unsigned)a.cout * 16u;
    a.w_bytes = 9u * (unsigned)a.cout * (unsigned)a.cin * 2u;
    a.stages = a.kc == 16 ? 4 : 3;
    CUtensorMap ta, tb;
    const cuuint64_t gdim_a[4] = {(cuuint64_t)a.cin, (cuuint64_t)a.wd, (cuuint64_t)a.h, (cuuint64_t)a.n};
    const cuuint64_t gstr_a[3] = {(cuuint64_t)a.cin * 2, (cuuint64_t)a.cin * 2 * a.wd,
                                  (cuuint64_t)a.cin * 2 * a.wd * a.h};
    const cuuint32_t box_a[4] = {8, (cuuint32_t)(a.bx + 2), 3, 1};
    const cuuint32_t one[4] = {1, 1, 1, 1};
    if (enc(&ta, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void *>(in), gdim_a, gstr_a, box_a, one,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return 1;
    const cuuint64_t gdim_b[3] = {(cuuint64_t)a.cin, (cuuint64_t)a.cout, 9};
    const cuuint64_t gstr_b[2] = {(cuuint64_t)a.cin * 2, (cuuint64_t)a.cin * 2 * a.cout};
    const cuuint32_t box_b[3] = {8, (cuuint32_t)a.cout, 1};
    if (enc(&tb, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(w), gdim_b, gstr_b, box_b, one,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return 1;
    const size_t smem = 1024 + ((a.w_bytes + 1023u) & ~1023u) + (size_t)a.stages * a.stage_bytes +
                        8 * (2 * TC_MAX_STAGES + 6) + 16;
    int rc = set_smem((const void *)k_conv3x3_tc_halo, smem);
    if (rc) return rc;
    int cap = 0;
    rc = conv_tc_occupancy(1, smem, 2u * a.tmem_cols, &cap);
    if (rc) return rc;
    k_conv3x3_tc_halo<<<std::min(a.tiles, cap), TC_THREADS, smem, st>>>(ta, tb, a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("conv3x3 (tcgen05, halo) launch failed: %s", cudaGetErrorString(e));
        return PIC_POISSON_ECUDA;
    }
    return PIC_POISSON_OK;
}

// Tile shape of a W-wide image: 128 pixels of a row (W a multiple of 128) or
// 128 / W whole rows (W = 16, 32 or 64); 0 when the tensor-core path does not
// take this width.
int conv_tc_tile_x(int wd) {
    if (wd % TC_M == 0) return TC_M;
    if (wd == 16 || wd == 32 || wd == 64) return wd;
    return 0;
}

}  // namespace

// The tensor-core convolution, or 1 when it does not apply (the caller then
// runs the mma.sync kernel): cout a multiple of 16 up to 128, cin a multiple of
// 16, a tileable width, 16-byte aligned tensors and the driver's tensor-map
// encoder available.  0 on success, a PIC_POISSON_* error otherwise.
int launch_conv3x3_tc(const void *in, int cin, const void *w, const float *bias, void *out, float *out32, int cout,
                      int n, int h, int wd, int relu, cudaStream_t st) {
    const int bx = conv_tc_tile_x(wd);
    if (!bx || cout % 16 || cout > 128 || cin % 16 || ((uintptr_t)in & 15) || ((uintptr_t)w & 15) ||
        ((uintptr_t)out & 15) || ((uintptr_t)out32 & 15))
        return 1;
    EncodeTiledFn enc = encoder();
    if (!enc) return 1;
    ConvTCArgs a{};
    a.n = n;
    a.h = h;
    a.wd = wd;
    a.cin = cin;
    a.cout = cout;
    a.kc = cin % 64 == 0 ? 64 : (cin % 32 == 0 ? 32 : 16);
    a.nchunks = cin / a.kc;
    a.bx = bx;
    a.by = TC_M / bx;
    a.tiles_x = wd / bx;
    a.tiles_y = (h + a.by - 1) / a.by;
    const long tiles = (long)n * a.tiles_y * a.tiles_x;
    if (tiles > 0x7fffffffL) return 1;
    a.tiles = (int)tiles;
    a.a_bytes = (unsigned)(TC_M * a.kc * 2);
    a.b_bytes = (unsigned)(cout * a.kc * 2);
    a.stage_bytes = (a.a_bytes + a.b_bytes + 1023u) & ~1023u;
    a.tmem_cols = cout <= 32 ? 32u : (cout <= 64 ? 64u : 128u);
    // kind::f16 instruction descriptor: FP32 accumulator (bits 4-5 = 1), BF16 A
    // and B (bits 7-9, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at
    // bits 17-22, M >> 4 at bits 24-28
    a.idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(cout >> 3) << 17) | ((unsigned)(TC_M >> 4) << 24);
    // rows of kc BF16 = 32, 64 or 128 bytes: the matching swizzle, 8 rows per group
    a.swz = a.kc == 64 ? 2u : (a.kc == 32 ? 4u : 6u);
    a.sbo = 8u * (unsigned)(a.kc * 2);
    a.bias = bias;
    a.out = (bf16 *)out;
    a.out32 = out32;
    a.relu = relu;
    // halo variant: one-row tiles and weights small enough to stay resident
    const unsigned w_all = 9u * (unsigned)cout * (unsigned)cin * 2u;
    if (a.by == 1 && w_all <= 48u * 1024u) return launch_halo(a, in, w, enc, st);
    const CUtensorMapSwizzle sw = a.kc == 64 ? CU_TENSOR_MAP_SWIZZLE_128B
                                             : (a.kc == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B);
    // activations: (c, x, y, n), zero fill outside
    CUtensorMap ta, tb;
    const cuuint64_t gdim_a[4] = {(cuuint64_t)cin, (cuuint64_t)wd, (cuuint64_t)h, (cuuint64_t)n};
    const cuuint64_t gstr_a[3] = {(cuuint64_t)cin * 2, (cuuint64_t)cin * 2 * wd, (cuuint64_t)cin * 2 * wd * h};
    const cuuint32_t box_a[4] = {(cuuint32_t)a.kc, (cuuint32_t)a.bx, (cuuint32_t)a.by, 1};
    const cuuint32_t one[4] = {1, 1, 1, 1};
    if (enc(&ta, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void *>(in), gdim_a, gstr_a, box_a, one,
            CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return 1;
    // weights [tap][cout][cin]: (c, co, tap)
    const cuuint64_t gdim_b[3] = {(cuuint64_t)cin, (cuuint64_t)cout, 9};
    const cuuint64_t gstr_b[2] = {(cuuint64_t)cin * 2, (cuuint64_t)cin * 2 * cout};
    const cuuint32_t box_b[3] = {(cuuint32_t)a.kc, (cuuint32_t)cout, 1};
    if (enc(&tb, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(w), gdim_b, gstr_b, box_b, one,
            CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return 1;
    a.stages = a.kc == 16 ? 8 : 4;
    const size_t smem = 1024 + (size_t)a.stages * a.stage_bytes + 8 * (2 * TC_MAX_STAGES + 5) + 16;
    int rc = set_smem((const void *)k_conv3x3_tc, smem);
    if (rc) return rc;
    int cap = 0;
    rc = conv_tc_occupancy(0, smem, 2u * a.tmem_cols, &cap);
    if (rc) return rc;
    const int grid = std::min(a.tiles, cap);
    k_conv3x3_tc<<<grid, TC_THREADS, smem, st>>>(ta, tb, a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("conv3x3 (tcgen05) launch failed: %s", cudaGetErrorString(e));
        return PIC_POISSON_ECUDA;
    }
    return PIC_POISSON_OK;
}

}  // namespace pp

// Status of the tensor-core convolution's bounded waits: 0 if none ran out
// since the last call, else 1 + the role (0 TMA, 1 MMA, 2 epilogue, 3 copy
// drain, 4 MMA drain) of the first that did; the flag is then cleared.
extern "C" int pic_nn_conv_tc_status(int *status) {
    pp::clear_error();
    if (!status) {
        pp::set_error("status is NULL");
        return PIC_POISSON_EINVAL;
    }
    int v = 0, zero = 0;
    PP_CUDA(cudaMemcpyFromSymbol(&v, pp::g_conv_tc_error, sizeof(int)));
    PP_CUDA(cudaMemcpyToSymbol(pp::g_conv_tc_error, &zero, sizeof(int)));
    *status = v;
    return PIC_POISSON_OK;
}
