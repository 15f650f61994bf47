// Mode-space residual and relative residual without any device allocation.
//
// Some callers cannot call cudaMalloc: a particle-in-cell code that reserves
// all device memory for particles at start-up and hands out nothing else, or a
// real-time step loop that may not pay cudaMalloc's implicit device-wide
// synchronisation.  For them pic_poisson_mode_residual_noalloc needs no plan:
// it builds the operator's coefficients inside the kernel from the
// descriptor's uniform geometry, and keeps its per-block partial sums in a
// fixed file-scope device array instead of a workspace.
#include <cmath>
#include <mutex>

#include <cuda.h>

#include "internal.h"

namespace pp {
namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_MAX_BLOCKS = 65536;                         // => at most 16,777,216 mode entries
constexpr long NA_MAX_ENTRIES = (long)NA_MAX_BLOCKS * NA_THREADS;
constexpr int NA_MAX_MODES = 129;                            // ntheta <= 256
constexpr int NA_MAX_DEVICES = 64;

// Partial sums of the two squared norms, one pair per block: 2 * 65536 doubles
// = 1 MiB, resident on every GPU that loads the library until the process exits.
static __device__ __align__(256) double g_noalloc_scratch[2 * NA_MAX_BLOCKS];

struct NAParams {
    int nr, nz, nm, nt;
    double r_in, dr, dz;
    double lam[NA_MAX_MODES];    // exact discrete azimuthal eigenvalues
};

__device__ __forceinline__ double na_block_sum(double v, double *red) {
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

// r = b - A_m u with the cell coefficients of the appendix (interior and
// Dirichlet face conductances, mu, lambda_m) evaluated in place; writes the
// block's Parseval-weighted squared norms of r and b into scratch.
__global__ void __launch_bounds__(NA_THREADS)
k_residual_noalloc(const NAParams P, const double2 *__restrict__ u, const double2 *__restrict__ b,
                   double2 *__restrict__ r_out, double *__restrict__ scratch, unsigned total) {
    __shared__ double red[NA_THREADS / 32];
    const unsigned e = blockIdx.x * blockDim.x + threadIdx.x;
    double ar = 0.0, ab = 0.0;
    if (e < total) {
        const unsigned nm = P.nm;
        const unsigned c = e / nm;
        const int m = (int)(e - c * nm);
        const int k = (int)(c / (unsigned)P.nr);
        const int i = (int)(c - (unsigned)k * P.nr);
        const double dr = P.dr, dz = P.dz;
        const double rm = P.r_in + i * dr, rp = P.r_in + (i + 1) * dr, rc = P.r_in + (i + 0.5) * dr;
        const double gw = (i > 0) ? rm * dz / dr : rm * dz / (0.5 * dr);
        const double ge = (i < P.nr - 1) ? rp * dz / dr : rp * dz / (0.5 * dr);
        const double cz = rc * dr / dz;
        const double tz = (P.nz == 1) ? 4.0 : ((k == 0 || k == P.nz - 1) ? 3.0 : 2.0);
        const double d = (gw + ge) + tz * cz + P.lam[m] * (dr * dz / rc);
        const size_t rowstride = (size_t)P.nr * nm;
        double sx = 0.0, sy = 0.0;
        if (k > 0) {
            const double2 v = u[e - rowstride];
            sx += v.x;
            sy += v.y;
        }
        if (k < P.nz - 1) {
            const double2 v = u[e + rowstride];
            sx += v.x;
            sy += v.y;
        }
        const double2 bq = b[e];
        double rx = fma(cz, sx, bq.x), ry = fma(cz, sy, bq.y);
        if (i > 0) {
            const double2 v = u[e - nm];
            rx = fma(gw, v.x, rx);
            ry = fma(gw, v.y, ry);
        }
        if (i < P.nr - 1) {
            const double2 v = u[e + nm];
            rx = fma(ge, v.x, rx);
            ry = fma(ge, v.y, ry);
        }
        const double2 uc = u[e];
        rx = fma(-d, uc.x, rx);
        ry = fma(-d, uc.y, ry);
        if (r_out) r_out[e] = make_double2(rx, ry);
        const double w = (m == 0 || 2 * m == P.nt) ? 1.0 : 2.0;
        ar = w * (rx * rx + ry * ry);
        ab = w * (bq.x * bq.x + bq.y * bq.y);
    }
    const double tr = na_block_sum(ar, red);
    if (threadIdx.x == 0) scratch[blockIdx.x] = tr;
    const double tb = na_block_sum(ab, red);
    if (threadIdx.x == 0) scratch[NA_MAX_BLOCKS + blockIdx.x] = tb;
}

// One CTA: deterministic sums of the nb partials of each norm; writes ||r|| / ||b||.
__global__ void __launch_bounds__(1024) k_finish_noalloc(const double *__restrict__ scratch, int nb, double *rel) {
    __shared__ double red[32];
    double sr = 0.0, sb = 0.0;
    for (int f = threadIdx.x; f < nb; f += blockDim.x) {
        sr += scratch[f];
        sb += scratch[NA_MAX_BLOCKS + f];
    }
    const double tr = na_block_sum(sr, red);
    const double tb = na_block_sum(sb, red);
    if (threadIdx.x == 0) *rel = tb > 0.0 ? sqrt(tr / tb) : sqrt(tr);
}

std::mutex g_na_mutex;
struct NAScratchAddr {
    unsigned long long ctx_id;   // context the address belongs to
    double *ptr;
};
NAScratchAddr g_na_addr[NA_MAX_DEVICES] = {};

using CtxGetCurrentFn = CUresult (*)(CUcontext *);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long *);
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;

// Unique id of the calling thread's current context (0 if none is current).
// A context created after a device reset gets a new id even where its handle
// value repeats, and the library's module -- with the scratch array -- may
// then be loaded at another address.  Called with g_na_mutex held.
int current_context_id(unsigned long long *id) {
    *id = 0;
    if (!g_ctx_get_current || !g_ctx_get_id) {
        cudaDriverEntryPointQueryResult q1, q2;
        void *f1 = nullptr, *f2 = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
            q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2) {
            set_error("driver entry points cuCtxGetCurrent / cuCtxGetId unavailable");
            return PIC_POISSON_ECUDA;
        }
        g_ctx_get_current = (CtxGetCurrentFn)f1;
        g_ctx_get_id = (CtxGetIdFn)f2;
    }
    CUcontext c = nullptr;
    if (g_ctx_get_current(&c) != CUDA_SUCCESS) {
        set_error("cuCtxGetCurrent failed");
        return PIC_POISSON_ECUDA;
    }
    if (c && g_ctx_get_id(c, id) != CUDA_SUCCESS) {
        set_error("cuCtxGetId failed");
        return PIC_POISSON_ECUDA;
    }
    return PIC_POISSON_OK;
}

int lookup_scratch(double **out) {
    void *p = nullptr;
    cudaError_t err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (err != cudaSuccess || !p) {
        set_error("cudaGetSymbolAddress(scratch) failed: %s", cudaGetErrorString(err));
        return PIC_POISSON_ECUDA;
    }
    *out = (double *)p;
    return PIC_POISSON_OK;
}

// Device address of the scratch array in the current context.  Host code
// cannot use the array's name as a device address, so the address is looked
// up with cudaGetSymbolAddress once per device and context, and again when
// the device's context has changed (for instance after cudaDeviceReset).
int noalloc_scratch(double **out) {
    int dev = 0;
    PP_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NA_MAX_DEVICES) {
        set_error("device ordinal %d beyond %d", dev, NA_MAX_DEVICES);
        return PIC_POISSON_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_na_mutex);
    unsigned long long id = 0;
    int rc = current_context_id(&id);
    if (rc) return rc;
    if (id != 0 && g_na_addr[dev].ptr && g_na_addr[dev].ctx_id == id) {
        *out = g_na_addr[dev].ptr;
        return PIC_POISSON_OK;
    }
    double *p = nullptr;
    rc = lookup_scratch(&p);   // also makes the runtime's context current if none was
    if (rc) return rc;
    if (id == 0) {
        rc = current_context_id(&id);
        if (rc) return rc;
    }
    g_na_addr[dev] = NAScratchAddr{id, p};
    *out = p;
    return PIC_POISSON_OK;
}

}  // namespace
}  // namespace pp

extern "C" int pic_poisson_mode_residual_noalloc(const pic_poisson_desc *desc, const double *uhat_dev,
                                                 const double *bhat_dev, double *rhat_dev, double *rel_res_dev,
                                                 void *stream) {
    using namespace pp;
    clear_error();
    if (!desc || !uhat_dev || !bhat_dev || !rel_res_dev) {
        set_error("desc, uhat_dev, bhat_dev and rel_res_dev must be non-NULL");
        return PIC_POISSON_EINVAL;
    }
    const pic_poisson_desc &d = *desc;
    if (d.nr < 1 || d.nz < 1 || d.ntheta < 2 || d.ntheta > 2 * (NA_MAX_MODES - 1) || (d.ntheta & (d.ntheta - 1)) ||
        !(d.r_in > 0) || !(d.r_out > d.r_in) || !(d.z1 > d.z0)) {
        set_error("invalid descriptor (sizes, ntheta a power of two <= %d, 0 < r_in < r_out, z0 < z1)",
                  2 * (NA_MAX_MODES - 1));
        return PIC_POISSON_EINVAL;
    }
    if (d.n_patches > 0 || d.z_faces) {
        set_error("pic_poisson_mode_residual_noalloc does not take a composite domain or non-uniform axial mesh "
                  "(n_patches must be 0, z_faces NULL)");
        return PIC_POISSON_EINVAL;
    }
    if (d.r_faces) {
        set_error("pic_poisson_mode_residual_noalloc needs a uniform radial mesh (r_faces must be NULL)");
        return PIC_POISSON_EINVAL;
    }
    const int nm = d.ntheta / 2 + 1;
    const long total = (long)d.nr * d.nz * nm;
    if (total > NA_MAX_ENTRIES) {
        set_error("pic_poisson_mode_residual_noalloc handles at most %ld mode entries (nr*nz*(ntheta/2+1)); "
                  "got %ld: use pic_poisson_mode_residual with a plan",
                  NA_MAX_ENTRIES, total);
        return PIC_POISSON_EINVAL;
    }
    double *scratch = nullptr;
    int rc = noalloc_scratch(&scratch);
    if (rc) return rc;
    NAParams P{};
    P.nr = d.nr;
    P.nz = d.nz;
    P.nm = nm;
    P.nt = d.ntheta;
    P.r_in = d.r_in;
    P.dr = (d.r_out - d.r_in) / d.nr;
    P.dz = (d.z1 - d.z0) / d.nz;
    if (!std::isfinite(d.theta_span) || !std::isfinite(d.r_in) || !std::isfinite(d.r_out) ||
        !std::isfinite(d.z0) || !std::isfinite(d.z1)) {
        set_error("r_in, r_out, z0, z1 and theta_span must be finite (theta_span <= 0 selects 2 pi)");
        return PIC_POISSON_EINVAL;
    }
    const double span = d.theta_span > 0 ? d.theta_span : 2.0 * 3.14159265358979323846;
    const double da = span / d.ntheta;
    for (int m = 0; m < nm; ++m) {
        const double s = std::sin(3.14159265358979323846 * m / d.ntheta);
        P.lam[m] = 4.0 / (da * da) * s * s;
    }
    const unsigned nb = (unsigned)((total + NA_THREADS - 1) / NA_THREADS);
    const cudaStream_t st = (cudaStream_t)stream;
    k_residual_noalloc<<<nb, NA_THREADS, 0, st>>>(P, (const double2 *)uhat_dev, (const double2 *)bhat_dev,
                                                  (double2 *)rhat_dev, scratch, (unsigned)total);
    k_finish_noalloc<<<1, 1024, 0, st>>>(scratch, (int)nb, rel_res_dev);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) {
        set_error("no-allocation residual launch failed: %s", cudaGetErrorString(err));
        return PIC_POISSON_ECUDA;
    }
    return PIC_POISSON_OK;
}
