// Cloud-in-cell deposit of macro-particles to the cell-corner nodes and the
// projection of nodal density to cell-centred charge: the steps before the
// Poisson solve in the paper's particle-in-cell cycle (Sec. 2, and Sec.
// "Warp-aggregated cylindrical CIC deposition", Eqs. cic_weights,
// particle_cic_update, warp_aggregated_cic).
//
// Deposit.  A particle in cell (i, j, k) at normalised position (xi, eta,
// zeta) adds W w_r w_alpha w_z / V_nu to each of the cell's eight corner
// nodes (w^(0) = 1 - t, w^(1) = t; V_nu the node's cylindrical control
// volume, from cell centre to cell centre in r and z and cut at the walls, a
// full dalpha in alpha).  Aggregation (Eq. warp_aggregated_cic): a thread
// first sums, in registers, its consecutive particles that share a cell;
// then lanes whose last cells agree -- runs of equal cell labels in lane
// order, which cell-sorted input makes long -- add their sums with a
// segmented scan of register shuffles, and the last lane of each run issues
// the run's eight FP64 atomic additions, each divided by the node's volume
// once.  The weights' products and the sums are double-float (df.h, about
// 48 bits, on the FP32 pipe); the particle's cell and offset and the final
// per-node values are binary64.  All weights and corners stay; only the
// order of the additions changes.  Particles outside the domain deposit
// nothing.
//
// Non-uniform faces and composite domains (k_deposit_faces): the cell comes
// from the face arrays (a bin lookup guesses, binary64 comparisons decide),
// the offsets from the cell's own faces; in a composite domain (Sec. 2.2) a
// particle in an inactive cell deposits nothing and a node's volume counts
// only its octants in active cells, so the projection below conserves the
// active cells' charge; inactive cells get rho = 0.
//
// Projection (Sec. 2, "volume-consistent projection to cell-centred
// charge"; the paper gives no formula -- the reading): each node's control
// volume is split into the octants inside its adjacent cells and an
// octant's charge goes to its cell, rho_q = charge * sum over the corners of
// q of n_nu V_(nu in q) / V_q.  The radial octant share is the exact r dr
// integral of the half cell (f_lo, f_hi below, f_lo + f_hi = 1), the
// azimuthal and axial ones are 1/2; so charge is conserved exactly:
// sum_q rho_q V_q = charge * sum_nu n_nu V_nu.
#include <cmath>

#include "df.h"
#include "plan.h"

namespace pp {
namespace {

struct DepositArgs {
    int nr, nt, nz;
    long long np;
    double r_in, z0, inv_dr, inv_da, inv_dz;
    float w_hi, w_lo;       // the weight W 2^-w_exp in double-float, in [1, 2)
    int w_exp;
    const double *r, *al, *z;
    const double *inv_vr;   // [nr + 1] 1 / (radial integral of r dr of node a's interval)
    const double *inv_vz;   // [nz + 1] 1 / (dalpha * axial length of node c's interval)
    double *nodes;          // (nz + 1, nt, nr + 1)
};

// Non-uniform faces or a composite domain (k_deposit_faces): the cell is found
// on the face arrays -- a lookup bin guesses it, exact comparisons settle it.
struct DepositGeo {
    const double *rf, *zf;          // faces [nr + 1], [nz + 1]
    const double *inv_wr, *inv_wz;  // 1 / cell widths
    const int *rbin, *zbin;         // cell at the lower end of each bin
    int nrbin, nzbin;
    float r0f, z0f, inv_rbw, inv_zbw;
    const unsigned char *act;       // composite: active flags [nz][nr] (null: all active)
    const double *inv_v2;           // composite: 1 / node volumes of active octants [nz + 1][nr + 1]
};

// Cell of coordinate x on faces f[0..n] (max{a : f[a] <= x}), or -1 outside
// [f[0], f[n]).  The binary32 bin lookup only guesses; the binary64
// comparisons against the faces decide, so the cell is exactly the one the
// face array defines (a guess off by any amount still ends right, the loops
// are bounded by n).
__device__ __forceinline__ int find_cell(double x, const double *f, int n, const int *bin, int nbin, float x0,
                                         float inv_bw) {
    if (!(x >= f[0] && x < f[n])) return -1;   // NaN included
    int b = (int)(((float)x - x0) * inv_bw);
    b = b < 0 ? 0 : (b >= nbin ? nbin - 1 : b);
    int a = bin[b];
    while (a > 0 && x < f[a]) --a;
    while (a < n - 1 && x >= f[a + 1]) ++a;
    return a;
}

constexpr int DEP_PPT = 4;   // consecutive particles per thread

// The eight corner contributions W w_r w_alpha w_z 2^-w_exp (corner index
// 4 dz + 2 dalpha + dr) of offsets (xr, xa, xz) in the cell, in double-float
// on the FP32 pipe -- the deposit's FP64 instructions were its bound.
__device__ __forceinline__ bool weights8(const DepositArgs &a, double xr, double xa, double xz, df c[8]) {
    const df r1 = split_scaled(xr, 1023), r0 = split_scaled(1.0 - xr, 1023);
    const df a1 = split_scaled(xa, 1023), a0 = split_scaled(1.0 - xa, 1023);
    const df z1 = split_scaled(xz, 1023), z0 = split_scaled(1.0 - xz, 1023);
    const df w = {a.w_hi, a.w_lo};
    const df wz0 = df_mul(w, z0), wz1 = df_mul(w, z1);
    const df q00 = df_mul(wz0, a0), q01 = df_mul(wz0, a1), q10 = df_mul(wz1, a0), q11 = df_mul(wz1, a1);
    c[0] = df_mul(q00, r0);
    c[1] = df_mul(q00, r1);
    c[2] = df_mul(q01, r0);
    c[3] = df_mul(q01, r1);
    c[4] = df_mul(q10, r0);
    c[5] = df_mul(q10, r1);
    c[6] = df_mul(q11, r0);
    c[7] = df_mul(q11, r1);
    return true;
}

// Cell and corner contributions of particle p; false when p is absent or
// outside.  The position arithmetic (cell, offset in the cell) is binary64.
__device__ __forceinline__ bool cic_weights(const DepositArgs &a, long long p, int &ir, int &ia, int &iz, df c[8]) {
    if (p >= a.np) return false;
    const double tr = (a.r[p] - a.r_in) * a.inv_dr, ta = a.al[p] * a.inv_da, tz = (a.z[p] - a.z0) * a.inv_dz;
    const double fr = floor(tr), fa = floor(ta), fz = floor(tz);
    // in range before any conversion (NaN compares false)
    if (!(fr >= 0.0 && fr < (double)a.nr && fa >= 0.0 && fa < (double)a.nt && fz >= 0.0 && fz < (double)a.nz))
        return false;
    ir = (int)fr;
    ia = (int)fa;
    iz = (int)fz;
    const double xr = tr - fr, xa = ta - fa, xz = tz - fz;   // exact, in [0, 1)
    return weights8(a, xr, xa, xz, c);
}

// The same on face arrays; false also for a particle in an inactive cell.
__device__ __forceinline__ bool cic_weights_faces(const DepositArgs &a, const DepositGeo &g, long long p, int &ir,
                                                  int &ia, int &iz, df c[8]) {
    if (p >= a.np) return false;
    const double r = a.r[p], z = a.z[p], ta = a.al[p] * a.inv_da;
    const double fa = floor(ta);
    if (!(fa >= 0.0 && fa < (double)a.nt)) return false;
    ir = find_cell(r, g.rf, a.nr, g.rbin, g.nrbin, g.r0f, g.inv_rbw);
    iz = find_cell(z, g.zf, a.nz, g.zbin, g.nzbin, g.z0f, g.inv_zbw);
    if (ir < 0 || iz < 0) return false;
    if (g.act && !g.act[(size_t)iz * a.nr + ir]) return false;   // inactive cell: nothing deposited
    ia = (int)fa;
    // the products may round to 1 at the upper face; the weights stay in [0, 1]
    const double xr = fmin((r - g.rf[ir]) * g.inv_wr[ir], 1.0), xz = fmin((z - g.zf[iz]) * g.inv_wz[iz], 1.0);
    return weights8(a, xr, ta - fa, xz, c);
}

// The eight atomic additions of a run's sums to the corners of cell (ir, ia, iz).
__device__ __forceinline__ void add_corners(const DepositArgs &a, int ir, int ia, int iz, const df c[8]) {
    const int ja = ia + 1 == a.nt ? 0 : ia + 1;
    const size_t rs = (size_t)a.nr + 1, ps = (size_t)a.nt * rs;
#pragma unroll
    for (int d = 0; d < 8; ++d) {
        const int nzi = iz + (d >> 2), nai = (d & 2) ? ja : ia, nri = ir + (d & 1);
        atomicAdd(a.nodes + (size_t)nzi * ps + (size_t)nai * rs + nri,
                  to_double(c[d], a.w_exp) * a.inv_vr[nri] * a.inv_vz[nzi]);
    }
}

// The same with the composite domain's node volumes of active octants.
__device__ __forceinline__ void add_corners_faces(const DepositArgs &a, const DepositGeo &g, int ir, int ia, int iz,
                                                  const df c[8]) {
    if (!g.inv_v2) {
        add_corners(a, ir, ia, iz, c);
        return;
    }
    const int ja = ia + 1 == a.nt ? 0 : ia + 1;
    const size_t rs = (size_t)a.nr + 1, ps = (size_t)a.nt * rs;
#pragma unroll
    for (int d = 0; d < 8; ++d) {
        const int nzi = iz + (d >> 2), nai = (d & 2) ? ja : ia, nri = ir + (d & 1);
        atomicAdd(a.nodes + (size_t)nzi * ps + (size_t)nai * rs + nri,
                  to_double(c[d], a.w_exp) * g.inv_v2[(size_t)nzi * rs + nri]);
    }
}

// Each thread takes DEP_PPT consecutive particles and sums those of one cell
// in registers (a cell change inside the chunk sends the finished run's sums
// straight to the nodes); then the threads' last runs are aggregated across
// the warp.
__global__ void __launch_bounds__(256) k_deposit(const DepositArgs a) {
    const long long t0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) * DEP_PPT;
    const int lane = threadIdx.x & 31;
    const unsigned full = 0xffffffffu;
    df acc[8];
#pragma unroll
    for (int d = 0; d < 8; ++d) acc[d] = {0.f, 0.f};
    int cr = 0, ca = 0, cz = 0;
    bool have = false;
#pragma unroll
    for (int t = 0; t < DEP_PPT; ++t) {
        df c[8];
        int ir, ia, iz;
        if (!cic_weights(a, t0 + t, ir, ia, iz, c)) continue;
        if (have && (ir != cr || ia != ca || iz != cz)) {
            add_corners(a, cr, ca, cz, acc);
            have = false;
        }
        if (!have) {
#pragma unroll
            for (int d = 0; d < 8; ++d) acc[d] = c[d];
            cr = ir;
            ca = ia;
            cz = iz;
            have = true;
        } else {
#pragma unroll
            for (int d = 0; d < 8; ++d) acc[d] = df_add(acc[d], c[d]);
        }
    }
    // runs of lanes with the same last cell (lanes with nothing left: a run each)
    const long long label = have ? ((long long)cz * a.nt + ca) * a.nr + cr : -1 - lane;
    const long long prev = __shfl_up_sync(full, label, 1);
    const unsigned heads = __ballot_sync(full, lane == 0 || prev != label);
    const unsigned upto = lane == 31 ? full : ((2u << lane) - 1u);
    const int start = 31 - __clz(heads & upto);   // first lane of this lane's run
#pragma unroll
    for (int d = 0; d < 8; ++d) {
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const df y = {__shfl_up_sync(full, acc[d].hi, off), __shfl_up_sync(full, acc[d].lo, off)};
            if (lane - off >= start) acc[d] = df_add(acc[d], y);
        }
    }
    const bool last = lane == 31 || ((heads >> (lane + 1)) & 1u);
    if (have && last) add_corners(a, cr, ca, cz, acc);
}

// The same on face arrays and composite domains (kept a separate kernel so
// that the plain one's code stays as it is).
__global__ void __launch_bounds__(256) k_deposit_faces(const DepositArgs a, const DepositGeo g) {
    const long long t0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) * DEP_PPT;
    const int lane = threadIdx.x & 31;
    const unsigned full = 0xffffffffu;
    df acc[8];
#pragma unroll
    for (int d = 0; d < 8; ++d) acc[d] = {0.f, 0.f};
    int cr = 0, ca = 0, cz = 0;
    bool have = false;
#pragma unroll
    for (int t = 0; t < DEP_PPT; ++t) {
        df c[8];
        int ir, ia, iz;
        if (!cic_weights_faces(a, g, t0 + t, ir, ia, iz, c)) continue;
        if (have && (ir != cr || ia != ca || iz != cz)) {
            add_corners_faces(a, g, cr, ca, cz, acc);
            have = false;
        }
        if (!have) {
#pragma unroll
            for (int d = 0; d < 8; ++d) acc[d] = c[d];
            cr = ir;
            ca = ia;
            cz = iz;
            have = true;
        } else {
#pragma unroll
            for (int d = 0; d < 8; ++d) acc[d] = df_add(acc[d], c[d]);
        }
    }
    // runs of lanes with the same last cell (lanes with nothing left: a run each)
    const long long label = have ? ((long long)cz * a.nt + ca) * a.nr + cr : -1 - lane;
    const long long prev = __shfl_up_sync(full, label, 1);
    const unsigned heads = __ballot_sync(full, lane == 0 || prev != label);
    const unsigned upto = lane == 31 ? full : ((2u << lane) - 1u);
    const int start = 31 - __clz(heads & upto);   // first lane of this lane's run
#pragma unroll
    for (int d = 0; d < 8; ++d) {
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const df y = {__shfl_up_sync(full, acc[d].hi, off), __shfl_up_sync(full, acc[d].lo, off)};
            if (lane - off >= start) acc[d] = df_add(acc[d], y);
        }
    }
    const bool last = lane == 31 || ((heads >> (lane + 1)) & 1u);
    if (have && last) add_corners_faces(a, g, cr, ca, cz, acc);
}

struct ProjectArgs {
    int nr, nt, nz, accumulate;
    double charge;
    const double *flo, *fhi;   // [nr] radial shares of a cell's lower / upper corner nodes
    const double *nodes;
    double *rho;
    const unsigned char *act;  // MASK: active flags [nz][nr]; inactive cells get no charge
};

template <bool MASK>
__global__ void __launch_bounds__(256) k_project(const ProjectArgs a) {
    const unsigned e = blockIdx.x * blockDim.x + threadIdx.x;   // (k, j, i), i fastest
    const unsigned nr = (unsigned)a.nr;
    if (e >= (unsigned)a.nz * a.nt * nr) return;
    const unsigned row = e / nr;
    const int i = (int)(e - row * nr);
    const int k = (int)(row / (unsigned)a.nt), j = (int)(row - (unsigned)k * a.nt);
    const int jn = j + 1 == a.nt ? 0 : j + 1;
    const size_t rs = nr + 1, ps = (size_t)a.nt * rs;
    const double *n0 = a.nodes + (size_t)k * ps, *n1 = n0 + ps;
    // the four (alpha, z) nodes at radius a = i and at a = i + 1
    const double lo = (n0[j * rs + i] + n0[jn * rs + i]) + (n1[j * rs + i] + n1[jn * rs + i]);
    const double hi = (n0[j * rs + i + 1] + n0[jn * rs + i + 1]) + (n1[j * rs + i + 1] + n1[jn * rs + i + 1]);
    double v = a.charge * 0.25 * (a.flo[i] * lo + a.fhi[i] * hi);
    if (MASK && !a.act[(size_t)k * nr + i]) v = 0.0;
    a.rho[e] = a.accumulate ? a.rho[e] + v : v;
}

}  // namespace
}  // namespace pp

using namespace pp;

namespace {
int single(const pic_poisson_plan_s *P, const char *what) {
    if (P->n != 1) {
        set_error("%s needs a single-problem plan (this plan holds %d problems)", what, P->n);
        return PIC_POISSON_EINVAL;
    }
    return PIC_POISSON_OK;
}
}  // namespace

extern "C" int pic_poisson_deposit(pic_poisson_plan_t plan, const double *r_dev, const double *alpha_dev,
                                   const double *z_dev, long long np, double weight, double *nodes_dev) {
    int rc = plan_enter(plan);
    if (rc) return rc;
    rc = single(plan, "pic_poisson_deposit");
    if (rc) return rc;
    if (np < 0 || (np > 0 && (!r_dev || !alpha_dev || !z_dev)) || !nodes_dev) {
        set_error("pic_poisson_deposit: NULL pointer or negative count");
        return PIC_POISSON_EINVAL;
    }
    const ProblemPlan &q = plan->pr[0];
    if (np == 0) return PIC_POISSON_OK;
    const LevelHost &h = q.lv[0];
    DepositArgs a{};
    a.nr = h.nr;
    a.nt = q.d.ntheta;
    a.nz = h.nz;
    a.np = np;
    a.r_in = q.d.r_in;
    a.z0 = q.d.z0;
    a.inv_dr = 1.0 / h.dr;
    a.inv_da = q.d.ntheta / q.d.theta_span;
    a.inv_dz = 1.0 / h.dz;
    // W = (w_hi + w_lo) 2^w_exp with w_hi + w_lo in [1, 2)
    int e2 = 0;
    const double m = std::frexp(weight, &e2);   // weight = m 2^e2, m in [0.5, 1)
    a.w_exp = e2 - 1;
    const double ws = 2.0 * m;
    a.w_hi = (float)ws;
    a.w_lo = (float)(ws - (double)a.w_hi);
    a.r = r_dev;
    a.al = alpha_dev;
    a.z = z_dev;
    a.inv_vr = q.dep_inv_vr;
    a.inv_vz = q.dep_inv_vz;
    a.nodes = nodes_dev;
    const bool gen = !q.uniform_r || !h.zf.empty() || q.act0;
    DepositGeo g{};
    if (gen) {
        g.rf = q.dep_rf;
        g.zf = q.dep_zf;
        g.inv_wr = q.dep_inv_wr;
        g.inv_wz = q.dep_inv_wz;
        g.rbin = q.dep_rbin;
        g.zbin = q.dep_zbin;
        g.nrbin = q.dep_nrbin;
        g.nzbin = q.dep_nzbin;
        g.r0f = (float)h.rf[0];
        g.z0f = (float)(h.zf.empty() ? q.d.z0 : h.zf[0]);
        g.inv_rbw = q.dep_inv_rbw;
        g.inv_zbw = q.dep_inv_zbw;
        g.act = q.act0;
        g.inv_v2 = q.dep_inv_v2;
    }
    const long long blocks = (np + 256LL * DEP_PPT - 1) / (256LL * DEP_PPT);
    if (blocks > 0x7fffffffLL) {
        set_error("pic_poisson_deposit: too many particles for one launch (%lld)", np);
        return PIC_POISSON_EINVAL;
    }
    if (gen) k_deposit_faces<<<(unsigned)blocks, 256, 0, plan->stream>>>(a, g);
    else k_deposit<<<(unsigned)blocks, 256, 0, plan->stream>>>(a);
    PP_CUDA(cudaGetLastError());
    return PIC_POISSON_OK;
}

extern "C" int pic_poisson_project(pic_poisson_plan_t plan, const double *nodes_dev, double charge, int accumulate,
                                   double *rho_dev) {
    int rc = plan_enter(plan);
    if (rc) return rc;
    rc = single(plan, "pic_poisson_project");
    if (rc) return rc;
    if (!nodes_dev || !rho_dev) {
        set_error("pic_poisson_project: NULL pointer");
        return PIC_POISSON_EINVAL;
    }
    const ProblemPlan &q = plan->pr[0];
    const LevelHost &h = q.lv[0];
    ProjectArgs a{};
    a.nr = h.nr;
    a.nt = q.d.ntheta;
    a.nz = h.nz;
    a.accumulate = accumulate ? 1 : 0;
    a.charge = charge;
    a.flo = q.dep_flo;
    a.fhi = q.dep_fhi;
    a.nodes = nodes_dev;
    a.rho = rho_dev;
    a.act = q.act0;
    const size_t n = (size_t)a.nz * a.nt * a.nr;
    if (q.act0) k_project<true><<<(unsigned)((n + 255) / 256), 256, 0, plan->stream>>>(a);
    else k_project<false><<<(unsigned)((n + 255) / 256), 256, 0, plan->stream>>>(a);
    PP_CUDA(cudaGetLastError());
    return PIC_POISSON_OK;
}
