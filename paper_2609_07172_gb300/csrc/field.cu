// Face-field reconstruction, the step that follows the Poisson solve in the
// paper's particle-in-cell cycle (Sec. 2: electric fields are stored on cell
// faces): E = -grad phi on every face of the three-dimensional cell grid,
// from the cell-centred potential.  Radial and axial faces use the distances
// of the operator's face conductances (appendix Eqs.
// interior_face_conductances, dirichlet_face_conductances): centre to centre
// between two cells, centre to face on a Dirichlet wall, where the potential
// is the wall value; azimuthal faces the arc r_i dalpha of the angular
// difference (Sec. 3.1), periodic.  So the face fluxes of a cell add up to its
// charge (discrete Gauss law): sum over faces of area E.n = rho V / eps0 for
// the discrete solution.
//
// One thread per cell, r fastest (coalesced): each cell writes its lower r,
// azimuthal (j + 1/2) and lower z face, and the cells next to the upper walls
// also the wall face.  The differences are binary64 (one subtraction and one
// multiplication by a precomputed inverse distance per face), so on this GPU
// the kernel is bound by the FP64 pipe rather than by its 4 arrays of traffic.
// Non-uniform axial faces and composite domains take a variant with an axial
// distance table and, for patches, exposed faces (k_face_field_gen).
#include "plan.h"

namespace pp {
namespace {

struct FieldArgs {
    int nr, nt, nz;
    double inv_dz, inv_hdz;                    // 1 / axial centre distance, 1 / centre-to-wall distance
    const double *inv_rd;                      // [nr + 1] 1 / radial distance across face a
    double phi_z0, phi_z1;
    const double *win, *wout;                  // [nz] r-wall potentials
    const double *inv_rda;                     // [nr] 1 / (r_i dalpha)
    const double *phi;                         // (nz, nt, nr)
    double *er, *ea, *ez;                      // (nz, nt, nr + 1), (nz, nt, nr), (nz + 1, nt, nr)
};

__global__ void __launch_bounds__(256) k_face_field(const FieldArgs a) {
    const unsigned e = blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned nr = (unsigned)a.nr, row_n = (unsigned)a.nz * (unsigned)a.nt;
    if (e >= row_n * nr) return;
    const unsigned row = e / nr;                     // k * nt + j
    const int i = (int)(e - row * nr);
    const int k = (int)(row / (unsigned)a.nt), j = (int)(row - (unsigned)k * a.nt);
    const double p = a.phi[e];
    // radial face i (between cells i - 1 and i; the inner wall for i = 0)
    const size_t fr = (size_t)row * (nr + 1) + i;
    const double pw = i > 0 ? a.phi[e - 1] : a.win[k];
    a.er[fr] = (pw - p) * a.inv_rd[i];
    if (i == a.nr - 1) a.er[fr + 1] = (p - a.wout[k]) * a.inv_rd[a.nr];
    // azimuthal face j + 1/2, periodic
    const int jn = j + 1 == a.nt ? 0 : j + 1;
    a.ea[e] = (p - a.phi[((size_t)k * a.nt + jn) * nr + i]) * a.inv_rda[i];
    // axial face k (between cells k - 1 and k; the wall z0 for k = 0)
    const size_t plane = (size_t)a.nt * nr;
    const double ps = k > 0 ? a.phi[e - plane] : a.phi_z0;
    a.ez[e] = (ps - p) * (k > 0 ? a.inv_dz : a.inv_hdz);
    if (k == a.nz - 1) a.ez[e + plane] = (p - a.phi_z1) * a.inv_hdz;
}

// The same on non-uniform axial faces and composite domains.  Axial
// distances come from a table like the radial ones.  With MASK (a composite
// domain, Sec. 2.2): a face between an active and an inactive cell is a
// Dirichlet face at phi_exposed, differenced from the active cell's centre
// to the face (the distance of the exposed face's conductance); faces with no
// active cell on either side, wall faces of inactive cells included, get
// E = 0.  The plain kernel above is unchanged for plain plans.
struct FieldGenArgs {
    FieldArgs a;
    const double *inv_zd;                      // [nz + 1] 1 / axial distance across face c
    const double *inv_half;                    // 1 / centre-to-face: r lower, r upper [nr]; z lower, z upper [nz]
    const unsigned char *act;                  // [nz][nr] active flags (MASK)
    double pe;                                 // phi_exposed
};

template <bool MASK>
__global__ void __launch_bounds__(256) k_face_field_gen(const FieldGenArgs g) {
    const FieldArgs &a = g.a;
    const unsigned e = blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned nr = (unsigned)a.nr, row_n = (unsigned)a.nz * (unsigned)a.nt;
    if (e >= row_n * nr) return;
    const unsigned row = e / nr;
    const int i = (int)(e - row * nr);
    const int k = (int)(row / (unsigned)a.nt), j = (int)(row - (unsigned)k * a.nt);
    const double p = a.phi[e];
    const bool ai = !MASK || g.act[(size_t)k * nr + i];
    const double *ihr_lo = g.inv_half, *ihr_hi = g.inv_half + a.nr;
    const double *ihz_lo = g.inv_half + 2 * a.nr, *ihz_hi = ihz_lo + a.nz;
    // radial face i
    const size_t fr = (size_t)row * (nr + 1) + i;
    double vr;
    if (i == 0) {
        vr = ai ? (a.win[k] - p) * a.inv_rd[0] : 0.0;
    } else {
        const bool aw = !MASK || g.act[(size_t)k * nr + i - 1];
        if (ai && aw) vr = (a.phi[e - 1] - p) * a.inv_rd[i];
        else if (aw) vr = (a.phi[e - 1] - g.pe) * ihr_hi[i - 1];   // exposed face east of cell i - 1
        else if (ai) vr = (g.pe - p) * ihr_lo[i];                  // exposed face west of cell i
        else vr = 0.0;
    }
    a.er[fr] = vr;
    if (i == a.nr - 1) a.er[fr + 1] = ai ? (p - a.wout[k]) * a.inv_rd[a.nr] : 0.0;
    // azimuthal face j + 1/2, periodic (both cells share the (r, z) cell's activity)
    const int jn = j + 1 == a.nt ? 0 : j + 1;
    a.ea[e] = ai ? (p - a.phi[((size_t)k * a.nt + jn) * nr + i]) * a.inv_rda[i] : 0.0;
    // axial face k
    const size_t plane = (size_t)a.nt * nr;
    double vz;
    if (k == 0) {
        vz = ai ? (a.phi_z0 - p) * g.inv_zd[0] : 0.0;
    } else {
        const bool as = !MASK || g.act[(size_t)(k - 1) * nr + i];
        if (ai && as) vz = (a.phi[e - plane] - p) * g.inv_zd[k];
        else if (as) vz = (a.phi[e - plane] - g.pe) * ihz_hi[k - 1];
        else if (ai) vz = (g.pe - p) * ihz_lo[k];
        else vz = 0.0;
    }
    a.ez[e] = vz;
    if (k == a.nz - 1) a.ez[e + plane] = ai ? (p - a.phi_z1) * g.inv_zd[a.nz] : 0.0;
}

}  // namespace
}  // namespace pp

using namespace pp;

extern "C" int pic_poisson_face_field(pic_poisson_plan_t plan, const double *phi_dev, double *er_dev, double *ea_dev,
                                      double *ez_dev) {
    int rc = plan_enter(plan);
    if (rc) return rc;
    if (plan->n != 1) {
        set_error("pic_poisson_face_field needs a single-problem plan (this plan holds %d problems)", plan->n);
        return PIC_POISSON_EINVAL;
    }
    if (!phi_dev || !er_dev || !ea_dev || !ez_dev) {
        set_error("NULL pointer");
        return PIC_POISSON_EINVAL;
    }
    const ProblemPlan &q = plan->pr[0];
    const LevelHost &h = q.lv[0];
    FieldArgs a{};
    a.nr = h.nr;
    a.nt = q.d.ntheta;
    a.nz = h.nz;
    a.inv_rd = q.finv_rd;
    a.inv_dz = 1.0 / h.dz;
    a.inv_hdz = 1.0 / (0.5 * h.dz);
    a.phi_z0 = q.d.phi_z0;
    a.phi_z1 = q.d.phi_z1;
    a.win = q.fwin;
    a.wout = q.fwout;
    a.inv_rda = q.finv_rda;
    a.phi = phi_dev;
    a.er = er_dev;
    a.ea = ea_dev;
    a.ez = ez_dev;
    const size_t n = (size_t)a.nz * a.nt * a.nr;
    const unsigned grid = (unsigned)((n + 255) / 256);
    if (h.act.empty() && h.zf.empty()) {
        k_face_field<<<grid, 256, 0, plan->stream>>>(a);
    } else {   // non-uniform axial faces and / or a composite domain
        FieldGenArgs g{};
        g.a = a;
        g.inv_zd = q.finv_zd;
        g.inv_half = q.finv_half;
        g.act = q.act0;
        g.pe = q.d.phi_exposed;
        if (q.act0) k_face_field_gen<true><<<grid, 256, 0, plan->stream>>>(g);
        else k_face_field_gen<false><<<grid, 256, 0, plan->stream>>>(g);
    }
    PP_CUDA(cudaGetLastError());
    return PIC_POISSON_OK;
}
