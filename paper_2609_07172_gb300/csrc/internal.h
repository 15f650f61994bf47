// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "pic_poisson.h"

namespace pp {

// ------------------------------------------------------------------ errors
void set_error(const char *fmt, ...);
void clear_error();

#define PP_CUDA(call)                                                                   \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess) {                                                        \
            ::pp::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),     \
                            __FILE__, __LINE__);                                        \
            return PIC_POISSON_ECUDA;                                                   \
        }                                                                               \
    } while (0)

#define PP_LAUNCH_CHECK()                                                               \
    do {                                                                                \
        cudaError_t e_ = cudaGetLastError();                                            \
        if (e_ != cudaSuccess) {                                                        \
            ::pp::set_error("kernel launch failed: %s (%s:%d)", cudaGetErrorString(e_), \
                            __FILE__, __LINE__);                                        \
            return PIC_POISSON_ECUDA;                                                   \
        }                                                                               \
    } while (0)

// ------------------------------------------------------------------ complex vector types
template <class T> struct V2t;
template <> struct V2t<double> { using type = double2; };
template <> struct V2t<float> { using type = float2; };
template <class T> using V2 = typename V2t<T>::type;

// ------------------------------------------------------------------ one multigrid level
// Coefficients of A_m on a uniform level (appendix Eqs. interior_face_conductances,
// dirichlet_face_conductances), separated by direction:
//   (A_m u)_(i,k) = (D0r_i + tz_k cz_i + lambda_m mu_i) u_(i,k)
//                   - cw_i u_(i-1,k) - ce_i u_(i+1,k) - cz_i (u_(i,k-1) + u_(i,k+1))
// with cw_0 = ce_(nr-1) = 0 (Dirichlet r faces fold into D0r) and the axial
// neighbour terms dropped on the wall rows, whose tz is 3 (one interior face plus
// a half-distance Dirichlet face of conductance 2 cz) instead of 2.
struct LevelHost {
    int nr = 0, nz = 0;
    double r0 = 0, dr = 0, z0 = 0, dz = 0;
    int ncls = 0;                 // distinct axial row classes: min(nz, 3)
    std::vector<double> cw, ce, cz, d0r, mu;   // per radial index
    std::vector<double> tz;       // per class
    std::vector<double> invd, diag;             // [ncls][nr][nm]
    std::vector<double> hw, he, hz;             // [ncls][nr][nm]: cw, ce, cz divided by diag
};

template <class T> struct LevelDev {
    int nr, nz, nm, ncls;
    const T *cw, *ce, *cz;        // [nr]
    const T *invd, *diag;         // [ncls][nr][nm]
    const T *hw, *he, *hz;        // [ncls][nr][nm] off-diagonal conductances / diag
    V2<T> *u;                     // iterate / correction, [nz][nr][nm]
    V2<T> *b;                     // right-hand side, [nz][nr][nm]
    V2<T> *bh;                    // right-hand side / diag, [nz][nr][nm]
};

// Coarsest level: separable direct solve (z eigenbasis, tridiagonal in r).
template <class T> struct CoarseDev {
    int nr, nz, nm;
    const T *V;                   // [nz][nz] orthonormal eigenvectors of the axial operator, V[k*nz+j]
    const T *e;                   // [nr] off-diagonal -ce_i of the radial operator
    const T *piv;                 // [nm][nz][nr] inverse pivots of the Thomas factorisation
    const T *cpr;                 // [nm][nz][nr] upper multipliers of the Thomas factorisation
};

// ------------------------------------------------------------------ kernels (launchers)
// All launchers enqueue on `st` and return cudaGetLastError().
struct FFTDev {
    int nt;                       // N_theta
    const double *tw;             // [max(M/2,1)] e^{-2 pi i t / M}, M = N_theta/2, as (cos, sin) pairs
    const double *tw2;            // [M+1] e^{-2 pi i m / N_theta}
};

// bh (may be null): also write bhat / diag using the level-0 table invd [ncls][nr][nm].
cudaError_t launch_forward(const double *rho, double2 *bhat, int nr, int nt, int nz, const FFTDev &f,
                           const double *s, const double *bD, double *partials, int *nblocks,
                           double2 *bh, const double *invd, int ncls, cudaStream_t st);
cudaError_t launch_inverse(const double2 *uhat, double *phi, int nr, int nt, int nz, const FFTDev &f,
                           cudaStream_t st);

template <class T>
cudaError_t launch_smooth(const LevelDev<T> &L, int color, cudaStream_t st);
// red_only: residual of the red fine cells only (valid right after a black half-sweep).
// init: 0 = coarse b only; 1 = also b_hat and u = 0; 2 = also b_hat and u = (red ? b_hat : 0).
template <class T>
cudaError_t launch_residual_restrict(const LevelDev<T> &L, const LevelDev<T> &C, int nt, bool red_only, int init,
                                     double *partials, int *nblocks, cudaStream_t st);
template <class T>
cudaError_t launch_residual(const LevelDev<T> &L, V2<T> *r, int nt, double *partials, int *nblocks,
                            cudaStream_t st);
template <class T>
cudaError_t launch_prolong(const LevelDev<T> &L, const LevelDev<T> &C, bool black_only, cudaStream_t st);
template <class T>
cudaError_t launch_coarse(const LevelDev<T> &L, const CoarseDev<T> &C, cudaStream_t st);

cudaError_t launch_defect(const LevelDev<double> &D, const LevelDev<float> &S, double sigma, int nt, bool init_red,
                          double *partials, int *nblocks, cudaStream_t st);
cudaError_t launch_update(const LevelDev<double> &D, const LevelDev<float> &S, double inv_sigma, cudaStream_t st);
cudaError_t launch_sum(const double *partials, int n, double *out, cudaStream_t st);

cudaError_t measure_fma(cudaStream_t st, double *fp64_gflops, double *fp32_gflops);

}  // namespace pp
