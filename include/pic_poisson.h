/*
 * pic_poisson -- batched Fourier-mode multigrid field solve for a cylindrical
 * electrostatic particle-in-cell method, on one GB300 (sm_103a).
 *
 * The solve (Sec. 3 "Exact Fourier-mode decomposition and batched
 * matrix-free multigrid"):
 *   1. a real DFT of the cell-centred charge density along the periodic
 *      azimuthal coordinate (Eq. azimuthal_dft, forward scale 1/N_theta),
 *      giving N_m = N_theta/2 + 1 complex modes (Sec. 3.1, last paragraph);
 *   2. for every mode m the shifted real operator A_m = A_0 + lambda_m M
 *      (Eqs. matrix_free_mode_operator, shifted_operator_family) with the
 *      exact discrete eigenvalue lambda_m = 4 sin^2(pi m / N_theta) / dalpha^2
 *      (Eq. discrete_azimuthal_eigenvalue), right-hand side
 *      b = s rho_hat + b^D delta_m0 (Eq. mode_rhs), solved for all modes
 *      together by matrix-free geometric multigrid V-cycles (Sec. 3.3);
 *   3. the inverse transform phi_j = sum_m phi_hat_m e^{i theta_m j}, no scale
 *      (Sec. 3.1, inverse transform).
 *
 * Geometry: a rectangular annular r-z cross-section with uniform spacing,
 * r in [r_in, r_out] (r_in > 0), z in [z0, z1], theta periodic over
 * theta_span.  Walls carry azimuthally invariant Dirichlet potentials; the
 * face conductances are those of the appendix (Eqs.
 * interior_face_conductances, dirichlet_face_conductances).
 *
 * Memory: every pointer argument named *_dev is caller-owned device memory
 * (for example a PyTorch tensor's data_ptr()); the library never frees it.
 * Real 3-D arrays are contiguous FP64, shape (nz, ntheta, nr), r fastest.
 * Mode-space arrays ("mode layout") are contiguous interleaved complex FP64,
 * element (k, i, m) at double offset 2*((k*nr + i)*N_m + m) (+0 real,
 * +1 imaginary): cell-major, mode-fast (Eq. mode_fast_layout with the mode
 * extent unpadded).  A plan owns its workspace (level vectors, coefficient
 * tables, coarse-grid factors), allocated at plan time with cudaMalloc and
 * released by pic_poisson_destroy.  All work is enqueued on the plan's
 * stream; functions that return a result to the host synchronise that stream.
 *
 * Errors: every function returns a PIC_POISSON_* status; no call aborts or
 * traps on the device.  pic_poisson_last_error() describes the most recent
 * failure on the calling thread.
 */
#ifndef PIC_POISSON_H
#define PIC_POISSON_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PIC_POISSON_OK 0
#define PIC_POISSON_EINVAL 1          /* bad descriptor, size or argument */
#define PIC_POISSON_ENOMEM 2          /* device or host allocation failed */
#define PIC_POISSON_ECUDA 3           /* a CUDA call failed (see last_error) */
#define PIC_POISSON_ENOTCONVERGED 4   /* tolerance not met in max_cycles; phi holds the last iterate */
#define PIC_POISSON_ENONFINITE 5      /* non-finite right-hand side or residual */

/* precision */
#define PIC_POISSON_FP64 0            /* every V-cycle in FP64 */
#define PIC_POISSON_MIXED 1           /* FP32 V-cycles inside an FP64 defect-correction loop */

/* flags */
#define PIC_POISSON_USE_INITIAL_GUESS 1u  /* phi_dev is read as the initial iterate */
#define PIC_POISSON_PROFILE 2u            /* time every kernel class with CUDA events (host-driven loop) */
#define PIC_POISSON_GRAPH 4u              /* run each solve as one CUDA graph: the convergence loop is a
                                             device-side while node (captured on the first solve; ignored
                                             together with PIC_POISSON_PROFILE) */
#define PIC_POISSON_HOST_STAGED 8u        /* pic_poisson_solve_host always copies through device staging
                                             buffers (default: mapped page-locked host buffers are read and
                                             written in place by the transforms) */

/* kernel classes, indices into pic_poisson_info.ms_phase / launches_phase */
#define PIC_POISSON_PHASE_FORWARD 0   /* azimuthal rFFT + right-hand side */
#define PIC_POISSON_PHASE_SMOOTH 1    /* red-black Gauss-Seidel half-sweeps, finest level */
#define PIC_POISSON_PHASE_SMOOTH_COARSE 2 /* red-black half-sweeps, coarser levels */
#define PIC_POISSON_PHASE_RESTRICT 3  /* residual + restriction (+ norm partials) */
#define PIC_POISSON_PHASE_COARSE 4    /* coarsest-level direct solve */
#define PIC_POISSON_PHASE_PROLONG 5   /* prolongation + correction */
#define PIC_POISSON_PHASE_NORM 6      /* norm reductions */
#define PIC_POISSON_PHASE_INVERSE 7   /* inverse azimuthal transform */
#define PIC_POISSON_PHASE_DEFECT 8    /* FP64 defect / update of the mixed loop */
#define PIC_POISSON_NPHASE 9

#define PIC_POISSON_MAX_LEVELS 16
#define PIC_POISSON_MAX_BATCH 64      /* problems per batched plan */
#define PIC_POISSON_MAX_PATCHES 64    /* rectangles of one composite domain */
#define PIC_POISSON_MAX_DENSE 1024    /* active cells of a composite domain's coarsest level */

typedef struct pic_poisson_plan_s *pic_poisson_plan_t;

typedef struct {
    int nr, ntheta, nz;        /* cells; ntheta a power of two in [2, 256] */
    double r_in, r_out;        /* radial walls, 0 < r_in < r_out */
    double z0, z1;             /* axial walls, z0 < z1 */
    double theta_span;         /* azimuthal period; <= 0 selects 2*pi */
    double phi_r_in, phi_r_out;/* Dirichlet potential on the r walls (used when the arrays below are NULL) */
    double phi_z0, phi_z1;     /* Dirichlet potential on the z walls */
    const double *phi_r_in_z;  /* host, nz values or NULL: inner r-wall potential per axial cell */
    const double *phi_r_out_z; /* host, nz values or NULL: outer r-wall potential per axial cell */
    const double *r_faces;     /* host, nr + 1 strictly increasing radial faces, or NULL: uniform from r_in
                                  to r_out.  Given, they define r_in and r_out (the fields above are
                                  ignored); cell centres are face midpoints and the coefficients follow
                                  the appendix's face-conductance formulas on them.  The axial spacing
                                  stays uniform.  The no-allocation residual needs uniform faces. */
    const double *z_faces;     /* host, nz + 1 strictly increasing axial faces, or NULL: uniform from z0
                                  to z1.  Given, they define z0 and z1; the coefficients are built row by
                                  row from them (per-row tables, a dense coarsest solve of at most
                                  PIC_POISSON_MAX_DENSE cells).  Not with smooth_fused or the
                                  no-allocation residual. */
    double eps0;               /* vacuum permittivity; <= 0 selects 8.8541878128e-12 F/m */
    int precision;             /* PIC_POISSON_FP64 or PIC_POISSON_MIXED */
    int max_cycles;            /* V-cycle cap; <= 0 selects 200 */
    int pre_sweeps;            /* red-black sweeps before restriction; < 0 selects 2 */
    int post_sweeps;           /* red-black sweeps after prolongation; < 0 selects 2 */
    int inner_cycles;          /* mixed precision: FP32 V-cycles per FP64 defect correction; <= 0 selects 2 */
    int smooth_threads;        /* threads per block of the smoother: 64, 128, 256 or 512; <= 0 selects 256 */
    int smooth_strip;          /* smoother work per thread: <= 0 one entry; 1, 2 or 4: that many rows of one
                                  parity at one (radial cell, mode), loads of the strip issued together */
    double omega;              /* over-relaxation of the red-black smoother, u <- u + omega (u_GS - u),
                                  0 < omega < 2; <= 0 selects 1 (plain Gauss-Seidel) */
    int smooth_fused;          /* mixed precision: 1 runs each pre- or post-smoothing of an FP32 level
                                  (1 or 2 sweeps, omega = 1, even nr) as one fused pass; 0 separate
                                  half-sweeps */
    int local_bottom;          /* 0: the level above the coarsest and the coarsest solve run per mode in
                                  one block's shared memory where they fit (omega = 1, 3 or more levels);
                                  -1: never (separate launches) */
    int fmg;                   /* FP64: 1 starts a solve with a full-multigrid pass: from a zero iterate,
                                  the right-hand side restricted to every level, coarsest solve, then
                                  prolongation and one V-cycle per level up to the finest; from a given
                                  iterate (PIC_POISSON_USE_INITIAL_GUESS, pic_poisson_solve_modes) the
                                  same on its correction equation (its level-0 residual restricted, the
                                  coarser levels as above, the correction prolongated into level 0);
                                  0: no such start */
    int inner_first;           /* mixed precision: FP32 V-cycles of the first defect correction of a solve;
                                  <= inner_cycles (0 included) selects inner_cycles.  A larger first
                                  correction can save one FP64 defect, update and convergence test */
    int n_patches;             /* composite domain (Sec. 2.2): the active r-z cells are the union of
                                  n_patches rectangles of the grid, 0 <= n_patches <= PIC_POISSON_MAX_PATCHES;
                                  0 selects the whole annulus */
    const int *patches;        /* host, 4 ints per patch: i0, i1, k0, k1 -- the cells i0 <= i < i1,
                                  k0 <= k < k1; non-empty, inside the grid, pairwise disjoint (patches
                                  may share faces: a shared face joins them).  A face between an active
                                  and an inactive cell is an exposed face: a Dirichlet face at
                                  phi_exposed with the centre-to-face distance, like a wall face; faces
                                  on the grid's walls keep the wall potentials.  Charge outside the
                                  patches is ignored and phi is returned as 0 there.  Coarsening halves
                                  a direction only while every patch boundary in it lies on a coarse
                                  face (protected faces); the coarsest level is solved densely and may
                                  hold at most PIC_POISSON_MAX_DENSE active cells.  smooth_fused
                                  takes composite domains (per-row coefficient classes); the
                                  no-allocation residual does not. */
    double phi_exposed;        /* Dirichlet potential of the exposed faces (V) */
    unsigned flags;            /* PIC_POISSON_* flags */
} pic_poisson_desc;

typedef struct {
    int status;                /* return code of the call */
    int cycles;                /* coarse-grid corrections applied (to this problem, in a batch) */
    int outer_iterations;      /* FP64 defect corrections (mixed precision) */
    int launches;              /* kernels this call launched */
    double rel_res0;           /* relative residual at the first convergence test: of the initial iterate
                                  (mixed) or after the first pre-smoothing (FP64) */
    double rel_res;            /* ||b - A phi|| / ||b|| of the returned iterate (3-D system, Parseval) */
    double ms_phase[PIC_POISSON_NPHASE];   /* device ms per kernel class (PROFILE flag) */
    int launches_phase[PIC_POISSON_NPHASE];/* launches per kernel class */
    double bytes_phase[PIC_POISSON_NPHASE];/* algorithmic (compulsory) DRAM bytes per kernel class */
    double flops_phase[PIC_POISSON_NPHASE];/* algorithmic floating-point operations per kernel class */
} pic_poisson_info;

#define PIC_POISSON_MAX_TUNE 96

typedef struct {
    int pre_sweeps, post_sweeps;           /* best smoothing schedule */
    int inner_cycles;                      /* best FP32 V-cycles per defect correction (mixed) */
    int inner_first;                       /* best FP32 V-cycles of the first correction (mixed) */
    int smooth_threads;                    /* best smoother block size */
    int smooth_strip;                      /* best smoother strip (0: one entry per thread) */
    double omega;                          /* best over-relaxation factor */
    int smooth_fused;                      /* best fused-smoother setting */
    int fmg;                               /* best full-multigrid start setting (FP64) */
    double ms;                             /* its median wall time per solve call */
    int tried;                             /* candidates timed (entries below) */
    double ms_tried[PIC_POISSON_MAX_TUNE];
    int pre_tried[PIC_POISSON_MAX_TUNE], post_tried[PIC_POISSON_MAX_TUNE];
    int inner_tried[PIC_POISSON_MAX_TUNE], threads_tried[PIC_POISSON_MAX_TUNE];
    int strip_tried[PIC_POISSON_MAX_TUNE];
    double omega_tried[PIC_POISSON_MAX_TUNE];
    int fused_tried[PIC_POISSON_MAX_TUNE];
    int fmg_tried[PIC_POISSON_MAX_TUNE];
    int first_tried[PIC_POISSON_MAX_TUNE];
} pic_poisson_tuning;

typedef struct {
    int levels;                            /* multigrid levels (1 = direct solve only) */
    int nr[PIC_POISSON_MAX_LEVELS];        /* cells per level */
    int nz[PIC_POISSON_MAX_LEVELS];
    int n_modes;                           /* N_theta / 2 + 1 */
    size_t workspace_bytes;                /* device bytes a plan allocates */
} pic_poisson_layout;

/*
 * Validate `desc` and describe the plan it would build (levels, sizes,
 * workspace).  Host only: touches no GPU.  2:1 coarsening in r and z while
 * both counts are even and at least 8 (Sec. 3.2 shared hierarchy); the
 * coarsest level is solved directly.  Returns PIC_POISSON_EINVAL for an
 * invalid descriptor.
 */
int pic_poisson_query(const pic_poisson_desc *desc, pic_poisson_layout *out);

/*
 * Level-0 coefficients of r-z cell (i, k) as the library computes them:
 * out[0..3] = conductance of the r-, r+, z-, z+ faces (Dirichlet faces use the
 * half-cell distance, appendix Eq. dirichlet_face_conductances),
 * out[4..7] = 1 for a Dirichlet face, else 0, out[8] = mu (Eq.
 * mode_mass_coefficient), out[9] = s (Eq. mode_rhs), out[10] = D0 (Eq.
 * base_diagonal_with_boundary), out[11] = b^D (Eq. boundary_rhs_appendix).
 * In a composite domain an exposed face is a Dirichlet face at phi_exposed,
 * and a cell outside the patches returns twelve zeros.
 * Host only.  `out` holds 12 doubles.
 */
int pic_poisson_cell_coeffs(const pic_poisson_desc *desc, int i, int k, double *out);

/*
 * Build a plan: coefficient tables for every level, coarsest-level factors,
 * workspace.  `stream` is a cudaStream_t (NULL = legacy default stream) on
 * which all of the plan's work is enqueued.  On success *out owns the plan.
 */
int pic_poisson_plan(const pic_poisson_desc *desc, void *stream, pic_poisson_plan_t *out);

/*
 * Build one plan for n independent problems (1 <= n <= PIC_POISSON_MAX_BATCH)
 * of different sizes and azimuthal resolutions.  Every kernel launch of a
 * solve covers all problems at once (per launch, each problem owns a range of
 * blocks), so n problems cost one launch per kernel and level, not n.  The
 * problems must share precision, max_cycles, sweeps, inner_cycles and flags.
 */
int pic_poisson_plan_batch(const pic_poisson_desc *descs, int n, void *stream, pic_poisson_plan_t *out);

/* Replace the plan's stream (later calls enqueue there). */
int pic_poisson_set_stream(pic_poisson_plan_t plan, void *stream);

/*
 * Full solve: rho_dev (nz, ntheta, nr) FP64 charge density -> phi_dev (same
 * shape) FP64 potential.  V-cycles run until the relative residual of the
 * three-dimensional system, ||b - A phi||_2 / ||b||_2, is <= tol (tol <= 0:
 * to the rounding floor -- until six convergence tests in a row have not
 * brought the residual below half of its value at the last halving, or
 * max_cycles).  The residual is
 * measured in mode space with Parseval weights 1 (m = 0, N/2) and 2 (others).
 * The convergence test runs on the device; without PIC_POISSON_GRAPH the host
 * reads its flag after every test (one small copy and stream synchronisation
 * per cycle), with it the whole solve is one graph launch.  For a plan with
 * several problems use pic_poisson_solve_batch (this call returns EINVAL).
 * rho_dev and phi_dev may not alias.  `info` may be NULL.  The norms are
 * binary64 sums of squares: right-hand sides whose entries lie outside about
 * 1e-150 .. 1e150 (underflowing or overflowing squares) are not supported.
 * The mixed form computes the forward transform in double-float arithmetic
 * (b to about 1e-14 relative; its result stays within 1e-10 of the FP64 one).
 */
int pic_poisson_solve(pic_poisson_plan_t plan, const double *rho_dev, double *phi_dev, double tol,
                      pic_poisson_info *info);

/*
 * Solve every problem of a batched plan: rho_dev[p] -> phi_dev[p] (host
 * arrays of n device pointers, layouts as for pic_poisson_solve).  Iterates
 * until every problem meets tol; a problem that does is not iterated further
 * (its kernels skip it), so each returned phi is the iterate whose residual is
 * reported.  infos
 * (n entries, may be NULL): per-problem status, cycles and residuals; the
 * timing, byte and launch counters are those of the whole batched solve.
 * Returns ENONFINITE if any problem has it, else ENOTCONVERGED if any, else OK.
 */
int pic_poisson_solve_batch(pic_poisson_plan_t plan, const double *const *rho_dev, double *const *phi_dev,
                            double tol, pic_poisson_info *infos);

/*
 * Autotuner: choose pre/post sweeps, inner_cycles (mixed precision),
 * smooth_threads and smooth_strip for the problems `descs` (as for
 * pic_poisson_plan_batch) by timing complete solves of rho_dev[p] -> phi_dev[p]
 * to `tol` (> 0).  Stage 1 times the schedules (1,1) (2,1) (1,2) (2,2) (3,2)
 * (2,3) (3,3), and for mixed precision 1 to 4 inner cycles each, at 256
 * threads and one entry per thread; stage 2 times 64, 128 and 512 threads for
 * the winner; stage 3 strips of 2 and 4 rows at the best block size; stage 4
 * over-relaxation omega = 1.1, 1.2, 1.3 with the schedules (1,1), (1,2),
 * (2,1), (2,2) at the best block size, strip and inner cycles; stage 5
 * (mixed precision; not with axial faces) the fused smoother with the same
 * four schedules and 1 to 6 inner cycles, or (FP64) the full-multigrid start
 * with the schedules (1,2),
 * (2,1), (2,2); stage 6 (mixed precision) 1 to 3 extra first-correction
 * cycles (inner_first) with the best setting and with one inner cycle fewer.
 * Each
 * candidate builds its own plan, runs
 * one untimed solve and `repeats` (1..16) timed ones; the score is the median
 * wall time of the solve call.  Results in *out; phi_dev is overwritten.
 * This is a project addition for choosing kernel schedules; the paper does
 * not specify its multigrid schedule.
 */
int pic_poisson_autotune(const pic_poisson_desc *descs, int n, const double *const *rho_dev,
                         double *const *phi_dev, double tol, void *stream, int repeats,
                         pic_poisson_tuning *out);

/*
 * As pic_poisson_solve, starting from the mode-layout iterate uhat_guess_dev
 * (e.g. a previous solution from pic_poisson_get_modes, or a learned guess)
 * instead of zero or the transform of phi.  Single-problem plans.  In a
 * composite domain the guess must be zero outside the patches (as the modes
 * of a previous solve are).
 */
int pic_poisson_solve_modes(pic_poisson_plan_t plan, const double *rho_dev, const double *uhat_guess_dev,
                            double *phi_dev, double tol, pic_poisson_info *info);

/*
 * uhat_dev (mode layout) = (1/N_theta) DFT of phi_dev along theta
 * (Eq. azimuthal_dft, without the s_q factor or Dirichlet term of
 * pic_poisson_forward): the mode coefficients of a potential.
 */
int pic_poisson_analyze(pic_poisson_plan_t plan, const double *phi_dev, double *uhat_dev);

/* uhat_dev (mode layout) = the mode-space iterate of the last solve (its
 * converged phi_hat), copied on the plan's stream. */
int pic_poisson_get_modes(pic_poisson_plan_t plan, double *uhat_dev);

/*
 * As pic_poisson_solve with host buffers (pinned or pageable); returns after
 * phi_host is written.  When both buffers are page-locked host memory mapped
 * into the device's address space (cudaHostAlloc / cudaMallocHost, or
 * cudaHostRegister with the mapped flag, under unified addressing) and the
 * plan lacks PIC_POISSON_HOST_STAGED, the forward transform reads rho_host
 * and the inverse transform writes phi_host in place over the CPU-GPU link,
 * so the transfers overlap the transforms' arithmetic.  Otherwise rho_host is
 * copied to a device staging buffer, the solve runs there and phi is copied
 * back; the staging buffers are part of the plan's workspace (allocated on
 * first use).
 */
int pic_poisson_solve_host(pic_poisson_plan_t plan, const double *rho_host, double *phi_host, double tol,
                           pic_poisson_info *info);

/*
 * Cloud-in-cell deposit of one species' macro-particles (the step before the
 * solve in the PIC cycle; Sec. "Warp-aggregated cylindrical CIC deposition",
 * Eqs. cic_weights, particle_cic_update, warp_aggregated_cic).  Particle p at
 * (r_dev[p], alpha_dev[p], z_dev[p]) (device FP64 arrays of np entries, alpha
 * in [0, theta_span)) in cell (i, j, k) at normalised position (xi, eta,
 * zeta) adds weight * w_r w_alpha w_z / V_nu to each of the cell's eight
 * corner nodes, w^(0) = 1 - t, w^(1) = t; V_nu is the node's cylindrical
 * control volume (cell centre to cell centre in r and z, cut at the walls;
 * dalpha in alpha).  The sums are ADDED to nodes_dev, the nodal number
 * density (nz + 1, ntheta, nr + 1) FP64 (node (c, j, a) at z-face c, alpha
 * j dalpha, r-face a), which the caller zeroes before a step's first species.
 * Each thread sums its 4 consecutive particles of one cell in registers, lanes
 * of a warp holding the same cell add their sums with register shuffles, and
 * one lane per run of equal cells issues the eight FP64 atomics, so
 * cell-sorted particles are cheapest; any order is correct (the order of the
 * additions, hence rounding, varies from run to run).  The weights' products
 * and those sums are double-float (about 48 significant bits, ~1e-14
 * relative); cell, offset and the atomics are binary64.
 * Particles outside the domain deposit nothing.  On non-uniform faces
 * (r_faces, z_faces) the cell is the one the face arrays define (max{a :
 * face[a] <= x}, found by a lookup guess and exact binary64 comparisons) and
 * the offsets use that cell's faces.  On a composite domain (patches) a
 * particle in an inactive cell deposits nothing and V_nu counts only the
 * node's octants in active cells, so the projection conserves the active
 * cells' charge exactly.  Single-problem plans; on the plan's stream
 * (asynchronous).
 */
int pic_poisson_deposit(pic_poisson_plan_t plan, const double *r_dev, const double *alpha_dev, const double *z_dev,
                        long long np, double weight, double *nodes_dev);

/*
 * Projection of nodal number density to cell-centred charge density
 * (Sec. 2; reading of the paper's "volume-consistent projection"): each
 * node's control volume is split into the octants in its adjacent cells and
 * an octant's charge goes to its cell,
 *   rho_q = charge * sum over the corners nu of q of n_nu V_(nu in q) / V_q,
 * which conserves charge exactly.  rho_dev (nz, ntheta, nr) FP64 is
 * overwritten (accumulate = 0) or added to (accumulate != 0; e.g. ions, then
 * electrons with the opposite charge).  On a composite domain inactive
 * cells get rho = 0.  Single-problem plans; on the plan's stream
 * (asynchronous).
 */
int pic_poisson_project(pic_poisson_plan_t plan, const double *nodes_dev, double charge, int accumulate,
                        double *rho_dev);

/*
 * Face-field reconstruction, the step after the solve in the PIC cycle
 * (Sec. 2: fields live on cell faces): E = -grad phi on every cell face from
 * the cell-centred potential phi_dev (nz, ntheta, nr), with the plan's wall
 * potentials on the Dirichlet faces.  Writes (caller device memory, FP64):
 *   er_dev (nz, ntheta, nr + 1): radial faces, face i between cells i - 1 and
 *          i (face 0 the inner wall, face nr the outer wall);
 *   ea_dev (nz, ntheta, nr): azimuthal faces j + 1/2 (periodic);
 *   ez_dev (nz + 1, ntheta, nr): axial faces, face k between cells k - 1 and k.
 * Distances as in the operator's face conductances (appendix Eqs.
 * interior_face_conductances, dirichlet_face_conductances): centre to centre,
 * centre to wall at a Dirichlet face, r_i dalpha azimuthally; so for the
 * discrete solution the face fluxes of every cell sum to rho V / eps0.
 * Non-uniform faces use their own centre distances.  On a composite domain
 * (Sec. 2.2) a face between an active and an inactive cell is differenced
 * from the active cell's centre to the face at phi_exposed (the exposed
 * face's Dirichlet distance), and faces with no active cell on either side
 * get E = 0.  Single-problem plans; enqueued on the plan's stream
 * (asynchronous).
 */
int pic_poisson_face_field(pic_poisson_plan_t plan, const double *phi_dev, double *er_dev, double *ea_dev,
                           double *ez_dev);

/*
 * Step a-1 alone: bhat_dev (mode layout) = s * rho_hat + b^D delta_m0 where
 * rho_hat is the forward DFT of rho_dev along theta with scale 1/N_theta
 * (Eqs. azimuthal_dft, mode_rhs).  Imaginary parts of m = 0 and m = N/2 are
 * written as exactly 0.
 */
int pic_poisson_forward(pic_poisson_plan_t plan, const double *rho_dev, double *bhat_dev);

/*
 * Step a-8 alone: phi_dev (nz, ntheta, nr) = sum over all N_theta modes of
 * phihat_m e^{i theta_m j}, using conjugate symmetry for m > N/2 and the real
 * parts of m = 0 and m = N/2 (Sec. 3.1, inverse transform; no scale).
 */
int pic_poisson_inverse(pic_poisson_plan_t plan, const double *phihat_dev, double *phi_dev);

/*
 * Mode-space residual: rhat_dev = bhat_dev - A_m uhat_dev for every mode
 * (Eq. matrix_free_mode_operator) and, if rel_res is non-NULL, the
 * Parseval-weighted ||r|| / ||b|| written to *rel_res (synchronises).
 * rhat_dev may be NULL when only the norm is wanted.
 */
int pic_poisson_mode_residual(pic_poisson_plan_t plan, const double *uhat_dev, const double *bhat_dev,
                              double *rhat_dev, double *rel_res);

/*
 * No-allocation variant of pic_poisson_mode_residual, for callers that cannot
 * call cudaMalloc: a particle-in-cell code that has handed all device memory to
 * its particle arrays at start-up, or a real-time step loop that may not pay
 * cudaMalloc's implicit device synchronisation.  The paper has no counterpart;
 * it is a library utility.
 *
 * Needs no plan: the coefficients of A_m are computed inside the kernel from
 * desc's uniform geometry (only nr, ntheta, nz, r_in, r_out, z0, z1 and
 * theta_span are read; r_faces must be NULL).  Writes rhat_dev = bhat_dev - A_m uhat_dev (mode
 * layout; rhat_dev may be NULL) and *rel_res_dev = Parseval-weighted
 * ||r|| / ||b|| (one device double) on `stream`, asynchronously: the results
 * are valid once the stream's work up to this call has completed.
 *
 * Allocates nothing: its per-block partial sums live in a fixed 1 MiB
 * file-scope device array that every GPU loading the library holds until the
 * process exits.  Limit: nr * nz * (ntheta/2 + 1) <= 16,777,216 mode entries
 * and ntheta <= 256; larger problems are rejected with PIC_POISSON_EINVAL.
 * The first call on a device looks up that array's device address with
 * cudaGetSymbolAddress (device current at the call); make that first call
 * before any stream capture.  The address is kept per device together with
 * the id of the context it was looked up in, and looked up again when the
 * current context differs (after cudaDeviceReset, for example).  Non-finite
 * r_in, r_out, z0, z1 or theta_span are rejected with PIC_POISSON_EINVAL
 * (theta_span <= 0 selects 2 pi).  Every call reuses the same array; each call
 * writes every partial it later reads, so nothing needs clearing, but calls
 * whose work overlaps on the GPU (different streams, or devices sharing a
 * context) race on the array and must be serialised by the caller.
 */
int pic_poisson_mode_residual_noalloc(const pic_poisson_desc *desc, const double *uhat_dev,
                                      const double *bhat_dev, double *rhat_dev, double *rel_res_dev,
                                      void *stream);

/* Release everything the plan owns.  NULL is accepted.
 * The stage calls pic_poisson_forward, pic_poisson_inverse,
 * pic_poisson_mode_residual and pic_poisson_solve_host need a single-problem
 * plan (EINVAL otherwise). */
int pic_poisson_destroy(pic_poisson_plan_t plan);

/* Description of the most recent failure on this thread ("" if none). */
const char *pic_poisson_last_error(void);

/*
 * Measure this GPU's FP64 and FP32 fused-multiply-add throughput (GFLOP/s,
 * 2 flops per FMA) with a register-resident kernel on `stream`: the ALU
 * roofline denominators for FP64-bound kernels.  Synchronises the stream.
 */
int pic_poisson_measure_fma_peaks(void *stream, double *fp64_gflops, double *fp32_gflops);

#ifdef __cplusplus
}
#endif

#endif /* PIC_POISSON_H */
