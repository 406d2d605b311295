/*
 * swnmg.h -- C ABI of the GB300 Newton multigrid library for steady shallow
 * water flow with topography and wet/dry areas (Wu & Tang, arXiv:1608.06721).
 *
 * The problem (Section 2.2): given a uniform 1D or 2D Cartesian mesh, the bed
 * z at cell centres, boundary data and an initial state, find the cell
 * averages U with R(U) = 0, where R is the well-balanced finite-volume
 * residual of eq. Res (eq. DSeqs with eq. totalFlux).
 *
 * Conventions for every entry point:
 *   - cell index i = ix + nx*iy (x fastest); 1D problems have ny = 1;
 *   - states and vectors are SoA device arrays of ncomp*n doubles, component c
 *     of cell i at [c*n + i]; 1D: (h, hu), 2D: (h, hu, hv);
 *   - device pointers are owned by the caller and must stay valid for the
 *     call; the context owns its workspace (allocated in swnmg_create, freed
 *     in swnmg_destroy);
 *   - all work is issued on the stream given to swnmg_create; a call returns
 *     after its results are complete on that stream unless stated otherwise;
 *   - functions never abort or trap: failures return a status code and
 *     swnmg_last_error() describes the last failure of that context;
 *   - there is no CPU fallback: without a usable CUDA device every call that
 *     needs one returns SWNMG_ERR_CUDA.
 */
#ifndef SWNMG_H
#define SWNMG_H

#include <stdint.h>

#ifdef __cplusplus
#define SWNMG_API extern "C" __attribute__((visibility("default")))
#else
#define SWNMG_API __attribute__((visibility("default")))
#endif

typedef enum {
  SWNMG_OK = 0,
  SWNMG_ERR_ARG = 1,            /* invalid argument or unsupported size */
  SWNMG_ERR_CUDA = 2,           /* CUDA runtime error (text in swnmg_last_error) */
  SWNMG_ERR_NOT_CONVERGED = 3,  /* max_newton reached */
  SWNMG_ERR_NONFINITE = 4,      /* NaN/Inf in the state or residual */
  SWNMG_ERR_DIVERGED = 5,       /* sum ||R_i||_1 grew 1e6x above its minimum */
  SWNMG_ERR_TIMEOUT = 6,        /* a device-side wait ran out of its bound */
  SWNMG_ERR_OOM = 7             /* device allocation failed */
} swnmg_status;

/* boundary kinds, Remark 2.3 */
enum {
  SWNMG_BC_WALL_REFLECT = 0,     /* h_g = h_I, u_n,g = -u_n,I, u_tau,g = u_tau,I */
  SWNMG_BC_WALL_SLIP = 1,        /* h_g = h_I, u_n,g = 0, u_tau,g = u_tau,I */
  SWNMG_BC_INFLOW_DISCHARGE = 2, /* subcritical inflow: discharge q and u_tau prescribed */
  SWNMG_BC_OUTFLOW_DEPTH = 3,    /* subcritical outflow: depth h prescribed */
  SWNMG_BC_SUPER_INFLOW = 4,     /* supercritical inflow: h, q, u_tau prescribed */
  SWNMG_BC_SUPER_OUTFLOW = 5,    /* supercritical outflow: ghost = interior */
  SWNMG_BC_AUTO_FROUDE = 6       /* open boundary: one of kinds 2-5 chosen per evaluation by the
                                    interior's Froude number (|u|^2 >= g h: supercritical) and the
                                    sign of its outward normal velocity (< 0: inflow); uses h, q, ut */
};

/* numerical fluxes, Remark 2.2 */
enum { SWNMG_FLUX_HLL = 0, SWNMG_FLUX_HLLC = 1, SWNMG_FLUX_LLF = 2, SWNMG_FLUX_ROE = 3 };
enum { SWNMG_INIT_CASCADE = 0, SWNMG_INIT_NONE = 1 };   /* Algorithm 1 Step 1, or warm start */
/* MIXED: FP32 multigrid inner solve.  MIXED_STEP1: MIXED, and Step 1's
 * BLU-SGS sweeps on the coarse levels (l >= 1) in FP32 (finite-difference
 * step 2^-12, singular-pivot guard 1e-6 max|D|; the state stays FP64).
 * Batches take MIXED_STEP1 as MIXED. */
enum { SWNMG_PREC_FP64 = 0, SWNMG_PREC_MIXED = 1, SWNMG_PREC_MIXED_STEP1 = 2 };

/* Boundary data of one side.  q is the discharge along the +axis direction
 * (hu on the W/E sides, hv on S/N), so an inflow through the west side has
 * q > 0; ut is the prescribed tangential velocity. */
typedef struct { int32_t kind; double h, q, ut; } swnmg_bc;

/* Uniform mesh on [x0,x1] x [y0,y1] (1D: [x0,x1], ny = 1), gravity g,
 * boundary sides ordered W, E, S, N.  nx (and ny) must be divisible by
 * 2^n_levels (the coarse meshes aggregate 2 or 2x2 cells, Section 2.3). */
typedef struct {
  int32_t dim, nx, ny;
  double x0, x1, y0, y1, g;
  swnmg_bc bc[4];
} swnmg_problem;

/* Solver parameters; swnmg_default_params gives the paper's values
 * (Section 3 preamble): alpha = 3, fd_eps = 1e-8, tau = 1, h_eps = 1e-6,
 * eps_r = 0.03, eps_p = 0.2, N_mg = 2 (1D) / 3 (2D), N_L = 3, V-cycle,
 * eps_f = 0.4 (Roe flux, Remark 2.2).
 *   llf_wetdry    1: add eps_r sqrt(g max h) to the LLF speed on every edge
 *   tol           stop when sum_i ||R_i||_1 < tol (Step 3)
 *   nu1, nu2      symmetric block-SGS sweeps before/after the coarse correction
 *   gamma         1: V-cycle, 2: W-cycle (Algorithm 0)
 *   coarse_sweeps 2D coarsest level: this many symmetric SGS sweeps
 *                 (1D coarsest levels are solved exactly)
 *   eps_p         Step 1 stops on level l once sum_i ||R_{i,l}||_1 < eps_p 2^-l;
 *                 eps_p < 0 selects the paper's rule (its remark on Step 1:
 *                 about one percent of the initial data's residual), i.e.
 *                 |eps_p| x sum_i ||R_i||_1 of the initial data on level 0
 *                 (per problem in a batch)
 *   max_blusgs    cap of BLU-SGS sweeps per level in Step 1
 *   smoother      order of the block SGS smoother: SWNMG_SMOOTH_LEX (0, the
 *                 paper's lexicographic sweeps, Section 2.3) or
 *                 SWNMG_SMOOTH_COLOUR (1, a variant that is not in the
 *                 paper: cells of colour (ix + iy) mod 2, colour 0 then 1
 *                 forward, 1 then 0 backward; its iterates differ) */
typedef struct {
  int32_t flux, llf_wetdry;
  double alpha, fd_eps, tau, h_eps, eps_r, eps_p, tol;
  int32_t n_levels, n_mg, nu1, nu2, gamma, coarse_sweeps, max_newton, max_blusgs,
      init_mode, precision;
  double eps_f;   /* Harten's entropy-fix width of the Roe flux (paper: 0.4) */
  int32_t smoother;
} swnmg_params;

enum { SWNMG_SMOOTH_LEX = 0, SWNMG_SMOOTH_COLOUR = 1 };

#define SWNMG_HIST 512
typedef struct {
  int32_t status, n_newton, n_vcycles;
  int32_t blusgs_sweeps[16];     /* Step 1 sweeps per level */
  double init_res, final_res;    /* sum ||R_i||_1 before Step 2 and at exit */
  double res_hist[SWNMG_HIST];   /* sum ||R_i||_1 after Newton step k+1 */
  double ms_step1, ms_newton;    /* wall time of Step 1 and of Steps 2-3 */
} swnmg_stats;

typedef struct swnmg_ctx swnmg_ctx;

/* Fills *out with the paper's parameters for dim (1 or 2). */
SWNMG_API swnmg_status swnmg_default_params(int32_t dim, swnmg_params* out);

/* Creates a solver context for one problem: validates sizes, allocates the
 * operator hierarchy and workspace on the current device, copies z_dev
 * (n doubles) and builds the coarse beds by averaging (Algorithm 1, Step 1).
 * stream: a cudaStream_t (NULL = legacy default stream). */
SWNMG_API swnmg_status swnmg_create(const swnmg_problem* prob, const swnmg_params* prm,
                                    const double* z_dev, void* stream, swnmg_ctx** out);

SWNMG_API swnmg_status swnmg_destroy(swnmg_ctx* ctx);

/* Text of the last failure of ctx (static storage when ctx is NULL). */
SWNMG_API const char* swnmg_last_error(const swnmg_ctx* ctx);

/* Replaces the parameters; n_levels, precision and dim-dependent sizes must
 * not change (SWNMG_ERR_ARG otherwise). */
SWNMG_API swnmg_status swnmg_set_params(swnmg_ctx* ctx, const swnmg_params* prm);

/* Puts a 2D context on a structured curvilinear quadrilateral mesh (the
 * meshes of Examples 3.4 and 3.5): eq. totalFlux with each edge's own length
 * |e_ij| and unit normal n_ij, and each cell's own area |K_i|.
 * vx_host, vy_host: (nx+1)*(ny+1) vertex coordinates each, vertex (a, b) at
 * index a + (nx+1)*b, copied; cell (ix, iy) has the corners (ix, iy),
 * (ix+1, iy), (ix+1, iy+1), (ix, iy+1), counter-clockwise.  Level l uses every
 * 2^l-th vertex.  Edges are the straight segments between vertices, the
 * normal points from the lower-index cell to the higher-index one, and the
 * edge frame's tangent is the normal turned by +90 degrees on W/E edges and
 * by -90 degrees on S/N edges, so that a boundary's q is the discharge along
 * that normal and its ut the velocity along that tangent.  Step 1 averages
 * the children by area, and swnmg_time_step uses |K_i|/dt per cell.  Call
 * it after swnmg_create, before solving; calling it again replaces the mesh.
 * SWNMG_ERR_ARG for a 1D context, a null pointer, or a mesh with a
 * zero-length edge or a cell of non-positive area on any level (the context
 * then stays on its uniform mesh).  swnmg_adjoint then returns SWNMG_ERR_ARG
 * (built for uniform meshes only).  Synchronises the stream. */
SWNMG_API swnmg_status swnmg_set_mesh(swnmg_ctx* ctx, const double* vx_host, const double* vy_host);

/* eq. Res on the finest mesh: R_dev (ncomp*n) = R(U_dev); rnorm_dev (n,
 * nullable) = ||R_i||_1; l1_host (nullable) = sum_i ||R_i||_1 (this one
 * synchronises the stream). */
SWNMG_API swnmg_status swnmg_residual(swnmg_ctx* ctx, const double* U_dev, double* R_dev,
                                      double* rnorm_dev, double* l1_host);

/* eq. NewtonREG assembled at U_dev: finite-difference blocks (eq. NumerDiff,
 * boundary edges with the ghost recomputed, epsilon = fd_eps) plus
 * alpha ||R_i||_1 on the diagonal, the Galerkin hierarchy of eq. ProjectAR and
 * the block LU factors, all kept in ctx for swnmg_vcycle / swnmg_sgs_sweep. */
SWNMG_API swnmg_status swnmg_jacobian(swnmg_ctx* ctx, const double* U_dev);

/* Copies the level-l operator to host memory in the layout
 * out[((i*5 + b)*nc + s)*nc + k], b = 0 diagonal (with the regularisation),
 * 1 W, 2 E, 3 S, 4 N (zero on the boundary); FP32 blocks are widened. */
SWNMG_API swnmg_status swnmg_get_blocks(swnmg_ctx* ctx, int32_t level, double* host_out);

/* Runs ncycles of Algorithm 0 (gamma-cycle, block SGS smoothing, restriction
 * and Galerkin operators of eq. ProjectAR, correction of eq. correction) on
 * A dU = rhs with the operators of the last swnmg_jacobian; dU_dev is the
 * initial guess and the result (ncomp*n doubles; FP32 internally in MIXED). */
SWNMG_API swnmg_status swnmg_vcycle(swnmg_ctx* ctx, const double* rhs_dev, double* dU_dev,
                                    int32_t ncycles);

/* One block Gauss-Seidel sweep (forward = lexicographic, 0 = reverse) of
 * the level-l operator on x_dev (ncomp*n_l doubles) for right-hand side
 * rhs_dev; the smoother of Section 2.3, exposed for testing. */
SWNMG_API swnmg_status swnmg_sgs_sweep(swnmg_ctx* ctx, int32_t level, const double* rhs_dev,
                                       double* x_dev, int32_t forward);

/* nsweeps symmetric BLU-SGS sweeps (Algorithm 1, Steps 1 and 2.1) on U_dev
 * at level l (ncomp*n_l doubles, bed = the averaged level-l bed):
 * U_i <- U_i - (alpha||R_i||_1 I + dR_i/dU_i)^{-1} R_i in lexicographic order
 * then reverse, each followed by the dry reset of Remark 2.5. */
SWNMG_API swnmg_status swnmg_blusgs(swnmg_ctx* ctx, double* U_dev, int32_t level,
                                    int32_t nsweeps);

/* Algorithm 1 (NMGM): U_dev holds the initial data on entry and the steady
 * state on return; st (nullable) receives the counters and residual history.
 * Returns SWNMG_OK on convergence (sum ||R_i||_1 < tol). */
SWNMG_API swnmg_status swnmg_solve(swnmg_ctx* ctx, double* U_dev, swnmg_stats* st);

/* One implicit (beta = 0) or semi-implicit (0 < beta < 1) time step of the
 * time-dependent equations, Remark 2.6:
 *   |K_i| (U^{n+1} - U^n)/dt + beta R(U^n) + (1 - beta) R(U^{n+1}) = 0,
 * with |K_i| the cell measure (the remark's displayed equation leaves it out
 * of the time difference; the finite-volume form has it).  The nonlinear
 * system is solved by Steps 2-3 of Algorithm 1 from U^{n+1} = U^n (no Step 1):
 * BLU-SGS and the multigrid work on the step's residual and its Jacobian
 * |K_i|/dt I + (1 - beta) J, regularised by alpha ||R_i||_1 of the step's
 * residual; the stop test is sum_i ||R_i||_1 < tol on that residual.
 *   U_dev  (ncomp*n) U^n on entry, U^{n+1} on return
 *   dt > 0, 0 <= beta < 1; st (nullable) as for swnmg_solve
 * Returns as swnmg_solve.  The context's other entry points stay steady. */
SWNMG_API swnmg_status swnmg_time_step(swnmg_ctx* ctx, double* U_dev, double dt, double beta,
                                       swnmg_stats* st);

/* Kernel classes timed by swnmg_set_timing (CUDA events on the context's
 * stream around each launch of that class). */
enum {
  SWNMG_T_RESIDUAL = 0,     /* residual (eq. Res) */
  SWNMG_T_JACOBIAN = 1,     /* FD Jacobian + regularisation, level 0 */
  SWNMG_T_GALERKIN = 2,     /* coarse operators and block LU of all levels */
  SWNMG_T_SGS_FINE = 3,     /* block SGS half-sweep on level 0 */
  SWNMG_T_SGS_COARSE = 4,   /* block SGS half-sweeps on levels >= 1 */
  SWNMG_T_TRANSFER = 5,     /* restriction, prolongation, zero fill */
  SWNMG_T_BLUSGS = 6,       /* BLU-SGS half-sweep on level 0 (Step 2.1) */
  SWNMG_T_UPDATE = 7,       /* Newton update */
  SWNMG_T_COARSE_EXACT = 8, /* exact coarsest-level solve */
  SWNMG_T_BLUSGS_COARSE = 9,/* BLU-SGS half-sweeps on levels >= 1 (Step 1) */
  SWNMG_T_COUNT = 10
};

/* Enables (1) or disables (0) per-class kernel timing and clears the totals. */
SWNMG_API swnmg_status swnmg_set_timing(swnmg_ctx* ctx, int32_t enable);

/* Accumulated device milliseconds, launch counts and cells processed (the
 * level's cells summed over the timed launches) per class since the last
 * swnmg_set_timing(ctx, 1); each array holds SWNMG_T_COUNT entries.
 * Synchronises the stream. */
SWNMG_API swnmg_status swnmg_get_timing(swnmg_ctx* ctx, double* ms_out, int64_t* launches_out,
                                        double* cells_out);

/* Total number of CUDA kernels this library has launched in this process
 * (all contexts); differences around a region count its launches. */
SWNMG_API int64_t swnmg_launch_count(void);

/* Failure detection (not in the paper).  Every device-side wait of the
 * wavefront sweeps (a strip waiting on its predecessor's progress flag, a
 * warp waiting on its staged operator copy, the BLU-SGS grid barrier) polls
 * at most `polls` times; then the sweep stops, sets a sticky flag, and the
 * call returns SWNMG_ERR_TIMEOUT (the context stays usable; the output of
 * the interrupted sweep is undefined).  polls <= 0 restores the default,
 * 2^22 polls, seconds of waiting.  The limit is process-wide, read when a
 * launch is enqueued (a captured CUDA graph keeps the value it was captured
 * with), and exists so that a test can make a wait run out; warps that gave
 * up still wait for their own in-flight copies, under a separate bound,
 * before they exit.  Returns the previous limit. */
SWNMG_API int32_t swnmg_set_wait_limit(int32_t polls);

/* Measures the FP64 issue rate of the current device (a measurement utility
 * with no counterpart in the paper; the roofline denominator of the kernels
 * bound by the FP64 pipe).  op 0: independent chains of fused multiply-adds,
 * op 1: of additions; eight chains per thread, eight blocks of 256 threads
 * per SM, best of three timed launches after a warm-up (CUDA events on the
 * legacy default stream).  *lane_ops_per_s receives the lane operations per
 * second (an FMA counts once).  Synchronises the device; SWNMG_ERR_ARG for
 * a bad op or a null pointer. */
SWNMG_API swnmg_status swnmg_fp64_rate(int32_t op, double* lane_ops_per_s);

/* The residual of swnmg_residual (eq. Res, same kernels, same bits) for
 * callers that cannot allocate device memory: code inside a runtime that
 * owns all device memory through its own pool, and loops that cannot take
 * cudaMalloc/cudaFree's implicit device synchronisation.  The paper has no
 * counterpart: it is an interface convenience only.  The call enqueues
 * kernels, so like any CUDA call it must not be made from a stream callback
 * or a cudaLaunchHostFunc function.
 *
 * Needs no context.  Inputs and outputs are the caller's device arrays: z
 * (n), U (ncomp*n), R (ncomp*n), rnorm (n, nullable: ||R_i||_1), l1_dev
 * (one double, nullable: sum_i ||R_i||_1).  Work is enqueued on `stream`
 * (a cudaStream_t, NULL = legacy default) and the call returns without
 * waiting.  Scratch comes from one fixed device array of 2^20 doubles
 * (8 MiB) that every GPU loading the library keeps until the process exits;
 * a grid needs 2*ncomp*(edges) + 1024 doubles of it (+ n when rnorm is
 * NULL): up to 294x294 cells in 2D with rnorm, 283x283 without.  Larger
 * grids return SWNMG_ERR_ARG with the reason in swnmg_last_error(NULL).
 *
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current).  With CUDA's lazy module
 * loading that lookup loads the library's device code and commits the 8 MiB,
 * which can block or fail (SWNMG_ERR_OOM when memory is short), so "allocates
 * nothing" holds from the second call on: make one untimed warm-up call per
 * device, before any stream capture.  The looked-up address is cached per
 * device for the life of the process and does not survive cudaDeviceReset
 * (or any reset of the primary context); do not call this function after
 * one.  All calls share the one array, so calls that may overlap on the GPU
 * (other streams, other host threads) race and must be serialised by the
 * caller. */
SWNMG_API swnmg_status swnmg_residual_noalloc(const swnmg_problem* prob, const swnmg_params* prm,
                                              const double* z_dev, const double* U_dev,
                                              double* R_dev, double* rnorm_dev, double* l1_dev,
                                              void* stream);

/* Discrete adjoint of the steady state (an extension; the paper solves the
 * forward problem only).  At a steady state U* (R(U*, z, q) = 0) and for a
 * loss L(U*, z, q) with gradient g = dL/dU, the implicit function theorem
 * gives dL/dz = (direct part) - lambda^T dR/dz and dL/dq = -lambda^T dR/dq,
 * where lambda solves J^T lambda = g and J is the regularised
 * finite-difference Jacobian of eq. NewtonREG at U* (the alpha||R_i||_1 term
 * vanishes at a steady state).  lambda is found by Algorithm 0 applied to
 * J^T: the transposed Galerkin hierarchy (P^T J^T P = (P^T J P)^T, eq.
 * ProjectAR) with block SGS on J^T, in FP64 whatever the precision of ctx.
 *
 *   U_dev     (ncomp*n) the steady state, usually the output of swnmg_solve
 *   g_dev     (ncomp*n) dL/dU
 *   lam_dev   (ncomp*n) out: lambda, cycles started from lambda = 0
 *   gz_dev    (n) out: -lambda^T dR/dz, one value per cell bed: the part of
 *             dL/dz that flows through U* (add the loss's direct dL/dz)
 *   gq_host   (4 doubles, nullable) out: -lambda^T dR/dq = dL/dq of each
 *             side's prescribed discharge (sides W, E, S, N; 0 unless the
 *             side is SWNMG_BC_INFLOW_DISCHARGE)
 *   max_cycles cycles of Algorithm 0 at most (>= 1)
 *   rtol      > 0: stop once sum_i ||(g - J^T lambda)_i||_1 <= rtol *
 *             sum_i ||g_i||_1 (checked after every cycle);
 *             <= 0: run exactly max_cycles cycles
 *   cycles_out (nullable) cycles run
 * dR/dz and dR/dq are central differences with step 1e-6 of the edge terms
 * of eq. Res.  The FP64 transposed hierarchy is allocated on the first call
 * and kept in ctx; the forward operators of swnmg_jacobian are left
 * untouched.  Returns SWNMG_ERR_NOT_CONVERGED (with the outputs written) if
 * rtol > 0 is not met within max_cycles, SWNMG_ERR_NONFINITE if the linear
 * residual is not finite.  Synchronises the stream. */
SWNMG_API swnmg_status swnmg_adjoint(swnmg_ctx* ctx, const double* U_dev, const double* g_dev,
                                     double* lam_dev, double* gz_dev, double* gq_host,
                                     int32_t max_cycles, double rtol, int32_t* cycles_out);

/* ---- batches: many independent 2D problems solved together --------------
 * The batched form of Algorithm 1 (an extension; the paper solves one
 * problem at a time).  B problems -- 2D, any sizes, each with its own bed,
 * boundary data and number of levels -- share the other solver parameters.
 * Every step of Algorithm 1 runs for all of them in lockstep: each kernel
 * launch covers every problem still iterating (a per-problem work list), so
 * the wavefront sweeps of small levels and small problems fill the GPU
 * together.  Each problem goes through exactly the steps, stop tests and
 * arithmetic of swnmg_solve on its own and ends bit-identical to it.
 * Restrictions: dim = 2, 1 <= B <= 256, one stream; the coarsest level of
 * every problem is solved by the guarded inverse (coarse_sweeps <= 0 and at
 * most 128 coarsest cells) or, for all problems alike, by coarse_sweeps
 * symmetric SGS sweeps (coarse_sweeps > 0). */
typedef struct swnmg_batch swnmg_batch;

/* Creates a batch: probs[B]; n_levels[B] replaces prm->n_levels per problem
 * (each nx, ny divisible by 2^n_levels[p]); z_dev[B] are the beds (n_p
 * doubles each, copied).  Allocates one context's workspace per problem. */
SWNMG_API swnmg_status swnmg_batch_create(const swnmg_problem* probs, const int32_t* n_levels, int32_t B,
                                          const swnmg_params* prm, const double* const* z_dev,
                                          void* stream, swnmg_batch** out);

SWNMG_API swnmg_status swnmg_batch_destroy(swnmg_batch* bt);

/* Text of the last failure of bt (static storage when bt is NULL). */
SWNMG_API const char* swnmg_batch_last_error(const swnmg_batch* bt);

/* Algorithm 1 for every problem: U_dev[p] (3*n_p doubles) holds the initial
 * data on entry and the steady state on return; stats (nullable) receives B
 * records.  Returns SWNMG_OK when every problem converged, otherwise the
 * status of the first problem that did not (all statuses are in stats). */
SWNMG_API swnmg_status swnmg_batch_solve(swnmg_batch* bt, double* const* U_dev, swnmg_stats* stats);

/* 1: run the N_mg cycles of each Newton step from a CUDA graph captured on
 * first use (one graph for the whole batch: the per-problem masks it reads
 * are device arrays); 0: launch them one by one.  Results are identical. */
SWNMG_API swnmg_status swnmg_batch_set_graph(swnmg_batch* bt, int32_t enable);

/* Autotuner: times the candidate shared-memory staging depths of the SGS
 * sweep and the candidate BLU-SGS grid sizes (a quarter of the SMs up to
 * the co-resident limit) on every level of this batch (BLU-SGS on scratch
 * copies of U_dev, which is not modified) and keeps the fastest per level.
 * sgs_chunk and blusgs_blocks (13 entries each, nullable) receive the
 * choices.  Tuning changes speed only, never results.  Synchronises. */
SWNMG_API swnmg_status swnmg_batch_tune(swnmg_batch* bt, double* const* U_dev, int32_t* sgs_chunk,
                                        int32_t* blusgs_blocks);

/* Sets the tuning by hand: sgs_chunk (13 entries, each 4, 8 or 16 in MIXED
 * precision and 2, 4 or 8 in FP64; NULL keeps them), blusgs_blocks for
 * every level (<= 0 keeps them; otherwise at most the co-resident limit). */
SWNMG_API swnmg_status swnmg_batch_set_tuning(swnmg_batch* bt, const int32_t* sgs_chunk,
                                              int32_t blusgs_blocks);

/* Number of cells of level l (0 if l is out of range). */
SWNMG_API int64_t swnmg_level_cells(const swnmg_ctx* ctx, int32_t level);

#endif /* SWNMG_H */
