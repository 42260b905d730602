/*
 * gbmg.h — C ABI of the GB300 geometric-multigrid Poisson library.
 *
 * The library solves the particle-mesh Poisson problem on a periodic 3-D mesh by
 * geometric multigrid V-cycles (arxiv 2607.10983, Sec. 2.3 "Geometric multigrid"):
 *
 *   flat operator  (GBMG_OP_FLAT7): A phi = F, A the second-order 7-point
 *                  Laplacian (Sec. 2.1, Eq. linsys), F mean-projected, phi zero mean.
 *   curvilinear    (GBMG_OP_CURV19): the moving-mesh Laplace-Beltrami operator
 *                  L = M / sqrt(g) of a deformation potential psi (Sec. 4.2-4.3,
 *                  Eq. LB and curv_linsys), M the conservative 19-point flux
 *                  divergence; L phi = delta - sum(delta sqrt g)/sum(sqrt g)
 *                  (Eq. solvability), phi zero mean.
 *
 * Conventions for every entry point
 *   - Fields are dense arrays of nx*ny*nz values, row-major [z][y][x] with x the
 *     fastest index, mesh spacing one cell on the finest level (h_l = 2^l on level l).
 *   - Pointers named *_dev are device pointers on the device that was current at
 *     mg_setup; pointers named *_host are host pointers (pinned or pageable).
 *   - The caller owns every buffer passed in; the library never keeps a pointer
 *     past the call.  The library owns its hierarchy workspace (allocated once in
 *     mg_setup, released in mg_destroy).
 *   - All GPU work is queued on the context's stream (mg_setup / mg_set_stream).
 *     Component calls return after queueing; solves wait for the stream.
 *   - Every function returns a gbmg_status and never throws or aborts.  CUDA errors
 *     map to GBMG_ERR_CUDA; mg_last_error() gives the message of the last failure
 *     in this thread.
 *   - dtype arguments select the element type of component calls: GBMG_F32 (float)
 *     or GBMG_F64 (double).
 */
#ifndef GBMG_H
#define GBMG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gbmg_ctx gbmg_ctx;

typedef enum {
  GBMG_OK = 0,
  GBMG_ERR_INVALID_ARG = 1, /* bad sizes, NULL pointers, unsupported option         */
  GBMG_ERR_CUDA = 2,        /* a CUDA runtime call or kernel launch failed            */
  GBMG_ERR_OOM = 3,         /* device or pinned-host allocation failed                */
  GBMG_ERR_NOT_CONVERGED = 4, /* max_vcycles reached above tol; phi holds the last iterate */
  GBMG_ERR_NONFINITE = 5,   /* a residual norm was NaN or inf; phi holds the last iterate */
  GBMG_ERR_DIVERGED = 6,    /* residual grew 10x over two cycles; phi holds the last iterate */
  GBMG_ERR_STATE = 7        /* call not valid in the context's current state          */
} gbmg_status;

typedef enum { GBMG_OP_FLAT7 = 0, GBMG_OP_CURV19 = 1 } gbmg_op;
/* GBMG_FP64: plain FP64 V-cycle, one kernel per operation (the baseline method).
 * GBMG_MIXED: FP32 V-cycle inside FP64-accurate defect correction (Sec. 3.2) whose
 *             residual and solution update use double-float (two-FP32) arithmetic. */
typedef enum { GBMG_FP64 = 0, GBMG_MIXED = 1 } gbmg_prec;
typedef enum { GBMG_SMOOTH_CHEBYSHEV = 0, GBMG_SMOOTH_JACOBI = 1 } gbmg_smoother;
typedef enum { GBMG_F32 = 0, GBMG_F64 = 1 } gbmg_dtype;

/* Solver options.  gbmg_default_opts fills the paper's defaults:
 * Chebyshev degree 3 on [2/alpha, 2] with alpha = 8 (Sec. 2.3, Eq. flat_chebyshev),
 * Jacobi omega = 2/3 with nu1 = nu2 = 2 (Sec. 2.3 Eq. flat_jacobi, Sec. 4.3.3),
 * mixed precision, fused level kernels. */
typedef struct {
  int op;        /* gbmg_op                                                        */
  int prec;      /* gbmg_prec                                                      */
  int smoother;  /* gbmg_smoother                                                  */
  int degree;    /* Chebyshev: operator applications per smoothing pass (>= 1)     */
  double alpha;  /* Chebyshev target interval [2/alpha, 2] of D^-1 A (alpha > 1)   */
  int nu1, nu2;  /* Jacobi sweeps before / after the coarse correction (>= 0)      */
  double omega;  /* Jacobi weight                                                  */
  int fused;     /* temporally blocked level kernels (GBMG_MIXED + Chebyshev):       */
                 /* 1: on levels of at least 2^18 cells, 2: on every level of at   */
                 /* least 16^3 (results are identical), 0: one kernel per operation; */
                 /* an odd nx selects 0 (the fused kernels work on pairs of x cells) */
  int krylov;    /* 0: each defect-correction step applies one V-cycle; k > 0 (<= 16,    */
                 /* flat + GBMG_MIXED + Chebyshev): k steps of conjugate gradients      */
                 /* preconditioned by the V-cycle (Sec. 3.2) on the FP32 error equation */
                 /* of each step; stats count defect-correction steps                  */
  int curv_sym;  /* GBMG_OP_CURV19 only.  0: the paper's scheme (Sec. 4.3.1): face fluxes */
                 /* with the tangential derivatives averaged onto the face; not exactly   */
                 /* symmetric for variable B, so adjoint solves use its exact transpose.  */
                 /* 1: symmetric variant: the same B^aa face terms, the cross terms on   */
                 /* the cell edges, -sum_{a!=b} E_a^T C_ab E_b with C_ab the mean of B^ab */
                 /* over the edge's four cells and E_a the a-difference averaged over   */
                 /* the edge's two b-positions; M = M^T, 19 points, the same Fourier     */
                 /* symbol for constant B; forward and adjoint solves use M itself.     */
  int coarse_store; /* flat + GBMG_MIXED only.  Storage of the correction that a coarse  */
                 /* level (fewer than 128^3 cells) hands up to the next finer level:     */
                 /* 0: FP32; 1: BF16; 2: FP16 (16-bit storage of coarse-level          */
                 /* corrections; the paper runs FP32 throughout, Sec. 3.3).              */
                 /* The value is rounded to that format before the prolongation; levels */
                 /* solved inside the shared-memory bottom cycle (16^3 and below) keep   */
                 /* FP32 within it.  Not supported by batches.                          */
} gbmg_opts;

typedef struct {
  int cycles;           /* V-cycles performed by the call                          */
  int status;           /* gbmg_status of the solve                                */
  double rel_res0;      /* ||F - A phi0|| / ||F|| before the first cycle           */
  double rel_res;       /* ||F - A phi|| / ||F|| after the last cycle              */
  double res_hist[64];  /* relative residual after cycle k (k < 64)                */
} gbmg_stats;

/* Fill *opts with the defaults listed above.  opts must not be NULL. */
void gbmg_default_opts(gbmg_opts* opts);

/* Create a solver for an nx x ny x nz periodic mesh (Sec. 2.3 hierarchy).
 *   levels: number of levels, 0 = as many as possible.  A level is coarsened while
 *           every side is even and half of it is at least 4, so n^3 with n a power
 *           of two gives log2(n) - 1 levels (Sec. 4.3.3); the coarsest level is solved
 *           exactly on the zero-mean subspace.  The coarsest level may hold at most
 *           512 cells.
 *   smoother_degree: Chebyshev degree (overrides opts->degree when > 0).
 *   opts: NULL = defaults.  cuda_stream: a cudaStream_t, NULL = legacy default stream.
 * Errors: GBMG_ERR_INVALID_ARG for sides < 4, a coarsest level above 512 cells or bad
 * options; GBMG_ERR_OOM when the hierarchy does not fit; *out is set only on success. */
gbmg_status mg_setup(gbmg_ctx** out, int nx, int ny, int nz, int levels, int smoother_degree,
                     const gbmg_opts* opts, void* cuda_stream);

/* Release everything the context owns.  NULL is ignored. */
void mg_destroy(gbmg_ctx* ctx);

/* Queue later work on `cuda_stream` (a cudaStream_t; NULL = legacy default stream). */
gbmg_status mg_set_stream(gbmg_ctx* ctx, void* cuda_stream);

/* Cycle graphs (default on).  A mixed fused flat solve (V-cycle or krylov corrections)
 * and a curvilinear solve run each V-cycle of the defect correction (Sec. 3.2) as one
 * CUDA graph launch: the cycle's launches are captured once per context (per buffer
 * parity or orientation, after one cycle has run eagerly) and replayed; the host still
 * checks convergence after every cycle.  Results are the same bits either way.
 * enable = 0 launches every kernel of every cycle from the host.  Timed kernel families
 * (mg_profile_begin) are timed inside the graphs by event nodes. */
gbmg_status mg_set_cycle_graphs(gbmg_ctx* ctx, int enable);

/* Curvilinear contexts only: set the deformation potential psi (nx*ny*nz doubles,
 * cell units, periodic).  psi is restricted to every level by full weighting and the
 * triad A = I + Hess psi, sqrt(g) = det A and B = sqrt(g) g^-1 are rebuilt per level
 * (Sec. 4.2, Eq. triad, Eq. metric; Appendix B); the coarsest operator is inverted
 * exactly.  Waits for the stream.  GBMG_ERR_INVALID_ARG if a coarsest volume element
 * is not positive (a folded mesh). */
gbmg_status mg_set_geometry(gbmg_ctx* ctx, const double* psi_dev);

/* Curvilinear contexts only: set the operator's coefficients directly instead of from psi.
 * J_dev: the volume element sqrt(g) of the finest level (nx*ny*nz floats, > 0); B_dev: the
 * six components of the symmetric B = sqrt(g) g^-1 (Sec. 4.3.1), 6 * nx*ny*nz floats packed
 * xx, yy, zz, xy, xz, yz.  The operator M of Sec. 4.3.1 is built from them on the finest
 * level; each coarser level takes the full-weighting restriction (Appendix B weights) of
 * the finer level's J and B (the paper rebuilds coarse geometry from a restricted psi
 * instead; with coefficients alone there is no psi to restrict).  The coarsest operator is
 * inverted exactly.  mg_solve then needs coeffs_dev = NULL; mg_solve_adjoint gives
 * source_bar but no psi_bar (GBMG_ERR_STATE).  Waits for the stream.  Errors as for
 * mg_set_geometry. */
gbmg_status mg_set_coefficients(gbmg_ctx* ctx, const float* J_dev, const float* B_dev);

/* Solve A phi = F (Sec. 2.1) or, on a curvilinear context, L phi = f (Sec. 4.3).
 * source_dev: F (nx*ny*nz doubles; its mean, or volume-weighted mean for the
 * curvilinear operator, is projected out; the buffer is not modified).  coeffs_dev:
 * NULL for the flat operator; on a curvilinear context the deformation potential psi
 * (as for mg_set_geometry) or NULL to keep the geometry already set.  phi_inout_dev: initial guess in (zeros = cold start, previous solution =
 * warm start, Sec. 3.1-3.2), zero-mean solution out.  V-cycles run until
 * ||F - A phi|| / ||F|| <= tol or max_vcycles cycles (max_vcycles <= 0 runs none and
 * only evaluates the residual).  The call waits for the stream and returns the
 * convergence status: GBMG_OK, or NOT_CONVERGED / NONFINITE / DIVERGED with phi still
 * written (last iterate, gauge applied).  stats: NULL or filled on return; the same
 * record is kept for mg_last_stats(). */
gbmg_status mg_solve(gbmg_ctx* ctx, const double* source_dev, const double* coeffs_dev,
                     double* phi_inout_dev, double tol, int max_vcycles, gbmg_stats* stats);

/* Vector-Jacobian product of the solve (Sec. 4.8, Eq. adj_rhs and Eq. adj_op) for the
 * scalar <phi_bar, phi(source, psi)>:
 *   flat: source_bar = P A^+ P phi_bar (A symmetric; P removes the mean);
 *   curvilinear: M^T lam = phi_bar - mean(phi_bar) is solved by the same multigrid on
 *   the exact transpose, source_bar = J (lam - sum(J lam)/sum(J)), and, if psi_bar_dev
 *   is not NULL, psi_bar = the gradient through the geometry, which needs the forward
 *   solution phi_dev and source_dev.  All fields nx*ny*nz doubles; psi_bar_dev must be
 *   NULL for the flat operator.  Convergence as in mg_solve; waits for the stream. */
gbmg_status mg_solve_adjoint(gbmg_ctx* ctx, const double* phi_bar_dev, double* source_bar_dev,
                             double* psi_bar_dev, const double* phi_dev, const double* source_dev,
                             double tol, int max_vcycles, gbmg_stats* stats);

/* Same solve with host buffers (nx*ny*nz doubles each, phi overwritten), waits for the
 * stream.  Mixed precision with page-locked buffers (cudaHostAlloc, cudaHostRegister):
 * the conversion kernels read F and the initial phi from host memory and write the
 * result there, over the host link, with no staging copy.  Otherwise F and phi are
 * copied to device staging buffers (allocated on the first such call, kept until
 * mg_destroy), solved there and phi copied back.  Results are identical either way. */
gbmg_status mg_solve_host(gbmg_ctx* ctx, const double* source_host, double* phi_inout_host,
                          double tol, int max_vcycles, gbmg_stats* stats);

/* A warm-started sequence of solves with host buffers (the time-stepping use of Sec. 3.2:
 * each solve starts from the previous solution, "recycling"):
 *   solve t = 0 .. count-1 of A phi_t = F_t - mean(F_t), initial guess phi_{t-1}
 *   (phi0_host for t = 0, or zero when phi0_host is NULL); phi_host[t] receives phi_t.
 * sources_host[t], phi_host[t], phi0_host: nx*ny*nz doubles each, page-locked for the
 * copies to run asynchronously (pageable memory works, with synchronous copies).  The
 * copy of F_{t+1} to the device and of phi_{t-1} back run on two copy streams of the
 * context while solve t runs on its stream; the iterate stays on the device between
 * solves.  Each solve equals mg_solve on the same data (results identical).
 * stats: NULL or count entries.  Returns GBMG_OK when every solve converged, else the
 * first non-converged status (the sequence still runs to the end); argument, state and
 * CUDA errors stop it.  Allocates two sources and two potentials on the device on the
 * first call (kept until mg_destroy).  Waits for all of it before returning. */
gbmg_status mg_solve_host_sequence(gbmg_ctx* ctx, int count, const double* const* sources_host,
                                   double* const* phi_host, const double* phi0_host, double tol,
                                   int max_vcycles, gbmg_stats* stats);

/* Warm-start predictor (Sec. 3.2 "Predictors"): the initial guess of the next solve from
 * earlier solutions of this context's mesh, FP64, nx*ny*nz values each.
 *   history_dev[0] = phi_{n-1} (most recent), history_dev[1] = phi_{n-2}, ...
 *   order 0: out = growth * phi_{n-1}   (recycling for growth = 1; the growth-scaled
 *            predictor, Eq. growth, with growth = D(a_n) / D(a_{n-1}))
 *   order 1: out = 2 phi_{n-1} - phi_{n-2}                (linear extrapolation)
 *   order 2: out = 3 phi_{n-1} - 3 phi_{n-2} + phi_{n-3}  (quadratic extrapolation)
 * Every product and sum is one correctly rounded FP64 operation, left to right as
 * written.  out_dev may be history_dev[0] (in place).  Queued on the context's stream.
 * Errors: GBMG_ERR_INVALID_ARG for order outside 0..2, n_history < order + 1 or NULL
 * pointers. */
gbmg_status mg_predict(gbmg_ctx* ctx, int order, double growth, const double* const* history_dev, int n_history,
                       double* out_dev);

/* One mesh-motion step (Sec. 4.4) on a GBMG_OP_CURV19 context:
 *   psidot solves L_psi[psidot] = kappa (m_init - sqrt(g) rho)   (Eq. calcdefp)
 *     with the curvilinear solver of mg_solve (same operator, same projection and gauge),
 *     the source first smoothed by smooth_passes passes of the separable [1/4, 1/2, 1/4]
 *     filter (the paper smooths the source without naming the filter);
 *   psi <- psi + dtau psidot - mean(psi + dtau psidot)             (Eq. defadvance).
 * rho_dev: mass density per unit computational volume on the finest level (FP64);
 * psi_inout_dev: the deformation potential, updated in place (FP64);
 * psidot_inout_dev: initial guess of psidot (warm start; zeros for a cold start) and the
 * solution out (FP64).  The geometry is set from the incoming psi; after the call the
 * context needs mg_set_geometry (or coeffs in mg_solve) before its next solve.  Waits for
 * the stream.  Returns the solve's convergence status; psi is advanced with the last
 * iterate of psidot in every case except argument and CUDA errors. */
gbmg_status mg_mesh_motion(gbmg_ctx* ctx, const double* rho_dev, double kappa, double m_init, int smooth_passes,
                           double dtau, double* psi_inout_dev, double* psidot_inout_dev, double tol, int max_vcycles,
                           gbmg_stats* stats);

/* ---------------------------------------------------------------------------------
 * Particle-mesh steps around the solve (Sec. 2.1: particles are deposited by
 * cloud-in-cell interpolation to form the source; a static force evaluation is paint,
 * solve, fourth-order gradient (mg_grad), read).  On the finest level of ctx.
 * pos_dev: n_particles x 3 FP32, columns x, y, z in cell units (node (i, j, k) at position
 * (i, j, k)); any position is wrapped onto the periodic mesh.  Per axis node floor(x)
 * gets weight 1 - f and node floor(x) + 1 weight f, f = x - floor(x), formed in FP64.
 * --------------------------------------------------------------------------------- */
/* rho_dev (FP64, nx*ny*nz) = sum over particles of mass_p x CIC weight; mass_dev (FP32,
 * n_particles) or, when NULL, the scalar `mass` for every particle.  rho_dev is
 * overwritten; the sum uses FP64 atomics, so its rounding depends on the order in which
 * particles land.  Queued on the context's stream. */
gbmg_status mg_cic_paint(gbmg_ctx* ctx, const float* pos_dev, const float* mass_dev, double mass,
                         long long n_particles, double* rho_dev);
/* out_dev[p * ncomp + c] = sum of the CIC weights times field_dev[c * nx*ny*nz + node]
 * (FP64, ncomp = 1..3 components, e.g. the output of mg_grad); corners summed in the order
 * dz, dy, dx, each product and sum correctly rounded.  The transpose of mg_cic_paint. */
gbmg_status mg_cic_read(gbmg_ctx* ctx, const double* field_dev, int ncomp, const float* pos_dev,
                        long long n_particles, double* out_dev);

/* Single-precision force at the particles (the paper's PM force evaluation runs in FP32):
 * phi (FP64) rounded to FP32, force grid -grad4 phi (the fourth-order gradient of mg_grad,
 * h = 1) in FP32, then CIC read in FP32 with the weights of mg_cic_paint.
 * force_out_dev: n_particles x 3 FP32 (x, y, z).  Allocates 16 bytes per cell of scratch on
 * first use (kept until mg_destroy).  Queued on the context's stream. */
gbmg_status mg_force(gbmg_ctx* ctx, const double* phi_dev, const float* pos_dev, long long n_particles,
                     float* force_out_dev);

/* Statistics of the last completed mg_solve on this context (waits for the stream). */
gbmg_status mg_last_stats(gbmg_ctx* ctx, gbmg_stats* stats);

/* Number of levels, and the sides of level `level` (0 = finest). */
int mg_num_levels(const gbmg_ctx* ctx);
gbmg_status mg_level_dims(const gbmg_ctx* ctx, int level, int* nx, int* ny, int* nz);

/* ---------------------------------------------------------------------------------
 * Batched solves: many independent flat problems, sizes may differ, solved in ONE
 * persistent cooperative kernel launch (each operation of the V-cycle is a grid-wide
 * phase over every active problem; converged problems drop out).  Each problem uses
 * the hierarchy of its own context, which must be flat, GBMG_MIXED, Chebyshev,
 * fused = 0, with at least two levels; all contexts share the smoother settings and
 * the device.  A context must not be used by another call while its batch solves.
 * Iterates equal those of mg_solve on each context up to the rounding of the means.
 * --------------------------------------------------------------------------------- */
typedef struct gbmg_batch gbmg_batch;

/* Build the batch tables for ctxs[0..count-1] (device tables allocated here). */
gbmg_status mg_batch_create(gbmg_batch** out, gbmg_ctx* const* ctxs, int count, void* cuda_stream);
void mg_batch_destroy(gbmg_batch* batch);
/* Persistent grid size in blocks (default and maximum: every block resident). */
gbmg_status mg_batch_set_blocks(gbmg_batch* batch, int blocks);
/* Tile size per level: the number of consecutive cells (whole x rows of one problem)
 * one block takes in each grid-wide phase on level l, for l < nlevels.  Each size is a
 * multiple of 256 in [1024, 65536]; the default is 4096.  Rebuilds the tile tables
 * (waits for the stream).  Sizes change the schedule and the summation order of the
 * per-problem norms and means, nothing else. */
gbmg_status mg_batch_set_tiles(gbmg_batch* batch, const int* tile_cells, int nlevels);
/* Current tile sizes of levels 0 .. nlevels-1 (0 beyond the deepest level). */
gbmg_status mg_batch_get_tiles(const gbmg_batch* batch, int* tile_cells, int nlevels);
/* on != 0: run each solve as a CUDA graph (captured at the first solve on a stream of
 * the batch's own, replayed while tol, max_vcycles, grid and tile sizes are unchanged;
 * ordered after earlier and before later work on the batch's stream).  Off by default. */
gbmg_status mg_batch_use_graph(gbmg_batch* batch, int on);
/* Number of levels of the deepest problem (length of the tile-size array). */
int mg_batch_num_levels(const gbmg_batch* batch);
/* Autotuner: times full solves and keeps the fastest settings, first the grid size
 * (1 .. resident blocks per SM, times the SM count), then, level by level, the tile
 * size (1024, 2048, ... 65536 cells).  Every trial starts from the initial guesses in
 * phi_dev (saved in temporary device buffers, released before returning); on return
 * phi_dev holds the solution from those guesses with the chosen settings.
 * *blocks_out and tiles_out[0 .. levels-1] (both nullable) receive the choice. */
gbmg_status mg_batch_autotune(gbmg_batch* batch, const double* const* source_dev, double* const* phi_dev,
                              double tol, int max_vcycles, int* blocks_out, int* tiles_out);
/* Solve every problem: source_dev[i] / phi_dev[i] as for mg_solve on ctxs[i] (phi is
 * the initial guess in and the solution out).  Waits for the stream.  stats (array of
 * count, nullable) per problem; times_ms (array of count, nullable) receives each
 * problem's completion time after the launch started, from the GPU clock.  Returns
 * GBMG_OK if every problem converged, else the first problem's failure status. */
gbmg_status mg_batch_solve(gbmg_batch* batch, const double* const* source_dev, double* const* phi_dev, double tol,
                           int max_vcycles, gbmg_stats* stats, double* times_ms);

/* ---------------------------------------------------------------------------------
 * Measurement.  While a kernel family is being timed, every launch of it is
 * bracketed by CUDA events on the context's stream (no extra synchronisation).
 * --------------------------------------------------------------------------------- */
typedef enum {
  GBMG_PROF_OFF = 0,
  GBMG_PROF_DOWN0 = 1,   /* finest level, fused pre-smoothing + residual + restriction  */
  GBMG_PROF_UP0 = 2,     /* finest level, fused prolongation + post-smoothing            */
  GBMG_PROF_DF0 = 3,     /* finest level, double-float update and residual               */
  GBMG_PROF_SMOOTH0 = 4, /* finest level, one-kernel-per-operation smoother steps        */
  GBMG_PROF_CURV0 = 5    /* finest level, curvilinear weighted-Jacobi sweeps             */
} gbmg_prof_family;

/* Start timing the kernel families whose bits (1 << family) are set in family_mask
 * (waits for the stream; clears earlier records).  Inside cycle graphs at most 8
 * launches of a family per cycle are timed. */
gbmg_status mg_profile_begin(gbmg_ctx* ctx, int family_mask);
/* Number of timed launches of `family` since mg_profile_begin and their summed device
 * time in milliseconds (waits for the stream; timing continues). */
gbmg_status mg_profile_read(gbmg_ctx* ctx, int family, int* launches, double* total_ms);
/* Stop timing and clear the records. */
gbmg_status mg_profile_end(gbmg_ctx* ctx);
/* Number of kernels this library has launched in the process so far. */
long long mg_launch_count(void);

/* Human-readable status; never NULL. */
const char* mg_status_string(gbmg_status s);
/* Message of the last error raised in the calling thread ("" if none). */
const char* mg_last_error(void);

/* ---------------------------------------------------------------------------------
 * Component calls: one operation of the V-cycle on level `level`, on caller buffers
 * of that level's size, in precision dtype.  They exist so that each kernel can be
 * checked on its own; they run the same kernels as mg_solve.
 * --------------------------------------------------------------------------------- */

/* out = A_l u: 7-point Laplacian with spacing h_l = 2^level (Sec. 2.1, rediscretised
 * per level, Sec. 2.3). */
gbmg_status mg_apply(gbmg_ctx* ctx, int level, int dtype, const void* u_dev, void* out_dev);

/* out = f - A_l u (Sec. 2.3, Eq. flat_residual). */
gbmg_status mg_residual(gbmg_ctx* ctx, int level, int dtype, const void* f_dev, const void* u_dev,
                        void* out_dev);

/* One smoothing pass of the configured smoother on A_l e = r, in place on e:
 * Chebyshev (Eq. flat_chebyshev, `degree` operator applications) or weighted Jacobi
 * (Eq. flat_jacobi, nu1 sweeps). */
gbmg_status mg_smooth(gbmg_ctx* ctx, int level, int dtype, void* e_inout_dev, const void* r_dev);

/* coarse = R fine: full weighting [1/4,1/2,1/4] per axis then decimation (Appendix B);
 * fine is level `level`, coarse is level+1. */
gbmg_status mg_restrict(gbmg_ctx* ctx, int level, int dtype, const void* fine_dev, void* coarse_dev);

/* fine += P coarse: trilinear prolongation (Sec. 2.3, Eq. coarse_correction);
 * fine is level `level`, coarse is level+1. */
gbmg_status mg_prolong_add(gbmg_ctx* ctx, int level, int dtype, const void* coarse_dev, void* fine_dev);

/* e = exact minimum-norm solution of A_c e = r on the coarsest level (Sec. 2.3
 * "directly on the coarsest level"): the pseudo-inverse, built at setup. */
gbmg_status mg_coarse_solve(gbmg_ctx* ctx, int dtype, const void* r_dev, void* e_dev);

/* One V-cycle (mu = 1) on the error equation A_0 e = r of the finest level in the
 * working precision of the context (GBMG_FP64: double, GBMG_MIXED: float), starting
 * from e = 0, with the configured smoother and fusion. */
gbmg_status mg_vcycle(gbmg_ctx* ctx, const void* r_dev, void* e_dev);

/* Curvilinear components (geometry must be set).  out = op(u) or op(u) / J on level
 * `level`, op = M (transpose 0) or its exact transpose M^T (transpose 1); with
 * opts.curv_sym, op = S (the symmetric variant) for either value. */
gbmg_status mg_curv_apply(gbmg_ctx* ctx, int level, int dtype, int transpose, int divide_by_J,
                          const void* u_dev, void* out_dev);
/* Copy the geometry of a level: J (n floats) and B packed xx, yy, zz, xy, xz, yz (6 n
 * floats); either pointer may be NULL. */
gbmg_status mg_curv_geometry(gbmg_ctx* ctx, int level, float* J_dev, float* B_dev);
/* The FP32 level kernels of that V-cycle, one launch each, on level `level` (n floats
 * per buffer, distinct buffers).  mg_curv_residual: out = r - op(u) / (h_l^2 J), the
 * residual of L = M / J (Sec. 4.3, Eq. curv_linsys) or of the transposed-solve operator
 * M^T / J.  mg_curv_smooth: one weighted-Jacobi sweep (Appendix B, Eq. jacobi)
 * e_out = e_in + omega (J r - op(e_in) / h_l^2) / D with D the stencil's diagonal
 * (op / h_l^2 applied to a unit vector), omega = opts.omega; e_in and e_out must differ.
 * e_in NULL: the iterate is zero, and the sweep is the pointwise one the V-cycle uses
 * for its first pre-smoothing sweep (the same values as a sweep of a zero array).
 * op as in mg_curv_apply. */
gbmg_status mg_curv_residual(gbmg_ctx* ctx, int level, int transpose, const float* r_dev, const float* u_dev,
                             float* out_dev);
gbmg_status mg_curv_smooth(gbmg_ctx* ctx, int level, int transpose, const float* e_in_dev, const float* r_dev,
                           float* e_out_dev);
/* One FP32 curvilinear V-cycle (weighted Jacobi nu1/nu2) on L e = r (transpose 0) or on
 * the transposed-solve operator M^T / J (transpose 1), from e = 0 (S / J for either
 * value with opts.curv_sym). */
gbmg_status mg_curv_vcycle(gbmg_ctx* ctx, int transpose, const float* r_dev, float* e_dev);

/* Finite-difference gradient on the finest level, spacing 1, periodic: order 4 is the
 * one-exchange fourth-order stencil (-u_{i+2} + 8u_{i+1} - 8u_{i-1} + u_{i-2})/12 of
 * the force evaluation (Sec. 3.4), order 2 the central difference (Sec. 4.1).
 * transpose 0: in = u (n doubles), out = grad u (3n doubles, component-major x, y, z);
 * transpose 1: in = w (3n floats, component-major), out = grad^T w (n doubles). */
gbmg_status mg_grad(gbmg_ctx* ctx, int order, int transpose, const void* in_dev, double* out_dev);
/* out_dev[0] = sum over cells and components of w . grad u (u n doubles, w 3n floats). */
gbmg_status mg_grad_dot(gbmg_ctx* ctx, int order, const double* u_dev, const float* w_dev, double* out_dev);

/* Double-float helpers of the mixed-precision path.  A double-float array stores each
 * value x as the float pair (hi, lo), hi = round(x), lo = round(x - hi): 2*n floats. */
gbmg_status mg_f64_to_df(gbmg_ctx* ctx, long long n, const double* x_dev, float* df_dev);
gbmg_status mg_df_to_f64(gbmg_ctx* ctx, long long n, const float* df_dev, double* x_dev);
/* r = (F - m) - A_0 phi on the finest level in double-float arithmetic, rounded to
 * float; F and phi are double-float arrays, m a double. */
gbmg_status mg_df_residual(gbmg_ctx* ctx, const float* F_df_dev, double m, const float* phi_df_dev,
                           float* r_dev);

/* ---------------------------------------------------------------------------------
 * Allocation-free call (the paper has no counterpart).  For callers that must not
 * allocate device memory: a time-step loop that runs inside a fixed, pre-reserved
 * memory budget, or code hosted by another framework whose allocator owns the
 * device.  It needs no context and no mg_setup.
 *
 * Writes rel_out_dev[0] = ||F - m - A phi|| / ||F - m|| (a device double), with
 * F = source_dev, phi = phi_dev (nx*ny*nz doubles on the current device),
 * m = mean(F) and A the 7-point periodic Laplacian with unit spacing: the quantity
 * mg_solve reports as rel_res0.  The residual is evaluated in double-float and rounded
 * to FP32 per cell; the squares are summed in compensated (double-float) sums per
 * plane and in FP64 across planes, so the ratio carries about 1e-7 relative error at
 * any mesh size.
 *
 * Scratch: one fixed array of 2 * GBMG_NOALLOC_MAX_NZ + 8 doubles (about 64 KiB) in
 * the library's own device memory, held by every GPU that loads the library until
 * the process exits.  nz above GBMG_NOALLOC_MAX_NZ (or a side below 4) is rejected
 * with GBMG_ERR_INVALID_ARG.  The first call on a device looks the array's address
 * up on that device, with that device current; make that first call before any
 * stream capture.  The address is kept for the life of the process: after a
 * cudaDeviceReset of a device the library's device memory there is gone, and this call
 * must not be used on that device again.  Every call overwrites the scratch entries it reads (nothing has
 * to start at zero) and the array keeps the last call's contents; all calls share
 * it, so calls that overlap on the GPU (unordered streams) race.  The work is
 * queued on cuda_stream (NULL = legacy default stream); the call does not wait.
 * No memory is allocated or freed. */
#define GBMG_NOALLOC_MAX_NZ 4096
gbmg_status mg_rel_residual_noalloc(int nx, int ny, int nz, const double* source_dev, const double* phi_dev,
                                    double* rel_out_dev, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* GBMG_H */
