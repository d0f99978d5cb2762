/*
 * nswe.h - C ABI of the GB300 (sm_103a) library for the high-order Newton
 * multigrid method (NMGM) with a simplified Jacobian for steady shallow water
 * equations (Hu, Li, Wang, Wang, arXiv 2505.10857).
 *
 * Scope: the quasi-one-dimensional model of Section 2 (Eq. 3-4), discretised
 * by the third-order finite-volume WENO scheme of Section 3.1, linearised by
 * the regularized Newton iteration of Section 3.2 with the finite-difference
 * Jacobian J5 or its simplified block-tridiagonal form J3 (Section 3.3), and
 * solved by the geometric multigrid of Section 3.4 inside the nested NMGM of
 * Algorithm 3; the two-dimensional model of Section 4 (J21 / J9) through the
 * same calls. Arithmetic is FP64, with an optional mixed-precision solve in
 * 1D and 2D (NSWE_PREC_MIXED). A 1D solve runs on one thread block (many
 * problems per launch) or, for latency, on a thread-block cluster
 * (nswe_ctx_set_solve_cluster). A continuous-batching server for streams of
 * 1D and 2D solves sits at the end of this header.
 *
 * Conventions
 *   - Cells and faces are 0-based: cell j of a level with N cells spans faces
 *     j and j+1; face f sits at x0 + f*dx, dx = (x1-x0)/N.
 *   - A state (U, R, dU) is two planes of N doubles: H (wet cross-section
 *     sigma*h) then Q (discharge).
 *   - A banded block Jacobian with nb blocks per row (nb = 3: offsets -1..1;
 *     nb = 5: offsets -2..2) is stored as
 *         J[(k*4 + l*2 + m)*N + j] = (dR_j / dU_{j+k-(nb-1)/2})_{l,m},
 *     2x2 blocks row-major, l = residual component, m = unknown component;
 *     blocks reaching outside the grid are zero.
 *   - Nested level l has N_l = N / 2^l cells (level 0 finest). The multigrid
 *     hierarchy aggregates pairs of cells (Eq. 15).
 *   - Unless stated otherwise, array arguments of compute calls are DEVICE
 *     pointers owned by the caller; calls are asynchronous on the context's
 *     stream. Problem-creation calls take HOST arrays and copy them.
 *   - No call aborts, traps or exits. Bad arguments return NSWE_EINVAL; CUDA
 *     failures return NSWE_ECUDA. Device-side conditions (NaN, non-positive
 *     depth, non-convergence) are reported through nswe_info.
 */
#ifndef NSWE_H
#define NSWE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  NSWE_OK = 0,
  NSWE_EINVAL = 1,    /* invalid argument (size, pointer, parameter)          */
  NSWE_ENOMEM = 2,    /* device or host allocation failed                     */
  NSWE_ECUDA = 3,     /* a CUDA runtime call failed                           */
  NSWE_ENOTCONV = 4,  /* Newton stopped at n_max with res >= tol              */
  NSWE_ENAN = 5,      /* NaN/Inf in the residual                              */
  NSWE_ENEGDEPTH = 6, /* non-positive wet cross-section H in the state        */
  NSWE_ESINGULAR = 7, /* exactly zero pivot in the coarsest direct solve     */
  NSWE_ETIMEOUT = 8    /* a wait ended before the awaited event              */
} nswe_status;

/* Boundary data (Section 5.1). The paper gives the data, not the discrete
 * treatment: the library fills two ghost cells per side with one state built
 * from the data and the adjacent interior cell (sigma_b = width at the
 * boundary face):
 *   DISCHARGE: (H, Q) = (H_edge, q)         e.g. upstream discharge
 *   DEPTH:     (H, Q) = (sigma_b*h, Q_edge)  e.g. downstream depth
 *   STATE:     (H, Q) = (sigma_b*h, q)       both given (Section 5.1.1)
 *   EXTRAP:    (H, Q) = (H_edge, Q_edge)                                    */
typedef enum {
  NSWE_BC_DISCHARGE = 1,
  NSWE_BC_DEPTH = 2,
  NSWE_BC_STATE = 3,
  NSWE_BC_EXTRAP = 4
} nswe_bc_kind;

typedef struct {
  int kind;  /* nswe_bc_kind */
  double h;  /* depth (DEPTH, STATE)    */
  double q;  /* discharge (DISCHARGE, STATE) */
} nswe_bc1d;

/* Two-dimensional boundary kinds (Section 5.2), one per boundary cell. The
 * library fills two ghost layers: REFLECT mirrors the interior with the
 * normal momentum negated (slip wall), INFLOW takes the given (h, hu, hv),
 * OUTFLOW copies the edge cell, DISCHARGE takes the given momenta and the
 * edge depth, DEPTH the given depth and the edge momenta. Corner ghosts apply
 * the x rule, then the y rule. */
#define NSWE_BC2_REFLECT 5
#define NSWE_BC2_INFLOW 6
#define NSWE_BC2_OUTFLOW 7
#define NSWE_BC2_DISCHARGE 8
#define NSWE_BC2_DEPTH 9

#define NSWE_MAX_LEVELS 16
#define NSWE_JAC_SIMPLIFIED 3 /* 1D J3: block tridiagonal (Section 3.3); 2D J9 */
#define NSWE_JAC_FULL 5       /* 1D J5: block pentadiagonal; 2D J21          */
/* 2D only, OR'd into nswe_params.jacobian (J9 or J21): the frozen
 * linearisation, an option beside Eq. 12 that the paper does not have. The
 * perturbed local residuals take the WENO nonlinear weights (Eq. 8) and the
 * characteristic eigenvectors of every reconstruction from the current
 * iterate, so only the candidate polynomials, the fluxes and the sources see
 * the perturbation. The residual and its steady state are unchanged; Newton
 * becomes a quasi-Newton iteration. Where a discontinuity meets a wall (the
 * wedge of Section 5.2.2) the derivatives of the nonlinear weights make the
 * Jacobian of Eq. 12 one on which block SOR diverges; with the weights
 * frozen it contracts at the paper's omega = 0.1. 1D calls refuse it
 * (NSWE_EINVAL). */
#define NSWE_JAC_FROZEN 0x100

/* Arithmetic of a Newton step. The paper computes in double precision
 * (NSWE_PREC_FP64). NSWE_PREC_MIXED is this library's addition: the residual
 * (Eq. 10 / Eq. 20), res, the stopping test and the update (Eq. 14) stay
 * FP64, while the coarse operators, the smoother and the coarsest LU run in
 * FP32. The FD Jacobian (Eq. 12-13) is evaluated in FP32 in 1D and, since
 * the 2D perturbation eps = 1e-6 (Section 5.2) leaves no significant digits
 * in an FP32 difference, evaluated in FP64 and stored in FP32 in 2D. The
 * Jacobian is an approximation of the true derivative either way, so the
 * Newton fixed point R(U) = 0 is the FP64 one; only the convergence path
 * changes. */
#define NSWE_PREC_FP64 0
#define NSWE_PREC_MIXED 1

/* Solver parameters (Section 5). nswe_params_default fills the paper's 1D
 * values: alpha 3, tau 0.6, omega 1, nu1 = nu2 = nu3 = 2, tol 1e-11. */
typedef struct {
  double alpha;   /* regularization weight, Eq. 13                          */
  double tau;     /* Newton damping, Eq. 14                                 */
  double omega;   /* SOR relaxation, Eq. 19                                 */
  double tol;     /* stop when res < tol (Algorithms 1, 3)                  */
  int nu1, nu2;   /* pre/post smoothing steps per level (Algorithm 2)       */
  int nu3;        /* V-cycles per Newton step (Algorithm 3)                 */
  int n_max;      /* Newton iteration cap per nested level                  */
  int jacobian;   /* NSWE_JAC_SIMPLIFIED (J3/J9) or NSWE_JAC_FULL (J5/J21);
                     2D: optionally | NSWE_JAC_FROZEN                        */
  int nest_start; /* nested level the solve starts on; <0: coarsest (Alg. 3)*/
  int precision;  /* NSWE_PREC_FP64 or NSWE_PREC_MIXED                      */
  int colours2d;  /* 2D smoothing of the cross stencils (J9, coarse 5-point):
                     0 = two symmetric passes of the stencil colouring;
                     K >= 3 = the directional schedule, the multicolour
                     analogue of the sweeps D1-D4 of Eq. 22: diagonal colours
                     (i + j) mod K ascending, (j - i + Nx - 1) mod K
                     ascending, both descending; K >= Nx + Ny - 1 is the
                     lexicographic sweep itself;
                     NSWE_COLOURS2D_AUTO = the choice of nswe_autotune_2d */
  double eps[NSWE_MAX_LEVELS]; /* FD perturbation per nested level, Eq. 12  */
} nswe_params;

/* Per-solve record filled by nswe_newton_solve*. */
typedef struct {
  int status;                        /* nswe_status of the finest level    */
  int iters[NSWE_MAX_LEVELS];        /* Newton iterations per nested level */
  double res[NSWE_MAX_LEVELS];       /* final res per nested level         */
  int level_status[NSWE_MAX_LEVELS]; /* nswe_status per nested level       */
  int total_iters;
  int vcycles;
  unsigned long long t_start_ns;     /* solve start: 1D the device global
                                        timer, 2D the host steady clock   */
  unsigned long long t_end_ns;       /* solve end, on the same clock       */
} nswe_info;

typedef struct nswe_ctx_s *nswe_ctx;
typedef struct nswe_prob_s *nswe_prob;

const char *nswe_status_str(int status);

/* Fills p with the paper's one-dimensional defaults for a problem of N cells
 * and `levels` multigrid levels; eps per level from the paper's values
 * (0.2/0.15/0.1/0.05 at N = 96/192/384/768, log2 progression between,
 * clipped to [0.05, 0.2]). */
nswe_status nswe_params_default(nswe_params *p, int N, int levels);

/* Context: binds a device and a CUDA stream (cudaStream_t passed as void*,
 * may be NULL for the legacy default stream, or a stream owned by the
 * caller, e.g. PyTorch's). Owns nothing the caller passes in. */
nswe_status nswe_ctx_create(nswe_ctx *out, int device, void *stream);
nswe_status nswe_ctx_set_stream(nswe_ctx ctx, void *stream);

/* Storage of the 2D Jacobian in nested solves (a layout choice, not in the
 * paper; results are the same bits either way): Newton levels of at least
 * min_cells cells that are solved by V-cycles keep J9 and its diagonal
 * inverses colour-major, each colour (i + j) mod 3 of the smoother one
 * contiguous plane, so that a colour pass reads only its third of J.
 * min_cells < 0: never. Default 131072 (512 x 256). The standalone calls
 * (nswe_jacobian_*, nswe_mg_vcycle*) always use the cell-contiguous layout
 * they document. */
nswe_status nswe_ctx_set_colour_major_2d(nswe_ctx ctx, int min_cells);
/* Work split of the 2D FD Jacobian (Eq. 12; results are the same bits either
 * way): on levels of at least min_cells cells one thread takes a cell and
 * builds its unperturbed reconstruction lines once for all stencil blocks;
 * on smaller levels one thread takes one (cell, block) item. min_cells < 0:
 * never per cell. Default 32768. Applies to nested solves and to the
 * standalone Jacobian calls of this context. */
nswe_status nswe_ctx_set_jacobian_cells_2d(nswe_ctx ctx, int min_cells);
/* How nswe_newton_solve_batch and nswe_newton_solve_batch_each run a batch
 * of several 2D problems (the paper solves one problem; results are the same
 * bits either way):
 *   NSWE_BATCH2D_CONCURRENT: each problem's solve is sequenced on its own
 *     stream by one of up to 8 host worker threads.
 *   NSWE_BATCH2D_LOCKSTEP (default): problems with the same precision, Jacobian
 *     stencil (J9 / J21) and smoothing schedule (nu1, nu2, nu3, omega,
 *     colours2d) share launches: each phase of a Newton step (Eq. 12-14) and
 *     each colour pass of its V-cycles (Algorithm 2) is one launch over all
 *     of them, each problem owning a range of the launch's blocks. Nested
 *     stage k runs Newton iterations on level s0 - k of every problem that
 *     has it (s0 its start level); a problem that meets its stopping test
 *     is masked off until the stage ends. A stage's Newton step is captured
 *     once as a CUDA graph and replayed; the host reads every problem's res
 *     and flag once per replay. Groups with different schedules run one
 *     after another. Timestamps in nswe_info are host times. */
#define NSWE_BATCH2D_CONCURRENT 0
#define NSWE_BATCH2D_LOCKSTEP 1
nswe_status nswe_ctx_set_batch_2d(nswe_ctx ctx, int mode);

/* Programmatic dependent launch of the 2D kernels (the paper has no
 * counterpart; results are the same bits either way), process-wide, on by
 * default: each 2D kernel launched from the host (the standalone calls,
 * nswe_mg_vcycle, nswe_mg_smooth, the autotuner) carries programmatic
 * stream serialization, so that it may begin launching while the kernel
 * before it on the stream still runs, and waits for that kernel's
 * completion on the device before it reads anything. Launches captured into
 * the CUDA graphs of the nested solves keep ordinary stream order.
 * enable: 1 on, 0 off; other values NSWE_EINVAL. */
nswe_status nswe_set_launch_overlap_2d(int enable);

/* Tail threshold of the 2D V-cycles (the paper has no counterpart; results
 * are the same bits whatever its value): from the first level of at most
 * max_cells cells down to the coarsest and back, a V-cycle runs as one
 * thread block per problem instead of one launch per colour pass. precision:
 * NSWE_PREC_FP64 (default 256 cells) or NSWE_PREC_MIXED (default 4096). */
nswe_status nswe_ctx_set_tail_2d(nswe_ctx ctx, int precision, int max_cells);

/* Autotuner of the 2D V-cycle (the paper has no counterpart): forms the
 * Jacobian of params (J9 / J21, frozen or Eq. 12, eps[0], alpha) at the
 * finest level of `prob` from U (DEVICE [3][Nx*Ny]) in params->precision,
 * then times, with CUDA events on the context stream, one untimed and `reps`
 * timed V-cycles (Algorithm 2 with params' nu1, nu2, omega) for every
 * smoothing schedule schedules[0..nsched) (colours2d values: 0 or K >= 3)
 * and every tail threshold tails[0..ntails) (cells), and writes the mean
 * milliseconds per V-cycle to ms[a * ntails + b] (HOST, may be NULL). The
 * fastest pair is recorded in the context for prob's size and precision and
 * returned in *best_schedule and *best_tail (HOST, may be NULL); a solve of
 * a problem of that size and precision with colours2d = NSWE_COLOURS2D_AUTO
 * then uses it (a size with nothing recorded: schedule 0 and the context's
 * tail). The tail threshold changes no result; the schedule changes the
 * smoothing, and so the Newton iterates, though not the steady state.
 * Standalone V-cycle calls take the recorded schedule but the context's
 * tail. Overwrites the problem's multigrid workspace; synchronises the
 * context stream. */
#define NSWE_COLOURS2D_AUTO (-1)
nswe_status nswe_autotune_2d(nswe_ctx ctx, nswe_prob prob, const double *U,
                             const nswe_params *params, const int *schedules,
                             int nsched, const int *tails, int ntails,
                             int reps, double *ms, int *best_schedule,
                             int *best_tail);
/* The schedule and tail nswe_autotune_2d recorded for Nx x Ny in
 * `precision`; NSWE_EINVAL if none. */
nswe_status nswe_ctx_get_tuned_2d(nswe_ctx ctx, int Nx, int Ny, int precision,
                                  int *schedule, int *tail);
nswe_status nswe_ctx_destroy(nswe_ctx ctx);

/* One-dimensional problem (Eq. 3-4) on [x0, x1] with N cells and `levels`
 * nested/multigrid levels (N divisible by 2^(levels-1), every level >= 4
 * cells, coarsest level at most 128 cells for the direct solve). HOST arrays,
 * copied to device memory owned by the problem:
 *   sigma_face[N+1]      channel width sigma at the finest faces;
 *   gauss_geom           for l = 0..levels-1 in turn, [3][2][N_l]:
 *                        sigma, d sigma/dx and db/dx at the two Gauss points
 *                        x_j - dx_l/(2 sqrt 3) and x_j + dx_l/(2 sqrt 3)
 *                        of each cell j of level l (Eq. 9);
 *   left, right          boundary data (nswe_bc1d).
 * The problem also owns the device workspace of the solver (Jacobians,
 * multigrid hierarchy, coarsest factorisation). */
nswe_status nswe_prob_create_1d(nswe_ctx ctx, nswe_prob *out, int N, int levels,
                                double x0, double x1, double g,
                                const double *sigma_face,
                                const double *gauss_geom,
                                const nswe_bc1d *left, const nswe_bc1d *right);
/* Re-uploads geometry and boundary data of an existing problem (same N and
 * levels) from HOST arrays. The arrays are checked and packed into the
 * problem's pinned staging buffer before the call returns (the caller may
 * reuse them at once); the copy to the device and the derived geometry then
 * run asynchronously on the context stream. A later upload to the same
 * problem first waits for that copy. EINVAL for non-finite data (nothing is
 * uploaded). */
nswe_status nswe_prob_set_geometry_1d(nswe_ctx ctx, nswe_prob prob,
                                      const double *sigma_face,
                                      const double *gauss_geom,
                                      const nswe_bc1d *left,
                                      const nswe_bc1d *right);

/* Numerical flux of a 1D problem's residual (Section 3.1 names both): HLL,
 * the paper's choice in 1D and the default, or LLF (the mean of the two
 * physical fluxes minus a (U_R - U_L) / 2, a the larger |u| + c), kept for
 * comparison. Applies to every later call on the problem; EINVAL for a 2D
 * problem or another value. The problems of one batched solve share a flux
 * (NSWE_EINVAL otherwise); LLF batches run in the default launch shape. */
#define NSWE_FLUX_HLL 0
#define NSWE_FLUX_LLF 1
nswe_status nswe_prob_set_flux_1d(nswe_ctx ctx, nswe_prob prob, int flux);

/* The same for `count` distinct 1D problems (HOST arrays of count entries
 * each): the packing and checks run in parallel on host threads, and no
 * upload starts unless every problem's data is valid. */
nswe_status nswe_prob_set_geometry_batch_1d(nswe_ctx ctx, int count,
                                            const nswe_prob *probs,
                                            const double *const *sigma_faces,
                                            const double *const *gauss_geoms,
                                            const nswe_bc1d *lefts,
                                            const nswe_bc1d *rights);
/* Two-dimensional problem (Eq. 1-2, Section 4) on [x0,x1] x [y0,y1] with
 * Nx x Ny cells and `levels` nested/multigrid levels (Nx, Ny divisible by
 * 2^(levels-1); every level at least 4 x 4 cells; coarsest level at most 512
 * cells for the dense direct solve). Cell (i, j) has index c = j*Nx + i; a 2D
 * state is three planes h, hu, hv of Nx*Ny doubles. HOST arrays, copied:
 *   gauss_geom   for l = 0..levels-1 in turn, [2][4][Ny_l*Nx_l]: db/dx and
 *                db/dy at the Gauss points (x_i -+ dx/(2 sqrt 3), y_j -+
 *                dy/(2 sqrt 3)), point q = 2*beta + gamma (beta: y, gamma: x);
 *   bc_kind      for l = 0..levels-1 in turn, [Ny_l left | Ny_l right |
 *                Nx_l bottom | Nx_l top] NSWE_BC2_* kinds;
 *   bc_state     [4][3] (h, hu, hv) data of the left, right, bottom, top sides.
 * 2D block operators use 3x3 blocks: J[(k*9 + l*3 + m)*n + c] =
 * (dR_c/dU_{c + off(k)})_{lm}, with the offset lists (dx, dy) sorted by dy then
 * dx: J9 (the cross of Eq. 21) (0,-2) (0,-1) (-2,0) (-1,0) (0,0) (1,0) (2,0)
 * (0,1) (0,2); J21 (the 21-cell stencil of Section 4.1): |dx| <= 2, |dy| <= 1
 * or |dx| <= 1, |dy| <= 2. */
nswe_status nswe_prob_create_2d(nswe_ctx ctx, nswe_prob *out, int Nx, int Ny,
                                int levels, double x0, double x1, double y0,
                                double y1, double g, const double *gauss_geom,
                                const int *bc_kind, const double *bc_state);
nswe_status nswe_prob_destroy(nswe_prob prob);
int nswe_prob_cells(nswe_prob prob, int level);
int nswe_prob_dim(nswe_prob prob);

/* Residual R_j = F_{j+1/2} - F_{j-1/2} - S_j (Eq. 10; not divided by dx)
 * of state U on nested level `level`: WENO3 reconstruction (Eq. 7-8, with
 * the linear weights that give third order), HLL flux, two-point Gauss
 * source of the cubic through four interface values (Eq. 9).
 *   U[2][N_l] in, R[2][N_l] out, res_l1 (device scalar, may be NULL) out =
 *   (1/N_l) sum_j ||R_j||_1 (Algorithm 1, step 7). */
nswe_status nswe_residual(nswe_ctx ctx, nswe_prob prob, int level,
                          const double *U, double *R, double *res_l1);

/* Regularized finite-difference Jacobian (Eq. 12-13) of the residual at U:
 * one-sided differences of the local residual with U_i perturbed by eps in
 * one component (ghost cells follow the perturbed interior cell), plus
 * alpha*||R_j||_1 on the diagonal block. The simplified call keeps the three
 * central blocks (J3, Section 3.3); the full call keeps all five (J5).
 *   U[2][N_l] in; R[2][N_l] out (the residual at U); J[nb][4][N_l] out;
 *   res_l1 (device scalar, may be NULL) out. */
nswe_status nswe_jacobian_simplified(nswe_ctx ctx, nswe_prob prob, int level,
                                     const double *U, double eps, double alpha,
                                     double *R, double *J, double *res_l1);
nswe_status nswe_jacobian_full(nswe_ctx ctx, nswe_prob prob, int level,
                               const double *U, double eps, double alpha,
                               double *R, double *J, double *res_l1);

/* 2D Jacobian of Eq. 12-13 under the frozen linearisation (NSWE_JAC_FROZEN;
 * not in the paper): nb = 9 (J9) or 21 (J21); U, R [3][n_l], J [nb][9][n_l],
 * res_l1 (device scalar, may be NULL) as in nswe_jacobian_simplified. A 1D
 * problem or another nb: NSWE_EINVAL. */
nswe_status nswe_jacobian_frozen(nswe_ctx ctx, nswe_prob prob, int level, int nb,
                                 const double *U, double eps, double alpha,
                                 double *R, double *J, double *res_l1);

/* The Jacobian of a NSWE_PREC_MIXED Newton step: R and res_l1 as in
 * nswe_residual (FP64); J the Jacobian of Eq. 12-13 stored in FP32, with the
 * regularization alpha*||R_j||_1 taken from the FP64 R. 1D: the perturbed
 * residuals are evaluated in FP32 from the FP64 state; nb = 3 (J3) or 5 (J5),
 * U, R [2][N_l] (double), J [nb][4][N_l] (float). 2D: evaluated in FP64,
 * rounded to FP32; nb = 9 (J9) or 21 (J21), U, R [3][n_l] (double),
 * J [nb][9][n_l] (float). res_l1 (device scalar, may be NULL) out. */
nswe_status nswe_jacobian_f32(nswe_ctx ctx, nswe_prob prob, int level, int nb,
                              const double *U, double eps, double alpha,
                              double *R, float *J, double *res_l1);

/* One multigrid V-cycle (Algorithm 2) for J dU = -R on nested level `level`
 * with the hierarchy level..levels-1: Galerkin coarse operators (Eq. 17),
 * nu1/nu2 symmetric multicolour block-SOR steps (Eq. 19; colours j mod C,
 * C = 2 for J3 and coarse levels, 3 for J5, visited 0..C-1 then C-1..0),
 * defect restriction (Eq. 17), prolongation (Eq. 18), and an exact solve by
 * LU with partial pivoting on the coarsest level.
 *   nb = 3 or 5; J[nb][4][N_l], R[2][N_l] in; dU[2][N_l] in/out. */
nswe_status nswe_mg_vcycle(nswe_ctx ctx, nswe_prob prob, int level, int nb,
                           const double *J, const double *R, double *dU,
                           const nswe_params *params);

/* The smoother of Algorithm 2 alone on one 2D level: params->nu1 steps of
 * the multicolour block SOR of Eq. 22 (relaxation params->omega, schedule
 * params->colours2d as in a V-cycle: K = 0 two symmetric passes of the
 * stencil colouring per step, K >= 3 the directional schedule), after the
 * inverse diagonal blocks of J are formed in the problem's workspace. No
 * coarse correction. 2D problems only (1D: NSWE_EINVAL).
 *   nb            9 (J9) or 21 (J21).
 *   J             DEVICE [nb][9][S]: cell-contiguous (colour_major = 0,
 *                 S = n_l, cell (i, j) at j*Nx + i), or, for J9 only,
 *                 colour-major (colour_major = 1) as the library stores large
 *                 Newton levels: the cells of colour (i + j) mod 3 form one
 *                 plane of Ny rows of W3 = ceil(Nx/3) slots, cell (i, j) at
 *                 ((i + j) mod 3 * Ny + j) * W3 + i / 3, S = 3 * Ny * W3.
 *   R             DEVICE [3][n_l] right-hand side of J dU = -R; dU DEVICE
 *                 [3][n_l] in/out (cell-contiguous in both layouts).
 *   launches      HOST, may be NULL: the number of colour-pass launches.
 * Asynchronous on the context stream. */
nswe_status nswe_mg_smooth(nswe_ctx ctx, nswe_prob prob, int level, int nb,
                           const double *J, const double *R, double *dU,
                           const nswe_params *params, int colour_major,
                           int *launches);

/* nswe_mg_vcycle in FP32, the linear solve of a NSWE_PREC_MIXED step: J, R
 * (float) in and dU (float) in/out in the layouts of nswe_mg_vcycle (nb = 3
 * or 5 in 1D, 9 or 21 in 2D). The coarse levels reuse the problem's
 * workspace, which this call overwrites. */
nswe_status nswe_mg_vcycle_f32(nswe_ctx ctx, nswe_prob prob, int level, int nb,
                               const float *J, const float *R, float *dU,
                               const nswe_params *params);

/* Nested NMGM (Algorithm 3). Starts on level s = params->nest_start (or the
 * coarsest): Newton iterations with a direct solve on the coarsest level,
 * with nu3 V-cycles from dU = 0 on other levels; damped update (Eq. 14);
 * then App. A interpolation to the next finer level, until level 0.
 *   U0[2][N_s] in (initial guess on level s), U[2][N_0] out.
 *   info (HOST pointer, may be NULL) is filled; the call synchronises the
 *   context stream when info != NULL. Returns the finest level's status. */
nswe_status nswe_newton_solve(nswe_ctx ctx, nswe_prob prob, const double *U0,
                              double *U, const nswe_params *params,
                              nswe_info *info);

/* Batched Algorithm 3: `count` independent problems of one dimension. 1D:
 * one launch, one thread block per problem. 2D: the solves run concurrently,
 * each sequenced by a host worker thread on its own stream (up to 8 at a
 * time) after the work already queued on the context stream; the call
 * returns when all have finished. A problem may appear once per batch
 * (NSWE_EINVAL otherwise, 2D). probs[], U0s[], Us[] are HOST arrays of count
 * entries (U0s[i], Us[i] device pointers as in nswe_newton_solve); infos
 * (HOST, may be NULL) receives count records and makes the 1D call
 * synchronous. */
nswe_status nswe_newton_solve_batch(nswe_ctx ctx, int count,
                                    const nswe_prob *probs,
                                    const double *const *U0s,
                                    double *const *Us,
                                    const nswe_params *params,
                                    nswe_info *infos);

/* Batched Algorithm 3 with parameters per problem (uneven instances sharing
 * one batch): params is a HOST array of `count` records, params[i] for
 * problem i, each checked as in nswe_newton_solve; everything else as in
 * nswe_newton_solve_batch. A 1D batch is one launch, which computes in one
 * arithmetic type: all records must then share `precision` (NSWE_EINVAL
 * otherwise), while J3 and J5 tasks, relaxation factors, smoothing counts,
 * tolerances and nested start levels may differ. In 2D each record may also
 * choose its own Jacobian (J9, J21, | NSWE_JAC_FROZEN) and precision. */
nswe_status nswe_newton_solve_batch_each(nswe_ctx ctx, int count,
                                         const nswe_prob *probs,
                                         const double *const *U0s,
                                         double *const *Us,
                                         const nswe_params *params,
                                         nswe_info *infos);

/* Launch shapes of the batched 1D solve kernel (one thread block per
 * problem): shape i has nswe_solve_shape_info(i) threads per block and is
 * built for that many resident blocks per SM. Which shape is fastest depends
 * on the precision, the problem sizes and the batch size; the context keeps
 * one shape per precision (shape 0 until changed), used by
 * nswe_newton_solve and nswe_newton_solve_batch on 1D problems. */
int nswe_solve_shape_count(void);
nswe_status nswe_solve_shape_info(int shape, int *threads, int *blocks_per_sm);
nswe_status nswe_ctx_set_solve_shape(nswe_ctx ctx, int precision, int shape);
nswe_status nswe_ctx_get_solve_shape(nswe_ctx ctx, int precision, int *shape);

/* Latency form of the 1D solve (the paper has no counterpart; Algorithm 3
 * itself is unchanged): with ctas >= 2, nswe_newton_solve and
 * nswe_newton_solve_batch give each 1D problem a thread-block cluster of
 * `ctas` CTAs (128 threads each) on as many SMs instead of one thread block.
 * The residual, Jacobian, update and the multigrid levels of at least
 * team_cells cells run on all CTAs of the cluster, with cluster barriers
 * between phases; the coarser levels and the coarsest LU run on its first
 * CTA. Every cell sees the same arithmetic as in the block form; the sum
 * that forms res is taken in another order, so res (and in rare cases the
 * Newton step at which it crosses tol) may differ in the last bits.
 * Worthwhile for few problems at a time (one solve's latency); a full batch
 * runs faster in the block form. ctas = 1 restores the block form (the
 * default); 2..16 (sizes above 8 need the GPU's non-portable cluster sizes);
 * team_cells >= 1; NSWE_EINVAL otherwise. LLF problems always run in the
 * block form. nswe_ctx_get_solve_cluster reads both settings (either
 * pointer may be NULL). */
nswe_status nswe_ctx_set_solve_cluster(nswe_ctx ctx, int ctas, int team_cells);
nswe_status nswe_ctx_get_solve_cluster(nswe_ctx ctx, int *ctas, int *team_cells);

/* Autotuner of the launch shape (the paper has no counterpart): solves the
 * given 1D batch once untimed and `reps` times timed (CUDA events on the
 * context stream) in every shape, records the fastest for params->precision
 * in the context, writes the mean milliseconds per batch of each shape to
 * ms[nswe_solve_shape_count()] (may be NULL) and the chosen shape to *best
 * (may be NULL). Arguments as nswe_newton_solve_batch; the solutions in Us
 * are overwritten. Synchronises the context stream. */
nswe_status nswe_autotune_solve_batch(nswe_ctx ctx, int count,
                                      const nswe_prob *probs,
                                      const double *const *U0s,
                                      double *const *Us,
                                      const nswe_params *params, int reps,
                                      double *ms, int *best);

/* Throughput probe of the FMA pipes (the paper has no counterpart): the
 * measured denominators of the arithmetic rooflines, since the FD Jacobian
 * (Eq. 12) and the multigrid sweeps of this library are bound by FP64 issue.
 * Launches `blocks` x `threads` threads on `stream` (cudaStream_t as void*),
 * each running `iters` rounds of 8 independent fused multiply-add chains in
 * FP64 (precision NSWE_PREC_FP64) or FP32 (NSWE_PREC_MIXED), and writes one
 * value per thread to `sink` (DEVICE, blocks*threads doubles or floats).
 * *flops (HOST, may be NULL) receives 2 * 8 * blocks * threads * iters; the
 * caller times the launch with CUDA events on the stream. Asynchronous.
 * threads must be a multiple of 32 in [32, 1024]; otherwise NSWE_EINVAL. */
nswe_status nswe_probe_fma(void *stream, int precision, int blocks,
                           int threads, int iters, void *sink, double *flops);

/* Allocation-free nested solve. The paper has no counterpart: this entry
 * point exists for callers that cannot call cudaMalloc, such as code running
 * after another allocator (e.g. a framework's caching allocator) has
 * reserved the device memory it may use, or real-time loops that must not
 * block on the device synchronisation cudaMalloc/cudaFree imply. It runs the
 * same solve as nswe_newton_solve on one problem of at most
 * NSWE_NOALLOC_MAX_CELLS cells, with the problem description and workspace
 * in a fixed device array of the library (about 3.4 MB, held by every GPU that
 * loads the library until the process exits); it allocates nothing.
 *   device       CUDA device index; it is made current for the call.
 *   stream       cudaStream_t as void* (NULL: legacy default stream).
 *   N, levels, x0, x1, g, left, right: as in nswe_prob_create_1d, with
 *                N <= NSWE_NOALLOC_MAX_CELLS (larger N returns NSWE_EINVAL).
 *   sigma_face   DEVICE [N+1] width at the finest faces.
 *   gauss_geom   DEVICE, the per-level Gauss-point geometry in the layout of
 *                nswe_prob_create_1d; read in place.
 *   U0, U        DEVICE, as in nswe_newton_solve.
 *   info         DEVICE pointer to one nswe_info, or NULL.
 * Asynchronous on `stream`. The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress); make that first call before any
 * stream capture. All calls share the array, which keeps the last call's
 * contents; calls that overlap on the GPU race and must be serialised by the
 * caller. The looked-up address is kept for the life of the process: after
 * cudaDeviceReset on a device the array may move, so this entry point must
 * not be called on that device again in the same process. */
#define NSWE_NOALLOC_MAX_CELLS 4096
nswe_status nswe_newton_solve_noalloc(int device, void *stream, int N,
                                      int levels, double x0, double x1,
                                      double g, const double *sigma_face,
                                      const double *gauss_geom,
                                      const nswe_bc1d *left,
                                      const nswe_bc1d *right,
                                      const double *U0, double *U,
                                      const nswe_params *params,
                                      nswe_info *info);

/* ------------------------------------------------------------------------
 * Continuous-batching solve server (1D). The paper has no counterpart: this
 * is the serving form of nswe_newton_solve_batch for a stream of requests of
 * different sizes. Each request is one nested solve (Algorithm 3) described
 * by host arrays, copied at submission. The server owns one device arena of
 * device_bytes and one pinned host arena of host_bytes; a request is
 * admitted, in submission order, once its footprint
 * (nswe_server_footprint_1d) fits, and its problem data and Newton /
 * multigrid workspace stay resident in its block until it completes.
 * Admitted requests are launched together, one thread block each, on an
 * idle stream among `streams`, at most max_batch per launch and one
 * precision per launch; launches on different streams overlap on the GPU.
 * A scheduler thread owned by the server issues all of its CUDA work; the
 * calls below are thread-safe. A solve's result does not depend on the
 * other requests it is launched with.
 *
 * 2D requests (nswe_server_submit_2d, when device_bytes_2d > 0) are served
 * by `streams` worker threads, each with its own stream: a request is
 * admitted, in submission order, once its footprint
 * (nswe_server_footprint_2d) fits in device_bytes_2d besides the 2D solves
 * running; its worker then builds the problem, runs the nested solve (the
 * host sequences each 2D Newton step) and copies the result back, and the
 * solves of different workers overlap on the GPU. Tickets, polling,
 * waiting and results are shared with the 1D requests.
 * ------------------------------------------------------------------------ */
typedef struct {
  size_t device_bytes; /* device arena for resident solves (>= 1 MiB)        */
  size_t host_bytes;   /* pinned staging arena (>= 1 MiB)                    */
  int streams;         /* concurrent launches, 1..16                         */
  int max_batch;       /* solves per launch, 1..65536                        */
  double batch_window_s; /* a launch that is not full waits until its oldest
                            request has waited this long (0: launch at once) */
  size_t device_bytes_2d; /* device bytes for 2D solves in flight (0: the
                             server refuses 2D requests)                  */
} nswe_server_config;

typedef struct { /* host steady-clock nanoseconds */
  unsigned long long t_submit_ns, t_admit_ns, t_launch_ns, t_done_ns;
} nswe_server_times;

typedef struct {
  long long submitted, completed, launches;
  int waiting, running;
  size_t device_bytes_used, device_bytes_peak;
} nswe_server_stats;

typedef struct nswe_server_s *nswe_server;

/* Device bytes a request of N cells, `levels` levels and nested start level
 * nest_start (<0: coarsest) occupies in the arena; 0 for invalid sizes. */
size_t nswe_server_footprint_1d(int N, int levels, int nest_start);

/* Device bytes a 2D request of Nx x Ny cells and `levels` levels asks of the
 * device allocator while it runs (problem, workspace, guess on the nested
 * start level nest_start (<0: coarsest) and result); 0 for invalid sizes. */
size_t nswe_server_footprint_2d(int Nx, int Ny, int levels, int nest_start);

/* Allocates the arenas, streams and the scheduler thread on `device`.
 * EINVAL for a bad config, ENOMEM if an arena cannot be allocated. A 1D
 * launch gives each request one thread block of 128 threads (FP64; the
 * launch shape 128 x 4 of nswe_solve_shape_info) or 256 threads (mixed
 * precision; 256 x 4), or a cluster (nswe_server_set_cluster). */
nswe_status nswe_server_create(nswe_server *out, int device,
                               const nswe_server_config *cfg);

/* Queues one solve. Arguments as nswe_prob_create_1d (HOST arrays) plus
 * U0 (HOST [2][N_s], N_s the cells of the nested start level) and params
 * (copied; eps per level, precision and jacobian per request). Returns a
 * ticket. EINVAL for invalid input, ENOMEM if the footprint exceeds an
 * arena (it could never be admitted), the server's error after a CUDA
 * failure. */
nswe_status nswe_server_submit_1d(nswe_server s, int N, int levels, double x0,
                                  double x1, double g,
                                  const double *sigma_face,
                                  const double *gauss_geom,
                                  const nswe_bc1d *left,
                                  const nswe_bc1d *right, const double *U0,
                                  const nswe_params *params,
                                  unsigned long long *ticket);

/* Queues one 2D solve. Arguments as nswe_prob_create_2d (HOST arrays) plus
 * U0 (HOST [3][n_s], n_s the cells of the nested start level) and params
 * (copied; the Jacobian choice, NSWE_JAC_FROZEN included, and precision per
 * request). Returns a ticket. EINVAL for invalid input or when the server
 * takes no 2D requests, ENOMEM if the footprint exceeds device_bytes_2d (it
 * could never be admitted), the server's error after a CUDA failure. */
nswe_status nswe_server_submit_2d(nswe_server s, int Nx, int Ny, int levels,
                                  double x0, double x1, double y0, double y1,
                                  double g, const double *gauss_geom,
                                  const int *bc_kind, const double *bc_state,
                                  const double *U0, const nswe_params *params,
                                  unsigned long long *ticket);

/* Tickets completed since the last poll (up to max, in completion order). */
nswe_status nswe_server_poll(nswe_server s, unsigned long long *tickets,
                             int max, int *count);

/* Blocks until at least min_completed tickets await polling, or timeout_s
 * seconds pass (NSWE_ETIMEOUT). */
nswe_status nswe_server_wait(nswe_server s, int min_completed,
                             double timeout_s);

/* Result of a completed ticket: U (HOST [2][N] in 1D, [3][Nx Ny] in 2D,
 * may be NULL), the solve record and the host timestamps; the ticket is
 * released. EINVAL for a ticket that is not (or no longer) complete. */
nswe_status nswe_server_take(nswe_server s, unsigned long long ticket,
                             double *U, nswe_info *info,
                             nswe_server_times *times);

nswe_status nswe_server_query(nswe_server s, nswe_server_stats *out);

/* Latency form for light load (see nswe_ctx_set_solve_cluster): a 1D launch
 * runs each of its problems on a thread-block cluster of `ctas` CTAs when the
 * 1D solves in flight, the launch's own included, are at most
 * max_in_flight; otherwise, and always with ctas = 1 (the default), one
 * thread block per problem. team_cells as in nswe_ctx_set_solve_cluster.
 * May be called at any time; applies from the next launch. EINVAL for ctas
 * outside 1..16, max_in_flight < 0 or team_cells < 1. */
nswe_status nswe_server_set_cluster(nswe_server s, int ctas, int max_in_flight,
                                    int team_cells);

/* Stops the scheduler after the launched work finishes, frees everything;
 * requests not yet launched are dropped. */
nswe_status nswe_server_destroy(nswe_server s);

/* The server's arena allocator, exposed for tests and for callers that
 * manage their own device pools: first fit over [0, bytes), offsets and
 * lengths rounded up to `align` (a power of two), freed blocks coalesced
 * with free neighbours. No device memory is involved. */
typedef struct nswe_arena_s *nswe_arena;
nswe_status nswe_arena_create(nswe_arena *out, size_t bytes, size_t align);
nswe_status nswe_arena_alloc(nswe_arena a, size_t bytes, size_t *offset);
nswe_status nswe_arena_free(nswe_arena a, size_t offset);
nswe_status nswe_arena_query(nswe_arena a, size_t *used, size_t *peak,
                             size_t *largest_free);
nswe_status nswe_arena_destroy(nswe_arena a);

#ifdef __cplusplus
}
#endif
#endif
