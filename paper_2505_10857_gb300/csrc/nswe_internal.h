// Internal declarations shared by the host side of the library and its CUDA
// kernels: the device-resident problem description and the kernel launchers.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "../../include/nswe.h"

namespace nswe {

#ifndef NSWE_THREADS
#define NSWE_THREADS 256           // threads per block of every 1D kernel
#endif
constexpr int kThreads = NSWE_THREADS;

// Launch shapes of the persistent solve kernel, (threads per block, resident
// blocks per SM it is built for): the register budget per thread follows
// from the pair (65536 registers per SM). Shape 0 is the default.
constexpr int kSolveShapes = 6;
constexpr int kSolveShapeThreads[kSolveShapes] = {256, 128, 256, 128, 160, 192};
constexpr int kSolveShapeBlocks[kSolveShapes] = {4, 8, 2, 4, 4, 4};
constexpr int kMaxCoarse = 128;    // max cells of the coarsest level (direct solve)
// Launch shapes of the serving server's 1D block launches, per precision:
// 128 x 4 in FP64 (128 registers a thread, no spills), 256 x 4 in mixed
// precision (the faster of the two there).
constexpr int kServerShapeFp64 = 3;
constexpr int kServerShapeMixed = 0;
static_assert(kSolveShapeThreads[kServerShapeFp64] == 128 && kSolveShapeBlocks[kServerShapeFp64] == 4,
              "FP64 server shape is 128 x 4");
static_assert(kSolveShapeThreads[kServerShapeMixed] == 256 && kSolveShapeBlocks[kServerShapeMixed] == 4,
              "mixed server shape is 256 x 4");
// The latency form of the solve kernel: one problem per thread-block cluster
// of up to kMaxClusterCtas CTAs of kClusterThreads threads.
constexpr int kClusterThreads = 128;
constexpr int kMaxClusterCtas = 16;

// One nested / multigrid level of a 1D problem. Geometry is read-only input;
// the rest is solver workspace owned by the problem.
struct LevelDev {
  int N;
  double dx;
  const double *sf;  // [N+1] width at faces
  const double *gq;  // [3][2][N] sigma, sigma_x, b_x at the two Gauss points
  double *U;         // [2][N] nested-level solution
  double *R;         // [2][N] residual / multigrid right-hand side
  double *J;         // [5][4][N] Jacobian (nb blocks used)
  double *Dinv;      // [4][N] inverse diagonal blocks
  double *dU;        // [2][N] multigrid correction
  double *gd;        // [4N+2] derived from the geometry by launch_geom_derive:
                     // 1/sigma at faces [N+1], sqrt(g/sigma) at faces [N+1],
                     // 1/sigma at the Gauss points [2][N]
};

struct ProbDev {
  int levels;
  double g;
  int bl, br;        // boundary kinds (nswe_bc_kind)
  double blh, blq, brh, brq;
  int flux;          // numerical flux: NSWE_FLUX_HLL (0) or NSWE_FLUX_LLF
  double *jw;        // Jacobian workspace: 16*(N+2) + 18*(N+1) doubles, finest N
  LevelDev lev[NSWE_MAX_LEVELS];
};

// Doubles of Jacobian workspace for a level of N cells.
__host__ __device__ inline size_t jw_doubles(size_t N) { return 16 * (N + 2) + 18 * (N + 1); }
// Doubles of derived geometry per level of N cells.
inline size_t gd_doubles(size_t N) { return 4 * N + 2; }

// ---------------------------------------------------------------- 2D
// Block stencils of 2D operators (offset tables in nswe_kernels_2d.cu).
constexpr int ST_J9 = 0, ST_J21 = 1, ST_P5 = 2, ST_P9 = 3;
inline int st_size_host(int st) { return st == ST_J9 ? 9 : st == ST_J21 ? 21 : st == ST_P5 ? 5 : 9; }
inline int st_coarse_host(int st) { return (st == ST_J9 || st == ST_P5) ? ST_P5 : ST_P9; }
inline int st_colours_host(int st) { return st == ST_J9 ? 3 : st == ST_J21 ? 9 : st == ST_P5 ? 2 : 4; }

struct Level2Dev {
  int Nx, Ny;
  double dx, dy;
  const double *gq;  // [2][4][n]: b_x, b_y at the Gauss points q = 2*beta + gamma
  const int *bck;    // [2*Ny + 2*Nx] boundary kinds: left, right, bottom, top
  double *U, *R, *dU;  // [3][n]
  double *J;           // [21][9][n]
  double *Dinv;        // [9][n]
};

struct ProbDev2 {
  int levels;
  double g;
  double bcs[12];    // (h, hu, hv) data per side
  Level2Dev lev[NSWE_MAX_LEVELS];
};

cudaError_t launch2_residual(const ProbDev2 *p, int level, int n, const double *U, double *R, double *res,
                             double *partials, cudaStream_t s);
// Multigrid launchers for T = double (FP64 path) and T = float (the multigrid
// of a mixed-precision step); the Jacobian may be stored in either.
// Storage of the 3x3 blocks (J, Dinv) of one level: cell-contiguous (cm = 0:
// stride n, cell (i, j) at j Nx + i) or colour-major for the J9 colouring
// (cm = 1): the cells of colour (i + j) mod 3 form one plane of Ny rows of
// W3 = ceil(Nx / 3) slots, cell (i, j) at slot i / 3 of row j of its plane,
// so that a colour pass reads one contiguous plane; stride 3 Ny W3 (at most
// two unused slots per row of a plane).
__host__ __device__ __forceinline__ size_t blk_stride(int cm, int Nx, int Ny) {
  return cm ? 3 * (size_t)Ny * (size_t)((Nx + 2) / 3) : (size_t)Nx * (size_t)Ny;
}
__host__ __device__ __forceinline__ size_t blk_pos(int cm, int Nx, int Ny, int i, int j) {
  return cm ? ((size_t)((i + j) % 3) * Ny + j) * (size_t)((Nx + 2) / 3) + (size_t)(i / 3) : (size_t)j * Nx + i;
}

// frozen: the frozen linearisation (weights and eigenvectors from U); cm:
// the storage of J (blk_pos); levels of at least cell_min cells (>= 0) take
// the one-cell-per-thread kernel, the others one (cell, block) item per
// thread (the same bits either way).
constexpr int kJac2CellMinDefault = 32768;
template <typename TJ>
cudaError_t launch2_jacobian(const ProbDev2 *p, int level, int n, int st, const double *U, double eps, double alpha,
                             const double *R, TJ *J, bool frozen, int cm, int cell_min, cudaStream_t s);
template <typename T>
cudaError_t launch2_coarse_op(int Nx, int Ny, int st, const T *Jf, T *Jc, int cm, cudaStream_t s);
template <typename T>
cudaError_t launch2_dinv(int Nx, int Ny, int st, const T *J, T *Dinv, int cm, cudaStream_t s);
// mode 0: cells of colour col of the stencil's colouring; mode 1 / 2: of the
// diagonal colourings (i + j) mod Kc / (j - i + Nx - 1) mod Kc.
template <typename T>
cudaError_t launch2_sor(int Nx, int Ny, int st, const T *J, const T *Dinv, const T *R, T *dU, double omega, int mode,
                        int Kc, int col, int reps, int cm, cudaStream_t s);
template <typename T>
cudaError_t launch2_restrict(int Nx, int Ny, int st, const T *J, const T *R, const T *dU, T *Rc, T *dUc, int cm,
                             cudaStream_t s);
template <typename T>
cudaError_t launch2_prolong(int Nx, int Ny, T *dU, const T *dUc, cudaStream_t s);
template <typename T>
cudaError_t launch2_dense_factor(int Nx, int Ny, int st, const T *J, T *A, int *piv, int *flag, cudaStream_t s);
template <typename T>
cudaError_t launch2_dense_solve(int n, const T *A, const int *piv, const T *R, T *x, T *dU, cudaStream_t s);
template <typename T>
cudaError_t launch2_update(int n, double *U, const T *dU, double tau, int *flag, cudaStream_t s);
cudaError_t launch2_to_f32(long count, const double *src, float *dst, cudaStream_t s);

// The levels ls..L of a 2D V-cycle (down-leg, coarsest solve with the dense
// factors A/piv, up-leg) run by one thread block: the levels of at most
// tail2_cells<T>() cells, where one launch per colour pass would cost
// more than the pass. One SM issues FP32 at 64x its FP64 rate, so the FP64
// tail stops at far smaller levels.
template <typename T>
#ifndef NSWE_TAIL_F64
#define NSWE_TAIL_F64 256
#endif
#ifndef NSWE_TAIL_F32
#define NSWE_TAIL_F32 4096
#endif
constexpr int tail2_cells() { return sizeof(T) == 4 ? NSWE_TAIL_F32 : NSWE_TAIL_F64; }
#ifndef NSWE_TAIL_THREADS
#define NSWE_TAIL_THREADS 1024
#endif
constexpr int kTail2Threads = NSWE_TAIL_THREADS;
template <typename T>
struct Tail2 {
  int ls, L;
  int Nx[NSWE_MAX_LEVELS], Ny[NSWE_MAX_LEVELS], st[NSWE_MAX_LEVELS];
  T *J[NSWE_MAX_LEVELS], *Dinv[NSWE_MAX_LEVELS], *R[NSWE_MAX_LEVELS], *dU[NSWE_MAX_LEVELS];
  const T *A;
  const int *piv;
  T *x;
};
template <typename T>
cudaError_t launch2_vcycle_tail(const Tail2<T> &t, int nu1, int nu2, double omega, int Kc, cudaStream_t s);
cudaError_t launch2_interp(const ProbDev2 *p, int coarse_level, int nc, const double *Uc, double *Uf,
                           cudaStream_t s);

// ---------------------------------------------------------------- batched 2D
// Lockstep batches of 2D problems: every phase of a Newton step and every
// colour pass of its V-cycles is one launch over all problems of the batch.
// A problem owns the launch's blocks [b0, b0 + nb) (the instance -> tile
// map); inside them the same device code as the single-problem kernels runs
// on that problem's arrays, with the same per-problem block count where the
// result depends on it (the residual's partial sums), so a batched solve is
// the same bits as the problem solved alone. done[prob] != 0 (a problem that
// has converged on its current nested level) skips the problem's blocks.
template <typename T>
struct BTask2 {
  int b0, nb, prob;      // blocks [b0, b0 + nb) of the launch; the problem's index in the batch
  int Nx, Ny, st, cm;    // the level: grid, stencil, storage of J and Dinv (blk_pos)
  T *J, *Dinv, *R, *dU;  // its multigrid arrays (R: the right-hand side in T)
  T *Jc, *Rc, *dUc;      // the next coarser level's: Galerkin operator, restriction, prolongation
  const ProbDev2 *P;     // residual / Jacobian / update: the problem and its nested level
  int level, frozen, msplit;
  double *U, *R64;       // state and FP64 residual of the Newton level
  double *partials;      // residual partial sums (nb of them)
  float *R32;            // FP32 copy of R64 (mixed precision)
  double eps, alpha, tau;
  T *A, *x;              // dense coarsest system and its solve buffer
  int *piv;
};
// Launchers: tasks is a DEVICE array of ntask tasks sorted by b0, blocks the
// launch's grid (the sum of their nb), done / flags / res DEVICE arrays
// indexed by the task's prob.
template <typename T>
struct Batch2Launch {
  const BTask2<T> *tasks;
  int ntask, blocks;
};
cudaError_t launchb2_residual(const Batch2Launch<double> &b, const int *done, double *res, cudaStream_t s);
template <typename TJ>
cudaError_t launchb2_jacobian(const Batch2Launch<TJ> &b, const int *done, int kind, bool frozen, cudaStream_t s);
constexpr int kB2JacItems = 0, kB2JacCells = 1;  // launchb2_jacobian kinds
int b2_jacobian_cell_threads();
cudaError_t launchb2_to_f32(const Batch2Launch<float> &b, const int *done, cudaStream_t s);
template <typename T>
cudaError_t launchb2_zero_du(const Batch2Launch<T> &b, const int *done, cudaStream_t s);
template <typename T>
cudaError_t launchb2_coarse_op(const Batch2Launch<T> &b, const int *done, cudaStream_t s);
template <typename T>
cudaError_t launchb2_dinv(const Batch2Launch<T> &b, const int *done, cudaStream_t s);
// one colour pass (mode, Kc, col, reps as launch2_sor) of every task; all
// tasks of the launch share the stencil st
template <typename T>
cudaError_t launchb2_sor(const Batch2Launch<T> &b, const int *done, int st, double omega, int mode, int Kc, int col,
                         int reps, cudaStream_t s);
constexpr int kB2SorThreads = 128, kB2SorCellsPerBlock = 40;  // three lanes per cell, ten cells per warp
template <typename T>
cudaError_t launchb2_restrict(const Batch2Launch<T> &b, const int *done, cudaStream_t s);
template <typename T>
cudaError_t launchb2_prolong(const Batch2Launch<T> &b, const int *done, cudaStream_t s);
// one block per task: the tail of each task's V-cycle (tails[i] for tasks[i])
template <typename T>
cudaError_t launchb2_vcycle_tail(const Tail2<T> *tails, const BTask2<T> *tasks, int ntask, const int *done, int nu1,
                                 int nu2, double omega, int Kc, cudaStream_t s);
template <typename T>
cudaError_t launchb2_dense_factor(const Batch2Launch<T> &zero, const Batch2Launch<T> &scatter, const BTask2<T> *tasks,
                                  int ntask, const int *done, int *flags, cudaStream_t s);
template <typename T>
cudaError_t launchb2_dense_solve(const BTask2<T> *tasks, int ntask, const int *done, cudaStream_t s);
template <typename T>
cudaError_t launchb2_update(const Batch2Launch<T> &b, const int *done, int *flags, cudaStream_t s);
int b2_grid(long items);  // blocks of kThreads for `items` grid-stride items (as the single launches)
// Programmatic dependent launch of the 2D kernels (process-wide; on by default).
void set_pdl_2d(int on);
int get_pdl_2d();
// Lockstep batched 2D solves (nswe_batch2d.cu): problems grouped by precision,
// Jacobian stencil and smoothing schedule; prms[each ? i : 0] are problem i's.
nswe_status solve2d_lockstep(nswe_ctx ctx, int count, const nswe_prob *probs, const double *const *U0s,
                             double *const *Us, const nswe_params *prms, bool each, nswe_info *infos);
// The parameters and tail threshold (cells) a 2D solve of `p` runs with:
// colours2d = NSWE_COLOURS2D_AUTO takes the schedule and tail that
// nswe_autotune_2d recorded for p's size and precision (none recorded:
// schedule 0 and the context's tail).
void resolve2d(const nswe_prob_s *p, const nswe_params &in, nswe_params &out, int &tail);

// One solve of a batch.
struct SolveTask {
  const ProbDev *prob;
  const double *U0;
  double *U;
  nswe_info *info;           // device record
  const nswe_params *prm;    // device copy of this solve's parameters, or
                             // null for the launch's parameters
  int derive;                // 1: fill prob's derived geometry first
  int *done;                 // null, or a flag set to 1 (system scope) once
                             // U and info are written: lets the host see
                             // each solve of a launch complete on its own
};

// Kernel launchers (stream-ordered, return cudaGetLastError()).
// Fills every level's gd from its sf and gq (after each geometry upload).
cudaError_t launch_geom_derive(const ProbDev *p, int finest_cells, cudaStream_t s);
// The derived geometry of tasks[0..count).prob, one block each.
cudaError_t launch_geom_derive_batch(const SolveTask *tasks, int count, cudaStream_t s);
cudaError_t launch_residual(const ProbDev *p, int level, int N, const double *U, double *R, double *res,
                            double *partials, cudaStream_t s);
cudaError_t launch_jacobian(const ProbDev *p, int level, int N, int nb, const double *U, double eps,
                            double alpha, double *R, double *J, double *res, double *partials,
                            cudaStream_t s);
// FP64 residual (R, res) then the FP32 Jacobian regularised with that R.
cudaError_t launch_jacobian_f32(const ProbDev *p, int level, int N, int nb, const double *U, double eps,
                                double alpha, double *R, float *J, double *res, double *partials,
                                cudaStream_t s);
// coarse_cells: cells of the coarsest level; coarse_nb: its block band (3 or 5).
cudaError_t launch_vcycle(const ProbDev *p, int level, int nb, const double *J, const double *R, double *dU,
                          const nswe_params &prm, int *status, int coarse_cells, int coarse_nb, cudaStream_t s);
cudaError_t launch_vcycle_f32(const ProbDev *p, int level, int nb, const float *J, const float *R, float *dU,
                              const nswe_params &prm, int *status, int coarse_cells, int coarse_nb, cudaStream_t s);
// max_coarse_cells: largest coarsest level over the tasks; prm.precision
// selects the FP64 or the mixed-precision solve kernel.
cudaError_t launch_solve(const SolveTask *tasks, int count, const nswe_params &prm, int max_coarse_cells,
                         cudaStream_t s);
// The same with the coarsest band sized for max_nb (3 or 5) whatever prm
// says (for batches whose tasks carry their own parameters), in launch shape
// `shape` (0 .. kSolveShapes-1).
// flux: the numerical flux of every task (NSWE_FLUX_HLL, or NSWE_FLUX_LLF,
// which runs in the default shape).
cudaError_t launch_solve_sized(const SolveTask *tasks, int count, const nswe_params &prm, int max_coarse_cells,
                               int max_nb, int shape, cudaStream_t s, int flux = NSWE_FLUX_HLL);
// One problem per cluster of `ctas` CTAs (2..kMaxClusterCtas, HLL flux):
// multigrid levels with at least team_cells cells run on the whole cluster.
cudaError_t launch_solve_cluster(const SolveTask *tasks, int count, const nswe_params &prm, int max_coarse_cells,
                                 int max_nb, int ctas, int team_cells, cudaStream_t s);
// Parameter checks shared by the entry points (eps of levels 0..first_level).
nswe_status check_params_1d(const nswe_params *p, int levels, int first_level);
// Parameter checks of a 2D solve (the frozen linearisation allowed).
nswe_status check_params_2d(const nswe_params *p, int levels, int first_level);
// 2D problem sizes (nswe_prob_create_2d): arena doubles and all device bytes.
size_t prob2d_arena_doubles(int Nx, int Ny, int levels);
size_t prob2d_device_bytes(int Nx, int Ny, int levels);

}  // namespace nswe

// A choice of nswe_autotune_2d: smoothing schedule and tail threshold of the
// 2D V-cycles of problems of Nx x Ny cells in one precision.
struct nswe_tuned2d {
  int Nx, Ny, precision, colours, tail;
};

// A context and a problem of the C ABI (include/nswe.h): host-side handles
// of device resources, shared by the host translation units.
struct nswe_ctx_s {
  int device;
  cudaStream_t stream;
  double *partials;      // [1024] per-block partial sums of res
  int *status;           // device status word of standalone V-cycles
  nswe::SolveTask *tasks;      // device task array
  nswe_info *infos;      // device info records
  nswe_params *prms;     // device per-task parameters (nswe_newton_solve_batch_each)
  int cap;               // capacity of tasks / infos / prms
  int solve_shape[2];    // launch shape of the 1D solve kernel per precision
  int solve_ctas = 1;    // 1D solves: CTAs per problem (1: a block per problem; 2..16: a cluster)
  int team_cells = 1024; // cluster form: multigrid levels with at least this many cells on every CTA
  int batch2d_lockstep = 1;  // 2D batches: 1 lockstep batched launches (default), 0 concurrent solves
  int cm2d_min_cells = 131072;  // 2D Newton levels of at least this many cells store J9 colour-major
  int jac2d_cell_min = nswe::kJac2CellMinDefault;  // 2D levels from which the per-cell Jacobian kernel runs
  // 2D V-cycles: levels of at most tail2[precision] cells run in the one-block tail (0 FP64, 1 mixed)
  int tail2[2] = {nswe::tail2_cells<double>(), nswe::tail2_cells<float>()};
  std::vector<nswe_tuned2d> tuned2;  // nswe_autotune_2d's choices per size and precision
};

struct nswe_prob_s {
  nswe_ctx ctx;
  int dim;               // 1 or 2
  int N, levels;         // 1D: cells of the finest level
  double x0, x1, g;
  nswe::ProbDev host;          // device pointers, host copy
  nswe::ProbDev *dev;          // device copy
  double *arena;
  size_t geo_doubles;    // geometry region at the front of the arena
  double *stage;         // 1D: pinned staging of the geometry upload [geo_doubles]
  cudaEvent_t staged;    // 1D: the last upload from `stage` has been copied
  // 2D
  int Nx, Ny;
  nswe::ProbDev2 host2;
  nswe::ProbDev2 *dev2;
  double *dense;         // coarsest dense LU factors [N3][N3]
  int *piv;              // [N3]
  double *xbuf;          // [N3]
  int *flag;             // device flag (zero pivot / non-positive depth)
  double *res_dev;       // device scalar
  double *res_host;      // pinned host scalar
  int *flag_host;        // pinned host flag
  cudaStream_t cap;      // 2D: stream on which a Newton step is captured
  double *partials2;     // 2D: [1024] per-block partial sums of res (per problem, so
                         // that several 2D solves can run concurrently)
};
