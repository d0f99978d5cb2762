// Internal declarations shared by the host side of the library and its CUDA
// kernels: the device-resident problem description and the kernel launchers.
#pragma once

#include <cuda_runtime.h>

#include "../../include/nswe.h"

namespace nswe {

#ifndef NSWE_THREADS
#define NSWE_THREADS 256           // threads per block of every 1D kernel
#endif
constexpr int kThreads = NSWE_THREADS;

// Launch shapes of the persistent solve kernel, (threads per block, resident
// blocks per SM it is built for): the register budget per thread follows
// from the pair (65536 registers per SM). Shape 0 is the default.
constexpr int kSolveShapes = 4;
constexpr int kSolveShapeThreads[kSolveShapes] = {256, 128, 256, 128};
constexpr int kSolveShapeBlocks[kSolveShapes] = {4, 8, 2, 4};
constexpr int kMaxCoarse = 128;    // max cells of the coarsest level (direct solve)

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
// Parameter checks shared by the entry points (eps of levels 0..first_level).
nswe_status check_params_1d(const nswe_params *p, int levels, int first_level);
// Parameter checks of a 2D solve (the frozen linearisation allowed).
nswe_status check_params_2d(const nswe_params *p, int levels, int first_level);
// 2D problem sizes (nswe_prob_create_2d): arena doubles and all device bytes.
size_t prob2d_arena_doubles(int Nx, int Ny, int levels);
size_t prob2d_device_bytes(int Nx, int Ny, int levels);

}  // namespace nswe
