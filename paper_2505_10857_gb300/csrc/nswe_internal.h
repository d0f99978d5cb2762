// Internal declarations shared by the host side of the library and its CUDA
// kernels: the device-resident problem description and the kernel launchers.
#pragma once

#include <cuda_runtime.h>

#include "../../include/nswe.h"

namespace nswe {

#ifndef NSWE_THREADS
#define NSWE_THREADS 256           // threads per block of every 1D kernel
#endif
#ifndef NSWE_SOLVE_MIN_BLOCKS
#define NSWE_SOLVE_MIN_BLOCKS 4    // resident blocks per SM the solve kernel is built for
#endif
constexpr int kThreads = NSWE_THREADS;
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
};

struct ProbDev {
  int levels;
  double g;
  int bl, br;        // boundary kinds (nswe_bc_kind)
  double blh, blq, brh, brq;
  double *jw;        // Jacobian workspace: 16*(N+2) + 18*(N+1) doubles, finest N
  LevelDev lev[NSWE_MAX_LEVELS];
};

// Doubles of Jacobian workspace for a level of N cells.
inline size_t jw_doubles(size_t N) { return 16 * (N + 2) + 18 * (N + 1); }

// One solve of a batch.
struct SolveTask {
  const ProbDev *prob;
  const double *U0;
  double *U;
  nswe_info *info;   // device record
};

// Kernel launchers (stream-ordered, return cudaGetLastError()).
cudaError_t launch_residual(const ProbDev *p, int level, int N, const double *U, double *R, double *res,
                            double *partials, cudaStream_t s);
cudaError_t launch_jacobian(const ProbDev *p, int level, int N, int nb, const double *U, double eps,
                            double alpha, double *R, double *J, double *res, double *partials,
                            cudaStream_t s);
// coarse_cells: cells of the coarsest level; coarse_nb: its block band (3 or 5).
cudaError_t launch_vcycle(const ProbDev *p, int level, int nb, const double *J, const double *R, double *dU,
                          const nswe_params &prm, int *status, int coarse_cells, int coarse_nb, cudaStream_t s);
// max_coarse_cells: largest coarsest level over the tasks.
cudaError_t launch_solve(const SolveTask *tasks, int count, const nswe_params &prm, int max_coarse_cells,
                         cudaStream_t s);

}  // namespace nswe
