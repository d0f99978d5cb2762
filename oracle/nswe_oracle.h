/*
 * CPU oracle for the high-order Newton multigrid method (NMGM) with a
 * simplified Jacobian for steady shallow water equations (Hu, Li, Wang,
 * Wang, arXiv 2505.10857).
 *
 * TEST INFRASTRUCTURE ONLY. This is a plain, slow, single-threaded FP64
 * restatement of the paper's equations and algorithms, used to check the
 * CUDA path. Only the test suite, the smoke check and the CPU-baseline leg of
 * the benchmark may load it. It shares no source with the CUDA library and
 * must never be used as a fallback for it.
 *
 * Build: plain C11, -O2 -ffp-contract=off (no fused multiply-add), so that
 * results are identical on x86-64 and aarch64 hosts.
 *
 * Conventions (0-based indices throughout; the paper is 1-based):
 *   - cell j of a 1D grid with N cells spans faces j and j+1; face f sits at
 *     x0 + f*dx.
 *   - a state vector is stored as two planes: H[0..N) then Q[0..N).
 *   - a block-banded Jacobian with nb blocks per row (offsets -h..h,
 *     h=(nb-1)/2) is stored as J[(k*4 + l*2 + m)*N + j] = (dR_j/dU_{j+k-h})_{lm}.
 */
#ifndef NSWE_ORACLE_H
#define NSWE_ORACLE_H

#define OR_BC_DISCHARGE 1 /* given Q; H extrapolated from the edge cell      */
#define OR_BC_DEPTH 2     /* given h (H = sigma_b*h); Q extrapolated          */
#define OR_BC_STATE 3     /* given h and Q                                     */
#define OR_BC_EXTRAP 4    /* both extrapolated (zeroth order)                  */

typedef struct {
  int N;
  double x0, x1, dx, g;
  const double *sig_face; /* [N+1] channel width at faces                     */
  const double *gq;       /* [3][2][N]: sigma, sigma_x, b_x at the 2 Gauss pts */
  int bcl_kind, bcr_kind;
  double bcl_h, bcl_q, bcr_h, bcr_q;
  int flux; /* numerical flux: 0 HLL (the paper's 1D choice), 1 LLF        */
} or_grid1d;

#endif
