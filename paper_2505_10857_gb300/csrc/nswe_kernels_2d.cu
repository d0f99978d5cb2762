// CUDA kernels (sm_103a) of the 2D NMGM (Section 4), FP64: the residual of
// Eq. 20 with dimension-by-dimension characteristic WENO3, LLF fluxes at the
// two Gauss points of each edge and the S2/S3 source quadratures; the FD
// Jacobians J21 and J9 (Eq. 21); Galerkin coarse operators by 2x2
// aggregation (Eq. 24); multicolour 3x3 block SOR (Eq. 22); restriction and
// prolongation (Eq. 24-25); a dense LU with partial pivoting on the coarsest
// grid; the App. A interpolation in tensor form (Eq. A.3).
//
// A 2D problem is large (512 x 256 cells = 131k cells, 85-200 MB of Jacobian),
// so every phase is a grid-wide kernel over cells; the host sequences them.
#include <atomic>
#include <cmath>
#include <type_traits>
#include <utility>

#include "nswe_internal.h"

namespace nswe {

// Programmatic dependent launch of the 2D kernels (on by default).
std::atomic<int> g_pdl2{1};
void set_pdl_2d(int on) { g_pdl2.store(on ? 1 : 0); }
int get_pdl_2d() { return g_pdl2.load(); }

// Stencil offset tables (dx, dy), sorted by dy then dx; index = position in
// the block storage J[(k*9 + l*3 + m)*n + c].
__constant__ int c_off_j9[9][2] = {{0, -2}, {0, -1}, {-2, 0}, {-1, 0}, {0, 0}, {1, 0}, {2, 0}, {0, 1}, {0, 2}};
__constant__ int c_off_j21[21][2] = {{-1, -2}, {0, -2}, {1, -2}, {-2, -1}, {-1, -1}, {0, -1}, {1, -1},
                                     {2, -1},  {-2, 0}, {-1, 0}, {0, 0},   {1, 0},   {2, 0},   {-2, 1},
                                     {-1, 1},  {0, 1},  {1, 1},  {2, 1},   {-1, 2},  {0, 2},   {1, 2}};
__constant__ int c_off_p5[5][2] = {{0, -1}, {-1, 0}, {0, 0}, {1, 0}, {0, 1}};
__constant__ int c_off_p9[9][2] = {{-1, -1}, {0, -1}, {1, -1}, {-1, 0}, {0, 0}, {1, 0}, {-1, 1}, {0, 1}, {1, 1}};

namespace {

// Programmatic dependent launch (sm_90 and later): every 2D kernel first
// waits until the kernel before it on the stream has completed and its
// writes are visible (griddepcontrol.wait), then lets the kernel after it
// begin launching (griddepcontrol.launch_dependents), so that a launch's
// set-up overlaps the previous kernel instead of following it. Both are
// no-ops for a launch without the programmatic-serialization attribute.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

constexpr double kZeta2 = 1e-6;
constexpr double kGs2 = 0.28867513459481288225;   // 1/(2 sqrt 3)
constexpr double kTq = 0.14433756729740644113;    // 1/(4 sqrt 3)
__device__ constexpr double kLag2[2][4] = {
    {(-kGs2 - 1.5) / 36.0, -(13.0 / 12.0) * (-kGs2 - 0.5), (13.0 / 12.0) * (-kGs2 + 0.5), -(-kGs2 + 1.5) / 36.0},
    {(kGs2 - 1.5) / 36.0, -(13.0 / 12.0) * (kGs2 - 0.5), (13.0 / 12.0) * (kGs2 + 0.5), -(kGs2 + 1.5) / 36.0}};

__device__ __forceinline__ int st_size(int st) { return st == ST_J9 ? 9 : st == ST_J21 ? 21 : st == ST_P5 ? 5 : 9; }
__device__ __forceinline__ int st_off(int st, int k, int d) {
  return st == ST_J9 ? c_off_j9[k][d] : st == ST_J21 ? c_off_j21[k][d] : st == ST_P5 ? c_off_p5[k][d] : c_off_p9[k][d];
}
__device__ __forceinline__ int st_center(int st) { return st == ST_J9 ? 4 : st == ST_J21 ? 10 : st == ST_P5 ? 2 : 4; }
__device__ __forceinline__ int st_coarse(int st) { return (st == ST_J9 || st == ST_P5) ? ST_P5 : ST_P9; }

struct Geo2 {
  int Nx, Ny;
  double dx, dy, g;
  const double *gq;
  const int *bck;
  const double *bcs;
};

__device__ __forceinline__ Geo2 make_geo2(const ProbDev2 &P, int l) {
  Geo2 G;
  G.Nx = P.lev[l].Nx;
  G.Ny = P.lev[l].Ny;
  G.dx = P.lev[l].dx;
  G.dy = P.lev[l].dy;
  G.g = P.g;
  G.gq = P.lev[l].gq;
  G.bck = P.lev[l].bck;
  G.bcs = P.bcs;
  return G;
}

// Largest colour pass (cells) that runs as k2_sor_split, per precision.
#ifndef NSWE_SOR_SPLIT_F64
#define NSWE_SOR_SPLIT_F64 (1L << 40)
#endif
#ifndef NSWE_SOR_SPLIT_F32
#define NSWE_SOR_SPLIT_F32 (1L << 40)
#endif
#ifndef NSWE_SOR_UNROLL
#define NSWE_SOR_UNROLL 1
#endif
constexpr long kSorSplitF64 = NSWE_SOR_SPLIT_F64, kSorSplitF32 = NSWE_SOR_SPLIT_F32;
// Largest number of (cell, block, component) items for which the Jacobian
// takes one component per item.
#ifndef NSWE_JAC_SPLIT_ITEMS
#define NSWE_JAC_SPLIT_ITEMS 65536
#endif
constexpr long kJacSplitItems = NSWE_JAC_SPLIT_ITEMS;

// Perturbation of one interior cell in one component (cp < 0: none).
struct Pert {
  int cp, m;
  double eps;
};

__device__ __forceinline__ void bc_post(int kind, const double *st, double o[3], int normal) {
  if (kind == NSWE_BC2_REFLECT) {
    o[normal] = -o[normal];
  } else if (kind == NSWE_BC2_DISCHARGE) {
    o[1] = st[1];
    o[2] = st[2];
  } else if (kind == NSWE_BC2_DEPTH) {
    o[0] = st[0];
  }
}

// Cell value with two ghost layers (x rule, then y rule at corners).
__device__ __forceinline__ void cellv(const Geo2 &G, const double *U, int i, int j, const Pert &p, double o[3]) {
  const int Nx = G.Nx, Ny = G.Ny, n = Nx * Ny;
  int xk = 0, xs = 0;
  if (i < 0 || i >= Nx) {
    xs = i < 0 ? 0 : 1;
    xk = G.bck[xs * Ny + min(max(j, 0), Ny - 1)];
    if (xk == NSWE_BC2_INFLOW) {
      o[0] = G.bcs[xs * 3];
      o[1] = G.bcs[xs * 3 + 1];
      o[2] = G.bcs[xs * 3 + 2];
      return;
    }
    i = (xk == NSWE_BC2_REFLECT) ? (i < 0 ? -1 - i : 2 * Nx - 1 - i) : (i < 0 ? 0 : Nx - 1);
  }
  if (j < 0 || j >= Ny) {
    const int ys = j < 0 ? 2 : 3;
    const int yk = G.bck[2 * Ny + (ys - 2) * Nx + i];
    if (yk == NSWE_BC2_INFLOW) {
      o[0] = G.bcs[ys * 3];
      o[1] = G.bcs[ys * 3 + 1];
      o[2] = G.bcs[ys * 3 + 2];
    } else {
      const int jj = (yk == NSWE_BC2_REFLECT) ? (j < 0 ? -1 - j : 2 * Ny - 1 - j) : (j < 0 ? 0 : Ny - 1);
      const int c = jj * Nx + i;
#pragma unroll
      for (int m = 0; m < 3; ++m) o[m] = (c == p.cp && m == p.m) ? U[m * n + c] + p.eps : U[m * n + c];
      bc_post(yk, G.bcs + ys * 3, o, 2);
    }
  } else {
    const int c = j * Nx + i;
#pragma unroll
    for (int m = 0; m < 3; ++m) o[m] = (c == p.cp && m == p.m) ? U[m * n + c] + p.eps : U[m * n + c];
  }
  if (xk) bc_post(xk, G.bcs + xs * 3, o, 1);
}

__device__ __forceinline__ void weno3_both(double a, double b, double c, double &up, double &um) {
  double d0 = c - b, d1 = b - a;
  double e0 = kZeta2 + d0 * d0, e1 = kZeta2 + d1 * d1;
  double s0 = e0 * e0, s1 = e1 * e1;
  double p0 = 1.5 * b - 0.5 * c, p1 = 0.5 * a + 0.5 * b;
  double q0 = 0.5 * b + 0.5 * c, q1 = -0.5 * a + 1.5 * b;
  double D1 = s1 + 2.0 * s0, D2 = 2.0 * s1 + s0;
  double inv = 1.0 / (D1 * D2);
  up = (s1 * p0 + 2.0 * s0 * p1) * (D2 * inv);
  um = (2.0 * s1 * q0 + s0 * q1) * (D1 * inv);
}

// WENO3 of the values (a, b, c) with the nonlinear weights of (a0, b0, c0):
// the frozen linearisation's reconstruction (weights as in weno3_both).
__device__ __forceinline__ void weno3_fixed(double a0, double b0, double c0, double a, double b, double c,
                                            double &up, double &um) {
  double d0 = c0 - b0, d1 = b0 - a0;
  double e0 = kZeta2 + d0 * d0, e1 = kZeta2 + d1 * d1;
  double s0 = e0 * e0, s1 = e1 * e1;
  double p0 = 1.5 * b - 0.5 * c, p1 = 0.5 * a + 0.5 * b;
  double q0 = 0.5 * b + 0.5 * c, q1 = -0.5 * a + 1.5 * b;
  double D1 = s1 + 2.0 * s0, D2 = 2.0 * s1 + s0;
  double inv = 1.0 / (D1 * D2);
  up = (s1 * p0 + 2.0 * s0 * p1) * (D2 * inv);
  um = (2.0 * s1 * q0 + s0 * q1) * (D1 * inv);
}

// One-sided characteristic WENO3 at the interface between line cells a and
// a+1; v[0..3] = cells a-1..a+2; side 0: U^-, side 1: U^+. FROZEN: the
// eigenvectors and the nonlinear weights come from b, the unperturbed values
// of the same cells (b is not read otherwise).
template <bool FROZEN>
__device__ __forceinline__ void char_rec(int dir, const double v[4][3], const double b[4][3], double g, int side,
                                         double out[3]) {
  const int in = dir == 0 ? 1 : 2, it = dir == 0 ? 2 : 1;
  const double(*r)[3] = FROZEN ? b : v;
  const double h = 0.5 * (r[1][0] + r[2][0]);
  const double ih = 1.0 / h;
  const double un = 0.5 * (r[1][in] + r[2][in]) * ih, ut = 0.5 * (r[1][it] + r[2][it]) * ih;
  const double c = sqrt(g * h), i2c = 0.5 / c;
  double W[3][3], Wb[3][3];
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    const double *u = v[side + s];
    W[s][0] = (un + c) * i2c * u[0] - i2c * u[in];
    W[s][1] = -ut * u[0] + u[it];
    W[s][2] = -(un - c) * i2c * u[0] + i2c * u[in];
    if (FROZEN) {
      const double *w = b[side + s];
      Wb[s][0] = (un + c) * i2c * w[0] - i2c * w[in];
      Wb[s][1] = -ut * w[0] + w[it];
      Wb[s][2] = -(un - c) * i2c * w[0] + i2c * w[in];
    }
  }
  double Wr[3];
#pragma unroll
  for (int f = 0; f < 3; ++f) {
    double up, um;
    if (FROZEN)
      weno3_fixed(Wb[0][f], Wb[1][f], Wb[2][f], W[0][f], W[1][f], W[2][f], up, um);
    else
      weno3_both(W[0][f], W[1][f], W[2][f], up, um);
    Wr[f] = side == 0 ? um : up;
  }
  out[0] = Wr[0] + Wr[2];
  out[in] = (un - c) * Wr[0] + (un + c) * Wr[2];
  out[it] = ut * Wr[0] + Wr[1] + ut * Wr[2];
}

__device__ __forceinline__ void llf(int dir, const double L[3], const double R[3], double g, double F[3]) {
  const int in = dir == 0 ? 1 : 2;
  const double iL = 1.0 / L[0], iR = 1.0 / R[0];
  const double uL = L[1] * iL, vL = L[2] * iL, uR = R[1] * iR, vR = R[2] * iR;
  const double pL = 0.5 * g * L[0] * L[0], pR = 0.5 * g * R[0] * R[0];
  double FL[3], FR[3];
  if (dir == 0) {
    FL[0] = L[1]; FL[1] = L[1] * uL + pL; FL[2] = L[1] * vL;
    FR[0] = R[1]; FR[1] = R[1] * uR + pR; FR[2] = R[1] * vR;
  } else {
    FL[0] = L[2]; FL[1] = L[2] * uL; FL[2] = L[2] * vL + pL;
    FR[0] = R[2]; FR[1] = R[2] * uR; FR[2] = R[2] * vR + pR;
  }
  const double a = fmax(fabs(L[in] * iL) + sqrt(g * L[0]), fabs(R[in] * iR) + sqrt(g * R[0]));
#pragma unroll
  for (int m = 0; m < 3; ++m) F[m] = 0.5 * (FL[m] + FR[m]) - 0.5 * a * (R[m] - L[m]);
}

// Interface values of one line of direction dir (dir 0: row r, positions
// a-3..a+3 along x; dir 1: column r, positions a-3..a+3 along y) at the
// interfaces a-3/2 .. a+3/2 (f = 0..3), sides U^- (0) and U^+ (1), of the
// (possibly perturbed) state; FROZEN: weights and eigenvectors from U itself.
template <bool FROZEN>
__device__ __forceinline__ void line_values2(const Geo2 &G, const double *U, int dir, int a, int r, const Pert &p,
                                             double out[4][2][3]) {
  double v[7][3];                 // line cells a-3 .. a+3
  double v0[FROZEN ? 7 : 1][3];   // the same cells unperturbed (FROZEN)
#pragma unroll
  for (int s = 0; s < 7; ++s) {
    if (dir == 0) cellv(G, U, a - 3 + s, r, p, v[s]);
    else cellv(G, U, r, a - 3 + s, p, v[s]);
  }
  if (FROZEN) {
    const Pert none{-1, 0, 0.0};
#pragma unroll
    for (int s = 0; s < 7; ++s) {
      if (dir == 0) cellv(G, U, a - 3 + s, r, none, v0[FROZEN ? s : 0]);
      else cellv(G, U, r, a - 3 + s, none, v0[FROZEN ? s : 0]);
    }
  }
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    // interface between cells k = a-2+f and k+1: v index of cell k-1 is f
    const double(*w)[3] = &v[f];
    const double(*w0)[3] = FROZEN ? &v0[FROZEN ? f : 0] : w;
    if (f > 0) char_rec<FROZEN>(dir, w, w0, G.g, 0, out[f][0]);
    if (f < 3) char_rec<FROZEN>(dir, w, w0, G.g, 1, out[f][1]);
  }
}

// The direction-dir part of R_ij from the interface values of its three
// lines (transverse positions r0-1, r0, r0+1): the edge fluxes at the two
// Gauss points of the faces a-1/2, a+1/2 (flux = right minus left) and the
// source component 1 + dir, -(1/4) sum g h b_dir (S / (dx dy)).
__device__ __forceinline__ void dir_part2(const Geo2 &G, int dir, int c, const double (*l0)[2][3],
                                          const double (*l1)[2][3], const double (*l2)[2][3], double flux[3],
                                          double &S) {
  const double(*ifv[3])[2][3] = {l0, l1, l2};
  const int n = G.Nx * G.Ny;
  double fl[2][3] = {{0, 0, 0}, {0, 0, 0}};
  double hq[2][4];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const double sg = q == 0 ? -kTq : kTq;
    double gv[4][2][3];
#pragma unroll
    for (int f = 0; f < 4; ++f)
#pragma unroll
      for (int sd = 0; sd < 2; ++sd) {
        if ((f == 0 && sd == 0) || (f == 3 && sd == 1)) continue;
#pragma unroll
        for (int m = 0; m < 3; ++m) gv[f][sd][m] = ifv[1][f][sd][m] + sg * (ifv[2][f][sd][m] - ifv[0][f][sd][m]);
      }
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      double F[3];
      llf(dir, gv[1 + e][0], gv[1 + e][1], G.g, F);
#pragma unroll
      for (int m = 0; m < 3; ++m) fl[e][m] += 0.5 * F[m];
    }
    hq[q][0] = gv[0][1][0];
    hq[q][1] = gv[1][1][0];
    hq[q][2] = gv[2][0][0];
    hq[q][3] = gv[3][0][0];
  }
#pragma unroll
  for (int m = 0; m < 3; ++m) flux[m] = fl[1][m] - fl[0][m];
  double acc = 0.0;
#pragma unroll
  for (int q = 0; q < 2; ++q)
#pragma unroll
    for (int pp = 0; pp < 2; ++pp) {
      const double hv = kLag2[pp][0] * hq[q][0] + kLag2[pp][1] * hq[q][1] + kLag2[pp][2] * hq[q][2] +
                        kLag2[pp][3] * hq[q][3];
      const int beta = dir == 0 ? q : pp, gamma = dir == 0 ? pp : q;
      acc += G.g * hv * G.gq[(dir * 4 + 2 * beta + gamma) * n + c];
    }
  S = -0.25 * acc;
}

// Local residual R_ij (Eq. 20) of the (possibly perturbed) state; FROZEN:
// the reconstructions take their weights and eigenvectors from U itself.
template <bool FROZEN>
__device__ void local_residual2(const Geo2 &G, const double *U, int i, int j, const Pert &p, double R[3]) {
  const int c = j * G.Nx + i;
  double flux[2][3], S[3] = {0.0, 0.0, 0.0};
#pragma unroll 1
  for (int dir = 0; dir < 2; ++dir) {
    const int a = dir == 0 ? i : j, r0 = dir == 0 ? j : i;
    double ifv[3][4][2][3];
#pragma unroll 1
    for (int t = 0; t < 3; ++t) line_values2<FROZEN>(G, U, dir, a, r0 - 1 + t, p, ifv[t]);
    dir_part2(G, dir, c, ifv[0], ifv[1], ifv[2], flux[dir], S[1 + dir]);
  }
#pragma unroll
  for (int m = 0; m < 3; ++m) R[m] = flux[0][m] / G.dx + flux[1][m] / G.dy - S[m];
}

// Interior cell whose state the (possibly ghost) position (i, j) reads, as in
// cellv, or -1 where it reads boundary data only (inflow ghosts).
__device__ __forceinline__ int cell_src(const Geo2 &G, int i, int j) {
  const int Nx = G.Nx, Ny = G.Ny;
  if (i < 0 || i >= Nx) {
    const int xs = i < 0 ? 0 : 1;
    const int xk = G.bck[xs * Ny + min(max(j, 0), Ny - 1)];
    if (xk == NSWE_BC2_INFLOW) return -1;
    i = (xk == NSWE_BC2_REFLECT) ? (i < 0 ? -1 - i : 2 * Nx - 1 - i) : (i < 0 ? 0 : Nx - 1);
  }
  if (j < 0 || j >= Ny) {
    const int ys = j < 0 ? 2 : 3;
    const int yk = G.bck[2 * Ny + (ys - 2) * Nx + i];
    if (yk == NSWE_BC2_INFLOW) return -1;
    j = (yk == NSWE_BC2_REFLECT) ? (j < 0 ? -1 - j : 2 * Ny - 1 - j) : (j < 0 ? 0 : Ny - 1);
  }
  return j * Nx + i;
}

// Whether the line (dir, a, r) of line_values2 reads interior cell cp.
__device__ __forceinline__ bool line_reads(const Geo2 &G, int dir, int a, int r, int cp) {
  bool hit = false;
#pragma unroll
  for (int s = 0; s < 7; ++s) hit |= (dir == 0 ? cell_src(G, a - 3 + s, r) : cell_src(G, r, a - 3 + s)) == cp;
  return hit;
}
__device__ double block_sum2(double v, double *red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    red[32] = s;
  }
  __syncthreads();
  return red[32];
}

// ---------------------------------------------------------------------------- kernels

// The residual of Eq. 20 by block `bid` of `nblk` (grid-stride over cells),
// its l1 partial sum stored in partials[bid].
__device__ __forceinline__ void residual_blocks2(const ProbDev2 *P, int level, const double *U, double *R,
                                                 double *partials, int bid, int nblk) {
  __shared__ double red[33];
  const Geo2 G = make_geo2(*P, level);
  const int n = G.Nx * G.Ny;
  const Pert np{-1, 0, 0.0};
  double acc = 0.0;
  for (int c = bid * blockDim.x + threadIdx.x; c < n; c += nblk * blockDim.x) {
    double r[3];
    local_residual2<false>(G, U, c % G.Nx, c / G.Nx, np, r);
    R[c] = r[0];
    R[n + c] = r[1];
    R[2 * n + c] = r[2];
    acc += fabs(r[0]) + fabs(r[1]) + fabs(r[2]);
  }
  const double s = block_sum2(acc, red);
  if (threadIdx.x == 0) partials[bid] = s;
}

__global__ void __launch_bounds__(kThreads) k2_residual(const ProbDev2 *P, int level, const double *U, double *R,
                                                        double *partials) {
  pdl_enter();
  residual_blocks2(P, level, U, R, partials, blockIdx.x, gridDim.x);
}

__global__ void k2_finish(const double *partials, int nparts, int n, double *res) {
  pdl_enter();
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < nparts; ++i) s += partials[i];
    *res = s / n;
  }
}

// One item = (cell, stencil block k): three perturbed local residuals
// (FROZEN: the frozen linearisation).
// msplit: one item per (cell, block, component m) instead of per (cell,
// block), for small grids where the kernel is bound by each thread's chain.
template <typename TJ, bool FROZEN>
__device__ __forceinline__ void jacobian_items2(const ProbDev2 *P, int level, int st, const double *U, double eps,
                                                double alpha, const double *R, TJ *J, int msplit, int cm, int first,
                                                int stride) {
  const Geo2 G = make_geo2(*P, level);
  const int n = G.Nx * G.Ny, K = st_size(st), kc = st_center(st);
  const double ieps = 1.0 / eps;
  const int items = n * K * (msplit ? 3 : 1);
  for (int it = first; it < items; it += stride) {
    const int c = it % n, kq = it / n, k = msplit ? kq % K : kq, i = c % G.Nx, j = c / G.Nx;
    const int m0 = msplit ? kq / K : 0, m1 = msplit ? m0 + 1 : 3;
    const size_t S = blk_stride(cm, G.Nx, G.Ny), pc = blk_pos(cm, G.Nx, G.Ny, i, j);
    const int pi = i + st_off(st, k, 0), pj = j + st_off(st, k, 1);
    if (pi < 0 || pi >= G.Nx || pj < 0 || pj >= G.Ny) {
      for (int l = 0; l < 3; ++l)
        for (int m = m0; m < m1; ++m) J[(size_t)(k * 9 + l * 3 + m) * S + pc] = TJ(0.0);
      continue;
    }
    const double R0[3] = {R[c], R[n + c], R[2 * n + c]};
    const double reg = (k == kc) ? alpha * (fabs(R0[0]) + fabs(R0[1]) + fabs(R0[2])) : 0.0;
    // The perturbed local residuals of Eq. 12, built line by line: a line
    // that does not read cell cp has the same interface values for the three
    // perturbations and is reconstructed once; a direction none of whose
    // lines read cp contributes the same flux and source to all three.
    const int cp = pj * G.Nx + pi;
    const Pert none{-1, 0, 0.0};
    double fd[2][3][3], sd[2][3];  // [dir][m][component], [dir][m]
#pragma unroll 1
    for (int dir = 0; dir < 2; ++dir) {
      const int a = dir == 0 ? i : j, r0 = dir == 0 ? j : i;
      double ifv[3][4][2][3];
      int reads = 0;
#pragma unroll 1
      for (int t = 0; t < 3; ++t) {
        if (line_reads(G, dir, a, r0 - 1 + t, cp)) reads |= 1 << t;
        else line_values2<FROZEN>(G, U, dir, a, r0 - 1 + t, none, ifv[t]);
      }
      if (!reads) {
        double f[3], sv;
        dir_part2(G, dir, c, ifv[0], ifv[1], ifv[2], f, sv);
#pragma unroll
        for (int m = 0; m < 3; ++m) {  // the same for every m (m0..m1-1 are read)
          fd[dir][m][0] = f[0];
          fd[dir][m][1] = f[1];
          fd[dir][m][2] = f[2];
          sd[dir][m] = sv;
        }
        continue;
      }
#pragma unroll 1
      for (int m = m0; m < m1; ++m) {
        const Pert p{cp, m, eps};
#pragma unroll 1
        for (int t = 0; t < 3; ++t)
          if (reads & (1 << t)) line_values2<FROZEN>(G, U, dir, a, r0 - 1 + t, p, ifv[t]);
        dir_part2(G, dir, c, ifv[0], ifv[1], ifv[2], fd[dir][m], sd[dir][m]);
      }
    }
    for (int m = m0; m < m1; ++m) {
      const double Sm[3] = {0.0, sd[0][m], sd[1][m]};
#pragma unroll
      for (int l = 0; l < 3; ++l) {
        const double Rp = fd[0][m][l] / G.dx + fd[1][m][l] / G.dy - Sm[l];
        double v = (Rp - R0[l]) * ieps;
        if (l == m) v += reg;
        J[(size_t)(k * 9 + l * 3 + m) * S + pc] = TJ(v);
      }
    }
  }
}

template <typename TJ, bool FROZEN>
__global__ void __launch_bounds__(kThreads) k2_jacobian(const ProbDev2 *P, int level, int st, const double *U,
                                                        double eps, double alpha, const double *R, TJ *J,
                                                        int msplit, int cm) {
  pdl_enter();
  jacobian_items2<TJ, FROZEN>(P, level, st, U, eps, alpha, R, J, msplit, cm, blockIdx.x * blockDim.x + threadIdx.x,
                              gridDim.x * blockDim.x);
}

template <typename T>
__device__ __forceinline__ void coarse_op_cells2(int Nx, int Ny, int st, const T *Jf, T *Jc, int cm, int first,
                                                 int stride) {
  const int Ncx = Nx / 2, Ncy = Ny / 2, nc = Ncx * Ncy, K = st_size(st), cs = st_coarse(st), Kc = st_size(cs);
  const size_t Sf = blk_stride(cm, Nx, Ny);
  for (int cc = first; cc < nc; cc += stride) {
    const int I = cc % Ncx, Jy = cc / Ncx;
    T acc[9][9];
    for (int t = 0; t < Kc; ++t)
      for (int e = 0; e < 9; ++e) acc[t][e] = T(0.0);
    for (int b = 0; b < 2; ++b)
      for (int a = 0; a < 2; ++a) {
        const int xi = 2 * I + a, yi = 2 * Jy + b;
        const size_t c = blk_pos(cm, Nx, Ny, xi, yi);
        for (int k = 0; k < K; ++k) {
          const int ex = xi + st_off(st, k, 0), ey = yi + st_off(st, k, 1);
          if (ex < 0 || ex >= Nx || ey < 0 || ey >= Ny) continue;
          const int ox = ex / 2 - I, oy = ey / 2 - Jy;
          int kk = -1;
          for (int t = 0; t < Kc; ++t)
            if (st_off(cs, t, 0) == ox && st_off(cs, t, 1) == oy) kk = t;
          if (kk < 0) continue;
          for (int e = 0; e < 9; ++e) acc[kk][e] += Jf[(size_t)(k * 9 + e) * Sf + c];
        }
      }
    for (int t = 0; t < Kc; ++t)
      for (int e = 0; e < 9; ++e) Jc[(size_t)(t * 9 + e) * nc + cc] = acc[t][e];
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k2_coarse_op(int Nx, int Ny, int st, const T *Jf, T *Jc, int cm) {
  pdl_enter();
  coarse_op_cells2<T>(Nx, Ny, st, Jf, Jc, cm, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

template <typename T>
__device__ __forceinline__ void dinv_cells2(int Nx, int Ny, int st, const T *J, T *Dinv, int cm, int first,
                                            int stride) {
  const int kc = st_center(st), ncell = Nx * Ny;
  const size_t n = blk_stride(cm, Nx, Ny);  // the stride of J and Dinv
  for (int q = first; q < ncell; q += stride) {
    const size_t c = blk_pos(cm, Nx, Ny, q % Nx, q / Nx);
    T a[9];
    for (int e = 0; e < 9; ++e) a[e] = J[(size_t)(kc * 9 + e) * n + c];
    const T c00 = a[4] * a[8] - a[5] * a[7], c01 = a[5] * a[6] - a[3] * a[8], c02 = a[3] * a[7] - a[4] * a[6];
    const T det = a[0] * c00 + a[1] * c01 + a[2] * c02;
    Dinv[0 * (size_t)n + c] = c00 / det;
    Dinv[1 * (size_t)n + c] = (a[2] * a[7] - a[1] * a[8]) / det;
    Dinv[2 * (size_t)n + c] = (a[1] * a[5] - a[2] * a[4]) / det;
    Dinv[3 * (size_t)n + c] = c01 / det;
    Dinv[4 * (size_t)n + c] = (a[0] * a[8] - a[2] * a[6]) / det;
    Dinv[5 * (size_t)n + c] = (a[2] * a[3] - a[0] * a[5]) / det;
    Dinv[6 * (size_t)n + c] = c02 / det;
    Dinv[7 * (size_t)n + c] = (a[1] * a[6] - a[0] * a[7]) / det;
    Dinv[8 * (size_t)n + c] = (a[0] * a[4] - a[1] * a[3]) / det;
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k2_dinv(int Nx, int Ny, int st, const T *J, T *Dinv, int cm) {
  pdl_enter();
  dinv_cells2<T>(Nx, Ny, st, J, Dinv, cm, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

// Block SOR update (Eq. 22) of cell (i, j), relaxation applied reps times
// (consecutive visits of a colour see the same neighbours).
template <typename T>
__device__ __forceinline__ void sor_cell2(int Nx, int Ny, int st, const T *J, const T *Dinv, const T *R, T *dU,
                                          double omega_d, int reps, int i, int j, int cm) {
  const T omega = T(omega_d);
  const int n = Nx * Ny, K = st_size(st), kc = st_center(st), c = j * Nx + i;
  const size_t S = blk_stride(cm, Nx, Ny), pc = blk_pos(cm, Nx, Ny, i, j);  // J, Dinv
  T r[3] = {R[c], R[n + c], R[2 * n + c]};
  for (int k = 0; k < K; ++k) {
    if (k == kc) continue;
    const int p = i + st_off(st, k, 0), q = j + st_off(st, k, 1);
    if (p < 0 || p >= Nx || q < 0 || q >= Ny) continue;
    const int cp = q * Nx + p;
    const T x0 = dU[cp], x1 = dU[n + cp], x2 = dU[2 * n + cp];
#pragma unroll
    for (int l = 0; l < 3; ++l) {  // a chain of fused multiply-adds (the order of sor_pass_split)
      r[l] = fma(J[(size_t)(k * 9 + l * 3 + 0) * S + pc], x0, r[l]);
      r[l] = fma(J[(size_t)(k * 9 + l * 3 + 1) * S + pc], x1, r[l]);
      r[l] = fma(J[(size_t)(k * 9 + l * 3 + 2) * S + pc], x2, r[l]);
    }
  }
  T t[3];
#pragma unroll
  for (int l = 0; l < 3; ++l)
    t[l] = Dinv[(size_t)(l * 3 + 0) * S + pc] * r[0] + Dinv[(size_t)(l * 3 + 1) * S + pc] * r[1] +
           Dinv[(size_t)(l * 3 + 2) * S + pc] * r[2];
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    T x = dU[l * n + c];
    for (int s = 0; s < reps; ++s) x = (T(1.0) - omega) * x - omega * t[l];
    dU[l * n + c] = x;
  }
}

// The cells of colour col, enumerated directly so that every lane of a warp
// updates a cell (an FP64 warp instruction costs the same whatever its
// active lanes): mode 0, the stencil's own colouring; mode 1, (i + j) mod Kc;
// mode 2, (j - i + Nx - 1) mod Kc. The J9 and 5-point colourings are mode 1
// with Kc = 3 and 2; the J21 and 9-point colourings are tensor products of
// residues, (i mod P) + P (j mod P) with P = 3 and 2.
__device__ __forceinline__ void sor_items(int Nx, int Ny, int st, int &mode, int &Kc, int col, int &P, int &W,
                                          int &items) {
  if (mode == 0 && (st == ST_J9 || st == ST_P5)) {
    mode = 1;
    Kc = st == ST_J9 ? 3 : 2;
  }
  if (mode == 0) {
    P = st == ST_J21 ? 3 : 2;
    const int a = col % P, b = col / P;
    W = Nx > a ? (Nx - a + P - 1) / P : 0;
    const int H = Ny > b ? (Ny - b + P - 1) / P : 0;
    items = W * H;
  } else {
    P = 0;
    W = (Nx + Kc - 1) / Kc;
    items = W * Ny;
  }
}

// One colour pass over the items first, first + stride, ... (a grid-wide or a
// block-wide stride).
template <typename T>
__device__ void sor_pass(int Nx, int Ny, int st, const T *J, const T *Dinv, const T *R, T *dU, double omega,
                         int mode, int Kc, int col, int reps, int first, int stride, int cm = 0) {
  int P, W, items;
  sor_items(Nx, Ny, st, mode, Kc, col, P, W, items);
  if (mode == 0) {
    const int a = col % P, b = col / P;
    for (int t = first; t < items; t += stride)
      sor_cell2(Nx, Ny, st, J, Dinv, R, dU, omega, reps, a + (t % W) * P, b + (t / W) * P, cm);
    return;
  }
  for (int t = first; t < items; t += stride) {
    const int j = t / W, m = t % W;
    const int a = mode == 1 ? col - j : j + Nx - 1 - col;
    const int i = ((a % Kc) + Kc) % Kc + m * Kc;
    if (i < Nx) sor_cell2(Nx, Ny, st, J, Dinv, R, dU, omega, reps, i, j, cm);
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k2_sor(int Nx, int Ny, int st, const T *J, const T *Dinv, const T *R,
                                                   T *dU, double omega, int mode, int Kc, int col, int reps, int cm) {
  pdl_enter();
  sor_pass<T>(Nx, Ny, st, J, Dinv, R, dU, omega, mode, Kc, col, reps, blockIdx.x * blockDim.x + threadIdx.x,
              gridDim.x * blockDim.x, cm);
}

// Cell (i, j) of item t of a colour pass (the enumeration of sor_pass);
// false if the item lies beyond the grid.
__device__ __forceinline__ bool sor_item_cell(int Nx, int mode, int Kc, int col, int P, int W, int t, int &i, int &j) {
  if (mode == 0) {
    i = col % P + (t % W) * P;
    j = col / P + (t / W) * P;
    return true;
  }
  j = t / W;
  const int a = mode == 1 ? col - j : j + Nx - 1 - col;
  i = ((a % Kc) + Kc) % Kc + (t % W) * Kc;
  return i < Nx;
}

// The same colour pass with three lanes per cell: lane l of a cell's group
// forms component l of r = R + sum_k J_k dU_k (the expression of sor_cell2,
// so the results are the same bits), the group exchanges r by shuffles, and
// lane l updates dU component l. Ten cells per warp (lanes 30, 31 idle). On
// small grids this spreads a pass over three times as many warps, each with a
// third of the dependent FP64 instructions: an FP64 warp instruction holds
// its SMSP's FP64 unit for tens of cycles, so the length of one thread's
// chain, not the total work, bounds such a pass.
// STC >= 0: the stencil fixed at compile time (the neighbour loop unrolls
// and its loads issue together); -1: the stencil st of the call.
template <typename T, int STC>
__device__ __forceinline__ void sor_pass_split(int Nx, int Ny, int st_arg, const T *J, const T *Dinv, const T *R,
                                               T *dU, double omega_d, int mode, int Kc, int col, int reps,
                                               int warp0, int warps, int cm) {
  const int st = STC >= 0 ? STC : st_arg;
  int P, W, items;
  sor_items(Nx, Ny, st, mode, Kc, col, P, W, items);
  const T omega = T(omega_d);
  const int lane = threadIdx.x & 31, g = lane / 3, l = lane - 3 * g, src = 3 * g;
  const int n = Nx * Ny, K = st_size(st), kc = st_center(st);
  for (int w = warp0; w * 10 < items; w += warps) {  // warp-uniform
    const int t = w * 10 + g;
    int i = 0, j = 0;
    const bool on = lane < 30 && t < items && sor_item_cell(Nx, mode, Kc, col, P, W, t, i, j);
    const int c = j * Nx + i;
    const size_t S = blk_stride(cm, Nx, Ny), pc = blk_pos(cm, Nx, Ny, i, j);  // J, Dinv
    T r = on ? R[l * n + c] : T(0.0);
    if (on)
#pragma unroll
      for (int k = 0; k < (STC >= 0 ? (STC == ST_J9 ? 9 : STC == ST_P5 ? 5 : 21) : K); ++k) {
        if (k == kc) continue;
        const int p = i + st_off(st, k, 0), q = j + st_off(st, k, 1);
        if (p < 0 || p >= Nx || q < 0 || q >= Ny) continue;
        const int cp = q * Nx + p;
        const T x0 = dU[cp], x1 = dU[n + cp], x2 = dU[2 * n + cp];
        r = fma(J[(size_t)(k * 9 + l * 3 + 0) * S + pc], x0, r);
        r = fma(J[(size_t)(k * 9 + l * 3 + 1) * S + pc], x1, r);
        r = fma(J[(size_t)(k * 9 + l * 3 + 2) * S + pc], x2, r);
      }
    const T r0 = __shfl_sync(0xffffffffu, r, min(src, 31));
    const T r1 = __shfl_sync(0xffffffffu, r, min(src + 1, 31));
    const T r2 = __shfl_sync(0xffffffffu, r, min(src + 2, 31));
    if (on) {
      const T tl = Dinv[(size_t)(l * 3 + 0) * S + pc] * r0 + Dinv[(size_t)(l * 3 + 1) * S + pc] * r1 +
                   Dinv[(size_t)(l * 3 + 2) * S + pc] * r2;
      T x = dU[l * n + c];
      for (int s = 0; s < reps; ++s) x = (T(1.0) - omega) * x - omega * tl;
      dU[l * n + c] = x;
    }
  }
}

template <typename T, int STC>
__global__ void __launch_bounds__(kThreads) k2_sor_split(int Nx, int Ny, int st, const T *J, const T *Dinv,
                                                         const T *R, T *dU, double omega, int mode, int Kc, int col,
                                                         int reps, int cm) {
  pdl_enter();
  sor_pass_split<T, STC>(Nx, Ny, st, J, Dinv, R, dU, omega, mode, Kc, col, reps,
                         (blockIdx.x * blockDim.x + threadIdx.x) >> 5, (gridDim.x * blockDim.x) >> 5, cm);
}

// A colour pass by the threads of one block (the tail kernel): in FP64 split
// as above; in FP32, where the dependent chains are short, one thread per
// cell measured faster.
template <typename T>
__device__ void sor_pass_block_split(int Nx, int Ny, int st, const T *J, const T *Dinv, const T *R, T *dU,
                                     double omega, int mode, int Kc, int col, int reps) {
  if (!std::is_same<T, double>::value) {
    sor_pass<T>(Nx, Ny, st, J, Dinv, R, dU, omega, mode, Kc, col, reps, threadIdx.x, blockDim.x);
    return;
  }
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (st == ST_J9)
    sor_pass_split<T, ST_J9>(Nx, Ny, st, J, Dinv, R, dU, omega, mode, Kc, col, reps, w, nw, 0);
  else if (st == ST_P5)
    sor_pass_split<T, ST_P5>(Nx, Ny, st, J, Dinv, R, dU, omega, mode, Kc, col, reps, w, nw, 0);
  else
    sor_pass_split<T, -1>(Nx, Ny, st, J, Dinv, R, dU, omega, mode, Kc, col, reps, w, nw, 0);
}

template <typename T>
__device__ void restrict_cells2(int Nx, int Ny, int st, const T *J, const T *R, const T *dU, T *Rc, T *dUc, int first,
                                int stride, int cm = 0) {
  const int n = Nx * Ny, Ncx = Nx / 2, nc = Ncx * (Ny / 2), K = st_size(st);
  const size_t S = blk_stride(cm, Nx, Ny);  // J
  for (int cc = first; cc < nc; cc += stride) {
    const int I = cc % Ncx, Jy = cc / Ncx;
    T s[3] = {T(0.0), T(0.0), T(0.0)};
    for (int b = 0; b < 2; ++b)
      for (int a = 0; a < 2; ++a) {
        const int xi = 2 * I + a, yi = 2 * Jy + b, c = yi * Nx + xi;
        const size_t pc = blk_pos(cm, Nx, Ny, xi, yi);
        T r[3] = {R[c], R[n + c], R[2 * n + c]};
        for (int k = 0; k < K; ++k) {
          const int p = xi + st_off(st, k, 0), q = yi + st_off(st, k, 1);
          if (p < 0 || p >= Nx || q < 0 || q >= Ny) continue;
          const int cp = q * Nx + p;
          const T x0 = dU[cp], x1 = dU[n + cp], x2 = dU[2 * n + cp];
#pragma unroll
          for (int l = 0; l < 3; ++l) {
            r[l] = fma(J[(size_t)(k * 9 + l * 3 + 0) * S + pc], x0, r[l]);
            r[l] = fma(J[(size_t)(k * 9 + l * 3 + 1) * S + pc], x1, r[l]);
            r[l] = fma(J[(size_t)(k * 9 + l * 3 + 2) * S + pc], x2, r[l]);
          }
        }
        s[0] += r[0];
        s[1] += r[1];
        s[2] += r[2];
      }
    // the oracle accumulates the four children in row-major fine order
    for (int l = 0; l < 3; ++l) {
      Rc[l * nc + cc] = s[l];
      dUc[l * nc + cc] = T(0.0);
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k2_restrict(int Nx, int Ny, int st, const T *J, const T *R, const T *dU,
                                                        T *Rc, T *dUc, int cm) {
  pdl_enter();
  restrict_cells2<T>(Nx, Ny, st, J, R, dU, Rc, dUc, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x,
                     cm);
}

template <typename T>
__device__ void prolong_cells2(int Nx, int Ny, T *dU, const T *dUc, int first, int stride) {
  const int n = Nx * Ny, Ncx = Nx / 2, nc = Ncx * (Ny / 2);
  for (int c = first; c < n; c += stride) {
    const int cc = (c / Nx / 2) * Ncx + (c % Nx) / 2;
    for (int l = 0; l < 3; ++l) dU[l * n + c] += dUc[l * nc + cc];
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k2_prolong(int Nx, int Ny, T *dU, const T *dUc) {
  pdl_enter();
  prolong_cells2<T>(Nx, Ny, dU, dUc, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

// Dense system A (row-major, unknown 3c+m) assembled from a block operator:
// zero it, then scatter the blocks.
template <typename T>
__global__ void __launch_bounds__(kThreads) k2_zero(long count, T *A) {
  pdl_enter();
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < count; t += (long)gridDim.x * blockDim.x) A[t] = T(0.0);
}

template <typename T>
__device__ __forceinline__ void scatter_items2(int Nx, int Ny, int st, const T *J, T *A, int first, int stride) {
  const int n = Nx * Ny, N3 = 3 * n, K = st_size(st);
  for (int t = first; t < n * K; t += stride) {
    const int c = t % n, k = t / n, i = c % Nx, j = c / Nx;
    const int p = i + st_off(st, k, 0), q = j + st_off(st, k, 1);
    if (p < 0 || p >= Nx || q < 0 || q >= Ny) continue;
    const int cp = q * Nx + p;
    for (int l = 0; l < 3; ++l)
      for (int m = 0; m < 3; ++m) A[(size_t)(3 * c + l) * N3 + 3 * cp + m] = J[(size_t)(k * 9 + l * 3 + m) * n + c];
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k2_scatter(int Nx, int Ny, int st, const T *J, T *A) {
  pdl_enter();
  scatter_items2<T>(Nx, Ny, st, J, A, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

// LU with partial pivoting (ties to the lowest row) of A (n x n, global
// memory), by the calling thread block. piv[k] = pivot row; flag = 1 on an
// exact zero pivot.
template <typename T>
__device__ void lu_block2(int N3, T *A, int *piv, int *flag) {
  __shared__ T sv[32];
  __shared__ int si[32];
  __shared__ int s_p;
  for (int k = 0; k < N3; ++k) {
    T best = T(-1.0);
    int bi = N3;
    for (int i = k + threadIdx.x; i < N3; i += blockDim.x) {
      const T v = fabs(A[(size_t)i * N3 + k]);
      if (v > best) {
        best = v;
        bi = i;
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const T ov = __shfl_down_sync(0xffffffffu, best, o);
      const int oi = __shfl_down_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) {
        best = ov;
        bi = oi;
      }
    }
    if ((threadIdx.x & 31) == 0) {
      sv[threadIdx.x >> 5] = best;
      si[threadIdx.x >> 5] = bi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      T b = sv[0];
      int p = si[0];
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
        if (sv[w] > b || (sv[w] == b && si[w] < p)) {
          b = sv[w];
          p = si[w];
        }
      s_p = p;
      piv[k] = p;
      if (A[(size_t)p * N3 + k] == T(0.0)) *flag = 1;
    }
    __syncthreads();
    const int p = s_p;
    // Swap only the active columns: earlier multipliers stay where they were
    // computed, which is what the interleaved forward solve expects.
    if (p != k)
      for (int c = k + threadIdx.x; c < N3; c += blockDim.x) {
        const T t = A[(size_t)k * N3 + c];
        A[(size_t)k * N3 + c] = A[(size_t)p * N3 + c];
        A[(size_t)p * N3 + c] = t;
      }
    __syncthreads();
    const T d = A[(size_t)k * N3 + k];
    for (int i = k + 1 + threadIdx.x; i < N3; i += blockDim.x) A[(size_t)i * N3 + k] = A[(size_t)i * N3 + k] / d;
    __syncthreads();
    const int rows = N3 - k - 1;
    for (int t = threadIdx.x; t < rows * rows; t += blockDim.x) {
      const int i = k + 1 + t / rows, c = k + 1 + t % rows;
      A[(size_t)i * N3 + c] -= A[(size_t)i * N3 + k] * A[(size_t)k * N3 + c];
    }
    __syncthreads();
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k2_lu(int N3, T *A, int *piv, int *flag) {
  pdl_enter();
  lu_block2<T>(N3, A, piv, flag);
}

// dU = -A^{-1} R with the factors (one warp; unknown 3c+m).
// Called by the 32 lanes of one warp (lane = threadIdx.x & 31).
template <typename T>
__device__ void lu_solve_warp(int n, const T *A, const int *piv, const T *R, T *x, T *dU) {
  const int N3 = 3 * n, lane = threadIdx.x & 31;
  for (int t = lane; t < n; t += 32)
    for (int m = 0; m < 3; ++m) x[3 * t + m] = -R[m * n + t];
  __syncwarp();
  for (int k = 0; k < N3; ++k) {
    const int p = piv[k];
    if (lane == 0 && p != k) {
      const T t = x[k];
      x[k] = x[p];
      x[p] = t;
    }
    __syncwarp();
    const T xk = x[k];
    for (int i = k + 1 + lane; i < N3; i += 32) x[i] -= A[(size_t)i * N3 + k] * xk;
    __syncwarp();
  }
  for (int i = N3 - 1; i >= 0; --i) {
    T s = T(0.0);
    for (int c = i + 1 + lane; c < N3; c += 32) s += A[(size_t)i * N3 + c] * x[c];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) x[i] = (x[i] - s) / A[(size_t)i * N3 + i];
    __syncwarp();
  }
  for (int t = lane; t < n; t += 32)
    for (int m = 0; m < 3; ++m) dU[m * n + t] = x[3 * t + m];
}

template <typename T>
__global__ void k2_lu_solve(int n, const T *A, const int *piv, const T *R, T *x, T *dU) {
  pdl_enter();
  if (threadIdx.x < 32) lu_solve_warp<T>(n, A, piv, R, x, dU);
}

// Smoothing of level l by the calling block, the same sequence of colour
// passes as the host's schedule (directional: four diagonal sweeps per step;
// otherwise two symmetric passes of the stencil colouring with consecutive
// visits of a colour fused).
__device__ __forceinline__ int st_ncolours(int st) { return st == ST_J9 ? 3 : st == ST_J21 ? 9 : st == ST_P5 ? 2 : 4; }

template <typename T>
__device__ void smooth_block(const Tail2<T> &t, int l, int steps, double omega, int Kc) {
  const int Nx = t.Nx[l], Ny = t.Ny[l], st = t.st[l];
  if (Kc >= 3 && (st == ST_J9 || st == ST_P5)) {
    for (int s = 0; s < steps; ++s)
      for (int d = 0; d < 4; ++d)
        for (int q = 0; q < Kc; ++q) {
          const int mode = (d % 2) + 1, col = d < 2 ? q : Kc - 1 - q;
          sor_pass_block_split<T>(Nx, Ny, st, t.J[l], t.Dinv[l], t.R[l], t.dU[l], omega, mode, Kc, col, 1);
          __syncthreads();
        }
    return;
  }
  const int C = st_ncolours(st);
  int prev = -1, reps = 0;
  for (int s = 0; s < steps; ++s)
    for (int pass = 0; pass < 4 * C; ++pass) {
      const int q = pass % (2 * C), col = q < C ? q : 2 * C - 1 - q;
      if (col == prev) {
        ++reps;
        continue;
      }
      if (prev >= 0) {
        sor_pass_block_split<T>(Nx, Ny, st, t.J[l], t.Dinv[l], t.R[l], t.dU[l], omega, 0, 0, prev, reps);
        __syncthreads();
      }
      prev = col;
      reps = 1;
    }
  if (prev >= 0) {
    sor_pass_block_split<T>(Nx, Ny, st, t.J[l], t.Dinv[l], t.R[l], t.dU[l], omega, 0, 0, prev, reps);
    __syncthreads();
  }
}

template <typename T>
__device__ void vcycle_tail_block2(const Tail2<T> &t, int nu1, int nu2, double omega, int Kc) {
  for (int l = t.ls; l < t.L; ++l) {
    smooth_block<T>(t, l, nu1, omega, Kc);
    restrict_cells2<T>(t.Nx[l], t.Ny[l], t.st[l], t.J[l], t.R[l], t.dU[l], t.R[l + 1], t.dU[l + 1], threadIdx.x,
                       blockDim.x);
    __syncthreads();
  }
  if (threadIdx.x < 32) lu_solve_warp<T>(t.Nx[t.L] * t.Ny[t.L], t.A, t.piv, t.R[t.L], t.x, t.dU[t.L]);
  __syncthreads();
  for (int l = t.L - 1; l >= t.ls; --l) {
    prolong_cells2<T>(t.Nx[l], t.Ny[l], t.dU[l], t.dU[l + 1], threadIdx.x, blockDim.x);
    __syncthreads();
    smooth_block<T>(t, l, nu2, omega, Kc);
  }
}

template <typename T>
__global__ void __launch_bounds__(kTail2Threads, 1) k2_vcycle_tail(Tail2<T> t, int nu1, int nu2, double omega,
                                                                  int Kc) {
  pdl_enter();
  vcycle_tail_block2<T>(t, nu1, nu2, omega, Kc);
}

__global__ void __launch_bounds__(kThreads) k2_to_f32(long count, const double *src, float *dst) {
  pdl_enter();
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < count; t += (long)gridDim.x * blockDim.x)
    dst[t] = float(src[t]);
}

template <typename T>
__device__ __forceinline__ void update_cells2(int n, double *U, const T *dU, double tau, int *flag, int first,
                                              int stride) {
  for (int c = first; c < n; c += stride) {
    const double h = U[c] + tau * double(dU[c]);
    U[c] = h;
    U[n + c] += tau * double(dU[n + c]);
    U[2 * n + c] += tau * double(dU[2 * n + c]);
    if (!(h > 0.0)) atomicOr(flag, 1);
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k2_update(int n, double *U, const T *dU, double tau, int *flag) {
  pdl_enter();
  update_cells2<T>(n, U, dU, tau, flag, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

__global__ void __launch_bounds__(kThreads) k2_interp(const ProbDev2 *P, int coarse_level, const double *Uc,
                                                      double *Uf) {
  pdl_enter();
  const Geo2 Gc = make_geo2(*P, coarse_level);
  const int Ncx = Gc.Nx, Ncy = Gc.Ny, Nfx = 2 * Ncx, nf = 4 * Ncx * Ncy;
  const double w[2][3] = {{0.125, 1.0, -0.125}, {-0.125, 1.0, 0.125}};
  const Pert np{-1, 0, 0.0};
  for (int cc = blockIdx.x * blockDim.x + threadIdx.x; cc < Ncx * Ncy; cc += gridDim.x * blockDim.x) {
    const int I = cc % Ncx, Jc = cc / Ncx;
    double nb[3][3][3];
    for (int q = -1; q <= 1; ++q)
      for (int p = -1; p <= 1; ++p) cellv(Gc, Uc, I + p, Jc + q, np, nb[q + 1][p + 1]);
    for (int b = 0; b < 2; ++b)
      for (int a = 0; a < 2; ++a) {
        const int cf = (2 * Jc + b) * Nfx + 2 * I + a;
        for (int m = 0; m < 3; ++m) {
          double s = 0.0;
          for (int q = 0; q < 3; ++q) {
            double row = 0.0;
            for (int p = 0; p < 3; ++p) row += w[a][p] * nb[q][p][m];
            s += w[b][q] * row;
          }
          Uf[m * nf + cf] = s;
        }
      }
  }
}

int grid2(long items) {
  long b = (items + kThreads - 1) / kThreads;
  return (int)(b < 1 ? 1 : (b > 4096 ? 4096 : b));
}

// Launches a 2D kernel. Launched from the host (not into a stream capture)
// and with the switch on, it carries programmatic stream serialization: it
// may begin launching while the previous kernel on the stream still runs,
// and waits for that kernel in pdl_enter(). Measured on the host-launched
// V-cycles this removes a quarter of their time on 64 x 32 to 256 x 128;
// replayed from a CUDA graph, where the gaps between kernel nodes are
// already short, the same edges made a nested solve 3 % slower, so launches
// into a capture keep ordinary stream order.
template <typename... KArgs, typename... Args>
void launchk2(void (*kern)(KArgs...), dim3 grid, dim3 block, cudaStream_t s, Args &&...args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  const bool pdl = g_pdl2.load(std::memory_order_relaxed) && cudaStreamIsCapturing(s, &cs) == cudaSuccess &&
                   cs == cudaStreamCaptureStatusNone;
  cfg.numAttrs = pdl ? 1 : 0;
  cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

}  // namespace

cudaError_t launch2_residual(const ProbDev2 *p, int level, int n, const double *U, double *R, double *res,
                             double *partials, cudaStream_t s) {
  const int grid = grid2(n) > 1024 ? 1024 : grid2(n);
  launchk2(k2_residual, grid, kThreads, s, p, level, U, R, partials);
  if (res) launchk2(k2_finish, 1, 32, s, partials, grid, n, res);
  return cudaGetLastError();
}

// The same Jacobian with one cell per thread (large grids): the six
// unperturbed reconstruction lines of the cell and its two direction parts
// are built once and serve all blocks and components; each perturbation
// rebuilds only the lines that read the perturbed cell (for J9, 60 line
// reconstructions per cell against 90 when each (cell, block) item builds
// its own). The same expressions on the same inputs as k2_jacobian, so the
// same bits. The lines live in local memory (about 1.9 KB a thread), which
// costs less than the saved FP64 work from about 32,768 cells on; below
// that the per-item kernel's nine- or 27-fold parallelism wins
// (kJac2CellMinDefault).
constexpr int kJacCellThreads = 128;
template <typename TJ, bool FROZEN>
__device__ __forceinline__ void jacobian_cells2(const ProbDev2 *P, int level, int st, const double *U, double eps,
                                                double alpha, const double *R, TJ *J, int cm, int first,
                                                int stride) {
  const Geo2 G = make_geo2(*P, level);
  const int n = G.Nx * G.Ny, K = st_size(st), kc = st_center(st);
  const double ieps = 1.0 / eps;
  const Pert none{-1, 0, 0.0};
  for (int c = first; c < n; c += stride) {
    const int i = c % G.Nx, j = c / G.Nx;
    const size_t S = blk_stride(cm, G.Nx, G.Ny), pc = blk_pos(cm, G.Nx, G.Ny, i, j);
    const double R0[3] = {R[c], R[n + c], R[2 * n + c]};
    double base[2][3][4][2][3], fb[2][3], sb[2];
#pragma unroll 1
    for (int dir = 0; dir < 2; ++dir) {
      const int a = dir == 0 ? i : j, r0 = dir == 0 ? j : i;
#pragma unroll 1
      for (int t = 0; t < 3; ++t) line_values2<FROZEN>(G, U, dir, a, r0 - 1 + t, none, base[dir][t]);
      dir_part2(G, dir, c, base[dir][0], base[dir][1], base[dir][2], fb[dir], sb[dir]);
    }
#pragma unroll 1
    for (int k = 0; k < K; ++k) {
      const int pi = i + st_off(st, k, 0), pj = j + st_off(st, k, 1);
      if (pi < 0 || pi >= G.Nx || pj < 0 || pj >= G.Ny) {
        for (int e = 0; e < 9; ++e) J[(size_t)(k * 9 + e) * S + pc] = TJ(0.0);
        continue;
      }
      const int cp = pj * G.Nx + pi;
      const double reg = (k == kc) ? alpha * (fabs(R0[0]) + fabs(R0[1]) + fabs(R0[2])) : 0.0;
      int reads[2];
#pragma unroll 1
      for (int dir = 0; dir < 2; ++dir) {
        const int a = dir == 0 ? i : j, r0 = dir == 0 ? j : i;
        reads[dir] = 0;
        for (int t = 0; t < 3; ++t)
          if (line_reads(G, dir, a, r0 - 1 + t, cp)) reads[dir] |= 1 << t;
      }
#pragma unroll 1
      for (int m = 0; m < 3; ++m) {
        const Pert p{cp, m, eps};
        double fd[2][3], sdv[2];
#pragma unroll 1
        for (int dir = 0; dir < 2; ++dir) {
          if (!reads[dir]) {
            fd[dir][0] = fb[dir][0];
            fd[dir][1] = fb[dir][1];
            fd[dir][2] = fb[dir][2];
            sdv[dir] = sb[dir];
            continue;
          }
          const int a = dir == 0 ? i : j, r0 = dir == 0 ? j : i;
          double tmp[3][4][2][3];
          const double(*l[3])[2][3];
#pragma unroll 1
          for (int t = 0; t < 3; ++t) {
            if (reads[dir] & (1 << t)) {
              line_values2<FROZEN>(G, U, dir, a, r0 - 1 + t, p, tmp[t]);
              l[t] = tmp[t];
            } else {
              l[t] = base[dir][t];
            }
          }
          dir_part2(G, dir, c, l[0], l[1], l[2], fd[dir], sdv[dir]);
        }
        const double Sm[3] = {0.0, sdv[0], sdv[1]};
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          const double Rp = fd[0][q] / G.dx + fd[1][q] / G.dy - Sm[q];
          double v = (Rp - R0[q]) * ieps;
          if (q == m) v += reg;
          J[(size_t)(k * 9 + q * 3 + m) * S + pc] = TJ(v);
        }
      }
    }
  }
}

template <typename TJ, bool FROZEN>
__global__ void __launch_bounds__(kJacCellThreads) k2_jacobian_cell(const ProbDev2 *P, int level, int st,
                                                                  const double *U, double eps, double alpha,
                                                                  const double *R, TJ *J, int cm) {
  pdl_enter();
  jacobian_cells2<TJ, FROZEN>(P, level, st, U, eps, alpha, R, J, cm, blockIdx.x * blockDim.x + threadIdx.x,
                              gridDim.x * blockDim.x);
}

template <typename TJ>
cudaError_t launch2_jacobian(const ProbDev2 *p, int level, int n, int st, const double *U, double eps, double alpha,
                             const double *R, TJ *J, bool frozen, int cm, int cell_min, cudaStream_t s) {
  if (cell_min >= 0 && n >= cell_min) {
    const int grid = (int)((n + kJacCellThreads - 1) / kJacCellThreads);
    if (frozen)
      launchk2(k2_jacobian_cell<TJ, true>, grid, kJacCellThreads, s, p, level, st, U, eps, alpha, R, J, cm);
    else
      launchk2(k2_jacobian_cell<TJ, false>, grid, kJacCellThreads, s, p, level, st, U, eps, alpha, R, J, cm);
    return cudaGetLastError();
  }
  const long items = (long)n * (st == ST_J21 ? 21 : 9);
  const int msplit = 3 * items <= kJacSplitItems ? 1 : 0;
  const int grid = grid2(items * (msplit ? 3 : 1));
  if (frozen)
    launchk2(k2_jacobian<TJ, true>, grid, kThreads, s, p, level, st, U, eps, alpha, R, J, msplit, cm);
  else
    launchk2(k2_jacobian<TJ, false>, grid, kThreads, s, p, level, st, U, eps, alpha, R, J, msplit, cm);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch2_coarse_op(int Nx, int Ny, int st, const T *Jf, T *Jc, int cm, cudaStream_t s) {
  launchk2(k2_coarse_op<T>, grid2((long)(Nx / 2) * (Ny / 2)), kThreads, s, Nx, Ny, st, Jf, Jc, cm);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch2_dinv(int Nx, int Ny, int st, const T *J, T *Dinv, int cm, cudaStream_t s) {
  launchk2(k2_dinv<T>, grid2((long)Nx * Ny), kThreads, s, Nx, Ny, st, J, Dinv, cm);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch2_sor(int Nx, int Ny, int st, const T *J, const T *Dinv, const T *R, T *dU, double omega, int mode,
                        int Kc, int col, int reps, int cm, cudaStream_t s) {
  // Items of the pass as the kernel enumerates them (see sor_items).
  long items;
  if (mode == 0 && (st == ST_J9 || st == ST_P5)) items = (long)((Nx + (st == ST_J9 ? 3 : 2) - 1) / (st == ST_J9 ? 3 : 2)) * Ny;
  else if (mode == 0) items = (long)((Nx + 2) / (st == ST_J21 ? 3 : 2) + 1) * ((Ny + 2) / (st == ST_J21 ? 3 : 2) + 1);
  else items = (long)((Nx + Kc - 1) / Kc) * Ny;
  if (items <= (std::is_same<T, double>::value ? kSorSplitF64 : kSorSplitF32)) {
    // three lanes per cell; one warp per block on small passes so that the
    // block scheduler spreads the warps over the SMs
    const long warps = (items + 9) / 10;
    const int bs = warps <= 4L * 152 ? 32 : 128;
    const unsigned grid = (unsigned)((warps * 32 + bs - 1) / bs);
    if (NSWE_SOR_UNROLL && st == ST_J9)
      launchk2(k2_sor_split<T, ST_J9>, grid, bs, s, Nx, Ny, st, J, Dinv, R, dU, omega, mode, Kc, col, reps, cm);
    else if (NSWE_SOR_UNROLL && st == ST_P5)
      launchk2(k2_sor_split<T, ST_P5>, grid, bs, s, Nx, Ny, st, J, Dinv, R, dU, omega, mode, Kc, col, reps, cm);
    else
      launchk2(k2_sor_split<T, -1>, grid, bs, s, Nx, Ny, st, J, Dinv, R, dU, omega, mode, Kc, col, reps, cm);
  } else {
    launchk2(k2_sor<T>, grid2(items), kThreads, s, Nx, Ny, st, J, Dinv, R, dU, omega, mode, Kc, col, reps, cm);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch2_restrict(int Nx, int Ny, int st, const T *J, const T *R, const T *dU, T *Rc, T *dUc, int cm,
                             cudaStream_t s) {
  launchk2(k2_restrict<T>, grid2((long)(Nx / 2) * (Ny / 2)), kThreads, s, Nx, Ny, st, J, R, dU, Rc, dUc, cm);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch2_prolong(int Nx, int Ny, T *dU, const T *dUc, cudaStream_t s) {
  launchk2(k2_prolong<T>, grid2((long)Nx * Ny), kThreads, s, Nx, Ny, dU, dUc);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch2_dense_factor(int Nx, int Ny, int st, const T *J, T *A, int *piv, int *flag, cudaStream_t s) {
  const long N3 = 3L * Nx * Ny;
  launchk2(k2_zero<T>, grid2(N3 * N3), kThreads, s, N3 * N3, A);
  launchk2(k2_scatter<T>, grid2((long)Nx * Ny * (st == ST_J21 ? 21 : 9)), kThreads, s, Nx, Ny, st, J, A);
  launchk2(k2_lu<T>, 1, kThreads, s, (int)N3, A, piv, flag);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch2_dense_solve(int n, const T *A, const int *piv, const T *R, T *x, T *dU, cudaStream_t s) {
  launchk2(k2_lu_solve<T>, 1, 32, s, n, A, piv, R, x, dU);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch2_update(int n, double *U, const T *dU, double tau, int *flag, cudaStream_t s) {
  launchk2(k2_update<T>, grid2(n), kThreads, s, n, U, dU, tau, flag);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch2_vcycle_tail(const Tail2<T> &t, int nu1, int nu2, double omega, int Kc, cudaStream_t s) {
  launchk2(k2_vcycle_tail<T>, 1, kTail2Threads, s, t, nu1, nu2, omega, Kc);
  return cudaGetLastError();
}

cudaError_t launch2_to_f32(long count, const double *src, float *dst, cudaStream_t s) {
  launchk2(k2_to_f32, grid2(count), kThreads, s, count, src, dst);
  return cudaGetLastError();
}

#define NSWE_2D_INSTANTIATE(T)                                                                                    \
  template cudaError_t launch2_jacobian<T>(const ProbDev2 *, int, int, int, const double *, double, double,      \
                                           const double *, T *, bool, int, int, cudaStream_t);                   \
  template cudaError_t launch2_coarse_op<T>(int, int, int, const T *, T *, int, cudaStream_t);                   \
  template cudaError_t launch2_dinv<T>(int, int, int, const T *, T *, int, cudaStream_t);                        \
  template cudaError_t launch2_sor<T>(int, int, int, const T *, const T *, const T *, T *, double, int, int, int, \
                                      int, int, cudaStream_t);                                                   \
  template cudaError_t launch2_restrict<T>(int, int, int, const T *, const T *, const T *, T *, T *, int,        \
                                           cudaStream_t);                                                        \
  template cudaError_t launch2_prolong<T>(int, int, T *, const T *, cudaStream_t);                               \
  template cudaError_t launch2_dense_factor<T>(int, int, int, const T *, T *, int *, int *, cudaStream_t);       \
  template cudaError_t launch2_dense_solve<T>(int, const T *, const int *, const T *, T *, T *, cudaStream_t);    \
  template cudaError_t launch2_update<T>(int, double *, const T *, double, int *, cudaStream_t);                 \
  template cudaError_t launch2_vcycle_tail<T>(const Tail2<T> &, int, int, double, int, cudaStream_t);
NSWE_2D_INSTANTIATE(double)
NSWE_2D_INSTANTIATE(float)
#undef NSWE_2D_INSTANTIATE

cudaError_t launch2_interp(const ProbDev2 *p, int coarse_level, int nc, const double *Uc, double *Uf,
                           cudaStream_t s) {
  launchk2(k2_interp, grid2(nc), kThreads, s, p, coarse_level, Uc, Uf);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------- batched (lockstep) kernels

namespace {

// The task owning this block (tasks sorted by b0) and the block's index in
// it; null when the task's problem is masked off.
template <typename T>
__device__ __forceinline__ const BTask2<T> *btask2(const BTask2<T> *tasks, int ntask, const int *done, int &lb) {
  int lo = 0, hi = ntask - 1;
  const int b = blockIdx.x;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tasks[mid].b0 <= b) lo = mid;
    else hi = mid - 1;
  }
  const BTask2<T> *t = tasks + lo;
  lb = b - t->b0;
  return (done && done[t->prob]) ? nullptr : t;
}

__global__ void __launch_bounds__(kThreads) kb2_residual(const BTask2<double> *tasks, int ntask, const int *done) {
  pdl_enter();
  int lb;
  const BTask2<double> *t = btask2(tasks, ntask, done, lb);
  if (t) residual_blocks2(t->P, t->level, t->U, t->R64, t->partials, lb, t->nb);
}

// One task per block: res[prob] = (sum of its partials, in order) / cells (as k2_finish).
__global__ void kb2_finish(const BTask2<double> *tasks, int ntask, const int *done, double *res) {
  pdl_enter();
  const BTask2<double> &t = tasks[blockIdx.x];
  if ((done && done[t.prob]) || threadIdx.x != 0) return;
  double s = 0.0;
  for (int i = 0; i < t.nb; ++i) s += t.partials[i];
  res[t.prob] = s / (t.Nx * t.Ny);
}

template <typename TJ, bool FROZEN>
__global__ void __launch_bounds__(kThreads) kb2_jacobian(const BTask2<TJ> *tasks, int ntask, const int *done) {
  pdl_enter();
  int lb;
  const BTask2<TJ> *t = btask2(tasks, ntask, done, lb);
  if (t)
    jacobian_items2<TJ, FROZEN>(t->P, t->level, t->st, t->U, t->eps, t->alpha, t->R64, t->J, t->msplit, t->cm,
                                lb * blockDim.x + threadIdx.x, t->nb * blockDim.x);
}

template <typename TJ, bool FROZEN>
__global__ void __launch_bounds__(kJacCellThreads) kb2_jacobian_cell(const BTask2<TJ> *tasks, int ntask,
                                                                   const int *done) {
  pdl_enter();
  int lb;
  const BTask2<TJ> *t = btask2(tasks, ntask, done, lb);
  if (t)
    jacobian_cells2<TJ, FROZEN>(t->P, t->level, t->st, t->U, t->eps, t->alpha, t->R64, t->J, t->cm,
                                lb * blockDim.x + threadIdx.x, t->nb * blockDim.x);
}

__global__ void __launch_bounds__(kThreads) kb2_to_f32(const BTask2<float> *tasks, int ntask, const int *done) {
  pdl_enter();
  int lb;
  const BTask2<float> *t = btask2(tasks, ntask, done, lb);
  if (!t) return;
  const long count = 3L * t->Nx * t->Ny;
  for (long c = lb * (long)blockDim.x + threadIdx.x; c < count; c += (long)t->nb * blockDim.x)
    t->R32[c] = float(t->R64[c]);
}

template <typename T>
__global__ void __launch_bounds__(kThreads) kb2_zero_du(const BTask2<T> *tasks, int ntask, const int *done) {
  pdl_enter();
  int lb;
  const BTask2<T> *t = btask2(tasks, ntask, done, lb);
  if (!t) return;
  const long count = 3L * t->Nx * t->Ny;
  for (long c = lb * (long)blockDim.x + threadIdx.x; c < count; c += (long)t->nb * blockDim.x) t->dU[c] = T(0.0);
}

template <typename T>
__global__ void __launch_bounds__(kThreads) kb2_coarse_op(const BTask2<T> *tasks, int ntask, const int *done) {
  pdl_enter();
  int lb;
  const BTask2<T> *t = btask2(tasks, ntask, done, lb);
  if (t) coarse_op_cells2<T>(t->Nx, t->Ny, t->st, t->J, t->Jc, t->cm, lb * blockDim.x + threadIdx.x, t->nb * blockDim.x);
}

template <typename T>
__global__ void __launch_bounds__(kThreads) kb2_dinv(const BTask2<T> *tasks, int ntask, const int *done) {
  pdl_enter();
  int lb;
  const BTask2<T> *t = btask2(tasks, ntask, done, lb);
  if (t) dinv_cells2<T>(t->Nx, t->Ny, t->st, t->J, t->Dinv, t->cm, lb * blockDim.x + threadIdx.x, t->nb * blockDim.x);
}

template <typename T, int STC>
__global__ void __launch_bounds__(kB2SorThreads) kb2_sor_split(const BTask2<T> *tasks, int ntask, const int *done,
                                                               int st, double omega, int mode, int Kc, int col,
                                                               int reps) {
  pdl_enter();
  int lb;
  const BTask2<T> *t = btask2(tasks, ntask, done, lb);
  if (t)
    sor_pass_split<T, STC>(t->Nx, t->Ny, st, t->J, t->Dinv, t->R, t->dU, omega, mode, Kc, col, reps,
                           (lb * blockDim.x + threadIdx.x) >> 5, (t->nb * blockDim.x) >> 5, t->cm);
}

template <typename T>
__global__ void __launch_bounds__(kThreads) kb2_restrict(const BTask2<T> *tasks, int ntask, const int *done) {
  pdl_enter();
  int lb;
  const BTask2<T> *t = btask2(tasks, ntask, done, lb);
  if (t)
    restrict_cells2<T>(t->Nx, t->Ny, t->st, t->J, t->R, t->dU, t->Rc, t->dUc, lb * blockDim.x + threadIdx.x,
                       t->nb * blockDim.x, t->cm);
}

template <typename T>
__global__ void __launch_bounds__(kThreads) kb2_prolong(const BTask2<T> *tasks, int ntask, const int *done) {
  pdl_enter();
  int lb;
  const BTask2<T> *t = btask2(tasks, ntask, done, lb);
  if (t) prolong_cells2<T>(t->Nx, t->Ny, t->dU, t->dUc, lb * blockDim.x + threadIdx.x, t->nb * blockDim.x);
}

template <typename T>
__global__ void __launch_bounds__(kTail2Threads, 1) kb2_vcycle_tail(const Tail2<T> *tails, const BTask2<T> *tasks,
                                                                   const int *done, int nu1, int nu2, double omega,
                                                                   int Kc) {
  pdl_enter();
  if (done && done[tasks[blockIdx.x].prob]) return;
  vcycle_tail_block2<T>(tails[blockIdx.x], nu1, nu2, omega, Kc);
}

template <typename T>
__global__ void __launch_bounds__(kThreads) kb2_dense_zero(const BTask2<T> *tasks, int ntask, const int *done) {
  pdl_enter();
  int lb;
  const BTask2<T> *t = btask2(tasks, ntask, done, lb);
  if (!t) return;
  const long N3 = 3L * t->Nx * t->Ny, count = N3 * N3;
  for (long c = lb * (long)blockDim.x + threadIdx.x; c < count; c += (long)t->nb * blockDim.x) t->A[c] = T(0.0);
}

template <typename T>
__global__ void __launch_bounds__(kThreads) kb2_scatter(const BTask2<T> *tasks, int ntask, const int *done) {
  pdl_enter();
  int lb;
  const BTask2<T> *t = btask2(tasks, ntask, done, lb);
  if (t) scatter_items2<T>(t->Nx, t->Ny, t->st, t->J, t->A, lb * blockDim.x + threadIdx.x, t->nb * blockDim.x);
}

template <typename T>
__global__ void __launch_bounds__(kThreads) kb2_lu(const BTask2<T> *tasks, const int *done, int *flags) {
  pdl_enter();
  const BTask2<T> &t = tasks[blockIdx.x];
  if (done && done[t.prob]) return;
  lu_block2<T>(3 * t.Nx * t.Ny, t.A, t.piv, flags + t.prob);
}

template <typename T>
__global__ void kb2_lu_solve(const BTask2<T> *tasks, const int *done) {
  pdl_enter();
  const BTask2<T> &t = tasks[blockIdx.x];
  if ((done && done[t.prob]) || threadIdx.x >= 32) return;
  lu_solve_warp<T>(t.Nx * t.Ny, t.A, t.piv, t.R, t.x, t.dU);
}

template <typename T>
__global__ void __launch_bounds__(kThreads) kb2_update(const BTask2<T> *tasks, int ntask, const int *done,
                                                       int *flags) {
  pdl_enter();
  int lb;
  const BTask2<T> *t = btask2(tasks, ntask, done, lb);
  if (t)
    update_cells2<T>(t->Nx * t->Ny, t->U, t->dU, t->tau, flags + t->prob, lb * blockDim.x + threadIdx.x,
                     t->nb * blockDim.x);
}

}  // namespace

int b2_grid(long items) { return grid2(items); }
int b2_jacobian_cell_threads() { return kJacCellThreads; }

cudaError_t launchb2_residual(const Batch2Launch<double> &b, const int *done, double *res, cudaStream_t s) {
  if (b.ntask == 0) return cudaSuccess;
  launchk2(kb2_residual, b.blocks, kThreads, s, b.tasks, b.ntask, done);
  launchk2(kb2_finish, b.ntask, 32, s, b.tasks, b.ntask, done, res);
  return cudaGetLastError();
}

template <typename TJ>
cudaError_t launchb2_jacobian(const Batch2Launch<TJ> &b, const int *done, int kind, bool frozen, cudaStream_t s) {
  if (b.ntask == 0) return cudaSuccess;
  if (kind == kB2JacCells) {
    if (frozen) launchk2(kb2_jacobian_cell<TJ, true>, b.blocks, kJacCellThreads, s, b.tasks, b.ntask, done);
    else launchk2(kb2_jacobian_cell<TJ, false>, b.blocks, kJacCellThreads, s, b.tasks, b.ntask, done);
  } else {
    if (frozen) launchk2(kb2_jacobian<TJ, true>, b.blocks, kThreads, s, b.tasks, b.ntask, done);
    else launchk2(kb2_jacobian<TJ, false>, b.blocks, kThreads, s, b.tasks, b.ntask, done);
  }
  return cudaGetLastError();
}

cudaError_t launchb2_to_f32(const Batch2Launch<float> &b, const int *done, cudaStream_t s) {
  if (b.ntask == 0) return cudaSuccess;
  launchk2(kb2_to_f32, b.blocks, kThreads, s, b.tasks, b.ntask, done);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launchb2_zero_du(const Batch2Launch<T> &b, const int *done, cudaStream_t s) {
  if (b.ntask == 0) return cudaSuccess;
  launchk2(kb2_zero_du<T>, b.blocks, kThreads, s, b.tasks, b.ntask, done);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launchb2_coarse_op(const Batch2Launch<T> &b, const int *done, cudaStream_t s) {
  if (b.ntask == 0) return cudaSuccess;
  launchk2(kb2_coarse_op<T>, b.blocks, kThreads, s, b.tasks, b.ntask, done);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launchb2_dinv(const Batch2Launch<T> &b, const int *done, cudaStream_t s) {
  if (b.ntask == 0) return cudaSuccess;
  launchk2(kb2_dinv<T>, b.blocks, kThreads, s, b.tasks, b.ntask, done);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launchb2_sor(const Batch2Launch<T> &b, const int *done, int st, double omega, int mode, int Kc, int col,
                         int reps, cudaStream_t s) {
  if (b.ntask == 0) return cudaSuccess;
  if (NSWE_SOR_UNROLL && st == ST_J9)
    launchk2(kb2_sor_split<T, ST_J9>, b.blocks, kB2SorThreads, s, b.tasks, b.ntask, done, st, omega, mode, Kc, col, reps);
  else if (NSWE_SOR_UNROLL && st == ST_P5)
    launchk2(kb2_sor_split<T, ST_P5>, b.blocks, kB2SorThreads, s, b.tasks, b.ntask, done, st, omega, mode, Kc, col, reps);
  else
    launchk2(kb2_sor_split<T, -1>, b.blocks, kB2SorThreads, s, b.tasks, b.ntask, done, st, omega, mode, Kc, col, reps);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launchb2_restrict(const Batch2Launch<T> &b, const int *done, cudaStream_t s) {
  if (b.ntask == 0) return cudaSuccess;
  launchk2(kb2_restrict<T>, b.blocks, kThreads, s, b.tasks, b.ntask, done);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launchb2_prolong(const Batch2Launch<T> &b, const int *done, cudaStream_t s) {
  if (b.ntask == 0) return cudaSuccess;
  launchk2(kb2_prolong<T>, b.blocks, kThreads, s, b.tasks, b.ntask, done);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launchb2_vcycle_tail(const Tail2<T> *tails, const BTask2<T> *tasks, int ntask, const int *done, int nu1,
                                 int nu2, double omega, int Kc, cudaStream_t s) {
  if (ntask == 0) return cudaSuccess;
  launchk2(kb2_vcycle_tail<T>, ntask, kTail2Threads, s, tails, tasks, done, nu1, nu2, omega, Kc);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launchb2_dense_factor(const Batch2Launch<T> &zero, const Batch2Launch<T> &scatter, const BTask2<T> *tasks,
                                  int ntask, const int *done, int *flags, cudaStream_t s) {
  if (ntask == 0) return cudaSuccess;
  launchk2(kb2_dense_zero<T>, zero.blocks, kThreads, s, zero.tasks, zero.ntask, done);
  launchk2(kb2_scatter<T>, scatter.blocks, kThreads, s, scatter.tasks, scatter.ntask, done);
  launchk2(kb2_lu<T>, ntask, kThreads, s, tasks, done, flags);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launchb2_dense_solve(const BTask2<T> *tasks, int ntask, const int *done, cudaStream_t s) {
  if (ntask == 0) return cudaSuccess;
  launchk2(kb2_lu_solve<T>, ntask, 32, s, tasks, done);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launchb2_update(const Batch2Launch<T> &b, const int *done, int *flags, cudaStream_t s) {
  if (b.ntask == 0) return cudaSuccess;
  launchk2(kb2_update<T>, b.blocks, kThreads, s, b.tasks, b.ntask, done, flags);
  return cudaGetLastError();
}

#define NSWE_B2_INSTANTIATE(T)                                                                                     \
  template cudaError_t launchb2_jacobian<T>(const Batch2Launch<T> &, const int *, int, bool, cudaStream_t);       \
  template cudaError_t launchb2_zero_du<T>(const Batch2Launch<T> &, const int *, cudaStream_t);                   \
  template cudaError_t launchb2_coarse_op<T>(const Batch2Launch<T> &, const int *, cudaStream_t);                 \
  template cudaError_t launchb2_dinv<T>(const Batch2Launch<T> &, const int *, cudaStream_t);                      \
  template cudaError_t launchb2_sor<T>(const Batch2Launch<T> &, const int *, int, double, int, int, int, int,     \
                                       cudaStream_t);                                                             \
  template cudaError_t launchb2_restrict<T>(const Batch2Launch<T> &, const int *, cudaStream_t);                  \
  template cudaError_t launchb2_prolong<T>(const Batch2Launch<T> &, const int *, cudaStream_t);                   \
  template cudaError_t launchb2_vcycle_tail<T>(const Tail2<T> *, const BTask2<T> *, int, const int *, int, int,   \
                                               double, int, cudaStream_t);                                        \
  template cudaError_t launchb2_dense_factor<T>(const Batch2Launch<T> &, const Batch2Launch<T> &,                 \
                                                const BTask2<T> *, int, const int *, int *, cudaStream_t);        \
  template cudaError_t launchb2_dense_solve<T>(const BTask2<T> *, int, const int *, cudaStream_t);                \
  template cudaError_t launchb2_update<T>(const Batch2Launch<T> &, const int *, int *, cudaStream_t);
NSWE_B2_INSTANTIATE(double)
NSWE_B2_INSTANTIATE(float)
#undef NSWE_B2_INSTANTIATE

}  // namespace nswe
