// CUDA kernels (sm_103a) of the 1D NMGM: WENO3 finite-volume residual,
// regularized FD Jacobian J3/J5, geometric multigrid V-cycle with
// multicolour block SOR, and the nested Newton solve (Algorithm 3), all FP64.
//
// Execution model: every building block is a "CTA-level" routine that loops
// over its work items with a block-wide stride, so the same code serves the
// standalone grid kernels (residual, Jacobian: many blocks per problem) and
// the persistent solve kernel, where one thread block runs a whole nested
// solve of one problem with __syncthreads() between phases and no host
// round trip. Problem data and workspace stay in device memory (L2 resident
// for the 1D sizes); the coarsest factorisation lives in shared memory.
#include <cooperative_groups.h>

#include <cmath>
#include <type_traits>

#include "nswe_internal.h"

namespace nswe {
namespace {

constexpr double kZeta = 1e-6;  // WENO epsilon (Section 3.1)

// Lagrange weights of the cubic through t = -3/2, -1/2, 1/2, 3/2 evaluated at
// the Gauss points t = -/+ 1/(2 sqrt 3) (Eq. 9). With t^2 = 1/12 the basis
// reduces to (t - 3/2)/36, -(13/12)(t - 1/2), (13/12)(t + 1/2), -(t + 3/2)/36.
constexpr double kGs = 0.28867513459481288225;  // 1/(2 sqrt 3)
__device__ constexpr double kLag[2][4] = {
    {(-kGs - 1.5) / 36.0, -(13.0 / 12.0) * (-kGs - 0.5), (13.0 / 12.0) * (-kGs + 0.5), -(-kGs + 1.5) / 36.0},
    {(kGs - 1.5) / 36.0, -(13.0 / 12.0) * (kGs - 0.5), (13.0 / 12.0) * (kGs + 0.5), -(kGs + 1.5) / 36.0}};

struct Geo {
  int N;
  double dx, g;
  const double *sf;   // [N+1] width at faces
  const double *gq;   // [3][2][N] sigma, sigma_x, b_x at the Gauss points
  const double *isf;  // [N+1] 1/sigma at faces
  const double *cgf;  // [N+1] sqrt(g/sigma) at faces
  const double *igq;  // [2][N] 1/sigma at the Gauss points
  int bl, br;
  double blh, blq, brh, brq;
  int flux;  // NSWE_FLUX_HLL or NSWE_FLUX_LLF
  // FP32 copies of the level's state and geometry, read by the FP32 Jacobian
  // passes instead of converting the FP64 values at every use (a conversion
  // from FP64 occupies the narrow FP64 pipe); nullptr: convert at use. The
  // copies hold exactly the converted values, so both give the same bits.
  const float *U32;    // [2][N]
  const float *isf32;  // [N+1]
  const float *cgf32;  // [N+1]
  const float *igq32;  // [2][N]
  const float *gq32;   // [2: sigma_x, b_x][2][N]
  float g32, hdx32;    // float(g), 0.5f * float(dx)
};

__device__ __forceinline__ Geo make_geo(const ProbDev &P, int l) {
  Geo G;
  G.U32 = G.isf32 = G.cgf32 = G.igq32 = G.gq32 = nullptr;
  G.g32 = G.hdx32 = 0.0f;
  G.N = P.lev[l].N;
  G.dx = P.lev[l].dx;
  G.g = P.g;
  G.sf = P.lev[l].sf;
  G.gq = P.lev[l].gq;
  G.isf = P.lev[l].gd;
  G.cgf = G.isf + G.N + 1;
  G.igq = G.cgf + G.N + 1;
  G.bl = P.bl;
  G.br = P.br;
  G.blh = P.blh;
  G.blq = P.blq;
  G.brh = P.brh;
  G.brq = P.brq;
  G.flux = P.flux;
  return G;
}

// Ghost state from the boundary data and the adjacent interior cell.
__device__ __forceinline__ void ghost(int kind, double bh, double bq, double sb, double He, double Qe,
                                      double &H, double &Q) {
  if (kind == NSWE_BC_DISCHARGE) {
    H = He;
    Q = bq;
  } else if (kind == NSWE_BC_DEPTH) {
    H = sb * bh;
    Q = Qe;
  } else if (kind == NSWE_BC_STATE) {
    H = sb * bh;
    Q = bq;
  } else {
    H = He;
    Q = Qe;
  }
}

// WENO3 in one cell from averages a, b, c (cells k-1, k, k+1), Eq. 7-8 with
// the linear weights (1/3, 2/3) for U^+_{k-1/2} and (2/3, 1/3) for
// U^-_{k+1/2}. With s_r = (zeta + beta_r)^2 the normalised weights are
// w0 = s1/(s1 + 2 s0), w1 = 2 s0/(s1 + 2 s0) and v0 = 2 s1/(2 s1 + s0),
// v1 = s0/(2 s1 + s0); both quotients share one reciprocal.
template <typename T>
__device__ __forceinline__ void weno3(T a, T b, T c, T &up, T &um) {
  T d0 = c - b, d1 = b - a;
  T e0 = T(kZeta) + d0 * d0, e1 = T(kZeta) + d1 * d1;
  T s0 = e0 * e0, s1 = e1 * e1;
  T p0 = T(1.5) * b - T(0.5) * c, p1 = T(0.5) * a + T(0.5) * b;   // U^(0), U^(1) at k-1/2
  T q0 = T(0.5) * b + T(0.5) * c, q1 = T(-0.5) * a + T(1.5) * b;  // U^(0), U^(1) at k+1/2
  T D1 = s1 + T(2.0) * s0, D2 = T(2.0) * s1 + s0;
  T inv = T(1.0) / (D1 * D2);
  up = (s1 * p0 + T(2.0) * s0 * p1) * (D2 * inv);
  um = (T(2.0) * s1 * q0 + s0 * q1) * (D1 * inv);
}

__device__ __forceinline__ double rsq(double x) { return rsqrt(x); }
__device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }

// Quantities of one interface state entering the HLL flux at a face of width
// sigma: velocity u = Q/H, celerity c = sqrt(g H/sigma) and physical flux
// F = (Q, Q^2/H + g H^2/(2 sigma)) (Eq. 4). One reciprocal square root
// r = H^(-1/2) gives both 1/H = r^2 and c = sqrt(g/sigma) H r; isg = 1/sigma
// and cg = sqrt(g/sigma) are per-face geometry. r2 = 1/H and the pressure
// term P = g H^2/(2 sigma) are kept, so that a state differing only in Q
// (fstate_q) costs one multiply and one fused multiply-add, with the same
// bits as a full evaluation.
template <typename T>
struct FState {
  T H, Q, u, c, F1, r2, P;
};

template <typename T>
__device__ __forceinline__ FState<T> fstate(T H, T Q, T isg, T cg, T g) {
  FState<T> s;
  s.H = H;
  s.Q = Q;
  const T r = rsq(H);
  s.r2 = r * r;
  s.u = Q * s.r2;
  const T h = H * isg;
  s.c = cg * (H * r);
  s.P = (T(0.5) * g * H) * h;
  s.F1 = fma(Q, s.u, s.P);
  return s;
}

// The state of `b` with its discharge replaced by Q.
template <typename T>
__device__ __forceinline__ FState<T> fstate_q(const FState<T> &b, T Q) {
  FState<T> s = b;
  s.Q = Q;
  s.u = Q * b.r2;
  s.F1 = fma(Q, s.u, b.P);
  return s;
}

// Ordering keys of FP64 values on the integer pipe (the FP64 pipe is the
// narrow one): for finite x, key(x) orders as x, with key(-0) = -1 just
// below key(+0) = 0. Selecting by key gives fmin / fmax of two finite values
// (either zero for a pair of zeros), and x >= 0 is key(x) >= -1.
__device__ __forceinline__ long long okey(double x) {
  const long long b = __double_as_longlong(x);
  return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ double kmin(double a, double b) { return okey(a) <= okey(b) ? a : b; }
__device__ __forceinline__ double kmax(double a, double b) { return okey(a) >= okey(b) ? a : b; }
__device__ __forceinline__ bool knonneg(double a) { return okey(a) >= -1LL; }
__device__ __forceinline__ bool knonpos(double a) { return okey(a) <= 0LL; }
__device__ __forceinline__ float kmin(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ float kmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ bool knonneg(float a) { return a >= 0.0f; }
__device__ __forceinline__ bool knonpos(float a) { return a <= 0.0f; }

// HLL flux of two interface states: S_L = min(u_L - c_L, u_R - c_R),
// S_R = max(u_L + c_L, u_R + c_R), upwind fluxes outside the fan, the HLL
// average inside.
template <typename T>
__device__ __forceinline__ void hll_states(const FState<T> &L, const FState<T> &R, T &F0, T &F1) {
  T SL = kmin(L.u - L.c, R.u - R.c);
  T SR = kmax(L.u + L.c, R.u + R.c);
  if (knonneg(SL)) {
    F0 = L.Q;
    F1 = L.F1;
  } else if (knonpos(SR)) {
    F0 = R.Q;
    F1 = R.F1;
  } else {
    T iw = T(1.0) / (SR - SL);
    F0 = (SR * L.Q - SL * R.Q + SL * SR * (R.H - L.H)) * iw;
    F1 = (SR * L.F1 - SL * R.F1 + SL * SR * (R.Q - L.Q)) * iw;
  }
}

// Numerical flux of two interface states: HLL, or LLF: the mean of the
// physical fluxes minus a (U_R - U_L) / 2, a = max(|u_L| + c_L, |u_R| + c_R).
// FLUX fixes the choice at compile time (NSWE_FLUX_HLL or NSWE_FLUX_LLF),
// or -1 takes it from `flux` (the standalone kernels).
template <int FLUX, typename T>
__device__ __forceinline__ void num_flux(const FState<T> &L, const FState<T> &R, int flux, T &F0, T &F1) {
  if (FLUX == NSWE_FLUX_LLF || (FLUX < 0 && flux == NSWE_FLUX_LLF)) {
    const T a = fmax(fabs(L.u) + L.c, fabs(R.u) + R.c);
    F0 = T(0.5) * (L.Q + R.Q) - T(0.5) * a * (R.H - L.H);
    F1 = T(0.5) * (L.F1 + R.F1) - T(0.5) * a * (R.Q - L.Q);
  } else {
    hll_states(L, R, F0, F1);
  }
}

// Five-cell window j-2..j+2 of one residual evaluation.
struct Win {
  double H[5], Q[5];
};

__device__ __forceinline__ void load_win(const Geo &G, const double *H, const double *Q, int j, Win &w) {
#pragma unroll
  for (int p = 0; p < 5; ++p) {
    int k = min(max(j - 2 + p, 0), G.N - 1);  // clamped: ghosts are filled later
    w.H[p] = H[k];
    w.Q[p] = Q[k];
  }
}

// Ghost positions of the window take the boundary state built from the
// window's (possibly perturbed) edge cell.
__device__ __forceinline__ void fill_ghosts(const Geo &G, int j, Win &w) {
  if (j < 2) {
    double He = (j == 0) ? w.H[2] : w.H[1];
    double Qe = (j == 0) ? w.Q[2] : w.Q[1];
    double Hg, Qg;
    ghost(G.bl, G.blh, G.blq, G.sf[0], He, Qe, Hg, Qg);
#pragma unroll
    for (int p = 0; p < 2; ++p)
      if (j - 2 + p < 0) {
        w.H[p] = Hg;
        w.Q[p] = Qg;
      }
  }
  if (j > G.N - 3) {
    double He = (j == G.N - 1) ? w.H[2] : w.H[3];
    double Qe = (j == G.N - 1) ? w.Q[2] : w.Q[3];
    double Hg, Qg;
    ghost(G.br, G.brh, G.brq, G.sf[G.N], He, Qe, Hg, Qg);
#pragma unroll
    for (int p = 3; p < 5; ++p)
      if (j - 2 + p >= G.N) {
        w.H[p] = Hg;
        w.Q[p] = Qg;
      }
  }
}

// Level data in the precision T of a pass: FP64 values as stored; FP32
// values from the copies when the level has them, else converted at use.
template <typename T> struct GeoT;
template <> struct GeoT<double> {
  static __device__ __forceinline__ double u(const Geo &G, const double *U, int i) { return U[i]; }
  static __device__ __forceinline__ double isf(const Geo &G, int f) { return G.isf[f]; }
  static __device__ __forceinline__ double cgf(const Geo &G, int f) { return G.cgf[f]; }
  static __device__ __forceinline__ double igq(const Geo &G, int i) { return G.igq[i]; }
  static __device__ __forceinline__ double sigx(const Geo &G, int i) { return G.gq[2 * G.N + i]; }
  static __device__ __forceinline__ double bx(const Geo &G, int i) { return G.gq[4 * G.N + i]; }
  static __device__ __forceinline__ double g(const Geo &G) { return G.g; }
  static __device__ __forceinline__ double hdx(const Geo &G) { return 0.5 * G.dx; }
};
template <> struct GeoT<float> {
  static __device__ __forceinline__ float u(const Geo &G, const double *U, int i) {
    return G.U32 ? G.U32[i] : float(U[i]);
  }
  static __device__ __forceinline__ float isf(const Geo &G, int f) { return G.isf32 ? G.isf32[f] : float(G.isf[f]); }
  static __device__ __forceinline__ float cgf(const Geo &G, int f) { return G.cgf32 ? G.cgf32[f] : float(G.cgf[f]); }
  static __device__ __forceinline__ float igq(const Geo &G, int i) { return G.igq32 ? G.igq32[i] : float(G.igq[i]); }
  static __device__ __forceinline__ float sigx(const Geo &G, int i) {
    return G.gq32 ? G.gq32[i] : float(G.gq[2 * G.N + i]);
  }
  static __device__ __forceinline__ float bx(const Geo &G, int i) {
    return G.gq32 ? G.gq32[2 * G.N + i] : float(G.gq[4 * G.N + i]);
  }
  static __device__ __forceinline__ float g(const Geo &G) { return G.isf32 ? G.g32 : float(G.g); }
  static __device__ __forceinline__ float hdx(const Geo &G) { return G.isf32 ? G.hdx32 : 0.5f * float(G.dx); }
};

// Two-point Gauss source of cell j (Eq. 9): S = (dx/2) sum_q [g h^2 sigma_x/2
// - g sigma h b_x] at the Gauss points, h = H_h/sigma, H_h the cubic through
// the interface values p0..p3 of H at t = -3/2, -1/2, 1/2, 3/2.
// With H_h = sigma h the second term is g H_h b_x; 1/sigma is per-cell
// geometry.
template <typename T>
__device__ __forceinline__ T source_at(const Geo &G, int j, T p0, T p1, T p2, T p3) {
  T S = T(0.0);
  const T g = GeoT<T>::g(G);
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    T Hh = T(kLag[q][0]) * p0 + T(kLag[q][1]) * p1 + T(kLag[q][2]) * p2 + T(kLag[q][3]) * p3;
    T sigx = GeoT<T>::sigx(G, q * G.N + j);
    T bx = GeoT<T>::bx(G, q * G.N + j);
    T h = Hh * GeoT<T>::igq(G, q * G.N + j);
    S += T(0.5) * g * h * h * sigx - g * Hh * bx;
  }
  return S * GeoT<T>::hdx(G);
}

// Local residual R_j (Eq. 10) from a filled window.
__device__ __forceinline__ void local_residual(const Geo &G, int j, const Win &w, double &R0, double &R1) {
  double upH[3], umH[3], upQ[3], umQ[3];
#pragma unroll
  for (int p = 0; p < 3; ++p) {
    weno3(w.H[p], w.H[p + 1], w.H[p + 2], upH[p], umH[p]);
    weno3(w.Q[p], w.Q[p + 1], w.Q[p + 2], upQ[p], umQ[p]);
  }
  double Fr0, Fr1, Fl0, Fl1;
  num_flux<-1>(fstate(umH[1], umQ[1], G.isf[j + 1], G.cgf[j + 1], G.g),
               fstate(upH[2], upQ[2], G.isf[j + 1], G.cgf[j + 1], G.g), G.flux, Fr0, Fr1);
  num_flux<-1>(fstate(umH[0], umQ[0], G.isf[j], G.cgf[j], G.g), fstate(upH[1], upQ[1], G.isf[j], G.cgf[j], G.g),
               G.flux, Fl0, Fl1);
  double S = source_at(G, j, upH[0], upH[1], umH[1], umH[2]);
  R0 = Fr0 - Fl0;
  R1 = Fr1 - Fl1 - S;
}

// ----------------------------------------------------------------------------
// Block-level helpers.

// Fixed-order block sum (warp shuffles, then warps in index order).
__device__ double block_sum(double v, double *red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    red[32] = s;
  }
  __syncthreads();
  double s = red[32];
  __syncthreads();
  return s;
}

// ----------------------------------------------------------------------------
// Teams: the threads that share one problem's phases. BlockTeam is one
// thread block (the batched form: one problem per block). ClusterTeam is a
// thread-block cluster of up to 16 CTAs on as many SMs (the latency form:
// one problem per cluster): the per-cell loops of a phase are strided over
// all its threads, phases are separated by cluster barriers (release /
// acquire at cluster scope, so the global writes of one phase are visible to
// every CTA in the next), and the coarse levels and the coarsest LU run on
// the leader CTA alone with block barriers. Every cluster barrier is reached
// by all threads of the cluster: the branches around them depend only on
// values that are the same in every CTA (sizes, and res, flags and counters
// reduced over the cluster).
struct BlockTeam {
  __device__ __forceinline__ int tid() const { return threadIdx.x; }
  __device__ __forceinline__ int size() const { return blockDim.x; }
  __device__ __forceinline__ void sync() const { __syncthreads(); }
  __device__ __forceinline__ bool lead() const { return true; }
  static constexpr bool kMulti = false;
  // the same sum in every thread (fixed order)
  __device__ __forceinline__ double sum(double v, double *red) const { return block_sum(v, red); }
  __device__ __forceinline__ bool any(bool b) const { return __syncthreads_or(b) != 0; }
  // the leader's value of a flag in every thread (after the leader wrote it)
  __device__ __forceinline__ int lead_value(const int *flag) const { return *flag; }
};

struct ClusterTeam {
  int rank, n;
  __device__ __forceinline__ int tid() const { return rank * (int)blockDim.x + (int)threadIdx.x; }
  __device__ __forceinline__ int size() const { return n * (int)blockDim.x; }
  __device__ __forceinline__ void sync() const { cooperative_groups::this_cluster().sync(); }
  __device__ __forceinline__ bool lead() const { return rank == 0; }
  static constexpr bool kMulti = true;
  // CTA partials in rank order: every thread adds the same values in the same
  // order. red[33] holds this CTA's partial until all CTAs have read it.
  __device__ double sum(double v, double *red) const {
    const double part = block_sum(v, red);
    if (threadIdx.x == 0) red[33] = part;
    sync();
    auto cl = cooperative_groups::this_cluster();
    double s = 0.0;
    for (int r = 0; r < n; ++r) s += *cl.map_shared_rank(red + 33, r);
    sync();
    return s;
  }
  __device__ bool any(bool b) const {
    __shared__ int s_any;
    const int mine = __syncthreads_or(b);
    if (threadIdx.x == 0) s_any = mine;
    sync();
    auto cl = cooperative_groups::this_cluster();
    int a = 0;
    for (int r = 0; r < n; ++r) a |= *cl.map_shared_rank(&s_any, r);
    sync();
    return a != 0;
  }
  __device__ int lead_value(const int *flag) const {
    const int v = *cooperative_groups::this_cluster().map_shared_rank(const_cast<int *>(flag), 0);
    sync();
    return v;
  }
};

// Residual of cells [first, N) with stride; returns sum_j ||R_j||_1.
__device__ double residual_cells(const Geo &G, const double *U, double *R, int first, int stride) {
  const double *H = U, *Q = U + G.N;
  double acc = 0.0;
  for (int j = first; j < G.N; j += stride) {
    Win w;
    load_win(G, H, Q, j, w);
    fill_ghosts(G, j, w);
    double R0, R1;
    local_residual(G, j, w, R0, R1);
    R[j] = R0;
    R[G.N + j] = R1;
    acc += fabs(R0) + fabs(R1);
  }
  return acc;
}

// The same residual with each block's five-cell windows staged in shared
// memory: the block reads cells t0-2 .. t0+B+1 of a tile of B = blockDim.x
// cells once, coalesced, and every thread builds its window from the tile.
// Thread tid of block bid takes cells bid*B + tid + k*nblk*B, the cells and
// the order of residual_cells with first = bid*B + tid, stride = nblk*B, so
// the partial sums are the same bits. sH, sQ: B + 4 doubles each.
__device__ double residual_cells_staged(const Geo &G, const double *U, double *R, int bid, int nblk, double *sH,
                                        double *sQ) {
  const int B = blockDim.x, N = G.N;
  const double *H = U, *Q = U + N;
  double acc = 0.0;
  for (int t0 = bid * B; t0 < N; t0 += nblk * B) {  // block-uniform
    __syncthreads();                                // the previous tile's windows are read
    for (int i = threadIdx.x; i < B + 4; i += B) {
      const int k = min(max(t0 - 2 + i, 0), N - 1);  // clamped as load_win: ghosts are filled later
      sH[i] = H[k];
      sQ[i] = Q[k];
    }
    __syncthreads();
    const int j = t0 + threadIdx.x;
    if (j < N) {
      Win w;
#pragma unroll
      for (int p = 0; p < 5; ++p) {
        w.H[p] = sH[threadIdx.x + p];
        w.Q[p] = sQ[threadIdx.x + p];
      }
      fill_ghosts(G, j, w);
      double R0, R1;
      local_residual(G, j, w, R0, R1);
      R[j] = R0;
      R[N + j] = R1;
      acc += fabs(R0) + fabs(R1);
    }
  }
  return acc;
}

// ----------------------------------------------------------------------------
// Regularized FD Jacobian (Eq. 12-13) in three passes that share work between
// neighbouring cells. Perturbing U_i in component m changes only the
// component-m reconstructions of cells i-1, i, i+1 (WENO3 is component-wise,
// ghost states copy the same component of the edge cell), hence only the
// fluxes of faces i-1..i+2 and the sources of cells i-1..i+1. So:
//   A  per cell k = -1..N: reconstructions of the base state and of the
//      three states with cell k-1, k or k+1 perturbed (same component);
//   B  per face f = 0..N: the base flux and the 8 fluxes with one of cells
//      f-2..f+1 perturbed in one component;
//   C  per block (j, i): R_j of the perturbed state from two face fluxes and
//      the Gauss source, minus the base R_j, over eps, plus alpha ||R_j||_1 I
//      on the diagonal.
// Each perturbed R_j is the same arithmetic on the same values as a full
// re-evaluation of the local residual, at a fraction of the cost.

template <typename T>
struct JW {
  T *rec;  // [2 comps][4 variants][2: up, um][N+2], cell k at k+1
  T *flx;  // [9 variants][2 comps][N+1]
  int N;
  __device__ __forceinline__ T &r(int m, int v, int o, int k) const {
    return rec[((m * 4 + v) * 2 + o) * (N + 2) + (k + 1)];
  }
  __device__ __forceinline__ T &f(int w, int l, int face) const { return flx[(w * 2 + l) * (N + 1) + face]; }
};

template <typename T>
__device__ __forceinline__ JW<T> jw_view(double *base, int N) {
  JW<T> W;
  W.rec = reinterpret_cast<T *>(base);
  W.flx = W.rec + 16 * (size_t)(N + 2);
  W.N = N;
  return W;
}

// Component m of cell kk (ghosts included) of the state with interior cell
// ip perturbed by eps in component m (ip = -1: no perturbation).
template <typename T>
__device__ __forceinline__ T pval(const Geo &G, const double *U, int m, int kk, int ip, double eps, T eps_t) {
  const int N = G.N;
  if (kk >= 0 && kk < N) {
    T x = GeoT<T>::u(G, U, m * N + kk);
    return kk == ip ? x + eps_t : x;
  }
  const int e = kk < 0 ? 0 : N - 1;
  double He = U[e], Qe = U[N + e];
  if (e == ip) {
    if (m == 0) He += eps;
    else Qe += eps;
  }
  double Hg, Qg;
  if (kk < 0) ghost(G.bl, G.blh, G.blq, G.sf[0], He, Qe, Hg, Qg);
  else ghost(G.br, G.brh, G.brq, G.sf[N], He, Qe, Hg, Qg);
  return T(m == 0 ? Hg : Qg);
}

// Pass A. Variant v = 0: base; v = 1, 2, 3: cell k + v - 2 perturbed.
template <typename T>
__device__ void jac_pass_a(const Geo &G, const double *U, double eps, const JW<T> &W, int first, int stride) {
  const int N = G.N, items = (N + 2) * 8;
  const T eps_t = T(eps);
  for (int it = first; it < items; it += stride) {
    const int k = it % (N + 2) - 1, mv = it / (N + 2), m = mv >> 2, v = mv & 3;
    int ip = -1;
    if (v > 0) {
      ip = k + v - 2;
      if (ip < 0 || ip >= N) continue;
    }
    T up, um;
    weno3<T>(pval<T>(G, U, m, k - 1, ip, eps, eps_t), pval<T>(G, U, m, k, ip, eps, eps_t),
             pval<T>(G, U, m, k + 1, ip, eps, eps_t), up, um);
    W.r(m, v, 0, k) = up;
    W.r(m, v, 1, k) = um;
  }
}

// Reconstruction variant of cell kk under a perturbation of cell i.
__device__ __forceinline__ int rec_variant(int i, int kk) {
  int d = i - kk;
  return (d >= -1 && d <= 1) ? d + 2 : 0;
}

// Pass B, one face per item. Variant w = 0: base; w = 1 + 2p + m: cell
// f - 2 + p perturbed in component m. The left state comes from cell f-1
// (perturbed for p = 0, 1, 2), the right state from cell f (p = 1, 2, 3);
// the per-state HLL quantities of the base states serve all variants that do
// not perturb that side.
template <typename T, int FLUX>
__device__ void jac_pass_b(const Geo &G, const JW<T> &W, int first, int stride) {
  const int N = G.N;
  const T g = GeoT<T>::g(G);
  for (int f = first; f <= N; f += stride) {
    const T isg = GeoT<T>::isf(G, f), cg = GeoT<T>::cgf(G, f);
    const FState<T> Lb = fstate<T>(W.r(0, 0, 1, f - 1), W.r(1, 0, 1, f - 1), isg, cg, g);
    const FState<T> Rb = fstate<T>(W.r(0, 0, 0, f), W.r(1, 0, 0, f), isg, cg, g);
    T F0, F1;
    num_flux<FLUX>(Lb, Rb, G.flux, F0, F1);
    W.f(0, 0, f) = F0;
    W.f(0, 1, f) = F1;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const int i = f - 2 + p;
      if (i < 0 || i >= N) continue;
#pragma unroll
      for (int m = 0; m < 2; ++m) {
        // a Q perturbation (m = 1) leaves H, 1/H, c and the pressure term of
        // the base state
        FState<T> Ls = Lb, Rs = Rb;
        if (p <= 2)
          Ls = m == 0 ? fstate<T>(W.r(0, p + 1, 1, f - 1), W.r(1, 0, 1, f - 1), isg, cg, g)
                      : fstate_q<T>(Lb, W.r(1, p + 1, 1, f - 1));
        if (p >= 1)
          Rs = m == 0 ? fstate<T>(W.r(0, p, 0, f), W.r(1, 0, 0, f), isg, cg, g) : fstate_q<T>(Rb, W.r(1, p, 0, f));
        num_flux<FLUX>(Ls, Rs, G.flux, F0, F1);
        const int w = 1 + 2 * p + m;
        W.f(w, 0, f) = F0;
        W.f(w, 1, f) = F1;
      }
    }
  }
}

// Flux variant at face `face` for a perturbation of cell i, component m.
__device__ __forceinline__ int flux_variant(int i, int m, int face) {
  int p = i - face + 2;
  return (p >= 0 && p <= 3) ? 1 + 2 * p + m : 0;
}

// Pass C, one cell j per item: the base R_j (written when Rout is given),
// then for each block k (cell i = j + k - hw) R_j of the state with U_i
// perturbed, from two face fluxes and the Gauss source, minus the base R_j,
// over eps, plus alpha ||R_j||_1 I on the diagonal. The regularisation uses
// Rreg when given (the FP64 residual of a mixed-precision step), else the
// pass's own base residual. Returns the partial sum of ||R_j||_1 of the
// cells that wrote R.
template <typename T>
__device__ double jac_pass_c(const Geo &G, int nb, double eps, double alpha, const JW<T> &W, const double *Rreg,
                             double *Rout, T *J, int first, int stride) {
  const int N = G.N, hw = (nb - 1) / 2;
  const T ieps = T(1.0) / T(eps);
  double acc = 0.0;
  for (int j = first; j < N; j += stride) {
    const T Sb = source_at<T>(G, j, W.r(0, 0, 0, j - 1), W.r(0, 0, 0, j), W.r(0, 0, 1, j), W.r(0, 0, 1, j + 1));
    const T R0 = W.f(0, 0, j + 1) - W.f(0, 0, j);
    const T R1 = W.f(0, 1, j + 1) - W.f(0, 1, j) - Sb;
    if (Rout) {
      Rout[j] = double(R0);
      Rout[N + j] = double(R1);
      acc += fabs(double(R0)) + fabs(double(R1));
    }
    const T reg = Rreg ? T(alpha * (fabs(Rreg[j]) + fabs(Rreg[N + j]))) : T(alpha) * (fabs(R0) + fabs(R1));
    for (int k = 0; k < nb; ++k) {
      const int i = j + k - hw;
      if (i < 0 || i >= N) {
#pragma unroll
        for (int e = 0; e < 4; ++e) J[(k * 4 + e) * N + j] = T(0.0);
        continue;
      }
#pragma unroll
      for (int m = 0; m < 2; ++m) {
        T S = Sb;
        if (m == 0) {
          const int v0 = rec_variant(i, j - 1), v1 = rec_variant(i, j), v2 = rec_variant(i, j + 1);
          S = source_at<T>(G, j, W.r(0, v0, 0, j - 1), W.r(0, v1, 0, j), W.r(0, v1, 1, j), W.r(0, v2, 1, j + 1));
        }
        const int wr = flux_variant(i, m, j + 1), wl = flux_variant(i, m, j);
        const T P0 = W.f(wr, 0, j + 1) - W.f(wl, 0, j);
        const T P1 = W.f(wr, 1, j + 1) - W.f(wl, 1, j) - S;
        T v0 = (P0 - R0) * ieps, v1 = (P1 - R1) * ieps;
        if (i == j) {
          if (m == 0) v0 += reg;
          else v1 += reg;
        }
        J[(k * 4 + 0 * 2 + m) * N + j] = v0;
        J[(k * 4 + 1 * 2 + m) * N + j] = v1;
      }
    }
  }
  return acc;
}

// ----------------------------------------------------------------------------
// FP64 residual in three passes over a compact workspace (the residual of a
// mixed-precision Newton step): reconstructions once per cell, fluxes once
// per face, then sources and differences per cell. Same arithmetic as the
// base variant of the Jacobian passes.
struct RW {
  double *rec;  // [2 comps][2: up, um][N+2], cell k at k+1
  double *flx;  // [2 comps][N+1]
  int N;
  __device__ __forceinline__ double &r(int m, int o, int k) const { return rec[(m * 2 + o) * (N + 2) + (k + 1)]; }
  __device__ __forceinline__ double &f(int l, int face) const { return flx[l * (N + 1) + face]; }
};

// FP32 copies of a mixed-precision level (Geo::U32 and the geometry): 10 N + 2
// floats placed after the FP64 residual's workspace, within jw_doubles(N).
__host__ __device__ inline size_t f32_area_offset(size_t N) {
  const size_t rw = (jw_doubles(N) / 2 + 2) / 2 * 2;
  return (rw + 4 * (N + 2) + 2 * (N + 1) + 3) / 4 * 4;
}

// Points G's FP32 copies at their place in the Jacobian workspace jw.
__device__ __forceinline__ float *attach_f32(Geo &G, double *jw) {
  float *A = reinterpret_cast<float *>(jw + f32_area_offset((size_t)G.N));
  const int N = G.N;
  G.U32 = A;
  G.isf32 = A + 2 * N;
  G.cgf32 = G.isf32 + N + 1;
  G.igq32 = G.cgf32 + N + 1;
  G.gq32 = G.igq32 + 2 * N;
  G.g32 = float(G.g);
  G.hdx32 = 0.5f * float(G.dx);
  return A;
}

// Writes the FP32 copies of state U and of G's geometry into A (attach_f32's
// layout), items strided.
__device__ void fill_f32(const Geo &G, const double *U, float *A, int first, int stride) {
  const int N = G.N;
  float *U32 = A, *isf = A + 2 * N, *cgf = isf + N + 1, *igq = cgf + N + 1, *gq = igq + 2 * N;
  for (int t = first; t < 4 * N; t += stride) {
    if (t < 2 * N) {
      U32[t] = float(U[t]);
      igq[t] = float(G.igq[t]);
    }
    if (t <= N) {
      isf[t] = float(G.isf[t]);
      cgf[t] = float(G.cgf[t]);
    }
    gq[t] = float(G.gq[2 * N + t]);  // sigma_x and b_x planes
  }
}

// Placed after the FP32 Jacobian workspace of the same level.
__device__ __forceinline__ RW rw_view(double *jw, int N) {
  RW W;
  W.rec = jw + (jw_doubles((size_t)N) / 2 + 2) / 2 * 2;
  W.flx = W.rec + 4 * (size_t)(N + 2);
  W.N = N;
  return W;
}

__device__ void res_pass_a(const Geo &G, const double *U, const RW &W, int first, int stride) {
  const int N = G.N, items = (N + 2) * 2;
  for (int it = first; it < items; it += stride) {
    const int k = it % (N + 2) - 1, m = it / (N + 2);
    double up, um;
    weno3<double>(pval<double>(G, U, m, k - 1, -1, 0.0, 0.0), pval<double>(G, U, m, k, -1, 0.0, 0.0),
                  pval<double>(G, U, m, k + 1, -1, 0.0, 0.0), up, um);
    W.r(m, 0, k) = up;
    W.r(m, 1, k) = um;
  }
}

template <int FLUX>
__device__ void res_pass_b(const Geo &G, const RW &W, int first, int stride) {
  for (int f = first; f <= G.N; f += stride) {
    double F0, F1;
    num_flux<FLUX>(fstate(W.r(0, 1, f - 1), W.r(1, 1, f - 1), G.isf[f], G.cgf[f], G.g),
                   fstate(W.r(0, 0, f), W.r(1, 0, f), G.isf[f], G.cgf[f], G.g), G.flux, F0, F1);
    W.f(0, f) = F0;
    W.f(1, f) = F1;
  }
}

__device__ double res_pass_c(const Geo &G, const RW &W, double *R, int first, int stride) {
  const int N = G.N;
  double acc = 0.0;
  for (int j = first; j < N; j += stride) {
    const double S = source_at<double>(G, j, W.r(0, 0, j - 1), W.r(0, 0, j), W.r(0, 1, j), W.r(0, 1, j + 1));
    const double R0 = W.f(0, j + 1) - W.f(0, j);
    const double R1 = W.f(1, j + 1) - W.f(1, j) - S;
    R[j] = R0;
    R[N + j] = R1;
    acc += fabs(R0) + fabs(R1);
  }
  return acc;
}

// Derived geometry of every level (1/sigma and sqrt(g/sigma) at faces, 1/sigma
// at the Gauss points), items strided over the finest level's faces.
__device__ void geom_derive_items(const ProbDev &P, int first, int stride) {
  for (int l = 0; l < P.levels; ++l) {
    const LevelDev &Lv = P.lev[l];
    const int N = Lv.N;
    double *isf = Lv.gd, *cgf = isf + N + 1, *igq = cgf + N + 1;
    for (int t = first; t <= N; t += stride) {
      isf[t] = 1.0 / Lv.sf[t];
      cgf[t] = sqrt(P.g * isf[t]);
    }
    for (int t = first; t < 2 * N; t += stride) {
      const int q = t / N, j = t % N;
      igq[t] = 1.0 / Lv.gq[(0 * 2 + q) * N + j];
    }
  }
}

// Inverse of the diagonal 2x2 blocks.
template <typename T>
__device__ void dinv_cells(int N, int nb, const T *J, T *Dinv, int first, int stride) {
  const int hw = (nb - 1) / 2;
  for (int j = first; j < N; j += stride) {
    T a = J[(hw * 4 + 0) * N + j], b = J[(hw * 4 + 1) * N + j];
    T c = J[(hw * 4 + 2) * N + j], d = J[(hw * 4 + 3) * N + j];
    T idet = T(1.0) / (a * d - b * c);
    Dinv[0 * N + j] = d * idet;
    Dinv[1 * N + j] = -b * idet;
    Dinv[2 * N + j] = -c * idet;
    Dinv[3 * N + j] = a * idet;
  }
}

// Galerkin coarse operator (Eq. 17): sums of fine blocks over aggregate pairs.
// An interior aggregate (2j, 2j+1) of a three-block fine level has the
// coarse blocks J_-1(2j), J_0(2j) + J_+1(2j) + J_-1(2j+1) + J_0(2j+1) and
// J_+1(2j+1), summed in the order of the general loop below.
template <typename T>
__device__ void coarse_op_cells(int Nf, int nbf, const T *Jf, int Nc, T *Jc, int first, int stride) {
  const int hf = (nbf - 1) / 2;
  for (int j = first; j < Nc; j += stride) {
    if (nbf == 3 && j > 0 && 2 * j + 2 < Nf) {
      const int x0 = 2 * j, x1 = 2 * j + 1;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        Jc[(0 * 4 + e) * Nc + j] = Jf[(0 * 4 + e) * Nf + x0];
        Jc[(1 * 4 + e) * Nc + j] =
            ((Jf[(1 * 4 + e) * Nf + x0] + Jf[(2 * 4 + e) * Nf + x0]) + Jf[(0 * 4 + e) * Nf + x1]) +
            Jf[(1 * 4 + e) * Nf + x1];
        Jc[(2 * 4 + e) * Nc + j] = Jf[(2 * 4 + e) * Nf + x1];
      }
      continue;
    }
    T a0[4] = {0, 0, 0, 0}, a1[4] = {0, 0, 0, 0}, a2[4] = {0, 0, 0, 0};
    for (int a = 0; a < 2; ++a) {
      int xi = 2 * j + a;
      if (xi >= Nf) break;
      for (int k = 0; k < nbf; ++k) {
        int eta = xi + k - hf;
        if (eta < 0 || eta >= Nf) continue;
        int kc = eta / 2 - j + 1;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          T v = Jf[(k * 4 + e) * Nf + xi];
          if (kc == 0) a0[e] += v;
          else if (kc == 1) a1[e] += v;
          else a2[e] += v;
        }
      }
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      Jc[(0 * 4 + e) * Nc + j] = a0[e];
      Jc[(1 * 4 + e) * Nc + j] = a1[e];
      Jc[(2 * 4 + e) * Nc + j] = a2[e];
    }
  }
}

// Block SOR update (Eq. 19) of the cells of one colour (j mod C == col),
// applied `reps` times in a row. Cells of one colour do not couple, so a
// repeated visit of the same colour sees the same neighbour values: the
// correction t is computed once and the relaxation applied reps times, which
// is exactly the sequence of reps separate passes. The neighbour sum is a
// chain of fused multiply-adds (two per product pair instead of a multiply,
// a fused multiply-add and an add).
template <typename T>
__device__ void sor_colour(int N, int nb, const T *J, const T *Dinv, const T *R, T *dU, double omega_d, int C,
                           int col, int reps, int first, int stride) {
  const T omega = T(omega_d);
  const int hw = (nb - 1) / 2;
  for (int j = col + C * first; j < N; j += C * stride) {
    T r0 = R[j], r1 = R[N + j];
    for (int k = 0; k < nb; ++k) {
      int i = j + k - hw;
      if (k == hw || i < 0 || i >= N) continue;
      T x0 = dU[i], x1 = dU[N + i];
      r0 = fma(J[(k * 4 + 0) * N + j], x0, r0);
      r0 = fma(J[(k * 4 + 1) * N + j], x1, r0);
      r1 = fma(J[(k * 4 + 2) * N + j], x0, r1);
      r1 = fma(J[(k * 4 + 3) * N + j], x1, r1);
    }
    T t0 = Dinv[0 * N + j] * r0 + Dinv[1 * N + j] * r1;
    T t1 = Dinv[2 * N + j] * r0 + Dinv[3 * N + j] * r1;
    T x0 = dU[j], x1 = dU[N + j];
    for (int r = 0; r < reps; ++r) {
      x0 = (T(1.0) - omega) * x0 - omega * t0;
      x1 = (T(1.0) - omega) * x1 - omega * t1;
    }
    dU[j] = x0;
    dU[N + j] = x1;
  }
}

// Defect restriction (Eq. 17) and zero coarse correction.
template <typename T>
__device__ void restrict_cells(int Nf, int nb, const T *J, const T *R, const T *dU, int Nc, T *Rc, T *dUc,
                               int first, int stride) {
  const int hw = (nb - 1) / 2;
  for (int j = first; j < Nc; j += stride) {
    T s0 = T(0.0), s1 = T(0.0);
    for (int a = 0; a < 2; ++a) {
      int xi = 2 * j + a;
      if (xi >= Nf) break;
      T r0 = R[xi], r1 = R[Nf + xi];
      for (int k = 0; k < nb; ++k) {
        int eta = xi + k - hw;
        if (eta < 0 || eta >= Nf) continue;
        T x0 = dU[eta], x1 = dU[Nf + eta];
        r0 = fma(J[(k * 4 + 0) * Nf + xi], x0, r0);
        r0 = fma(J[(k * 4 + 1) * Nf + xi], x1, r0);
        r1 = fma(J[(k * 4 + 2) * Nf + xi], x0, r1);
        r1 = fma(J[(k * 4 + 3) * Nf + xi], x1, r1);
      }
      s0 += r0;
      s1 += r1;
    }
    Rc[j] = s0;
    Rc[Nc + j] = s1;
    dUc[j] = T(0.0);
    dUc[Nc + j] = T(0.0);
  }
}

// Prolongation (Eq. 18).
template <typename T>
__device__ void prolong_cells(int Nf, T *dU, int Nc, const T *dUc, int first, int stride) {
  for (int xi = first; xi < Nf; xi += stride) {
    dU[xi] += dUc[xi / 2];
    dU[Nf + xi] += dUc[Nc + xi / 2];
  }
}

// App. A (Eq. A.2): fine averages from the coarse quadratic; the domain ends
// use the coarse level's ghost states.
__device__ void interp_cells(const Geo &Gc, const double *Uc, double *Uf, int first, int stride) {
  const int Nc = Gc.N, Nf = 2 * Nc;
  const double *Hc = Uc, *Qc = Uc + Nc;
  for (int c = first; c < Nc; c += stride) {
    double hm, qm, hp, qp;
    double h0 = Hc[c], q0 = Qc[c];
    if (c > 0) {
      hm = Hc[c - 1];
      qm = Qc[c - 1];
    } else {
      ghost(Gc.bl, Gc.blh, Gc.blq, Gc.sf[0], Hc[0], Qc[0], hm, qm);
    }
    if (c < Nc - 1) {
      hp = Hc[c + 1];
      qp = Qc[c + 1];
    } else {
      ghost(Gc.br, Gc.brh, Gc.brq, Gc.sf[Nc], Hc[Nc - 1], Qc[Nc - 1], hp, qp);
    }
    Uf[2 * c] = hm / 8.0 + h0 - hp / 8.0;
    Uf[2 * c + 1] = -hm / 8.0 + h0 + hp / 8.0;
    Uf[Nf + 2 * c] = qm / 8.0 + q0 - qp / 8.0;
    Uf[Nf + 2 * c + 1] = -qm / 8.0 + q0 + qp / 8.0;
  }
}

// ----------------------------------------------------------------------------
// Coarsest direct solve: LU with partial pivoting (ties to the lowest row) of
// the block-banded system, unknown u = 2j + m, in LAPACK-style band storage
// (kl sub-diagonals, 2 kl super-diagonals after fill-in). A banded matrix
// keeps its zeros outside the band through the elimination, so this performs
// the same pivots and updates as a dense LU. The elimination is a sequence of
// n pivot steps; one warp runs it, its lanes covering the entries of a step
// (the kl multipliers, the kl x 2kl updated entries, the 2kl back-substitution
// updates). GB300 issues an FP64 warp instruction at the same cost whatever
// its active lanes, so spreading each step over lanes, rather than running it
// on one thread, divides the FP64 work of the solve by about the band width.
// Every entry sees the same operations in the same order as in a serial
// elimination.

template <typename T>
struct Band {
  T *ab;    // [ldab][n]
  int *piv;      // [n]
  T *x;     // [n]
  T *rinv;  // [n] reciprocals of the pivots
  int n, kl, ldab;
  __device__ __forceinline__ T &A(int r, int c) const { return ab[(2 * kl + r - c) * n + c]; }
};

// Order key of |a|: for non-negative floating-point values the bit patterns,
// read as unsigned integers, are ordered as the values (NaN keys are dropped
// to 0, so a NaN never wins a pivot search).
__device__ __forceinline__ unsigned long long abs_key(double a) {
  return a == a ? (unsigned long long)(__double_as_longlong(a) & 0x7fffffffffffffffLL) : 0ull;
}
__device__ __forceinline__ unsigned long long abs_key(float a) {
  return a == a ? (unsigned long long)(__float_as_uint(a) & 0x7fffffffu) : 0ull;
}

// Factorisation by warp 0 (lanes 0..31, all of them calling). Returns true if
// a pivot was exactly zero.
template <typename T>
__device__ bool band_lu_warp(const Band<T> &B) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int n = B.n, kl = B.kl, w2 = 2 * kl, upd = kl * w2;
  bool sing = false;
  for (int k = 0; k < n; ++k) {
    const int imax = min(n - 1, k + kl), cmax = min(n - 1, k + w2);
    // Pivot: the first row of largest |A(i, k)|, i = k..imax (kl <= 7).
    unsigned long long key = 0;
    int p = 0x7fffffff;
    if (lane <= kl && k + lane <= imax) {
      key = abs_key(B.A(k + lane, k));
      p = k + lane;
    }
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) {
      const unsigned long long ok = __shfl_xor_sync(FULL, key, o);
      const int op = __shfl_xor_sync(FULL, p, o);
      if (ok > key || (ok == key && op < p)) {
        key = ok;
        p = op;
      }
    }
    p = __shfl_sync(FULL, p, 0);
    if (lane == 0) B.piv[k] = p;
    if (p != k)
      for (int c = k + lane; c <= cmax; c += 32) {
        const T t = B.A(k, c);
        B.A(k, c) = B.A(p, c);
        B.A(p, c) = t;
      }
    __syncwarp();
    // One division for 1/d (lane 0) and the multipliers A(k+i, k)/d (lane i).
    const T d = B.A(k, k);
    const bool mrow = lane >= 1 && lane <= kl && k + lane <= imax;
    const T q = (lane == 0 ? T(1.0) : (mrow ? B.A(k + lane, k) : T(0.0))) / d;
    if (lane == 0) {
      B.rinv[k] = q;
      if (d == T(0.0)) sing = true;
    }
    if (mrow) B.A(k + lane, k) = q;
    // A(k+i, k+c) -= l_i A(k, k+c), i = 1..kl, c = 1..2kl.
    for (int e0 = 0; e0 < upd; e0 += 32) {
      const int e = e0 + lane, i = 1 + e / w2, c = 1 + e % w2;
      const T l = __shfl_sync(FULL, q, min(i, 31));
      if (e < upd && k + i <= imax && k + c <= cmax) B.A(k + i, k + c) -= l * B.A(k, k + c);
    }
    __syncwarp();
  }
  return __shfl_sync(FULL, sing, 0);
}

// x (B.x, length n) := A^{-1} x with the stored factors, by warp 0. The back
// substitution is column oriented: once x_i is known, the rows above it take
// their A(r, i) x_i terms, so each row subtracts its terms from the farthest
// column to the nearest, the order of the row-oriented loop.
template <typename T>
__device__ void band_lu_solve_warp(const Band<T> &B) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int n = B.n, kl = B.kl;
  for (int k = 0; k < n; ++k) {
    const int p = B.piv[k];
    if (p != k && lane == 0) {
      const T t = B.x[k];
      B.x[k] = B.x[p];
      B.x[p] = t;
    }
    __syncwarp();
    const T xk = B.x[k];
    if (lane >= 1 && lane <= kl && k + lane < n) B.x[k + lane] -= B.A(k + lane, k) * xk;
    __syncwarp();
  }
  for (int i = n - 1; i >= 0; --i) {
    T xi = T(0.0);
    if (lane == 0) {
      xi = B.x[i] * B.rinv[i];
      B.x[i] = xi;
    }
    xi = __shfl_sync(FULL, xi, 0);
    const int r = i - lane;
    if (lane >= 1 && lane <= 2 * kl && r >= 0) B.x[r] -= B.A(r, i) * xi;
    __syncwarp();
  }
}

// FP32 instantiation: one thread runs the elimination with the active rows in
// registers (a window of kl+1 rows). FP32 instructions issue at full rate, so
// the serial recurrence is shorter than its warp-parallel form, whose
// shuffles and warp barriers then dominate.
template <int KL, typename T>
__device__ bool band_lu_serial(const Band<T> &B) {
  constexpr int W = 2 * KL + 1;
  const int n = B.n;
  T w[KL + 1][W];
#pragma unroll
  for (int i = 0; i <= KL; ++i)
#pragma unroll
    for (int c = 0; c < W; ++c) w[i][c] = (i < n && c < n) ? B.A(i, c) : T(0.0);
  bool sing = false;
  for (int k = 0; k < n; ++k) {
    int p = 0;
    T best = fabs(w[0][0]);
#pragma unroll
    for (int i = 1; i <= KL; ++i)
      if (k + i < n && fabs(w[i][0]) > best) {
        best = fabs(w[i][0]);
        p = i;
      }
    B.piv[k] = k + p;
#pragma unroll
    for (int i = 1; i <= KL; ++i)
      if (p == i)
#pragma unroll
        for (int c = 0; c < W; ++c) {
          T t = w[0][c];
          w[0][c] = w[i][c];
          w[i][c] = t;
        }
    const T d = w[0][0];
    if (d == T(0.0)) sing = true;
    B.rinv[k] = T(1.0) / d;
#pragma unroll
    for (int i = 1; i <= KL; ++i)
      if (k + i < n) {
        const T l = w[i][0] / d;
        B.A(k + i, k) = l;
#pragma unroll
        for (int c = 1; c < W; ++c) w[i][c] -= l * w[0][c];
      }
#pragma unroll
    for (int c = 0; c < W; ++c)
      if (k + c < n) B.A(k, k + c) = w[0][c];
    // Slide the window one row and one column.
#pragma unroll
    for (int i = 0; i < KL; ++i) {
#pragma unroll
      for (int c = 0; c < W - 1; ++c) w[i][c] = w[i + 1][c + 1];
      w[i][W - 1] = T(0.0);
    }
    const int r = k + KL + 1;
#pragma unroll
    for (int c = 0; c < W; ++c) w[KL][c] = (r < n && k + 1 + c < n) ? B.A(r, k + 1 + c) : T(0.0);
  }
  return sing;
}

// The same serial factorisation working on the band storage in place (any
// kl); used for the 5-block Jacobian of a direct solve on the coarsest level.
template <typename T>
__device__ bool band_lu_serial_smem(const Band<T> &B) {
  const int n = B.n, kl = B.kl;
  bool sing = false;
  for (int k = 0; k < n; ++k) {
    const int imax = min(n - 1, k + kl), cmax = min(n - 1, k + 2 * kl);
    int p = k;
    for (int i = k + 1; i <= imax; ++i)
      if (fabs(B.A(i, k)) > fabs(B.A(p, k))) p = i;
    B.piv[k] = p;
    if (p != k)
      for (int c = k; c <= cmax; ++c) {
        T t = B.A(k, c);
        B.A(k, c) = B.A(p, c);
        B.A(p, c) = t;
      }
    const T d = B.A(k, k);
    if (d == T(0.0)) sing = true;
    B.rinv[k] = T(1.0) / d;
    for (int i = k + 1; i <= imax; ++i) {
      const T l = B.A(i, k) / d;
      B.A(i, k) = l;
      for (int c = k + 1; c <= cmax; ++c) B.A(i, c) -= l * B.A(k, c);
    }
  }
  return sing;
}

// x (B.x, length n) := A^{-1} x with the stored factors (one thread).
template <int KL, typename T>
__device__ void band_lu_solve_serial(const Band<T> &B) {
  constexpr int W = 2 * KL + 1;
  const int n = B.n;
  T X[KL + 1];
#pragma unroll
  for (int i = 0; i <= KL; ++i) X[i] = i < n ? B.x[i] : T(0.0);
  for (int k = 0; k < n; ++k) {
    const int p = B.piv[k] - k;
#pragma unroll
    for (int i = 1; i <= KL; ++i)
      if (p == i) {
        T t = X[0];
        X[0] = X[i];
        X[i] = t;
      }
#pragma unroll
    for (int i = 1; i <= KL; ++i)
      if (k + i < n) X[i] -= B.A(k + i, k) * X[0];
    B.x[k] = X[0];
#pragma unroll
    for (int i = 0; i < KL; ++i) X[i] = X[i + 1];
    X[KL] = (k + KL + 1 < n) ? B.x[k + KL + 1] : T(0.0);
  }
  T Y[W - 1];  // Y[c] = x[i + 1 + c]
#pragma unroll
  for (int c = 0; c < W - 1; ++c) Y[c] = T(0.0);
  for (int i = n - 1; i >= 0; --i) {
    T s = B.x[i];
#pragma unroll
    for (int c = W - 2; c >= 1; --c)
      if (i + 1 + c < n) s -= B.A(i, i + 1 + c) * Y[c];
    if (i + 1 < n) s -= B.A(i, i + 1) * Y[0];
    const T xi = s * B.rinv[i];
    B.x[i] = xi;
#pragma unroll
    for (int c = W - 2; c >= 1; --c) Y[c] = Y[c - 1];
    Y[0] = xi;
  }
}

// Assemble the band matrix from J (all threads), then factor (warp 0 in
// FP64, thread 0 in FP32). Returns true if a pivot was exactly zero (all
// threads).
__shared__ int s_sing;

template <typename T>
__device__ bool band_factor(Band<T> &B, int N, int nb, const T *J) {
  const int hw = (nb - 1) / 2;
  B.n = 2 * N;
  B.kl = 2 * hw + 1;
  B.ldab = 3 * B.kl + 1;
  const int n = B.n;
  for (int t = threadIdx.x; t < B.ldab * n; t += blockDim.x) B.ab[t] = T(0.0);
  __syncthreads();
  for (int t = threadIdx.x; t < N * nb * 4; t += blockDim.x) {
    int j = t % N, ke = t / N, k = ke / 4, e = ke % 4, l = e / 2, m = e % 2;
    int i = j + k - hw;
    if (i < 0 || i >= N) continue;
    B.A(2 * j + l, 2 * i + m) = J[(k * 4 + e) * N + j];
  }
  __syncthreads();
  if constexpr (std::is_same<T, double>::value) {
    if (threadIdx.x < 32) {
      const bool sing = band_lu_warp<T>(B);
      if (threadIdx.x == 0) s_sing = sing ? 1 : 0;
    }
  } else {
    if (threadIdx.x == 0) s_sing = (B.kl == 3 ? band_lu_serial<3, T>(B) : band_lu_serial_smem<T>(B)) ? 1 : 0;
  }
  __syncthreads();
  return s_sing != 0;
}

// dU = -J^{-1} R with the stored factors (warp 0 solves in FP64, thread 0 in
// FP32; all threads call).
template <typename T>
__device__ void band_solve(const Band<T> &B, int N, const T *R, T *dU) {
  for (int t = threadIdx.x; t < N; t += blockDim.x) {
    B.x[2 * t] = -R[t];
    B.x[2 * t + 1] = -R[N + t];
  }
  __syncthreads();
  if constexpr (std::is_same<T, double>::value) {
    if (threadIdx.x < 32) band_lu_solve_warp<T>(B);
  } else if (threadIdx.x == 0) {
    if (B.kl == 3) band_lu_solve_serial<3, T>(B);
    else band_lu_solve_serial<5, T>(B);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < N; t += blockDim.x) {
    dU[t] = B.x[2 * t];
    dU[N + t] = B.x[2 * t + 1];
  }
  __syncthreads();
}

// ----------------------------------------------------------------------------
// Multigrid hierarchy view: level l0 (the system being solved) uses the
// caller's J/R/dU, levels l0+1..L the problem's workspace.
// In the FP32 instantiation the workspace arrays (sized for FP64) hold FP32
// values.
template <typename T>
struct MG {
  int l0, L;
  int N[NSWE_MAX_LEVELS], nb[NSWE_MAX_LEVELS];
  T *J[NSWE_MAX_LEVELS], *Dinv[NSWE_MAX_LEVELS], *R[NSWE_MAX_LEVELS], *dU[NSWE_MAX_LEVELS];
};

template <typename T>
__device__ void mg_bind(MG<T> &mg, const ProbDev &P, int l0, int nb0, const T *J, const T *R, T *dU) {
  mg.l0 = l0;
  mg.L = P.levels - 1;
  for (int l = l0; l <= mg.L; ++l) {
    mg.N[l] = P.lev[l].N;
    mg.nb[l] = (l == l0) ? nb0 : 3;
    mg.J[l] = (l == l0) ? const_cast<T *>(J) : reinterpret_cast<T *>(P.lev[l].J);
    mg.R[l] = (l == l0) ? const_cast<T *>(R) : reinterpret_cast<T *>(P.lev[l].R);
    mg.dU[l] = (l == l0) ? dU : reinterpret_cast<T *>(P.lev[l].dU);
    mg.Dinv[l] = reinterpret_cast<T *>(P.lev[l].Dinv);
  }
}

// First multigrid level run by the leader CTA alone: a cluster team runs
// the levels with at least team_cells cells (from l0 down) on all its CTAs
// and the coarser ones, with the coarsest solve, on the leader; a block team
// runs every level (the coarsest solve is level L).
template <typename T, class TM>
__device__ __forceinline__ int team_split(const MG<T> &mg, int team_cells) {
  if constexpr (!TM::kMulti) return mg.L;
  int lt = mg.l0;
  while (lt < mg.L && mg.N[lt] >= team_cells) ++lt;
  return lt;
}

// Coarse operators, diagonal inverses and the coarsest factorisation; done
// once per Newton step since J is fixed during its V-cycles. Returns whether
// a pivot was exactly zero, in every thread of the team.
template <typename T, class TM = BlockTeam>
__device__ bool mg_setup(const MG<T> &mg, Band<T> &B, const TM &team = TM(), int team_cells = 0) {
  const int lt = team_split<T, TM>(mg, team_cells);
  for (int l = mg.l0 + 1; l < lt; ++l) {
    coarse_op_cells(mg.N[l - 1], mg.nb[l - 1], mg.J[l - 1], mg.N[l], mg.J[l], team.tid(), team.size());
    team.sync();
  }
  if (team.lead())
    for (int l = max(mg.l0 + 1, lt); l <= mg.L; ++l) {
      coarse_op_cells(mg.N[l - 1], mg.nb[l - 1], mg.J[l - 1], mg.N[l], mg.J[l], threadIdx.x, blockDim.x);
      __syncthreads();
    }
  for (int l = mg.l0; l < lt; ++l) dinv_cells(mg.N[l], mg.nb[l], mg.J[l], mg.Dinv[l], team.tid(), team.size());
  bool sing = false;
  if (team.lead()) {
    for (int l = lt; l < mg.L; ++l) dinv_cells(mg.N[l], mg.nb[l], mg.J[l], mg.Dinv[l], threadIdx.x, blockDim.x);
    sing = band_factor(B, mg.N[mg.L], mg.nb[mg.L], mg.J[mg.L]);
  }
  if constexpr (TM::kMulti) {
    team.sync();  // the team's inverses and the leader's factors and flag are done
    sing = team.lead_value(&s_sing) != 0;
  }
  return sing;
}

// `steps` symmetric multicolour SOR steps (colours 0..C-1 then C-1..0 each);
// consecutive visits of one colour run as one pass.
template <typename T, class TM = BlockTeam>
__device__ void sor_smooth(const MG<T> &mg, int l, int steps, double omega, const TM &team = TM()) {
  const int nb = mg.nb[l], C = (nb - 1) / 2 + 1;
  int prev = -1, reps = 0;
  for (int s = 0; s < steps; ++s)
    for (int pass = 0; pass < 2 * C; ++pass) {
      const int col = pass < C ? pass : 2 * C - 1 - pass;
      if (col == prev) {
        ++reps;
        continue;
      }
      if (prev >= 0) {
        sor_colour(mg.N[l], nb, mg.J[l], mg.Dinv[l], mg.R[l], mg.dU[l], omega, C, prev, reps, team.tid(),
                   team.size());
        team.sync();
      }
      prev = col;
      reps = 1;
    }
  if (prev >= 0) {
    sor_colour(mg.N[l], nb, mg.J[l], mg.Dinv[l], mg.R[l], mg.dU[l], omega, C, prev, reps, team.tid(), team.size());
    team.sync();
  }
}

// Algorithm 2 from level l0, unrolled over levels. A cluster team smooths,
// restricts and prolongs the levels l0..lt-1; the leader CTA runs the
// V-cycle below them (levels lt..L) between two cluster barriers.
template <typename T, class TM = BlockTeam>
__device__ void mg_vcycle(const MG<T> &mg, const Band<T> &B, const nswe_params &prm, const TM &team = TM(),
                          int team_cells = 0) {
  const int lt = team_split<T, TM>(mg, team_cells);
  for (int l = mg.l0; l < lt; ++l) {
    sor_smooth(mg, l, prm.nu1, prm.omega, team);
    restrict_cells(mg.N[l], mg.nb[l], mg.J[l], mg.R[l], mg.dU[l], mg.N[l + 1], mg.R[l + 1], mg.dU[l + 1],
                   team.tid(), team.size());
    team.sync();
  }
  if (team.lead()) {
    for (int l = lt; l < mg.L; ++l) {
      sor_smooth(mg, l, prm.nu1, prm.omega);
      restrict_cells(mg.N[l], mg.nb[l], mg.J[l], mg.R[l], mg.dU[l], mg.N[l + 1], mg.R[l + 1], mg.dU[l + 1],
                     threadIdx.x, blockDim.x);
      __syncthreads();
    }
    band_solve(B, mg.N[mg.L], mg.R[mg.L], mg.dU[mg.L]);
    for (int l = mg.L - 1; l >= lt; --l) {
      prolong_cells(mg.N[l], mg.dU[l], mg.N[l + 1], mg.dU[l + 1], threadIdx.x, blockDim.x);
      __syncthreads();
      sor_smooth(mg, l, prm.nu2, prm.omega);
    }
  }
  if constexpr (TM::kMulti) team.sync();
  for (int l = lt - 1; l >= mg.l0; --l) {
    prolong_cells(mg.N[l], mg.dU[l], mg.N[l + 1], mg.dU[l + 1], team.tid(), team.size());
    team.sync();
    sor_smooth(mg, l, prm.nu2, prm.omega, team);
  }
}

// Band storage in dynamic shared memory, sized by the host for the coarsest
// level: ab [ldab_cap * n_cap], x [n_cap], rinv [n_cap], piv [n_cap].
extern __shared__ double g_dyn_smem[];

template <typename T>
__device__ __forceinline__ Band<T> band_view(int n_cap, int ldab_cap) {
  Band<T> B;
  B.ab = reinterpret_cast<T *>(g_dyn_smem);
  B.x = B.ab + (size_t)ldab_cap * n_cap;
  B.rinv = B.x + n_cap;
  B.piv = reinterpret_cast<int *>(B.rinv + n_cap);
  B.n = B.kl = B.ldab = 0;
  return B;
}

// ----------------------------------------------------------------------------
// Kernels.

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// NSWE_RESIDUAL_SMEM (default 1): the standalone residual stages its WENO
// windows in shared memory (residual_cells_staged); 0 reads them through L1.
#ifndef NSWE_RESIDUAL_SMEM
#define NSWE_RESIDUAL_SMEM 1
#endif

__global__ void __launch_bounds__(kThreads) k_residual(const ProbDev *P, int level, const double *U, double *R,
                                                       double *partials) {
  __shared__ double red[33];
  Geo G = make_geo(*P, level);
#if NSWE_RESIDUAL_SMEM
  __shared__ double sH[kThreads + 4], sQ[kThreads + 4];
  double acc = residual_cells_staged(G, U, R, blockIdx.x, gridDim.x, sH, sQ);
#else
  double acc = residual_cells(G, U, R, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
#endif
  double s = block_sum(acc, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) k_finish_res(const double *partials, int n, int N, double *res) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += partials[i];
    *res = s / N;
  }
}

__global__ void __launch_bounds__(kThreads) k_geom_derive(const ProbDev *P) {
  geom_derive_items(*P, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

// The derived geometry of many problems in one launch: block b derives
// tasks[b].prob.
__global__ void __launch_bounds__(kThreads) k_geom_derive_batch(const SolveTask *tasks) {
  geom_derive_items(*tasks[blockIdx.x].prob, threadIdx.x, blockDim.x);
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_jac_a(const ProbDev *P, int level, const double *U, double eps) {
  Geo G = make_geo(*P, level);
  jac_pass_a<T>(G, U, eps, jw_view<T>(P->jw, G.N), blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_jac_b(const ProbDev *P, int level) {
  Geo G = make_geo(*P, level);
  jac_pass_b<T, -1>(G, jw_view<T>(P->jw, G.N), blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_jac_c(const ProbDev *P, int level, int nb, double eps, double alpha,
                                                    const double *Rreg, double *R, T *J, double *partials) {
  __shared__ double red[33];
  Geo G = make_geo(*P, level);
  double acc = jac_pass_c<T>(G, nb, eps, alpha, jw_view<T>(P->jw, G.N), Rreg, R, J,
                             blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
  double s = block_sum(acc, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_vcycle(const ProbDev *P, int level, int nb, const T *J, const T *R,
                                                     T *dU, nswe_params prm, int *status, int n_cap, int ldab_cap) {
  MG<T> mg;
  mg_bind<T>(mg, *P, level, nb, J, R, dU);
  Band<T> B = band_view<T>(n_cap, ldab_cap);
  bool sing = mg_setup<T>(mg, B);
  __syncthreads();
  mg_vcycle<T>(mg, B, prm);
  if (threadIdx.x == 0) *status = sing ? NSWE_ESINGULAR : NSWE_OK;
}

// The team of the calling thread and the index of its problem: a block per
// problem, or a cluster per problem (clusters tile the grid along x).
template <class TM>
__device__ __forceinline__ TM make_team(int &task_index);
template <>
__device__ __forceinline__ BlockTeam make_team<BlockTeam>(int &task_index) {
  task_index = blockIdx.x;
  return BlockTeam{};
}
template <>
__device__ __forceinline__ ClusterTeam make_team<ClusterTeam>(int &task_index) {
  const auto cl = cooperative_groups::this_cluster();
  ClusterTeam t{(int)cl.block_rank(), (int)cl.num_blocks()};
  task_index = blockIdx.x / t.n;
  return t;
}

// Algorithm 3 for one problem per team (a thread block, or a cluster of
// blocks: TM). T is the precision of the Jacobian and the multigrid solve of
// each Newton step: with T = double the whole step is FP64; with T = float
// the residual, the convergence test and the update U += tau dU stay FP64
// while the FD Jacobian (Eq. 12-13), the coarse operators, the smoother and
// the coarsest LU run in FP32. FLUX: the numerical flux of every task of the
// launch (compile-time, so that the HLL kernels carry no LLF code).
// team_cells: a cluster team runs the multigrid levels with at least that
// many cells on all its CTAs, the others on the leader CTA.
template <typename T, int THREADS, int MINB, int FLUX, class TM = BlockTeam>
__global__ void __launch_bounds__(THREADS, MINB)
    k_solve(const SolveTask *tasks, nswe_params launch_prm, int n_cap, int ldab_cap, int team_cells) {
  constexpr bool kMixed = std::is_same<T, float>::value;
  __shared__ double red[34];
  __shared__ nswe_params s_prm;
  const unsigned long long t_start = global_ns();
  int ti;
  const TM team = make_team<TM>(ti);
  const SolveTask task = tasks[ti];
  const ProbDev &P = *task.prob;
  if (threadIdx.x == 0) s_prm = task.prm ? *task.prm : launch_prm;
  if (task.derive) geom_derive_items(P, team.tid(), team.size());
  team.sync();  // (a cluster team: also every CTA has started before any shared-memory access across CTAs)
  const nswe_params &prm = s_prm;
  const int L = P.levels - 1;
  const int s0 = (prm.nest_start < 0 || prm.nest_start > L) ? L : prm.nest_start;
  const int nb = prm.jacobian == NSWE_JAC_FULL ? 5 : 3;
  Band<T> B = band_view<T>(n_cap, ldab_cap);

  int iters[NSWE_MAX_LEVELS], lstat[NSWE_MAX_LEVELS];
  double lres[NSWE_MAX_LEVELS];
  for (int l = 0; l < NSWE_MAX_LEVELS; ++l) {
    iters[l] = 0;
    lstat[l] = NSWE_OK;
    lres[l] = 0.0;
  }
  int vcycles = 0, total = 0, fatal = 0;

  {
    const int Ns = P.lev[s0].N;
    for (int t = team.tid(); t < 2 * Ns; t += team.size()) P.lev[s0].U[t] = task.U0[t];
    team.sync();
  }

  for (int l = s0; l >= 0 && !fatal; --l) {
    const LevelDev &Lv = P.lev[l];
    Geo G = make_geo(P, l);
    const int N = G.N;
    if (l < s0) {
      interp_cells(make_geo(P, l + 1), P.lev[l + 1].U, Lv.U, team.tid(), team.size());
      team.sync();
    }
    // Mixed path: the FP32 Jacobian reads FP32 copies of the state (kept up
    // to date by the update) and of the level's geometry.
    float *U32 = nullptr;
    if constexpr (kMixed) {
      U32 = attach_f32(G, P.jw);
      fill_f32(G, Lv.U, U32, team.tid(), team.size());
      team.sync();
    }
    const JW<T> W = jw_view<T>(P.jw, N);
    T *const J = reinterpret_cast<T *>(Lv.J);
    T *const dU = reinterpret_cast<T *>(Lv.dU);
    // Right-hand side of the linear solve: the FP64 residual itself, or its
    // FP32 copy in the unused upper part of J's storage (J takes 4 nb N of
    // the 40 N floats there).
    T *const Rs = kMixed ? J + (size_t)4 * nb * N : reinterpret_cast<T *>(Lv.R);
    // FP64 path: R, J and res at the current state in one pass (Eq. 10,
    // 12-13). Mixed path: only the FP64 residual and res here.
    auto residual_step = [&]() -> double {
      double acc;
      if constexpr (kMixed) {
        const RW RWv = rw_view(P.jw, N);
        res_pass_a(G, Lv.U, RWv, team.tid(), team.size());
        team.sync();
        res_pass_b<FLUX>(G, RWv, team.tid(), team.size());
        team.sync();
        acc = res_pass_c(G, RWv, Lv.R, team.tid(), team.size());
      } else {
        jac_pass_a<T>(G, Lv.U, prm.eps[l], W, team.tid(), team.size());
        team.sync();
        jac_pass_b<T, FLUX>(G, W, team.tid(), team.size());
        team.sync();
        acc = jac_pass_c<T>(G, nb, prm.eps[l], prm.alpha, W, nullptr, Lv.R, J, team.tid(), team.size());
      }
      return team.sum(acc, red) / N;
    };
    double res = residual_step();
    int n = 0, st = NSWE_OK;
    while (true) {
      if constexpr (kMixed) {
        // FP32 Jacobian at the current state, regularised with the FP64 R.
        jac_pass_a<T>(G, Lv.U, prm.eps[l], W, team.tid(), team.size());
        team.sync();
        jac_pass_b<T, FLUX>(G, W, team.tid(), team.size());
        team.sync();
        jac_pass_c<T>(G, nb, prm.eps[l], prm.alpha, W, Lv.R, nullptr, J, team.tid(), team.size());
        for (int t = team.tid(); t < 2 * N; t += team.size()) Rs[t] = T(Lv.R[t]);
        team.sync();
      }
      MG<T> mg;
      mg_bind<T>(mg, P, l, nb, J, Rs, dU);
      bool sing = mg_setup<T, TM>(mg, B, team, team_cells);
      team.sync();
      if (sing) {
        st = NSWE_ESINGULAR;
        break;
      }
      if (l == L) {
        if (team.lead()) band_solve<T>(B, N, Rs, dU);
        if constexpr (TM::kMulti) team.sync();
      } else {
        for (int t = team.tid(); t < 2 * N; t += team.size()) dU[t] = T(0.0);
        team.sync();
        for (int m = 0; m < prm.nu3; ++m) {
          mg_vcycle<T, TM>(mg, B, prm, team, team_cells);
          ++vcycles;
        }
      }
      bool bad = false;
      for (int j = team.tid(); j < N; j += team.size()) {
        double h = Lv.U[j] + prm.tau * double(dU[j]);
        Lv.U[j] = h;
        Lv.U[N + j] += prm.tau * double(dU[N + j]);
        if constexpr (kMixed) {
          U32[j] = float(h);
          U32[N + j] = float(Lv.U[N + j]);
        }
        if (!(h > 0.0)) bad = true;
      }
      bad = team.any(bad);
      ++n;
      if (bad) {
        st = NSWE_ENEGDEPTH;
        break;
      }
      // res of the new state (on the FP64 path its Jacobian serves the next
      // step and is not needed once res < tol).
      res = residual_step();
      if (!(res == res) || isinf(res)) {
        st = NSWE_ENAN;
        break;
      }
      if (res < prm.tol) break;
      if (n >= prm.n_max) {
        st = NSWE_ENOTCONV;
        break;
      }
    }
    iters[l] = n;
    lres[l] = res;
    lstat[l] = st;
    total += n;
    if (st == NSWE_ENAN || st == NSWE_ENEGDEPTH || st == NSWE_ESINGULAR) fatal = st;
  }

  if (!fatal) {
    const int N0 = P.lev[0].N;
    for (int t = team.tid(); t < 2 * N0; t += team.size()) task.U[t] = P.lev[0].U[t];
  }
  if (threadIdx.x == 0 && team.lead() && task.info) {
    nswe_info inf;
    for (int l = 0; l < NSWE_MAX_LEVELS; ++l) {
      inf.iters[l] = iters[l];
      inf.res[l] = lres[l];
      inf.level_status[l] = lstat[l];
    }
    inf.status = fatal ? fatal : lstat[0];
    inf.total_iters = total;
    inf.vcycles = vcycles;
    inf.t_start_ns = t_start;
    inf.t_end_ns = global_ns();
    *task.info = inf;
  }
  if (task.done) {
    // Every thread's result writes are visible system-wide before the flag.
    __threadfence_system();
    team.sync();
    if (threadIdx.x == 0 && team.lead()) *reinterpret_cast<volatile int *>(task.done) = 1;
  }
  if constexpr (TM::kMulti) team.sync();  // no CTA leaves while another may read its shared memory
}

int grid_for(int items) {
  int b = (items + kThreads - 1) / kThreads;
  return b < 1 ? 1 : (b > 1024 ? 1024 : b);
}

}  // namespace

cudaError_t launch_geom_derive(const ProbDev *p, int finest_cells, cudaStream_t s) {
  k_geom_derive<<<grid_for(2 * finest_cells + 1), kThreads, 0, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_geom_derive_batch(const SolveTask *tasks, int count, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  k_geom_derive_batch<<<count, kThreads, 0, s>>>(tasks);
  return cudaGetLastError();
}

cudaError_t launch_residual(const ProbDev *p, int level, int N, const double *U, double *R, double *res,
                            double *partials, cudaStream_t s) {
  int grid = grid_for(N);
  k_residual<<<grid, kThreads, 0, s>>>(p, level, U, R, partials);
  if (res) k_finish_res<<<1, 32, 0, s>>>(partials, grid, N, res);
  return cudaGetLastError();
}

cudaError_t launch_jacobian(const ProbDev *p, int level, int N, int nb, const double *U, double eps,
                            double alpha, double *R, double *J, double *res, double *partials, cudaStream_t s) {
  k_jac_a<double><<<grid_for((N + 2) * 8), kThreads, 0, s>>>(p, level, U, eps);
  k_jac_b<double><<<grid_for(N + 1), kThreads, 0, s>>>(p, level);
  const int grid = grid_for(N * nb);
  k_jac_c<double><<<grid, kThreads, 0, s>>>(p, level, nb, eps, alpha, nullptr, R, J, partials);
  if (res) k_finish_res<<<1, 32, 0, s>>>(partials, grid, N, res);
  return cudaGetLastError();
}

cudaError_t launch_jacobian_f32(const ProbDev *p, int level, int N, int nb, const double *U, double eps,
                                double alpha, double *R, float *J, double *res, double *partials, cudaStream_t s) {
  // The residual's reduction has consumed `partials` (stream order) before
  // the FP32 pass C reuses it (it writes zeros there).
  cudaError_t e = launch_residual(p, level, N, U, R, res, partials, s);
  if (e != cudaSuccess) return e;
  k_jac_a<float><<<grid_for((N + 2) * 8), kThreads, 0, s>>>(p, level, U, eps);
  k_jac_b<float><<<grid_for(N + 1), kThreads, 0, s>>>(p, level);
  k_jac_c<float><<<grid_for(N * nb), kThreads, 0, s>>>(p, level, nb, eps, alpha, R, nullptr, J, partials);
  return cudaGetLastError();
}

size_t band_smem_bytes(int n_cap, int ldab_cap) {
  return sizeof(double) * ((size_t)ldab_cap * n_cap + 2 * (size_t)n_cap) + sizeof(int) * (size_t)n_cap;
}

cudaError_t launch_vcycle(const ProbDev *p, int level, int nb, const double *J, const double *R, double *dU,
                          const nswe_params &prm, int *status, int coarse_cells, int coarse_nb, cudaStream_t s) {
  const int n_cap = 2 * coarse_cells, ldab_cap = 3 * (coarse_nb == 5 ? 5 : 3) + 1;
  k_vcycle<double><<<1, kThreads, band_smem_bytes(n_cap, ldab_cap), s>>>(p, level, nb, J, R, dU, prm, status,
                                                                        n_cap, ldab_cap);
  return cudaGetLastError();
}

cudaError_t launch_vcycle_f32(const ProbDev *p, int level, int nb, const float *J, const float *R, float *dU,
                              const nswe_params &prm, int *status, int coarse_cells, int coarse_nb, cudaStream_t s) {
  const int n_cap = 2 * coarse_cells, ldab_cap = 3 * (coarse_nb == 5 ? 5 : 3) + 1;
  k_vcycle<float><<<1, kThreads, band_smem_bytes(n_cap, ldab_cap), s>>>(p, level, nb, J, R, dU, prm, status,
                                                                       n_cap, ldab_cap);
  return cudaGetLastError();
}

cudaError_t launch_solve(const SolveTask *tasks, int count, const nswe_params &prm, int max_coarse_cells,
                         cudaStream_t s) {
  return launch_solve_sized(tasks, count, prm, max_coarse_cells, prm.jacobian == NSWE_JAC_FULL ? 5 : 3, 0, s);
}

namespace {
template <int SHAPE, int FLUX = NSWE_FLUX_HLL>
void launch_shape(const SolveTask *tasks, int count, const nswe_params &prm, int n_cap, int ldab_cap, size_t smem,
                  cudaStream_t s) {
  constexpr int TH = kSolveShapeThreads[SHAPE], MB = kSolveShapeBlocks[SHAPE];
  if (prm.precision == NSWE_PREC_MIXED)
    k_solve<float, TH, MB, FLUX><<<count, TH, smem, s>>>(tasks, prm, n_cap, ldab_cap, 0);
  else
    k_solve<double, TH, MB, FLUX><<<count, TH, smem, s>>>(tasks, prm, n_cap, ldab_cap, 0);
}
}  // namespace

namespace {
template <typename T>
cudaError_t launch_cluster_t(const SolveTask *tasks, int count, const nswe_params &prm, int n_cap, int ldab_cap,
                             size_t smem, int ctas, int team_cells, cudaStream_t s) {
  auto kern = k_solve<T, kClusterThreads, 1, NSWE_FLUX_HLL, ClusterTeam>;
  if (ctas > 8) {
    const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)count * (unsigned)ctas, 1, 1);
  cfg.blockDim = dim3(kClusterThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)ctas;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, tasks, prm, n_cap, ldab_cap, team_cells);
}
}  // namespace

cudaError_t launch_solve_cluster(const SolveTask *tasks, int count, const nswe_params &prm, int max_coarse_cells,
                                 int max_nb, int ctas, int team_cells, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  const int n_cap = 2 * max_coarse_cells, ldab_cap = 3 * (max_nb == 5 ? 5 : 3) + 1;
  const size_t smem = band_smem_bytes(n_cap, ldab_cap);
  if (prm.precision == NSWE_PREC_MIXED)
    return launch_cluster_t<float>(tasks, count, prm, n_cap, ldab_cap, smem, ctas, team_cells, s);
  return launch_cluster_t<double>(tasks, count, prm, n_cap, ldab_cap, smem, ctas, team_cells, s);
}

cudaError_t launch_solve_sized(const SolveTask *tasks, int count, const nswe_params &prm, int max_coarse_cells,
                               int max_nb, int shape, cudaStream_t s, int flux) {
  const int n_cap = 2 * max_coarse_cells, ldab_cap = 3 * (max_nb == 5 ? 5 : 3) + 1;
  const size_t smem = band_smem_bytes(n_cap, ldab_cap);
  if (flux == NSWE_FLUX_LLF) {  // a comparison option: the default shape only
    launch_shape<0, NSWE_FLUX_LLF>(tasks, count, prm, n_cap, ldab_cap, smem, s);
    return cudaGetLastError();
  }
  switch (shape) {
  case 1: launch_shape<1>(tasks, count, prm, n_cap, ldab_cap, smem, s); break;
  case 2: launch_shape<2>(tasks, count, prm, n_cap, ldab_cap, smem, s); break;
  case 3: launch_shape<3>(tasks, count, prm, n_cap, ldab_cap, smem, s); break;
  case 4: launch_shape<4>(tasks, count, prm, n_cap, ldab_cap, smem, s); break;
  case 5: launch_shape<5>(tasks, count, prm, n_cap, ldab_cap, smem, s); break;
  default: launch_shape<0>(tasks, count, prm, n_cap, ldab_cap, smem, s); break;
  }
  return cudaGetLastError();
}

}  // namespace nswe
