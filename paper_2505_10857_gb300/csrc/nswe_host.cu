// Host side of the C ABI declared in include/nswe.h: contexts, problems
// (device arena with geometry and solver workspace), argument checking and
// kernel launches. No compute happens here.
#include <cmath>
#include <cstring>
#include <new>
#include <algorithm>
#include <atomic>
#include <chrono>
#include <thread>
#include <type_traits>
#include <vector>

#include "nswe_internal.h"

using namespace nswe;

namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess || prev != dev) cudaSetDevice(dev);
    else prev = -1;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

size_t round_up(size_t n) { return (n + 31) & ~size_t(31); }  // 256-byte slots

bool valid_bc(const nswe_bc1d *b) {
  return b && b->kind >= NSWE_BC_DISCHARGE && b->kind <= NSWE_BC_EXTRAP && std::isfinite(b->h) &&
         std::isfinite(b->q);
}

nswe_status check_params(const nswe_params *p, const nswe_prob_s *pr, int first_level) {
  if (!p) return NSWE_EINVAL;
  if (!(p->tau > 0.0 && p->tau <= 1.0) || !(p->alpha >= 0.0) || !(p->omega > 0.0 && p->omega < 2.0) ||
      !(p->tol > 0.0))
    return NSWE_EINVAL;
  if (p->nu1 < 0 || p->nu2 < 0 || p->nu3 < 1 || p->n_max < 1 || p->nu1 > 1000 || p->nu2 > 1000 ||
      p->nu3 > 1000)
    return NSWE_EINVAL;
  const int jb = p->jacobian & ~NSWE_JAC_FROZEN;
  if (jb != NSWE_JAC_SIMPLIFIED && jb != NSWE_JAC_FULL) return NSWE_EINVAL;
  if ((p->jacobian & NSWE_JAC_FROZEN) && pr && pr->dim != 2) return NSWE_EINVAL;  // 2D only
  if (p->precision != NSWE_PREC_FP64 && p->precision != NSWE_PREC_MIXED) return NSWE_EINVAL;
  if (p->colours2d != 0 && p->colours2d != NSWE_COLOURS2D_AUTO && (p->colours2d < 3 || p->colours2d > 4096))
    return NSWE_EINVAL;
  if (pr) {
    for (int l = 0; l <= first_level && l < pr->levels; ++l)
      if (!(p->eps[l] > 0.0) || !std::isfinite(p->eps[l])) return NSWE_EINVAL;
  }
  return NSWE_OK;
}

}  // namespace

// Doubles of a 2D problem's device arena (geometry, boundary kinds, state,
// Jacobian and multigrid workspace of every level, coarsest dense LU).
size_t nswe::prob2d_arena_doubles(int Nx, int Ny, int levels) {
  size_t doubles = 0, nk = 0;
  for (int l = 0; l < levels; ++l) {
    const size_t n = (size_t)(Nx >> l) * (Ny >> l);
    // Dinv: room for the colour-major stride (blk_stride <= n + 2 Ny)
    doubles += round_up(8 * n) + 3 * round_up(3 * n) + round_up(189 * n) + round_up(9 * n + 27 * (size_t)(Ny >> l));
    nk += 2 * (size_t)((Nx >> l) + (Ny >> l));
  }
  const size_t N3 = 3 * (size_t)(Nx >> (levels - 1)) * (Ny >> (levels - 1));
  return doubles + round_up(N3 * N3) + round_up(N3) + 2 * round_up(nk);
}

// All device bytes nswe_prob_create_2d requests for such a problem.
size_t nswe::prob2d_device_bytes(int Nx, int Ny, int levels) {
  const size_t N3 = 3 * (size_t)(Nx >> (levels - 1)) * (Ny >> (levels - 1));
  return sizeof(double) * prob2d_arena_doubles(Nx, Ny, levels) + sizeof(ProbDev2) + sizeof(int) * (N3 + 64) +
         sizeof(int) * 4 + sizeof(double) * 4 + sizeof(double) * 1024;
}

nswe_status nswe::check_params_2d(const nswe_params *p, int levels, int first_level) {
  nswe_status st = check_params(p, nullptr, 0);
  if (st != NSWE_OK) return st;
  for (int l = 0; l <= first_level && l < levels; ++l)
    if (!(p->eps[l] > 0.0) || !std::isfinite(p->eps[l])) return NSWE_EINVAL;
  return NSWE_OK;
}

nswe_status nswe::check_params_1d(const nswe_params *p, int levels, int first_level) {
  nswe_status st = check_params(p, nullptr, 0);
  if (st != NSWE_OK) return st;
  if (p->jacobian & NSWE_JAC_FROZEN) return NSWE_EINVAL;  // 2D only
  for (int l = 0; l <= first_level && l < levels; ++l)
    if (!(p->eps[l] > 0.0) || !std::isfinite(p->eps[l])) return NSWE_EINVAL;
  return NSWE_OK;
}

namespace {

nswe_status ensure_cap(nswe_ctx ctx, int count) {
  if (count <= ctx->cap) return NSWE_OK;
  int cap = count < 64 ? 64 : count;
  SolveTask *t = nullptr;
  nswe_info *i = nullptr;
  nswe_params *q = nullptr;
  if (cudaMalloc(&t, sizeof(SolveTask) * cap) != cudaSuccess) return NSWE_ENOMEM;
  if (cudaMalloc(&i, sizeof(nswe_info) * cap) != cudaSuccess || cudaMalloc(&q, sizeof(nswe_params) * cap) != cudaSuccess) {
    cudaFree(t);
    cudaFree(i);
    return NSWE_ENOMEM;
  }
  // Buffers may still be read by queued work on the context stream.
  cudaStreamSynchronize(ctx->stream);
  cudaFree(ctx->tasks);
  cudaFree(ctx->infos);
  cudaFree(ctx->prms);
  ctx->tasks = t;
  ctx->infos = i;
  ctx->prms = q;
  ctx->cap = cap;
  return NSWE_OK;
}

// Geometry upload of a 1D problem in two phases. Pack: the per-level face
// widths and Gauss-point geometry into the problem's pinned staging buffer
// (after the previous upload from it has been copied), with the finiteness
// check; host work only. Issue: the asynchronous copies of the staged
// geometry and of the problem record, and the derived-geometry kernel, on
// the context stream.
nswe_status pack_geometry(nswe_prob p, const double *sigma_face, const double *gauss_geom) {
  if (!p->stage) {
    if (cudaMallocHost(&p->stage, sizeof(double) * p->geo_doubles) != cudaSuccess) return NSWE_ENOMEM;
    if (cudaEventCreateWithFlags(&p->staged, cudaEventDisableTiming) != cudaSuccess) return NSWE_ECUDA;
  } else if (cudaEventSynchronize(p->staged) != cudaSuccess) {
    return NSWE_ECUDA;
  }
  double *geo = p->stage;
  size_t off = 0;
  for (int l = 0; l < p->levels; ++l) {
    const int Nl = p->N >> l;
    for (int f = 0; f <= Nl; ++f) geo[off + f] = sigma_face[(size_t)f << l];
    for (size_t f = Nl + 1; f < round_up(Nl + 1); ++f) geo[off + f] = 0.0;
    off += round_up(Nl + 1);
  }
  size_t src = 0;
  for (int l = 0; l < p->levels; ++l) {
    const int Nl = p->N >> l;
    std::memcpy(&geo[off], gauss_geom + src, sizeof(double) * 6 * Nl);
    for (size_t f = 6 * (size_t)Nl; f < round_up(6 * (size_t)Nl); ++f) geo[off + f] = 0.0;
    src += 6 * (size_t)Nl;
    off += round_up(6 * (size_t)Nl);
  }
  for (size_t i = 0; i < off; ++i)
    if (!std::isfinite(geo[i])) return NSWE_EINVAL;
  return NSWE_OK;
}

nswe_status issue_geometry(nswe_prob p, const nswe_bc1d *left, const nswe_bc1d *right, bool derive = true) {
  p->host.bl = left->kind;
  p->host.br = right->kind;
  p->host.blh = left->h;
  p->host.blq = left->q;
  p->host.brh = right->h;
  p->host.brq = right->q;
  cudaStream_t s = p->ctx->stream;
  if (cudaMemcpyAsync(p->arena, p->stage, sizeof(double) * p->geo_doubles, cudaMemcpyHostToDevice, s) !=
          cudaSuccess ||
      cudaEventRecord(p->staged, s) != cudaSuccess)
    return NSWE_ECUDA;
  if (cudaMemcpyAsync(p->dev, &p->host, sizeof(ProbDev), cudaMemcpyHostToDevice, s) != cudaSuccess)
    return NSWE_ECUDA;
  if (derive && launch_geom_derive(p->dev, p->N, s) != cudaSuccess) return NSWE_ECUDA;
  return NSWE_OK;
}

nswe_status upload_geometry(nswe_prob p, const double *sigma_face, const double *gauss_geom,
                            const nswe_bc1d *left, const nswe_bc1d *right) {
  nswe_status st = pack_geometry(p, sigma_face, gauss_geom);
  return st != NSWE_OK ? st : issue_geometry(p, left, right);
}

// ---------------------------------------------------------------- 2D host side

// Symmetric multicolour smoothing of 2D level l: one step = colours 0..C-1,
// C-1..0, twice; consecutive visits of a colour run as one pass.
// One level of a 2D multigrid hierarchy in arithmetic T: in the FP32
// instantiation (the multigrid of a mixed-precision step) the level's FP64
// workspace arrays hold FP32 values.
template <typename T>
struct Lev2 {
  int Nx, Ny;
  T *J, *Dinv, *R, *dU;
  int cm;  // storage of J and Dinv (blk_pos)
};

template <typename T>
Lev2<T> lev2_view(const Level2Dev &L) {
  return Lev2<T>{L.Nx, L.Ny, reinterpret_cast<T *>(L.J), reinterpret_cast<T *>(L.Dinv), reinterpret_cast<T *>(L.R),
                 reinterpret_cast<T *>(L.dU), 0};
}

// launches (may be NULL): incremented once per colour-pass launch.
template <typename T>
cudaError_t smooth2(const Lev2<T> &Lv, int st, int steps, double omega, int Kc, cudaStream_t s,
                    int *launches = nullptr) {
  cudaError_t e = cudaSuccess;
  if (Kc >= 3 && (st == ST_J9 || st == ST_P5)) {
    // Directional schedule (the multicolour analogue of D1-D4): diagonal
    // colourings (i + j) mod Kc ascending, (j - i + Nx - 1) mod Kc ascending,
    // then both descending.
    for (int t = 0; t < steps; ++t)
      for (int d = 0; d < 4; ++d)
        for (int q = 0; q < Kc; ++q) {
          const int mode = (d % 2) + 1, col = d < 2 ? q : Kc - 1 - q;
          if ((e = launch2_sor<T>(Lv.Nx, Lv.Ny, st, Lv.J, Lv.Dinv, Lv.R, Lv.dU, omega, mode, Kc, col, 1, Lv.cm, s)))
            return e;
          if (launches) ++*launches;
        }
    return e;
  }
  const int C = st_colours_host(st);
  int prev = -1, reps = 0;
  for (int t = 0; t < steps; ++t)
    for (int pass = 0; pass < 4 * C; ++pass) {
      const int q = pass % (2 * C), col = q < C ? q : 2 * C - 1 - q;
      if (col == prev) {
        ++reps;
        continue;
      }
      if (prev >= 0 &&
          (e = launch2_sor<T>(Lv.Nx, Lv.Ny, st, Lv.J, Lv.Dinv, Lv.R, Lv.dU, omega, 0, 0, prev, reps, Lv.cm, s)))
        return e;
      if (prev >= 0 && launches) ++*launches;
      prev = col;
      reps = 1;
    }
  if (prev >= 0) {
    e = launch2_sor<T>(Lv.Nx, Lv.Ny, st, Lv.J, Lv.Dinv, Lv.R, Lv.dU, omega, 0, 0, prev, reps, Lv.cm, s);
    if (launches) ++*launches;
  }
  return e;
}

// Multigrid hierarchy from level l0 (stencil st0) to the coarsest: the
// level-l0 arrays are J, R, dU given by the caller.
template <typename T>
struct MG2 {
  int l0, L;
  int st[NSWE_MAX_LEVELS];
  Lev2<T> lv[NSWE_MAX_LEVELS];
};

// cm0: the storage of level l0's J and Dinv (blk_pos); the coarser levels
// are cell-contiguous.
template <typename T>
MG2<T> mg2_bind(const nswe_prob_s *p, int l0, int st0, const T *J, const T *R, T *dU, int cm0) {
  MG2<T> m;
  m.l0 = l0;
  m.L = p->levels - 1;
  for (int l = l0; l <= m.L; ++l) {
    m.lv[l] = lev2_view<T>(p->host2.lev[l]);
    m.st[l] = l == l0 ? st0 : st_coarse_host(m.st[l - 1]);
  }
  m.lv[l0].J = const_cast<T *>(J);
  m.lv[l0].R = const_cast<T *>(R);
  m.lv[l0].dU = dU;
  m.lv[l0].cm = cm0;
  return m;
}

template <typename T>
cudaError_t mg2_setup(nswe_prob_s *p, const MG2<T> &m, cudaStream_t s) {
  cudaError_t e;
  for (int l = m.l0 + 1; l <= m.L; ++l)
    if ((e = launch2_coarse_op<T>(m.lv[l - 1].Nx, m.lv[l - 1].Ny, m.st[l - 1], m.lv[l - 1].J, m.lv[l].J,
                                  m.lv[l - 1].cm, s)))
      return e;
  for (int l = m.l0; l < m.L; ++l)
    if ((e = launch2_dinv<T>(m.lv[l].Nx, m.lv[l].Ny, m.st[l], m.lv[l].J, m.lv[l].Dinv, m.lv[l].cm, s))) return e;
  return launch2_dense_factor<T>(m.lv[m.L].Nx, m.lv[m.L].Ny, m.st[m.L], m.lv[m.L].J,
                                 reinterpret_cast<T *>(p->dense), p->piv, p->flag, s);
}

// Algorithm 2 from level l0: grid-wide kernels on the large levels; from the
// first level of at most `tail` cells down to the coarsest and back up, one
// block-persistent launch (the same bits either way).
template <typename T>
cudaError_t mg2_vcycle(nswe_prob_s *p, const MG2<T> &m, const nswe_params &prm, cudaStream_t s, int tail) {
  cudaError_t e;
  int ls = m.L;  // first level handled by the tail launch
  for (int l = m.l0; l < m.L; ++l) {
    if (m.lv[l].Nx * m.lv[l].Ny <= tail) {
      ls = l;
      break;
    }
    if ((e = smooth2<T>(m.lv[l], m.st[l], prm.nu1, prm.omega, prm.colours2d, s))) return e;
    if ((e = launch2_restrict<T>(m.lv[l].Nx, m.lv[l].Ny, m.st[l], m.lv[l].J, m.lv[l].R, m.lv[l].dU, m.lv[l + 1].R,
                                 m.lv[l + 1].dU, m.lv[l].cm, s)))
      return e;
  }
  Tail2<T> t;
  t.ls = ls;
  t.L = m.L;
  for (int l = ls; l <= m.L; ++l) {
    t.Nx[l] = m.lv[l].Nx;
    t.Ny[l] = m.lv[l].Ny;
    t.st[l] = m.st[l];
    t.J[l] = m.lv[l].J;
    t.Dinv[l] = m.lv[l].Dinv;
    t.R[l] = m.lv[l].R;
    t.dU[l] = m.lv[l].dU;
  }
  t.A = reinterpret_cast<const T *>(p->dense);
  t.piv = p->piv;
  t.x = reinterpret_cast<T *>(p->xbuf);
  if ((e = launch2_vcycle_tail<T>(t, prm.nu1, prm.nu2, prm.omega, prm.colours2d, s))) return e;
  for (int l = ls - 1; l >= m.l0; --l) {
    if ((e = launch2_prolong<T>(m.lv[l].Nx, m.lv[l].Ny, m.lv[l].dU, m.lv[l + 1].dU, s))) return e;
    if ((e = smooth2<T>(m.lv[l], m.st[l], prm.nu2, prm.omega, prm.colours2d, s))) return e;
  }
  return cudaSuccess;
}

// Algorithm 3 for one 2D problem, sequenced from the host (one synchronisation
// per Newton step for the convergence test).
// T = double: the FP64 path; T = float: mixed precision (FP64 residual,
// stopping test and update; the FD Jacobian evaluated in FP64 and stored in
// FP32, FP32 multigrid with the FP32 right-hand side in the upper half of
// J's storage).
template <typename T>
nswe_status solve2d_t(nswe_prob_s *p, const double *U0, double *U, const nswe_params &prm_in, nswe_info *info,
                      cudaStream_t s) {
  nswe_params prm;
  int tail;
  resolve2d(p, prm_in, prm, tail);
  const int L = p->levels - 1;
  const int s0 = (prm.nest_start < 0 || prm.nest_start > L) ? L : prm.nest_start;
  const int st0 = (prm.jacobian & ~NSWE_JAC_FROZEN) == NSWE_JAC_FULL ? ST_J21 : ST_J9;
  const bool frozen = (prm.jacobian & NSWE_JAC_FROZEN) != 0;
  nswe_info inf;
  std::memset(&inf, 0, sizeof(inf));
  const int ns = p->host2.lev[s0].Nx * p->host2.lev[s0].Ny;
  if (cudaMemcpyAsync(p->host2.lev[s0].U, U0, sizeof(double) * 3 * ns, cudaMemcpyDeviceToDevice, s)) return NSWE_ECUDA;
  int fatal = 0;
  for (int l = s0; l >= 0 && !fatal; --l) {
    const Level2Dev &Lv = p->host2.lev[l];
    const int n = Lv.Nx * Lv.Ny;
    if (l < s0 && launch2_interp(p->dev2, l + 1, p->host2.lev[l + 1].Nx * p->host2.lev[l + 1].Ny,
                                 p->host2.lev[l + 1].U, Lv.U, s))
      return NSWE_ECUDA;
    if (launch2_residual(p->dev2, l, n, Lv.U, Lv.R, p->res_dev, p->partials2, s)) return NSWE_ECUDA;
    // One Newton step of this level (Eq. 12-14 with Algorithm 2): the same
    // launches every iteration, so they are captured once into a CUDA graph
    // and replayed; the host only waits for the residual and the flag.
    constexpr bool kMixed = std::is_same<T, float>::value;
    const int K = st0 == ST_J21 ? 21 : 9;
    // Colour-major J9 and Dinv on large levels solved by V-cycles (not on
    // the tail's levels, nor on the coarsest, whose J the dense LU reads).
    const int minc = p->ctx->cm2d_min_cells;
    const int cm = (l < L && st0 == ST_J9 && minc >= 0 && n >= minc && n > tail) ? 1 : 0;
    T *const J = reinterpret_cast<T *>(Lv.J);
    T *const dU = reinterpret_cast<T *>(Lv.dU);
    T *const Rs = kMixed ? J + (size_t)K * 9 * blk_stride(cm, Lv.Nx, Lv.Ny) : reinterpret_cast<T *>(Lv.R);
    auto step = [&](cudaStream_t q) -> cudaError_t {
      cudaError_t e;
      if ((e = launch2_jacobian<T>(p->dev2, l, n, st0, Lv.U, prm.eps[l], prm.alpha, Lv.R, J, frozen, cm,
                                   p->ctx->jac2d_cell_min, q)))
        return e;
      if constexpr (kMixed) {
        if ((e = launch2_to_f32(3L * n, Lv.R, reinterpret_cast<float *>(Rs), q))) return e;
      }
      if ((e = cudaMemsetAsync(p->flag, 0, sizeof(int), q))) return e;
      MG2<T> m = mg2_bind<T>(p, l, st0, J, Rs, dU, cm);
      if (l == L) {
        if ((e = launch2_dense_factor<T>(Lv.Nx, Lv.Ny, st0, J, reinterpret_cast<T *>(p->dense), p->piv, p->flag, q)) ||
            (e = launch2_dense_solve<T>(n, reinterpret_cast<const T *>(p->dense), p->piv, Rs,
                                        reinterpret_cast<T *>(p->xbuf), dU, q)))
          return e;
      } else {
        if ((e = mg2_setup<T>(p, m, q))) return e;
        if ((e = cudaMemsetAsync(dU, 0, sizeof(T) * 3 * n, q))) return e;
        for (int v = 0; v < prm.nu3; ++v)
          if ((e = mg2_vcycle<T>(p, m, prm, q, tail))) return e;
      }
      if ((e = launch2_update<T>(n, Lv.U, dU, prm.tau, p->flag, q))) return e;
      if ((e = launch2_residual(p->dev2, l, n, Lv.U, Lv.R, p->res_dev, p->partials2, q))) return e;
      if ((e = cudaMemcpyAsync(p->res_host, p->res_dev, sizeof(double), cudaMemcpyDeviceToHost, q))) return e;
      return cudaMemcpyAsync(p->flag_host, p->flag, sizeof(int), cudaMemcpyDeviceToHost, q);
    };
    if (!p->cap && cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking) != cudaSuccess) return NSWE_ECUDA;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    if (cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return NSWE_ECUDA;
    const cudaError_t ce = step(p->cap);
    if (cudaStreamEndCapture(p->cap, &graph) != cudaSuccess || ce != cudaSuccess ||
        cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return NSWE_ECUDA;
    }
    cudaGraphDestroy(graph);
    int it = 0, st = NSWE_OK;
    double res = 0.0;
    while (true) {
      if (cudaGraphLaunch(exec, s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGraphExecDestroy(exec);
        return NSWE_ECUDA;
      }
      if (l != L) inf.vcycles += prm.nu3;
      res = *p->res_host;
      ++it;
      if (*p->flag_host) {
        st = NSWE_ENEGDEPTH;  // non-positive depth or an exact zero pivot
        break;
      }
      if (!(res == res) || std::isinf(res)) {
        st = NSWE_ENAN;
        break;
      }
      if (res < prm.tol) break;
      if (it >= prm.n_max) {
        st = NSWE_ENOTCONV;
        break;
      }
    }
    cudaGraphExecDestroy(exec);
    inf.iters[l] = it;
    inf.res[l] = res;
    inf.level_status[l] = st;
    inf.total_iters += it;
    if (st == NSWE_ENAN || st == NSWE_ENEGDEPTH) fatal = st;
  }
  if (!fatal) {
    const int n0 = p->Nx * p->Ny;
    if (cudaMemcpyAsync(U, p->host2.lev[0].U, sizeof(double) * 3 * n0, cudaMemcpyDeviceToDevice, s)) return NSWE_ECUDA;
  }
  inf.status = fatal ? fatal : inf.level_status[0];
  if (info) *info = inf;
  return (nswe_status)inf.status;
}

nswe_status solve2d(nswe_prob_s *p, const double *U0, double *U, const nswe_params &prm, nswe_info *info,
                    cudaStream_t s) {
  return prm.precision == NSWE_PREC_MIXED ? solve2d_t<float>(p, U0, U, prm, info, s)
                                          : solve2d_t<double>(p, U0, U, prm, info, s);
}

// A batch of 2D solves. Each 2D solve is sequenced from the host with one
// synchronisation per Newton step and mostly small kernels, so the solves of
// a batch run concurrently: up to kSolve2DWorkers host threads, each with its
// own stream, take the problems in turn. The workers' streams first wait for
// the work already queued on the context stream; the call returns once every
// solve has finished.
constexpr int kSolve2DWorkers = 8;

// Host steady clock in ns: the time stamps of 2D solves, which the host sequences.
unsigned long long host_ns() {
  return (unsigned long long)std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

// prms[each ? i : 0] are problem i's parameters.
nswe_status solve2d_batch(nswe_ctx ctx, int count, const nswe_prob *probs, const double *const *U0s,
                          double *const *Us, const nswe_params *prms, bool each, nswe_info *infos) {
  if (count > 1 && ctx->batch2d_lockstep) return solve2d_lockstep(ctx, count, probs, U0s, Us, prms, each, infos);
  if (count == 1) {
    nswe_info inf;
    const unsigned long long t0 = host_ns();
    nswe_status st = solve2d(probs[0], U0s[0], Us[0], prms[0], &inf, ctx->stream);
    if (infos) {
      if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return NSWE_ECUDA;
      inf.t_start_ns = t0;
      inf.t_end_ns = host_ns();
      infos[0] = inf;
    }
    return st;
  }
  cudaEvent_t ready = nullptr;
  if (cudaEventCreateWithFlags(&ready, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventRecord(ready, ctx->stream) != cudaSuccess) {
    if (ready) cudaEventDestroy(ready);
    return NSWE_ECUDA;
  }
  std::vector<nswe_status> status(count, NSWE_OK);
  std::vector<nswe_info> rec(count);
  std::atomic<int> next{0};
  std::atomic<bool> cuda_error{false};
  const int workers = count < kSolve2DWorkers ? count : kSolve2DWorkers;
  std::vector<std::thread> pool;
  for (int w = 0; w < workers; ++w)
    pool.emplace_back([&] {
      cudaStream_t s = nullptr;
      if (cudaSetDevice(ctx->device) != cudaSuccess ||
          cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
          cudaStreamWaitEvent(s, ready, 0) != cudaSuccess) {
        cuda_error = true;
        if (s) cudaStreamDestroy(s);
        return;
      }
      for (int i = next++; i < count; i = next++) {
        std::memset(&rec[i], 0, sizeof(nswe_info));
        const unsigned long long t0 = host_ns();
        status[i] = solve2d(probs[i], U0s[i], Us[i], prms[each ? i : 0], &rec[i], s);
        if (status[i] == NSWE_ECUDA || cudaStreamSynchronize(s) != cudaSuccess) cuda_error = true;
        rec[i].t_start_ns = t0;
        rec[i].t_end_ns = host_ns();
      }
      if (cudaStreamSynchronize(s) != cudaSuccess) cuda_error = true;
      cudaStreamDestroy(s);
    });
  for (auto &t : pool) t.join();
  cudaEventDestroy(ready);
  if (cuda_error) return NSWE_ECUDA;
  int worst = NSWE_OK;
  for (int i = 0; i < count; ++i) {
    if (infos) infos[i] = rec[i];
    if (status[i] != NSWE_OK && worst == NSWE_OK) worst = status[i];
  }
  return (nswe_status)worst;
}

// One 2D V-cycle from `level` in arithmetic T (a direct solve when `level`
// is the coarsest).
template <typename T>
nswe_status vcycle2d_entry(nswe_ctx ctx, nswe_prob prob, int level, int nb, const T *J, const T *R, T *dU,
                           const nswe_params &prm_in) {
  if (nb != 9 && nb != 21) return NSWE_EINVAL;
  nswe_params prm;
  int tail;
  resolve2d(prob, prm_in, prm, tail);
  tail = ctx->tail2[std::is_same<T, float>::value ? 1 : 0];  // the standalone call's own precision
  MG2<T> m = mg2_bind<T>(prob, level, nb == 21 ? ST_J21 : ST_J9, J, R, dU, 0);
  cudaMemsetAsync(prob->flag, 0, sizeof(int), ctx->stream);
  if (level == prob->levels - 1) {
    const int n = nswe_prob_cells(prob, level);
    return (launch2_dense_factor<T>(m.lv[level].Nx, m.lv[level].Ny, m.st[level], J,
                                    reinterpret_cast<T *>(prob->dense), prob->piv, prob->flag, ctx->stream) ||
            launch2_dense_solve<T>(n, reinterpret_cast<const T *>(prob->dense), prob->piv, R,
                                   reinterpret_cast<T *>(prob->xbuf), dU, ctx->stream))
               ? NSWE_ECUDA
               : NSWE_OK;
  }
  return (mg2_setup<T>(prob, m, ctx->stream) || mg2_vcycle<T>(prob, m, prm, ctx->stream, tail)) ? NSWE_ECUDA
                                                                                                : NSWE_OK;
}

}  // namespace

void nswe::resolve2d(const nswe_prob_s *p, const nswe_params &in, nswe_params &out, int &tail) {
  out = in;
  const int prec = in.precision == NSWE_PREC_MIXED ? 1 : 0;
  tail = p->ctx->tail2[prec];
  if (in.colours2d != NSWE_COLOURS2D_AUTO) return;
  out.colours2d = 0;
  for (const nswe_tuned2d &t : p->ctx->tuned2)
    if (t.Nx == p->Nx && t.Ny == p->Ny && t.precision == prec) {
      out.colours2d = t.colours;
      tail = t.tail;
    }
}

extern "C" {

const char *nswe_status_str(int s) {
  switch (s) {
  case NSWE_OK: return "ok";
  case NSWE_EINVAL: return "invalid argument";
  case NSWE_ENOMEM: return "out of memory";
  case NSWE_ECUDA: return "CUDA runtime error";
  case NSWE_ENOTCONV: return "Newton iteration did not converge within n_max";
  case NSWE_ENAN: return "NaN or Inf in the residual";
  case NSWE_ENEGDEPTH: return "non-positive wet cross-section";
  case NSWE_ESINGULAR: return "singular coarsest system";
  case NSWE_ETIMEOUT: return "wait timed out";
  default: return "unknown status";
  }
}

nswe_status nswe_params_default(nswe_params *p, int N, int levels) {
  if (!p || N < 1 || levels < 1 || levels > NSWE_MAX_LEVELS) return NSWE_EINVAL;
  std::memset(p, 0, sizeof(*p));
  p->alpha = 3.0;
  p->tau = 0.6;
  p->omega = 1.0;
  p->tol = 1e-11;
  p->nu1 = p->nu2 = p->nu3 = 2;
  p->n_max = 2000;
  p->jacobian = NSWE_JAC_SIMPLIFIED;
  p->nest_start = -1;
  for (int l = 0; l < NSWE_MAX_LEVELS; ++l) {
    double n = (double)(N >> (l < levels ? l : levels - 1));
    double e = 0.2 - 0.05 * std::log2(n / 96.0);
    p->eps[l] = e < 0.05 ? 0.05 : (e > 0.2 ? 0.2 : e);
  }
  return NSWE_OK;
}

nswe_status nswe_ctx_create(nswe_ctx *out, int device, void *stream) {
  if (!out) return NSWE_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return NSWE_EINVAL;
  DeviceGuard g(device);
  nswe_ctx c = new (std::nothrow) nswe_ctx_s();
  if (!c) return NSWE_ENOMEM;
  c->device = device;
  c->stream = (cudaStream_t)stream;
  if (cudaMalloc(&c->partials, sizeof(double) * 1024) != cudaSuccess ||
      cudaMalloc(&c->status, sizeof(int) * 4) != cudaSuccess) {
    cudaFree(c->partials);
    delete c;
    return NSWE_ENOMEM;
  }
  *out = c;
  return NSWE_OK;
}

nswe_status nswe_ctx_set_colour_major_2d(nswe_ctx ctx, int min_cells) {
  if (!ctx) return NSWE_EINVAL;
  ctx->cm2d_min_cells = min_cells;
  return NSWE_OK;
}

nswe_status nswe_ctx_set_batch_2d(nswe_ctx ctx, int mode) {
  if (!ctx || (mode != NSWE_BATCH2D_CONCURRENT && mode != NSWE_BATCH2D_LOCKSTEP)) return NSWE_EINVAL;
  ctx->batch2d_lockstep = mode == NSWE_BATCH2D_LOCKSTEP ? 1 : 0;
  return NSWE_OK;
}

nswe_status nswe_ctx_set_jacobian_cells_2d(nswe_ctx ctx, int min_cells) {
  if (!ctx) return NSWE_EINVAL;
  ctx->jac2d_cell_min = min_cells;
  return NSWE_OK;
}

nswe_status nswe_ctx_set_stream(nswe_ctx ctx, void *stream) {
  if (!ctx) return NSWE_EINVAL;
  ctx->stream = (cudaStream_t)stream;
  return NSWE_OK;
}

nswe_status nswe_ctx_destroy(nswe_ctx ctx) {
  if (!ctx) return NSWE_EINVAL;
  DeviceGuard g(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  cudaFree(ctx->partials);
  cudaFree(ctx->status);
  cudaFree(ctx->tasks);
  cudaFree(ctx->infos);
  cudaFree(ctx->prms);
  delete ctx;
  return NSWE_OK;
}

nswe_status nswe_prob_create_1d(nswe_ctx ctx, nswe_prob *out, int N, int levels, double x0, double x1, double g,
                                const double *sigma_face, const double *gauss_geom, const nswe_bc1d *left,
                                const nswe_bc1d *right) {
  if (!out) return NSWE_EINVAL;
  *out = nullptr;
  if (!ctx || !sigma_face || !gauss_geom || !valid_bc(left) || !valid_bc(right)) return NSWE_EINVAL;
  if (levels < 1 || levels > NSWE_MAX_LEVELS || N < 4 || N > (1 << 26)) return NSWE_EINVAL;
  if (N % (1 << (levels - 1)) != 0) return NSWE_EINVAL;
  const int NL = N >> (levels - 1);
  if (NL < 4 || NL > kMaxCoarse) return NSWE_EINVAL;
  if (!(x1 > x0) || !(g > 0.0) || !std::isfinite(x0) || !std::isfinite(x1) || !std::isfinite(g))
    return NSWE_EINVAL;
  DeviceGuard dg(ctx->device);
  nswe_prob p = new (std::nothrow) nswe_prob_s();
  if (!p) return NSWE_ENOMEM;
  p->ctx = ctx;
  p->dim = 1;
  p->N = N;
  p->levels = levels;
  p->x0 = x0;
  p->x1 = x1;
  p->g = g;
  size_t geo = 0, work = 0;
  for (int l = 0; l < levels; ++l) {
    size_t Nl = (size_t)(N >> l);
    geo += round_up(Nl + 1) + round_up(6 * Nl);
    work += round_up(2 * Nl) * 3 + round_up(20 * Nl) + round_up(4 * Nl) + round_up(gd_doubles(Nl));
  }
  work += round_up(jw_doubles((size_t)N));
  p->geo_doubles = geo;
  if (cudaMalloc(&p->arena, sizeof(double) * (geo + work)) != cudaSuccess) {
    delete p;
    return NSWE_ENOMEM;
  }
  if (cudaMalloc(&p->dev, sizeof(ProbDev)) != cudaSuccess) {
    cudaFree(p->arena);
    delete p;
    return NSWE_ENOMEM;
  }
  ProbDev &h = p->host;
  std::memset(&h, 0, sizeof(h));
  h.levels = levels;
  h.g = g;
  double *a = p->arena;
  for (int l = 0; l < levels; ++l) {
    int Nl = N >> l;
    h.lev[l].N = Nl;
    h.lev[l].dx = (x1 - x0) / Nl;
    h.lev[l].sf = a;
    a += round_up(Nl + 1);
  }
  for (int l = 0; l < levels; ++l) {
    int Nl = N >> l;
    h.lev[l].gq = a;
    a += round_up(6 * (size_t)Nl);
  }
  for (int l = 0; l < levels; ++l) {
    size_t Nl = (size_t)(N >> l);
    h.lev[l].U = a;
    a += round_up(2 * Nl);
    h.lev[l].R = a;
    a += round_up(2 * Nl);
    h.lev[l].dU = a;
    a += round_up(2 * Nl);
    h.lev[l].J = a;
    a += round_up(20 * Nl);
    h.lev[l].Dinv = a;
    a += round_up(4 * Nl);
    h.lev[l].gd = a;
    a += round_up(gd_doubles(Nl));
  }
  h.jw = a;
  a += round_up(jw_doubles((size_t)N));
  nswe_status st = upload_geometry(p, sigma_face, gauss_geom, left, right);
  if (st != NSWE_OK) {
    cudaStreamSynchronize(ctx->stream);
    cudaFree(p->arena);
    cudaFree(p->dev);
    delete p;
    return st;
  }
  *out = p;
  return NSWE_OK;
}

nswe_status nswe_prob_set_geometry_1d(nswe_ctx ctx, nswe_prob prob, const double *sigma_face,
                                      const double *gauss_geom, const nswe_bc1d *left, const nswe_bc1d *right) {
  if (!ctx || !prob || prob->ctx != ctx || !sigma_face || !gauss_geom || !valid_bc(left) || !valid_bc(right))
    return NSWE_EINVAL;
  DeviceGuard dg(ctx->device);
  return upload_geometry(prob, sigma_face, gauss_geom, left, right);
}

nswe_status nswe_prob_set_flux_1d(nswe_ctx ctx, nswe_prob prob, int flux) {
  if (!ctx || !prob || prob->ctx != ctx || prob->dim != 1 || (flux != NSWE_FLUX_HLL && flux != NSWE_FLUX_LLF))
    return NSWE_EINVAL;
  DeviceGuard dg(ctx->device);
  prob->host.flux = flux;
  return cudaMemcpyAsync(prob->dev, &prob->host, sizeof(ProbDev), cudaMemcpyHostToDevice, ctx->stream) ==
                 cudaSuccess
             ? NSWE_OK
             : NSWE_ECUDA;
}

nswe_status nswe_prob_set_geometry_batch_1d(nswe_ctx ctx, int count, const nswe_prob *probs,
                                            const double *const *sigma_faces, const double *const *gauss_geoms,
                                            const nswe_bc1d *lefts, const nswe_bc1d *rights) {
  if (!ctx || count < 0 || (count > 0 && (!probs || !sigma_faces || !gauss_geoms || !lefts || !rights)))
    return NSWE_EINVAL;
  for (int i = 0; i < count; ++i) {
    if (!probs[i] || probs[i]->ctx != ctx || probs[i]->dim != 1 || !sigma_faces[i] || !gauss_geoms[i] ||
        !valid_bc(&lefts[i]) || !valid_bc(&rights[i]))
      return NSWE_EINVAL;
    for (int k = 0; k < i; ++k)
      if (probs[k] == probs[i]) return NSWE_EINVAL;  // one staging buffer per problem
  }
  if (count == 0) return NSWE_OK;
  DeviceGuard dg(ctx->device);
  // Pack every problem (host work, in parallel), then issue the copies: no
  // upload starts unless every problem's data is valid.
  std::vector<nswe_status> st(count, NSWE_OK);
  std::atomic<int> next{0};
  const unsigned hw = std::thread::hardware_concurrency();
  const int workers = std::max(1, std::min(count, std::min(16, (int)(hw ? hw : 1))));
  auto work = [&] {
    cudaSetDevice(ctx->device);
    for (int i = next++; i < count; i = next++) st[i] = pack_geometry(probs[i], sigma_faces[i], gauss_geoms[i]);
  };
  std::vector<std::thread> pool;
  for (int w = 1; w < workers; ++w) pool.emplace_back(work);
  work();
  for (auto &t : pool) t.join();
  for (int i = 0; i < count; ++i)
    if (st[i] != NSWE_OK) return st[i];
  for (int i = 0; i < count; ++i) {
    nswe_status e = issue_geometry(probs[i], &lefts[i], &rights[i], false);
    if (e != NSWE_OK) return e;
  }
  // the derived geometry of all problems in one launch (the context's task
  // array addresses them; later users of the array are ordered on the stream)
  nswe_status e = ensure_cap(ctx, count);
  if (e != NSWE_OK) return e;
  std::vector<SolveTask> tasks(count);
  for (int i = 0; i < count; ++i) {
    std::memset(&tasks[i], 0, sizeof(SolveTask));
    tasks[i].prob = probs[i]->dev;
  }
  if (cudaMemcpyAsync(ctx->tasks, tasks.data(), sizeof(SolveTask) * count, cudaMemcpyHostToDevice, ctx->stream) !=
          cudaSuccess ||
      launch_geom_derive_batch(ctx->tasks, count, ctx->stream) != cudaSuccess)
    return NSWE_ECUDA;
  return NSWE_OK;
}

nswe_status nswe_prob_destroy(nswe_prob prob) {
  if (!prob) return NSWE_EINVAL;
  DeviceGuard dg(prob->ctx->device);
  cudaStreamSynchronize(prob->ctx->stream);
  if (prob->staged) cudaEventDestroy(prob->staged);
  if (prob->stage) cudaFreeHost(prob->stage);
  cudaFree(prob->arena);
  cudaFree(prob->dev);
  cudaFree(prob->dev2);
  cudaFree(prob->piv);
  cudaFree(prob->flag);
  cudaFree(prob->res_dev);
  cudaFreeHost(prob->res_host);
  cudaFreeHost(prob->flag_host);
  cudaFree(prob->partials2);
  if (prob->cap) cudaStreamDestroy(prob->cap);
  delete prob;
  return NSWE_OK;
}

int nswe_prob_cells(nswe_prob prob, int level) {
  if (!prob || level < 0 || level >= prob->levels) return -1;
  if (prob->dim == 2) return (prob->Nx >> level) * (prob->Ny >> level);
  return prob->N >> level;
}

int nswe_prob_dim(nswe_prob prob) { return prob ? prob->dim : 0; }

nswe_status nswe_prob_create_2d(nswe_ctx ctx, nswe_prob *out, int Nx, int Ny, int levels, double x0, double x1,
                                double y0, double y1, double g, const double *gauss_geom, const int *bc_kind,
                                const double *bc_state) {
  if (!out) return NSWE_EINVAL;
  *out = nullptr;
  if (!ctx || !gauss_geom || !bc_kind || !bc_state) return NSWE_EINVAL;
  if (levels < 1 || levels > NSWE_MAX_LEVELS || Nx < 4 || Ny < 4 || (long)Nx * Ny > (1L << 26)) return NSWE_EINVAL;
  if (Nx % (1 << (levels - 1)) || Ny % (1 << (levels - 1))) return NSWE_EINVAL;
  const int NLx = Nx >> (levels - 1), NLy = Ny >> (levels - 1);
  if (NLx < 4 || NLy < 4 || NLx * NLy > 512) return NSWE_EINVAL;
  if (!(x1 > x0) || !(y1 > y0) || !(g > 0.0) || !std::isfinite(x0) || !std::isfinite(x1) || !std::isfinite(y0) ||
      !std::isfinite(y1) || !std::isfinite(g))
    return NSWE_EINVAL;
  for (int i = 0; i < 12; ++i)
    if (!std::isfinite(bc_state[i])) return NSWE_EINVAL;
  size_t nk = 0, ng = 0;
  for (int l = 0; l < levels; ++l) {
    nk += 2 * (size_t)((Nx >> l) + (Ny >> l));
    ng += 8 * (size_t)(Nx >> l) * (Ny >> l);
  }
  for (size_t i = 0; i < nk; ++i)
    if (bc_kind[i] < NSWE_BC2_REFLECT || bc_kind[i] > NSWE_BC2_DEPTH) return NSWE_EINVAL;
  for (size_t i = 0; i < ng; ++i)
    if (!std::isfinite(gauss_geom[i])) return NSWE_EINVAL;
  DeviceGuard dg(ctx->device);
  nswe_prob p = new (std::nothrow) nswe_prob_s();
  if (!p) return NSWE_ENOMEM;
  p->ctx = ctx;
  p->dim = 2;
  p->Nx = Nx;
  p->Ny = Ny;
  p->levels = levels;
  p->x0 = x0;
  p->x1 = x1;
  p->g = g;
  const size_t doubles = prob2d_arena_doubles(Nx, Ny, levels);
  const size_t N3 = 3 * (size_t)NLx * NLy;
  bool ok = cudaMalloc(&p->arena, sizeof(double) * doubles) == cudaSuccess &&
            cudaMalloc(&p->dev2, sizeof(ProbDev2)) == cudaSuccess &&
            cudaMalloc(&p->piv, sizeof(int) * (N3 + 64)) == cudaSuccess &&
            cudaMalloc(&p->flag, sizeof(int) * 4) == cudaSuccess &&
            cudaMalloc(&p->res_dev, sizeof(double) * 4) == cudaSuccess &&
            cudaMalloc(&p->partials2, sizeof(double) * 1024) == cudaSuccess &&
            cudaMallocHost(&p->res_host, sizeof(double) * 4) == cudaSuccess &&
            cudaMallocHost(&p->flag_host, sizeof(int) * 4) == cudaSuccess;
  if (!ok) {
    cudaFree(p->arena);
    cudaFree(p->dev2);
    cudaFree(p->piv);
    cudaFree(p->flag);
    cudaFree(p->res_dev);
    cudaFreeHost(p->res_host);
    cudaFreeHost(p->flag_host);
    delete p;
    return NSWE_ENOMEM;
  }
  ProbDev2 &h = p->host2;
  std::memset(&h, 0, sizeof(h));
  h.levels = levels;
  h.g = g;
  for (int i = 0; i < 12; ++i) h.bcs[i] = bc_state[i];
  double *a = p->arena;
  std::vector<double> geo;
  std::vector<int> kinds(bc_kind, bc_kind + nk);
  size_t gsrc = 0, ksrc = 0;
  int *kind_dev = reinterpret_cast<int *>(a);
  a += 2 * round_up(nk);
  for (int l = 0; l < levels; ++l) {
    Level2Dev &Lv = h.lev[l];
    Lv.Nx = Nx >> l;
    Lv.Ny = Ny >> l;
    Lv.dx = (x1 - x0) / Lv.Nx;
    Lv.dy = (y1 - y0) / Lv.Ny;
    const size_t n = (size_t)Lv.Nx * Lv.Ny;
    Lv.gq = a;
    if (cudaMemcpyAsync(a, gauss_geom + gsrc, sizeof(double) * 8 * n, cudaMemcpyHostToDevice, ctx->stream)) ok = false;
    gsrc += 8 * n;
    a += round_up(8 * n);
    Lv.bck = kind_dev + ksrc;
    ksrc += 2 * (size_t)(Lv.Nx + Lv.Ny);
    Lv.U = a;
    a += round_up(3 * n);
    Lv.R = a;
    a += round_up(3 * n);
    Lv.dU = a;
    a += round_up(3 * n);
    Lv.J = a;
    a += round_up(189 * n);
    Lv.Dinv = a;
    a += round_up(9 * n + 27 * (size_t)Lv.Ny);  // as prob2d_arena_doubles
  }
  p->dense = a;
  a += round_up(N3 * N3);
  p->xbuf = a;
  a += round_up(N3);
  if (cudaMemcpyAsync(kind_dev, kinds.data(), sizeof(int) * nk, cudaMemcpyHostToDevice, ctx->stream)) ok = false;
  if (cudaMemcpyAsync(p->dev2, &p->host2, sizeof(ProbDev2), cudaMemcpyHostToDevice, ctx->stream)) ok = false;
  if (!ok || cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
    nswe_prob_destroy(p);
    return NSWE_ECUDA;
  }
  *out = p;
  return NSWE_OK;
}

nswe_status nswe_residual(nswe_ctx ctx, nswe_prob prob, int level, const double *U, double *R, double *res_l1) {
  if (!ctx || !prob || prob->ctx != ctx || !U || !R || level < 0 || level >= prob->levels) return NSWE_EINVAL;
  DeviceGuard dg(ctx->device);
  if (prob->dim == 2)
    return launch2_residual(prob->dev2, level, nswe_prob_cells(prob, level), U, R, res_l1, ctx->partials,
                            ctx->stream) == cudaSuccess
               ? NSWE_OK
               : NSWE_ECUDA;
  int N = prob->N >> level;
  return launch_residual(prob->dev, level, N, U, R, res_l1, ctx->partials, ctx->stream) == cudaSuccess
             ? NSWE_OK
             : NSWE_ECUDA;
}

static nswe_status jacobian_common(nswe_ctx ctx, nswe_prob prob, int level, int nb, const double *U, double eps,
                                   double alpha, double *R, double *J, double *res, bool frozen = false) {
  if (!ctx || !prob || prob->ctx != ctx || !U || !R || !J || level < 0 || level >= prob->levels) return NSWE_EINVAL;
  if (!(eps > 0.0) || !std::isfinite(eps) || !(alpha >= 0.0) || !std::isfinite(alpha)) return NSWE_EINVAL;
  DeviceGuard dg(ctx->device);
  if (prob->dim == 2) {
    const int n = nswe_prob_cells(prob, level);
    if (launch2_residual(prob->dev2, level, n, U, R, res, ctx->partials, ctx->stream) ||
        launch2_jacobian<double>(prob->dev2, level, n, nb == 5 ? ST_J21 : ST_J9, U, eps, alpha, R, J, frozen, 0,
                                 ctx->jac2d_cell_min, ctx->stream))
      return NSWE_ECUDA;
    return NSWE_OK;
  }
  int N = prob->N >> level;
  return launch_jacobian(prob->dev, level, N, nb, U, eps, alpha, R, J, res, ctx->partials, ctx->stream) ==
                 cudaSuccess
             ? NSWE_OK
             : NSWE_ECUDA;
}

nswe_status nswe_jacobian_simplified(nswe_ctx ctx, nswe_prob prob, int level, const double *U, double eps,
                                     double alpha, double *R, double *J, double *res_l1) {
  return jacobian_common(ctx, prob, level, 3, U, eps, alpha, R, J, res_l1);
}

nswe_status nswe_jacobian_full(nswe_ctx ctx, nswe_prob prob, int level, const double *U, double eps,
                               double alpha, double *R, double *J, double *res_l1) {
  return jacobian_common(ctx, prob, level, 5, U, eps, alpha, R, J, res_l1);
}

nswe_status nswe_jacobian_frozen(nswe_ctx ctx, nswe_prob prob, int level, int nb, const double *U, double eps,
                                 double alpha, double *R, double *J, double *res_l1) {
  if (!prob || prob->dim != 2 || (nb != 9 && nb != 21)) return NSWE_EINVAL;
  return jacobian_common(ctx, prob, level, nb == 21 ? 5 : 3, U, eps, alpha, R, J, res_l1, true);
}

nswe_status nswe_jacobian_f32(nswe_ctx ctx, nswe_prob prob, int level, int nb, const double *U, double eps,
                              double alpha, double *R, float *J, double *res_l1) {
  if (!ctx || !prob || prob->ctx != ctx || !U || !R || !J || level < 0 || level >= prob->levels) return NSWE_EINVAL;
  if (!(eps > 0.0) || !std::isfinite(eps) || !(alpha >= 0.0) || !std::isfinite(alpha)) return NSWE_EINVAL;
  DeviceGuard dg(ctx->device);
  if (prob->dim == 2) {
    if (nb != 9 && nb != 21) return NSWE_EINVAL;
    const int n = nswe_prob_cells(prob, level);
    return (launch2_residual(prob->dev2, level, n, U, R, res_l1, ctx->partials, ctx->stream) ||
            launch2_jacobian<float>(prob->dev2, level, n, nb == 21 ? ST_J21 : ST_J9, U, eps, alpha, R, J, false, 0,
                                    ctx->jac2d_cell_min, ctx->stream))
               ? NSWE_ECUDA
               : NSWE_OK;
  }
  if (nb != 3 && nb != 5) return NSWE_EINVAL;
  const int N = prob->N >> level;
  return launch_jacobian_f32(prob->dev, level, N, nb, U, eps, alpha, R, J, res_l1, ctx->partials, ctx->stream) ==
                 cudaSuccess
             ? NSWE_OK
             : NSWE_ECUDA;
}

nswe_status nswe_mg_vcycle_f32(nswe_ctx ctx, nswe_prob prob, int level, int nb, const float *J, const float *R,
                               float *dU, const nswe_params *params) {
  if (!ctx || !prob || prob->ctx != ctx || !J || !R || !dU || level < 0 || level >= prob->levels) return NSWE_EINVAL;
  nswe_status st = check_params(params, nullptr, 0);
  if (st != NSWE_OK) return st;
  DeviceGuard dg(ctx->device);
  if (prob->dim == 2) return vcycle2d_entry<float>(ctx, prob, level, nb, J, R, dU, *params);
  if (nb != 3 && nb != 5) return NSWE_EINVAL;
  const int coarse = prob->N >> (prob->levels - 1);
  const int coarse_nb = (level == prob->levels - 1) ? nb : 3;
  return launch_vcycle_f32(prob->dev, level, nb, J, R, dU, *params, ctx->status, coarse, coarse_nb, ctx->stream) ==
                 cudaSuccess
             ? NSWE_OK
             : NSWE_ECUDA;
}

nswe_status nswe_mg_vcycle(nswe_ctx ctx, nswe_prob prob, int level, int nb, const double *J, const double *R,
                           double *dU, const nswe_params *params) {
  if (!ctx || !prob || prob->ctx != ctx || !J || !R || !dU || level < 0 || level >= prob->levels) return NSWE_EINVAL;
  nswe_status st = check_params(params, nullptr, 0);
  if (st != NSWE_OK) return st;
  DeviceGuard dg(ctx->device);
  if (prob->dim == 2) return vcycle2d_entry<double>(ctx, prob, level, nb, J, R, dU, *params);
  if (nb != 3 && nb != 5) return NSWE_EINVAL;
  const int coarse = prob->N >> (prob->levels - 1);
  const int coarse_nb = (level == prob->levels - 1) ? nb : 3;
  return launch_vcycle(prob->dev, level, nb, J, R, dU, *params, ctx->status, coarse, coarse_nb, ctx->stream) ==
                 cudaSuccess
             ? NSWE_OK
             : NSWE_ECUDA;
}

nswe_status nswe_mg_smooth(nswe_ctx ctx, nswe_prob prob, int level, int nb, const double *J, const double *R,
                           double *dU, const nswe_params *params, int colour_major, int *launches) {
  if (!ctx || !prob || prob->ctx != ctx || !J || !R || !dU || level < 0 || level >= prob->levels) return NSWE_EINVAL;
  if (prob->dim != 2 || (nb != 9 && nb != 21) || (colour_major != 0 && colour_major != 1) ||
      (colour_major && nb != 9))
    return NSWE_EINVAL;
  nswe_status st = check_params(params, nullptr, 0);
  if (st != NSWE_OK) return st;
  DeviceGuard dg(ctx->device);
  const Level2Dev &L = prob->host2.lev[level];
  const int stc = nb == 21 ? ST_J21 : ST_J9;
  nswe_params prm;
  int tail;
  resolve2d(prob, *params, prm, tail);
  Lev2<double> Lv{L.Nx, L.Ny, const_cast<double *>(J), L.Dinv, const_cast<double *>(R), dU, colour_major};
  int count = 0;
  if (launch2_dinv<double>(L.Nx, L.Ny, stc, J, L.Dinv, colour_major, ctx->stream) != cudaSuccess ||
      smooth2<double>(Lv, stc, prm.nu1, prm.omega, prm.colours2d, ctx->stream, &count) != cudaSuccess)
    return NSWE_ECUDA;
  if (launches) *launches = count;
  return NSWE_OK;
}

nswe_status nswe_set_launch_overlap_2d(int enable) {
  if (enable != 0 && enable != 1) return NSWE_EINVAL;
  set_pdl_2d(enable);
  return NSWE_OK;
}

nswe_status nswe_ctx_set_tail_2d(nswe_ctx ctx, int precision, int max_cells) {
  if (!ctx || (precision != NSWE_PREC_FP64 && precision != NSWE_PREC_MIXED) || max_cells < 0) return NSWE_EINVAL;
  ctx->tail2[precision == NSWE_PREC_MIXED ? 1 : 0] = max_cells;
  return NSWE_OK;
}

nswe_status nswe_ctx_get_tuned_2d(nswe_ctx ctx, int Nx, int Ny, int precision, int *schedule, int *tail) {
  if (!ctx || (precision != NSWE_PREC_FP64 && precision != NSWE_PREC_MIXED)) return NSWE_EINVAL;
  const int prec = precision == NSWE_PREC_MIXED ? 1 : 0;
  for (const nswe_tuned2d &t : ctx->tuned2)
    if (t.Nx == Nx && t.Ny == Ny && t.precision == prec) {
      if (schedule) *schedule = t.colours;
      if (tail) *tail = t.tail;
      return NSWE_OK;
    }
  return NSWE_EINVAL;  // nothing recorded for this size and precision
}

}  // extern "C"

namespace {

// Times `reps` V-cycles from the finest level of `prob` for every (schedule,
// tail) pair, the Jacobian formed once from U in the precision of `prm`.
template <typename T>
nswe_status autotune2d_t(nswe_ctx ctx, nswe_prob prob, const double *U, const nswe_params &prm,
                         const int *schedules, int nsched, const int *tails, int ntails, int reps, double *ms,
                         int *best_s, int *best_t) {
  const int n = prob->Nx * prob->Ny;
  const int st = (prm.jacobian & ~NSWE_JAC_FROZEN) == NSWE_JAC_FULL ? ST_J21 : ST_J9;
  const int K = st == ST_J21 ? 21 : 9;
  const bool frozen = (prm.jacobian & NSWE_JAC_FROZEN) != 0;
  cudaStream_t s = ctx->stream;
  double *R64 = nullptr;
  T *J = nullptr, *R = nullptr, *dU = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  nswe_status status = NSWE_OK;
  if (cudaMalloc(&R64, sizeof(double) * 3 * n) || cudaMalloc(&J, sizeof(T) * (size_t)K * 9 * n) ||
      cudaMalloc(&R, sizeof(T) * 3 * n) || cudaMalloc(&dU, sizeof(T) * 3 * n) || cudaEventCreate(&e0) ||
      cudaEventCreate(&e1))
    status = NSWE_ENOMEM;
  if (status == NSWE_OK &&
      (launch2_residual(prob->dev2, 0, n, U, R64, nullptr, prob->partials2, s) ||
       launch2_jacobian<T>(prob->dev2, 0, n, st, U, prm.eps[0], prm.alpha, R64, J, frozen, 0, ctx->jac2d_cell_min, s)))
    status = NSWE_ECUDA;
  if (status == NSWE_OK) {
    if constexpr (std::is_same<T, float>::value) {
      if (launch2_to_f32(3L * n, R64, R, s)) status = NSWE_ECUDA;
    } else {
      if (cudaMemcpyAsync(R, R64, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, s)) status = NSWE_ECUDA;
    }
  }
  MG2<T> m = mg2_bind<T>(prob, 0, st, J, R, dU, 0);
  if (status == NSWE_OK && mg2_setup<T>(prob, m, s)) status = NSWE_ECUDA;
  double best = 0.0;
  for (int a = 0; a < nsched && status == NSWE_OK; ++a)
    for (int b = 0; b < ntails && status == NSWE_OK; ++b) {
      nswe_params q = prm;
      q.colours2d = schedules[a];
      float t = 0.f;
      if (cudaMemsetAsync(dU, 0, sizeof(T) * 3 * n, s) || mg2_vcycle<T>(prob, m, q, s, tails[b]) ||  // untimed
          cudaEventRecord(e0, s)) {
        status = NSWE_ECUDA;
        break;
      }
      for (int r = 0; r < reps && status == NSWE_OK; ++r)
        if (mg2_vcycle<T>(prob, m, q, s, tails[b])) status = NSWE_ECUDA;
      if (status != NSWE_OK || cudaEventRecord(e1, s) || cudaEventSynchronize(e1) ||
          cudaEventElapsedTime(&t, e0, e1)) {
        status = NSWE_ECUDA;
        break;
      }
      const double per = (double)t / reps;
      if (ms) ms[a * ntails + b] = per;
      if ((a == 0 && b == 0) || per < best) {
        best = per;
        *best_s = schedules[a];
        *best_t = tails[b];
      }
    }
  cudaStreamSynchronize(s);
  cudaFree(R64);
  cudaFree(J);
  cudaFree(R);
  cudaFree(dU);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return status;
}

}  // namespace

extern "C" {

nswe_status nswe_autotune_2d(nswe_ctx ctx, nswe_prob prob, const double *U, const nswe_params *params,
                             const int *schedules, int nsched, const int *tails, int ntails, int reps, double *ms,
                             int *best_schedule, int *best_tail) {
  if (!ctx || !prob || prob->ctx != ctx || prob->dim != 2 || !U || !params || !schedules || !tails || nsched < 1 ||
      ntails < 1 || nsched > 64 || ntails > 64 || reps < 1 || reps > 100)
    return NSWE_EINVAL;
  nswe_status st = check_params(params, prob, 0);
  if (st != NSWE_OK) return st;
  for (int a = 0; a < nsched; ++a)
    if (schedules[a] != 0 && (schedules[a] < 3 || schedules[a] > 4096)) return NSWE_EINVAL;
  for (int b = 0; b < ntails; ++b)
    if (tails[b] < 0) return NSWE_EINVAL;
  if (prob->levels < 2) return NSWE_EINVAL;  // a V-cycle needs a coarser level
  DeviceGuard dg(ctx->device);
  int bs = 0, bt = 0;
  st = params->precision == NSWE_PREC_MIXED
           ? autotune2d_t<float>(ctx, prob, U, *params, schedules, nsched, tails, ntails, reps, ms, &bs, &bt)
           : autotune2d_t<double>(ctx, prob, U, *params, schedules, nsched, tails, ntails, reps, ms, &bs, &bt);
  if (st != NSWE_OK) return st;
  const int prec = params->precision == NSWE_PREC_MIXED ? 1 : 0;
  bool found = false;
  for (nswe_tuned2d &t : ctx->tuned2)
    if (t.Nx == prob->Nx && t.Ny == prob->Ny && t.precision == prec) {
      t.colours = bs;
      t.tail = bt;
      found = true;
    }
  if (!found) ctx->tuned2.push_back({prob->Nx, prob->Ny, prec, bs, bt});
  if (best_schedule) *best_schedule = bs;
  if (best_tail) *best_tail = bt;
  return NSWE_OK;
}

// Batched Algorithm 3; params[each ? i : 0] are problem i's parameters.
static nswe_status solve_batch_common(nswe_ctx ctx, int count, const nswe_prob *probs, const double *const *U0s,
                                      double *const *Us, const nswe_params *params, bool each, nswe_info *infos) {
  if (!ctx || count < 0 || (count > 0 && (!probs || !U0s || !Us || !params))) return NSWE_EINVAL;
  if (count == 0) return NSWE_OK;
  if (count > (1 << 20)) return NSWE_EINVAL;
  std::vector<SolveTask> tasks(count);
  int nb = 3;
  for (int i = 0; i < count; ++i) {
    nswe_prob p = probs[i];
    const nswe_params *q = params + (each ? i : 0);
    if (!p || p->ctx != ctx || !U0s[i] || !Us[i]) return NSWE_EINVAL;
    if (p->dim != probs[0]->dim) return NSWE_EINVAL;
    int s0 = (q->nest_start >= 0 && q->nest_start < p->levels) ? q->nest_start : p->levels - 1;
    nswe_status st = check_params(q, p, s0);
    if (st != NSWE_OK) return st;
    // one 1D launch computes in one arithmetic type, with one numerical flux
    if (p->dim == 1 && (q->precision != params[0].precision || p->host.flux != probs[0]->host.flux))
      return NSWE_EINVAL;
    if ((q->jacobian & ~NSWE_JAC_FROZEN) == NSWE_JAC_FULL) nb = 5;
  }
  DeviceGuard dg(ctx->device);
  if (probs[0]->dim == 2) {
    for (int i = 1; i < count; ++i)
      for (int k = 0; k < i; ++k)
        if (probs[k] == probs[i]) return NSWE_EINVAL;  // one problem's workspace cannot serve two solves at once
    return solve2d_batch(ctx, count, probs, U0s, Us, params, each, infos);
  }
  nswe_status st = ensure_cap(ctx, count);
  if (st != NSWE_OK) return st;
  cudaStream_t s = ctx->stream;
  if (each && cudaMemcpyAsync(ctx->prms, params, sizeof(nswe_params) * count, cudaMemcpyHostToDevice, s) !=
                  cudaSuccess)
    return NSWE_ECUDA;
  int max_coarse = 4;
  for (int i = 0; i < count; ++i) {
    const int c = probs[i]->N >> (probs[i]->levels - 1);
    if (c > max_coarse) max_coarse = c;
    tasks[i].prob = probs[i]->dev;
    tasks[i].U0 = U0s[i];
    tasks[i].U = Us[i];
    tasks[i].info = ctx->infos + i;
    tasks[i].prm = each ? ctx->prms + i : nullptr;
    tasks[i].derive = 0;
    tasks[i].done = nullptr;
  }
  if (cudaMemcpyAsync(ctx->tasks, tasks.data(), sizeof(SolveTask) * count, cudaMemcpyHostToDevice, s) !=
      cudaSuccess)
    return NSWE_ECUDA;
  const int shape = ctx->solve_shape[params->precision == NSWE_PREC_MIXED ? 1 : 0];
  const cudaError_t le =
      (ctx->solve_ctas > 1 && probs[0]->host.flux == NSWE_FLUX_HLL)
          ? launch_solve_cluster(ctx->tasks, count, *params, max_coarse, nb, ctx->solve_ctas, ctx->team_cells, s)
          : launch_solve_sized(ctx->tasks, count, *params, max_coarse, nb, shape, s, probs[0]->host.flux);
  if (le != cudaSuccess) return NSWE_ECUDA;
  if (infos) {
    if (cudaMemcpyAsync(infos, ctx->infos, sizeof(nswe_info) * count, cudaMemcpyDeviceToHost, s) != cudaSuccess)
      return NSWE_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return NSWE_ECUDA;
    int worst = NSWE_OK;
    for (int i = 0; i < count; ++i)
      if (infos[i].status != NSWE_OK && worst == NSWE_OK) worst = infos[i].status;
    return (nswe_status)worst;
  }
  return NSWE_OK;
}

nswe_status nswe_newton_solve_batch(nswe_ctx ctx, int count, const nswe_prob *probs, const double *const *U0s,
                                    double *const *Us, const nswe_params *params, nswe_info *infos) {
  return solve_batch_common(ctx, count, probs, U0s, Us, params, false, infos);
}

nswe_status nswe_newton_solve_batch_each(nswe_ctx ctx, int count, const nswe_prob *probs, const double *const *U0s,
                                         double *const *Us, const nswe_params *params, nswe_info *infos) {
  return solve_batch_common(ctx, count, probs, U0s, Us, params, true, infos);
}

nswe_status nswe_newton_solve(nswe_ctx ctx, nswe_prob prob, const double *U0, double *U, const nswe_params *params,
                              nswe_info *info) {
  return nswe_newton_solve_batch(ctx, 1, &prob, &U0, &U, params, info);
}

int nswe_solve_shape_count(void) { return kSolveShapes; }

nswe_status nswe_solve_shape_info(int shape, int *threads, int *blocks_per_sm) {
  if (shape < 0 || shape >= kSolveShapes) return NSWE_EINVAL;
  if (threads) *threads = kSolveShapeThreads[shape];
  if (blocks_per_sm) *blocks_per_sm = kSolveShapeBlocks[shape];
  return NSWE_OK;
}

nswe_status nswe_ctx_set_solve_shape(nswe_ctx ctx, int precision, int shape) {
  if (!ctx || (precision != NSWE_PREC_FP64 && precision != NSWE_PREC_MIXED) || shape < 0 || shape >= kSolveShapes)
    return NSWE_EINVAL;
  ctx->solve_shape[precision == NSWE_PREC_MIXED ? 1 : 0] = shape;
  return NSWE_OK;
}

nswe_status nswe_ctx_set_solve_cluster(nswe_ctx ctx, int ctas, int team_cells) {
  if (!ctx || ctas < 1 || ctas > kMaxClusterCtas || team_cells < 1) return NSWE_EINVAL;
  ctx->solve_ctas = ctas;
  ctx->team_cells = team_cells;
  return NSWE_OK;
}

nswe_status nswe_ctx_get_solve_cluster(nswe_ctx ctx, int *ctas, int *team_cells) {
  if (!ctx) return NSWE_EINVAL;
  if (ctas) *ctas = ctx->solve_ctas;
  if (team_cells) *team_cells = ctx->team_cells;
  return NSWE_OK;
}

nswe_status nswe_ctx_get_solve_shape(nswe_ctx ctx, int precision, int *shape) {
  if (!ctx || !shape || (precision != NSWE_PREC_FP64 && precision != NSWE_PREC_MIXED)) return NSWE_EINVAL;
  *shape = ctx->solve_shape[precision == NSWE_PREC_MIXED ? 1 : 0];
  return NSWE_OK;
}

nswe_status nswe_autotune_solve_batch(nswe_ctx ctx, int count, const nswe_prob *probs, const double *const *U0s,
                                      double *const *Us, const nswe_params *params, int reps, double *ms,
                                      int *best) {
  if (!ctx || !params || count < 1 || reps < 1 || reps > 100) return NSWE_EINVAL;
  if (probs[0] == nullptr || probs[0]->dim != 1) return NSWE_EINVAL;
  const int prec = params->precision == NSWE_PREC_MIXED ? 1 : 0;
  const int keep = ctx->solve_shape[prec];
  DeviceGuard dg(ctx->device);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return NSWE_ECUDA;
  }
  nswe_status st = NSWE_OK;
  int arg = 0;
  double tbest = 0.0;
  for (int shape = 0; shape < kSolveShapes && st == NSWE_OK; ++shape) {
    ctx->solve_shape[prec] = shape;
    st = nswe_newton_solve_batch(ctx, count, probs, U0s, Us, params, nullptr);  // untimed first run
    if (st != NSWE_OK) break;
    if (cudaEventRecord(e0, ctx->stream) != cudaSuccess) st = NSWE_ECUDA;
    for (int r = 0; r < reps && st == NSWE_OK; ++r) st = nswe_newton_solve_batch(ctx, count, probs, U0s, Us, params, nullptr);
    float t = 0.f;
    if (st == NSWE_OK && (cudaEventRecord(e1, ctx->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                          cudaEventElapsedTime(&t, e0, e1) != cudaSuccess))
      st = NSWE_ECUDA;
    if (st != NSWE_OK) break;
    const double per = (double)t / reps;
    if (ms) ms[shape] = per;
    if (shape == 0 || per < tbest) {
      tbest = per;
      arg = shape;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx->solve_shape[prec] = st == NSWE_OK ? arg : keep;
  if (st == NSWE_OK && best) *best = arg;
  return st;
}

}  // extern "C"
