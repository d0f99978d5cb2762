// Host side of the C ABI declared in include/nswe.h: contexts, problems
// (device arena with geometry and solver workspace), argument checking and
// kernel launches. No compute happens here.
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "nswe_internal.h"

using namespace nswe;

struct nswe_ctx_s {
  int device;
  cudaStream_t stream;
  double *partials;      // [1024] per-block partial sums of res
  int *status;           // device status word of standalone V-cycles
  SolveTask *tasks;      // device task array
  nswe_info *infos;      // device info records
  int cap;               // capacity of tasks / infos
};

struct nswe_prob_s {
  nswe_ctx ctx;
  int N, levels;
  double x0, x1, g;
  ProbDev host;          // device pointers, host copy
  ProbDev *dev;          // device copy
  double *arena;
  size_t geo_doubles;    // geometry region at the front of the arena
};

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
  if (p->jacobian != NSWE_JAC_SIMPLIFIED && p->jacobian != NSWE_JAC_FULL) return NSWE_EINVAL;
  if (pr) {
    for (int l = 0; l <= first_level && l < pr->levels; ++l)
      if (!(p->eps[l] > 0.0) || !std::isfinite(p->eps[l])) return NSWE_EINVAL;
  }
  return NSWE_OK;
}

nswe_status ensure_cap(nswe_ctx ctx, int count) {
  if (count <= ctx->cap) return NSWE_OK;
  int cap = count < 64 ? 64 : count;
  SolveTask *t = nullptr;
  nswe_info *i = nullptr;
  if (cudaMalloc(&t, sizeof(SolveTask) * cap) != cudaSuccess) return NSWE_ENOMEM;
  if (cudaMalloc(&i, sizeof(nswe_info) * cap) != cudaSuccess) {
    cudaFree(t);
    return NSWE_ENOMEM;
  }
  // Buffers may still be read by queued work on the context stream.
  cudaStreamSynchronize(ctx->stream);
  cudaFree(ctx->tasks);
  cudaFree(ctx->infos);
  ctx->tasks = t;
  ctx->infos = i;
  ctx->cap = cap;
  return NSWE_OK;
}

nswe_status upload_geometry(nswe_prob p, const double *sigma_face, const double *gauss_geom,
                            const nswe_bc1d *left, const nswe_bc1d *right) {
  std::vector<double> geo(p->geo_doubles, 0.0);
  size_t off = 0;
  for (int l = 0; l < p->levels; ++l) {
    int Nl = p->N >> l;
    for (int f = 0; f <= Nl; ++f) geo[off + f] = sigma_face[(size_t)f << l];
    off += round_up(Nl + 1);
  }
  size_t src = 0;
  for (int l = 0; l < p->levels; ++l) {
    int Nl = p->N >> l;
    std::memcpy(&geo[off], gauss_geom + src, sizeof(double) * 6 * Nl);
    src += 6 * (size_t)Nl;
    off += round_up(6 * (size_t)Nl);
  }
  for (size_t i = 0; i < off; ++i)
    if (!std::isfinite(geo[i])) return NSWE_EINVAL;
  p->host.bl = left->kind;
  p->host.br = right->kind;
  p->host.blh = left->h;
  p->host.blq = left->q;
  p->host.brh = right->h;
  p->host.brq = right->q;
  cudaStream_t s = p->ctx->stream;
  if (cudaMemcpyAsync(p->arena, geo.data(), sizeof(double) * off, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return NSWE_ECUDA;
  if (cudaMemcpyAsync(p->dev, &p->host, sizeof(ProbDev), cudaMemcpyHostToDevice, s) != cudaSuccess)
    return NSWE_ECUDA;
  return NSWE_OK;
}

}  // namespace

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
  p->N = N;
  p->levels = levels;
  p->x0 = x0;
  p->x1 = x1;
  p->g = g;
  size_t geo = 0, work = 0;
  for (int l = 0; l < levels; ++l) {
    size_t Nl = (size_t)(N >> l);
    geo += round_up(Nl + 1) + round_up(6 * Nl);
    work += round_up(2 * Nl) * 3 + round_up(20 * Nl) + round_up(4 * Nl);
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

nswe_status nswe_prob_destroy(nswe_prob prob) {
  if (!prob) return NSWE_EINVAL;
  DeviceGuard dg(prob->ctx->device);
  cudaStreamSynchronize(prob->ctx->stream);
  cudaFree(prob->arena);
  cudaFree(prob->dev);
  delete prob;
  return NSWE_OK;
}

int nswe_prob_cells(nswe_prob prob, int level) {
  if (!prob || level < 0 || level >= prob->levels) return -1;
  return prob->N >> level;
}

nswe_status nswe_residual(nswe_ctx ctx, nswe_prob prob, int level, const double *U, double *R, double *res_l1) {
  if (!ctx || !prob || prob->ctx != ctx || !U || !R || level < 0 || level >= prob->levels) return NSWE_EINVAL;
  DeviceGuard dg(ctx->device);
  int N = prob->N >> level;
  return launch_residual(prob->dev, level, N, U, R, res_l1, ctx->partials, ctx->stream) == cudaSuccess
             ? NSWE_OK
             : NSWE_ECUDA;
}

static nswe_status jacobian_common(nswe_ctx ctx, nswe_prob prob, int level, int nb, const double *U, double eps,
                                   double alpha, double *R, double *J, double *res) {
  if (!ctx || !prob || prob->ctx != ctx || !U || !R || !J || level < 0 || level >= prob->levels) return NSWE_EINVAL;
  if (!(eps > 0.0) || !std::isfinite(eps) || !(alpha >= 0.0) || !std::isfinite(alpha)) return NSWE_EINVAL;
  DeviceGuard dg(ctx->device);
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

nswe_status nswe_mg_vcycle(nswe_ctx ctx, nswe_prob prob, int level, int nb, const double *J, const double *R,
                           double *dU, const nswe_params *params) {
  if (!ctx || !prob || prob->ctx != ctx || !J || !R || !dU || level < 0 || level >= prob->levels) return NSWE_EINVAL;
  if (nb != 3 && nb != 5) return NSWE_EINVAL;
  nswe_status st = check_params(params, nullptr, 0);
  if (st != NSWE_OK) return st;
  DeviceGuard dg(ctx->device);
  const int coarse = prob->N >> (prob->levels - 1);
  const int coarse_nb = (level == prob->levels - 1) ? nb : 3;
  return launch_vcycle(prob->dev, level, nb, J, R, dU, *params, ctx->status, coarse, coarse_nb, ctx->stream) ==
                 cudaSuccess
             ? NSWE_OK
             : NSWE_ECUDA;
}

nswe_status nswe_newton_solve_batch(nswe_ctx ctx, int count, const nswe_prob *probs, const double *const *U0s,
                                    double *const *Us, const nswe_params *params, nswe_info *infos) {
  if (!ctx || count < 0 || (count > 0 && (!probs || !U0s || !Us))) return NSWE_EINVAL;
  if (count == 0) return NSWE_OK;
  if (count > (1 << 20)) return NSWE_EINVAL;
  std::vector<SolveTask> tasks(count);
  for (int i = 0; i < count; ++i) {
    nswe_prob p = probs[i];
    if (!p || p->ctx != ctx || !U0s[i] || !Us[i]) return NSWE_EINVAL;
    int s0 = (params && params->nest_start >= 0 && params->nest_start < p->levels) ? params->nest_start
                                                                                     : p->levels - 1;
    nswe_status st = check_params(params, p, s0);
    if (st != NSWE_OK) return st;
  }
  DeviceGuard dg(ctx->device);
  nswe_status st = ensure_cap(ctx, count);
  if (st != NSWE_OK) return st;
  int max_coarse = 4;
  for (int i = 0; i < count; ++i) {
    const int c = probs[i]->N >> (probs[i]->levels - 1);
    if (c > max_coarse) max_coarse = c;
    tasks[i].prob = probs[i]->dev;
    tasks[i].U0 = U0s[i];
    tasks[i].U = Us[i];
    tasks[i].info = ctx->infos + i;
  }
  cudaStream_t s = ctx->stream;
  if (cudaMemcpyAsync(ctx->tasks, tasks.data(), sizeof(SolveTask) * count, cudaMemcpyHostToDevice, s) !=
      cudaSuccess)
    return NSWE_ECUDA;
  if (launch_solve(ctx->tasks, count, *params, max_coarse, s) != cudaSuccess) return NSWE_ECUDA;
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

nswe_status nswe_newton_solve(nswe_ctx ctx, nswe_prob prob, const double *U0, double *U, const nswe_params *params,
                              nswe_info *info) {
  return nswe_newton_solve_batch(ctx, 1, &prob, &U0, &U, params, info);
}

}  // extern "C"
