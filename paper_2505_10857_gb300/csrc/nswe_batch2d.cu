// Lockstep batched solves of many 2D problems (Algorithm 3 for each): every
// phase of a Newton step (the FD Jacobian of Eq. 12-13, the Galerkin
// operators of Eq. 24, each colour pass of the block SOR of Eq. 22, the
// restriction and prolongation of Eq. 24-25, the coarsest direct solve, the
// update of Eq. 14 and the residual of Eq. 20) is one launch over all the
// problems of the batch, each owning a contiguous range of the launch's
// blocks. Problems of different sizes advance through their nested levels
// together: stage k runs one Newton iteration per replay on level s0_i - k of
// every problem i that has it, and a problem that meets its stopping test is
// masked off (its blocks return at once) until the stage ends, so its Newton
// iterates are exactly those of the problem solved alone. The launches of a
// stage's Newton step are captured once into a CUDA graph and replayed; the
// host reads back every problem's residual norm and flag once per replay.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "nswe_internal.h"

using namespace nswe;

namespace {

struct DevGuard {
  int prev = -1;
  explicit DevGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess || prev != dev) cudaSetDevice(dev);
    else prev = -1;
  }
  ~DevGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

unsigned long long now_ns() {
  return (unsigned long long)std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

constexpr long kJacSplitItemsHost = 65536;  // as the single-problem Jacobian launcher

// Items of one colour pass (the largest over the colours of the schedule),
// as the kernels enumerate them.
long sor_items_host(int Nx, int Ny, int st, int Kc) {
  if (Kc >= 3 && (st == ST_J9 || st == ST_P5)) return (long)((Nx + Kc - 1) / Kc) * Ny;
  if (st == ST_J9) return (long)((Nx + 2) / 3) * Ny;
  if (st == ST_P5) return (long)((Nx + 1) / 2) * Ny;
  const int P = st == ST_J21 ? 3 : 2;
  return (long)((Nx + P - 1) / P) * ((Ny + P - 1) / P);
}

// Task records of the launch groups of a stage; flatten() lays the groups
// out one after another (each group's tasks contiguous, sorted by b0).
template <typename T>
struct TaskPool {
  struct Group {
    std::vector<BTask2<T>> tasks;
    size_t first = 0;
    int blocks = 0;
  };
  std::vector<Group> groups;
  std::vector<BTask2<T>> host;
  int begin() {
    groups.emplace_back();
    return (int)groups.size() - 1;
  }
  void add(int g, BTask2<T> t, int nb) {
    t.b0 = groups[g].blocks;
    t.nb = nb;
    groups[g].blocks += nb;
    groups[g].tasks.push_back(t);
  }
  void flatten() {
    host.clear();
    for (auto &G : groups) {
      G.first = host.size();
      host.insert(host.end(), G.tasks.begin(), G.tasks.end());
    }
  }
};

template <typename T>
struct StageData {
  TaskPool<T> pool;
  TaskPool<double> pool64;  // residual tasks (FP64 arrays whatever T)
  int g_res = -1, g_jac[2][2] = {{-1, -1}, {-1, -1}}, g_f32 = -1, g_upd = -1;
  int g_direct_zero = -1, g_direct_scatter = -1, g_direct = -1;
  int g_vc_zero = -1, g_vc_scatter = -1, g_vc_lu = -1, g_zero_du = -1;
  std::vector<int> g_cop, g_dinv, g_sor, g_restrict, g_prolong;  // per depth
  std::vector<int> sor_st;                                        // stencil of each depth's passes
  int g_tail = -1;
  std::vector<Tail2<T>> tails;
  BTask2<T> *dev = nullptr;
  BTask2<double> *dev64 = nullptr;
  Tail2<T> *dev_tails = nullptr;
  Batch2Launch<T> launch(int g) const {
    if (g < 0) return Batch2Launch<T>{nullptr, 0, 0};
    const auto &G = pool.groups[g];
    return Batch2Launch<T>{dev + G.first, (int)G.tasks.size(), G.blocks};
  }
  Batch2Launch<double> launch64(int g) const {
    if (g < 0) return Batch2Launch<double>{nullptr, 0, 0};
    const auto &G = pool64.groups[g];
    return Batch2Launch<double>{dev64 + G.first, (int)G.tasks.size(), G.blocks};
  }
  ~StageData() {
    cudaFree(dev);
    cudaFree(dev64);
    cudaFree(dev_tails);
  }
};

// One colour pass of the smoothing schedule of a V-cycle level (the host
// order of smooth2 in the single-problem path): directional for the cross
// stencils with Kc >= 3, otherwise two symmetric passes of the stencil's
// own colouring with consecutive visits of a colour fused.
template <typename F>
void for_each_pass(int st, int steps, int Kc, F &&pass) {
  if (Kc >= 3 && (st == ST_J9 || st == ST_P5)) {
    for (int t = 0; t < steps; ++t)
      for (int d = 0; d < 4; ++d)
        for (int q = 0; q < Kc; ++q) pass((d % 2) + 1, Kc, d < 2 ? q : Kc - 1 - q, 1);
    return;
  }
  const int C = st_colours_host(st);
  int prev = -1, reps = 0;
  for (int t = 0; t < steps; ++t)
    for (int p = 0; p < 4 * C; ++p) {
      const int q = p % (2 * C), col = q < C ? q : 2 * C - 1 - q;
      if (col == prev) {
        ++reps;
        continue;
      }
      if (prev >= 0) pass(0, 0, prev, reps);
      prev = col;
      reps = 1;
    }
  if (prev >= 0) pass(0, 0, prev, reps);
}

// tails[i]: the tail threshold (cells) of problem i's V-cycles.
template <typename T>
nswe_status lockstep_t(nswe_ctx ctx, int count, const nswe_prob *probs, const double *const *U0s, double *const *Us,
                       const nswe_params *prms, const int *tails, bool each, nswe_info *infos) {
  constexpr bool kMixed = std::is_same<T, float>::value;
  const nswe_params &P0 = prms[0];
  const int st0 = (P0.jacobian & ~NSWE_JAC_FROZEN) == NSWE_JAC_FULL ? ST_J21 : ST_J9;
  const int K = st0 == ST_J21 ? 21 : 9;
  cudaStream_t s = ctx->stream;
  std::vector<nswe_info> rec(count);
  std::vector<int> s0(count), fatal(count, 0);
  for (int i = 0; i < count; ++i) {
    std::memset(&rec[i], 0, sizeof(nswe_info));
    const nswe_params &p = prms[each ? i : 0];
    const int L = probs[i]->levels - 1;
    s0[i] = (p.nest_start < 0 || p.nest_start > L) ? L : p.nest_start;
  }
  // batch-owned device state: mask, flags, residual norms (and pinned mirrors)
  int *done = nullptr, *flags = nullptr, *done_h = nullptr, *flags_h = nullptr;
  double *res = nullptr, *res_h = nullptr;
  cudaStream_t cap = nullptr;
  auto release = [&]() {
    cudaFree(done);
    cudaFree(flags);
    cudaFree(res);
    cudaFreeHost(done_h);
    cudaFreeHost(flags_h);
    cudaFreeHost(res_h);
    if (cap) cudaStreamDestroy(cap);
  };
  if (cudaMalloc(&done, sizeof(int) * count) || cudaMalloc(&flags, sizeof(int) * count) ||
      cudaMalloc(&res, sizeof(double) * count) || cudaMallocHost(&done_h, sizeof(int) * count) ||
      cudaMallocHost(&flags_h, sizeof(int) * count) || cudaMallocHost(&res_h, sizeof(double) * count) ||
      cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking)) {
    release();
    return NSWE_ENOMEM;
  }
  const unsigned long long t0 = now_ns();
  for (int i = 0; i < count; ++i) {
    const Level2Dev &Lv = probs[i]->host2.lev[s0[i]];
    if (cudaMemcpyAsync(Lv.U, U0s[i], sizeof(double) * 3 * Lv.Nx * Lv.Ny, cudaMemcpyDeviceToDevice, s)) {
      release();
      return NSWE_ECUDA;
    }
  }
  const int stages = 1 + *std::max_element(s0.begin(), s0.end());
  nswe_status err = NSWE_OK;
  for (int k = 0; k < stages && err == NSWE_OK; ++k) {
    std::vector<int> act, lev;
    for (int i = 0; i < count; ++i)
      if (!fatal[i] && s0[i] - k >= 0) {
        act.push_back(i);
        lev.push_back(s0[i] - k);
      }
    if (act.empty()) break;
    StageData<T> sd;
    // ---- the tasks of this stage
    sd.g_res = sd.pool64.begin();
    for (int g = 0; g < 2; ++g)
      for (int f = 0; f < 2; ++f) sd.g_jac[g][f] = sd.pool.begin();
    if (kMixed) sd.g_f32 = sd.pool.begin();
    sd.g_upd = sd.pool.begin();
    sd.g_direct_zero = sd.pool.begin();
    sd.g_direct_scatter = sd.pool.begin();
    sd.g_direct = sd.pool.begin();
    sd.g_vc_zero = sd.pool.begin();
    sd.g_vc_scatter = sd.pool.begin();
    sd.g_vc_lu = sd.pool.begin();
    sd.g_zero_du = sd.pool.begin();
    sd.g_tail = sd.pool.begin();
    int depths = 0;  // grid-wide V-cycle depths of the stage
    struct VC {
      int i, l, ls, L, cm;
    };
    std::vector<VC> vcs;
    for (size_t a = 0; a < act.size(); ++a) {
      const int i = act[a], l = lev[a];
      nswe_prob_s *p = probs[i];
      const nswe_params &prm = prms[each ? i : 0];
      const int L = p->levels - 1;
      const Level2Dev &Lv = p->host2.lev[l];
      const int n = Lv.Nx * Lv.Ny;
      const int minc = ctx->cm2d_min_cells;
      const int cm = (l < L && st0 == ST_J9 && minc >= 0 && n >= minc && n > tails[i]) ? 1 : 0;
      T *const J = reinterpret_cast<T *>(Lv.J);
      T *const dU = reinterpret_cast<T *>(Lv.dU);
      T *const Rs = kMixed ? J + (size_t)K * 9 * blk_stride(cm, Lv.Nx, Lv.Ny) : reinterpret_cast<T *>(Lv.R);
      BTask2<T> t;
      std::memset(&t, 0, sizeof(t));
      t.prob = i;
      t.Nx = Lv.Nx;
      t.Ny = Lv.Ny;
      t.st = st0;
      t.cm = cm;
      t.J = J;
      t.Dinv = reinterpret_cast<T *>(Lv.Dinv);
      t.R = Rs;
      t.dU = dU;
      t.P = p->dev2;
      t.level = l;
      t.frozen = (prm.jacobian & NSWE_JAC_FROZEN) != 0;
      t.U = Lv.U;
      t.R64 = Lv.R;
      t.partials = p->partials2;
      t.R32 = reinterpret_cast<float *>(Rs);
      t.eps = prm.eps[l];
      t.alpha = prm.alpha;
      t.tau = prm.tau;
      t.A = reinterpret_cast<T *>(p->dense);
      t.x = reinterpret_cast<T *>(p->xbuf);
      t.piv = p->piv;
      {  // residual (the block count of launch2_residual)
        BTask2<double> r;
        std::memset(&r, 0, sizeof(r));
        r.prob = i;
        r.Nx = Lv.Nx;
        r.Ny = Lv.Ny;
        r.P = p->dev2;
        r.level = l;
        r.U = Lv.U;
        r.R64 = Lv.R;
        r.partials = p->partials2;
        const int g = b2_grid(n);
        sd.pool64.add(sd.g_res, r, g > 1024 ? 1024 : g);
      }
      {  // Jacobian: one cell per thread on large levels, else one (cell, block) item
        const bool cells = ctx->jac2d_cell_min >= 0 && n >= ctx->jac2d_cell_min;
        BTask2<T> j = t;
        int nb;
        if (cells) {
          const int th = b2_jacobian_cell_threads();
          nb = (n + th - 1) / th;
        } else {
          const long items = (long)n * K;
          j.msplit = 3 * items <= kJacSplitItemsHost ? 1 : 0;
          nb = b2_grid(items * (j.msplit ? 3 : 1));
        }
        sd.pool.add(sd.g_jac[cells ? 1 : 0][t.frozen ? 1 : 0], j, nb);
      }
      if (kMixed) sd.pool.add(sd.g_f32, t, b2_grid(3L * n));
      sd.pool.add(sd.g_upd, t, b2_grid(n));
      if (l == L) {  // Newton on the coarsest grid: dense LU of the regularized system
        const long N3 = 3L * n;
        sd.pool.add(sd.g_direct_zero, t, b2_grid(N3 * N3));
        sd.pool.add(sd.g_direct_scatter, t, b2_grid((long)n * K));
        sd.pool.add(sd.g_direct, t, 1);
        continue;
      }
      // V-cycles: the first level of at most tails[i] cells starts the tail
      int ls = L;
      for (int m = l; m < L; ++m)
        if (p->host2.lev[m].Nx * p->host2.lev[m].Ny <= tails[i]) {
          ls = m;
          break;
        }
      vcs.push_back({i, l, ls, L, cm});
      depths = std::max(depths, ls - l);
    }
    sd.g_cop.resize(16);
    for (int d = 0; d < 16; ++d) sd.g_cop[d] = sd.pool.begin();
    sd.g_dinv.resize(16);
    for (int d = 0; d < 16; ++d) sd.g_dinv[d] = sd.pool.begin();
    sd.g_sor.resize(16);
    for (int d = 0; d < 16; ++d) sd.g_sor[d] = sd.pool.begin();
    sd.g_restrict.resize(16);
    for (int d = 0; d < 16; ++d) sd.g_restrict[d] = sd.pool.begin();
    sd.g_prolong.resize(16);
    for (int d = 0; d < 16; ++d) sd.g_prolong[d] = sd.pool.begin();
    sd.sor_st.assign(16, st0);
    for (int d = 1; d < 16; ++d) sd.sor_st[d] = st_coarse_host(sd.sor_st[d - 1]);
    for (const VC &v : vcs) {
      nswe_prob_s *p = probs[v.i];
      const nswe_params &prm = prms[each ? v.i : 0];
      (void)prm;
      int st = st0;
      for (int m = v.l; m <= v.L; ++m) {
        const int d = m - v.l;
        const Level2Dev &Lm = p->host2.lev[m];
        const int n = Lm.Nx * Lm.Ny;
        BTask2<T> t;
        std::memset(&t, 0, sizeof(t));
        t.prob = v.i;
        t.Nx = Lm.Nx;
        t.Ny = Lm.Ny;
        t.st = st;
        t.cm = d == 0 ? v.cm : 0;
        if (d == 0) {
          const Level2Dev &Lv = p->host2.lev[v.l];
          t.J = reinterpret_cast<T *>(Lv.J);
          t.R = kMixed ? t.J + (size_t)K * 9 * blk_stride(v.cm, Lv.Nx, Lv.Ny) : reinterpret_cast<T *>(Lv.R);
        } else {
          t.J = reinterpret_cast<T *>(Lm.J);
          t.R = reinterpret_cast<T *>(Lm.R);
        }
        t.Dinv = reinterpret_cast<T *>(Lm.Dinv);
        t.dU = reinterpret_cast<T *>(Lm.dU);
        if (m < v.L) {
          const Level2Dev &Lc = p->host2.lev[m + 1];
          t.Jc = reinterpret_cast<T *>(Lc.J);
          t.Rc = reinterpret_cast<T *>(Lc.R);
          t.dUc = reinterpret_cast<T *>(Lc.dU);
        }
        t.A = reinterpret_cast<T *>(p->dense);
        t.x = reinterpret_cast<T *>(p->xbuf);
        t.piv = p->piv;
        if (m < v.L) {
          sd.pool.add(sd.g_cop[d], t, b2_grid((long)(Lm.Nx / 2) * (Lm.Ny / 2)));
          sd.pool.add(sd.g_dinv[d], t, b2_grid(n));
        } else {  // the coarsest: dense factors
          const long N3 = 3L * n;
          sd.pool.add(sd.g_vc_zero, t, b2_grid(N3 * N3));
          sd.pool.add(sd.g_vc_scatter, t, b2_grid((long)n * st_size_host(st)));
          sd.pool.add(sd.g_vc_lu, t, 1);
        }
        if (d == 0) sd.pool.add(sd.g_zero_du, t, b2_grid(3L * n));
        if (m < v.ls) {
          const long items = sor_items_host(Lm.Nx, Lm.Ny, st, P0.colours2d);
          sd.pool.add(sd.g_sor[d], t, (int)((items + kB2SorCellsPerBlock - 1) / kB2SorCellsPerBlock));
          sd.pool.add(sd.g_restrict[d], t, b2_grid((long)(Lm.Nx / 2) * (Lm.Ny / 2)));
          sd.pool.add(sd.g_prolong[d], t, b2_grid(n));
        }
        st = st_coarse_host(st);
      }
      // the tail of this problem's V-cycle (one block)
      Tail2<T> tl;
      std::memset(&tl, 0, sizeof(tl));
      tl.ls = v.ls;
      tl.L = v.L;
      int stl = st0;
      for (int m = v.l; m <= v.L; ++m) {
        if (m >= v.ls) {
          const Level2Dev &Lm = p->host2.lev[m];
          tl.Nx[m] = Lm.Nx;
          tl.Ny[m] = Lm.Ny;
          tl.st[m] = stl;
          if (m == v.l) {
            const Level2Dev &Lv = p->host2.lev[v.l];
            tl.J[m] = reinterpret_cast<T *>(Lv.J);
            tl.R[m] = kMixed ? tl.J[m] + (size_t)K * 9 * blk_stride(v.cm, Lv.Nx, Lv.Ny) : reinterpret_cast<T *>(Lv.R);
          } else {
            tl.J[m] = reinterpret_cast<T *>(Lm.J);
            tl.R[m] = reinterpret_cast<T *>(Lm.R);
          }
          tl.Dinv[m] = reinterpret_cast<T *>(Lm.Dinv);
          tl.dU[m] = reinterpret_cast<T *>(Lm.dU);
        }
        stl = st_coarse_host(stl);
      }
      tl.A = reinterpret_cast<const T *>(p->dense);
      tl.piv = p->piv;
      tl.x = reinterpret_cast<T *>(p->xbuf);
      BTask2<T> tt;
      std::memset(&tt, 0, sizeof(tt));
      tt.prob = v.i;
      sd.pool.add(sd.g_tail, tt, 1);
      sd.tails.push_back(tl);
    }
    // ---- upload the task tables
    sd.pool.flatten();
    sd.pool64.flatten();
    const size_t nt = sd.pool.host.size(), nt64 = sd.pool64.host.size();
    if ((nt && cudaMalloc(&sd.dev, sizeof(BTask2<T>) * nt)) || (nt64 && cudaMalloc(&sd.dev64, sizeof(BTask2<double>) * nt64)) ||
        (!sd.tails.empty() && cudaMalloc(&sd.dev_tails, sizeof(Tail2<T>) * sd.tails.size()))) {
      err = NSWE_ENOMEM;
      break;
    }
    if ((nt && cudaMemcpyAsync(sd.dev, sd.pool.host.data(), sizeof(BTask2<T>) * nt, cudaMemcpyHostToDevice, s)) ||
        (nt64 && cudaMemcpyAsync(sd.dev64, sd.pool64.host.data(), sizeof(BTask2<double>) * nt64,
                                 cudaMemcpyHostToDevice, s)) ||
        (!sd.tails.empty() && cudaMemcpyAsync(sd.dev_tails, sd.tails.data(), sizeof(Tail2<T>) * sd.tails.size(),
                                              cudaMemcpyHostToDevice, s))) {
      err = NSWE_ECUDA;
      break;
    }
    // ---- interpolation to this stage's levels, and their residuals
    for (size_t a = 0; a < act.size() && k > 0; ++a) {
      nswe_prob_s *p = probs[act[a]];
      const int l = lev[a];
      if (launch2_interp(p->dev2, l + 1, p->host2.lev[l + 1].Nx * p->host2.lev[l + 1].Ny, p->host2.lev[l + 1].U,
                         p->host2.lev[l].U, s)) {
        err = NSWE_ECUDA;
        break;
      }
    }
    if (err) break;
    for (int i = 0; i < count; ++i) done_h[i] = 1;
    for (int i : act) done_h[i] = 0;
    if (cudaMemcpyAsync(done, done_h, sizeof(int) * count, cudaMemcpyHostToDevice, s) ||
        launchb2_residual(sd.launch64(sd.g_res), done, res, s)) {
      err = NSWE_ECUDA;
      break;
    }
    // ---- one batched Newton step, captured
    const double omega = P0.omega;
    const int Kc = P0.colours2d;
    auto step = [&](cudaStream_t q) -> cudaError_t {
      cudaError_t e;
      if ((e = cudaMemcpyAsync(done, done_h, sizeof(int) * count, cudaMemcpyHostToDevice, q))) return e;
      if ((e = cudaMemsetAsync(flags, 0, sizeof(int) * count, q))) return e;
      for (int g = 0; g < 2; ++g)
        for (int f = 0; f < 2; ++f)
          if ((e = launchb2_jacobian<T>(sd.launch(sd.g_jac[g][f]), done, g ? kB2JacCells : kB2JacItems, f == 1, q)))
            return e;
      if constexpr (kMixed) {
        if ((e = launchb2_to_f32(sd.launch(sd.g_f32), done, q))) return e;
      }
      // Newton on the coarsest grid
      const auto dz = sd.launch(sd.g_direct);
      if ((e = launchb2_dense_factor<T>(sd.launch(sd.g_direct_zero), sd.launch(sd.g_direct_scatter), dz.tasks,
                                        dz.ntask, done, flags, q)) ||
          (e = launchb2_dense_solve<T>(dz.tasks, dz.ntask, done, q)))
        return e;
      // V-cycles: Galerkin operators and inverse diagonal blocks, coarsest factors, then nu3 cycles
      for (int d = 0; d < 16; ++d)
        if ((e = launchb2_coarse_op<T>(sd.launch(sd.g_cop[d]), done, q))) return e;
      for (int d = 0; d < 16; ++d)
        if ((e = launchb2_dinv<T>(sd.launch(sd.g_dinv[d]), done, q))) return e;
      const auto lu = sd.launch(sd.g_vc_lu);
      if ((e = launchb2_dense_factor<T>(sd.launch(sd.g_vc_zero), sd.launch(sd.g_vc_scatter), lu.tasks, lu.ntask,
                                        done, flags, q)))
        return e;
      if ((e = launchb2_zero_du<T>(sd.launch(sd.g_zero_du), done, q))) return e;
      const auto tail = sd.launch(sd.g_tail);
      for (int v = 0; v < P0.nu3; ++v) {
        for (int d = 0; d < depths; ++d) {
          const auto b = sd.launch(sd.g_sor[d]);
          for_each_pass(sd.sor_st[d], P0.nu1, Kc, [&](int mode, int kc, int col, int reps) {
            if (!e) e = launchb2_sor<T>(b, done, sd.sor_st[d], omega, mode, kc, col, reps, q);
          });
          if (e || (e = launchb2_restrict<T>(sd.launch(sd.g_restrict[d]), done, q))) return e;
        }
        if ((e = launchb2_vcycle_tail<T>(sd.dev_tails, tail.tasks, tail.ntask, done, P0.nu1, P0.nu2, omega, Kc, q)))
          return e;
        for (int d = depths - 1; d >= 0; --d) {
          if ((e = launchb2_prolong<T>(sd.launch(sd.g_prolong[d]), done, q))) return e;
          const auto b = sd.launch(sd.g_sor[d]);
          for_each_pass(sd.sor_st[d], P0.nu2, Kc, [&](int mode, int kc, int col, int reps) {
            if (!e) e = launchb2_sor<T>(b, done, sd.sor_st[d], omega, mode, kc, col, reps, q);
          });
          if (e) return e;
        }
      }
      if ((e = launchb2_update<T>(sd.launch(sd.g_upd), done, flags, q))) return e;
      if ((e = launchb2_residual(sd.launch64(sd.g_res), done, res, q))) return e;
      if ((e = cudaMemcpyAsync(res_h, res, sizeof(double) * count, cudaMemcpyDeviceToHost, q))) return e;
      return cudaMemcpyAsync(flags_h, flags, sizeof(int) * count, cudaMemcpyDeviceToHost, q);
    };
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    if (cudaStreamSynchronize(s) != cudaSuccess ||
        cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      err = NSWE_ECUDA;
      break;
    }
    const cudaError_t ce = step(cap);
    if (cudaStreamEndCapture(cap, &graph) != cudaSuccess || ce != cudaSuccess ||
        cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      err = NSWE_ECUDA;
      break;
    }
    cudaGraphDestroy(graph);
    std::vector<int> it(count, 0);
    std::vector<double> last(count, 0.0);
    int open = (int)act.size();
    while (open > 0) {
      if (cudaGraphLaunch(exec, s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
        err = NSWE_ECUDA;
        break;
      }
      const unsigned long long tnow = now_ns();
      for (size_t a = 0; a < act.size(); ++a) {
        const int i = act[a], l = lev[a];
        if (done_h[i]) continue;
        const nswe_params &prm = prms[each ? i : 0];
        const int L = probs[i]->levels - 1;
        if (l != L) rec[i].vcycles += prm.nu3;
        const double r = res_h[i];
        ++it[i];
        int st = -1;
        if (flags_h[i]) st = NSWE_ENEGDEPTH;
        else if (!(r == r) || std::isinf(r)) st = NSWE_ENAN;
        else if (r < prm.tol) st = NSWE_OK;
        else if (it[i] >= prm.n_max) st = NSWE_ENOTCONV;
        if (st < 0) continue;
        done_h[i] = 1;
        --open;
        rec[i].iters[l] = it[i];
        rec[i].res[l] = r;
        rec[i].level_status[l] = st;
        rec[i].total_iters += it[i];
        if (st == NSWE_ENAN || st == NSWE_ENEGDEPTH) fatal[i] = st;
        if (l == 0 || fatal[i]) rec[i].t_end_ns = tnow;
      }
    }
    cudaGraphExecDestroy(exec);
  }
  // results and records
  if (err == NSWE_OK) {
    for (int i = 0; i < count; ++i) {
      nswe_prob_s *p = probs[i];
      if (!fatal[i] && cudaMemcpyAsync(Us[i], p->host2.lev[0].U, sizeof(double) * 3 * p->Nx * p->Ny,
                                       cudaMemcpyDeviceToDevice, s)) {
        err = NSWE_ECUDA;
        break;
      }
    }
  }
  if (err == NSWE_OK && cudaStreamSynchronize(s) != cudaSuccess) err = NSWE_ECUDA;
  release();
  if (err != NSWE_OK) return err;
  int worst = NSWE_OK;
  for (int i = 0; i < count; ++i) {
    rec[i].status = fatal[i] ? fatal[i] : rec[i].level_status[0];
    rec[i].t_start_ns = t0;
    if (!rec[i].t_end_ns) rec[i].t_end_ns = now_ns();
    if (infos) infos[i] = rec[i];
    if (rec[i].status != NSWE_OK && worst == NSWE_OK) worst = rec[i].status;
  }
  return (nswe_status)worst;
}

// Problems that can share lockstep launches: the same precision, Jacobian
// stencil and smoothing schedule (the colour passes of a launch are common).
bool same_group(const nswe_params &a, const nswe_params &b) {
  return a.precision == b.precision &&
         ((a.jacobian & ~NSWE_JAC_FROZEN) == NSWE_JAC_FULL) == ((b.jacobian & ~NSWE_JAC_FROZEN) == NSWE_JAC_FULL) &&
         a.nu1 == b.nu1 && a.nu2 == b.nu2 && a.nu3 == b.nu3 && a.omega == b.omega && a.colours2d == b.colours2d;
}

}  // namespace

namespace nswe {

nswe_status solve2d_lockstep(nswe_ctx ctx, int count, const nswe_prob *probs, const double *const *U0s,
                             double *const *Us, const nswe_params *prms, bool each, nswe_info *infos) {
  DevGuard dg(ctx->device);
  // each problem's schedule and tail threshold (colours2d = AUTO resolved per size)
  std::vector<nswe_params> res(count);
  std::vector<int> tail(count);
  for (int i = 0; i < count; ++i) resolve2d(probs[i], prms[each ? i : 0], res[i], tail[i]);
  std::vector<int> group(count, -1);
  int ngroups = 0;
  std::vector<int> rep;
  for (int i = 0; i < count; ++i) {
    for (int g = 0; g < ngroups && group[i] < 0; ++g)
      if (same_group(res[rep[g]], res[i])) group[i] = g;
    if (group[i] < 0) {
      group[i] = ngroups++;
      rep.push_back(i);
    }
  }
  int worst = NSWE_OK;
  for (int g = 0; g < ngroups; ++g) {
    std::vector<nswe_prob> pg;
    std::vector<const double *> u0g;
    std::vector<double *> ug;
    std::vector<nswe_params> prg;
    std::vector<int> idx, tg;
    for (int i = 0; i < count; ++i)
      if (group[i] == g) {
        pg.push_back(probs[i]);
        u0g.push_back(U0s[i]);
        ug.push_back(Us[i]);
        prg.push_back(res[i]);
        tg.push_back(tail[i]);
        idx.push_back(i);
      }
    std::vector<nswe_info> ig(pg.size());
    const bool mixed = prg[0].precision == NSWE_PREC_MIXED;
    const nswe_status st = mixed ? lockstep_t<float>(ctx, (int)pg.size(), pg.data(), u0g.data(), ug.data(),
                                                     prg.data(), tg.data(), true, ig.data())
                                 : lockstep_t<double>(ctx, (int)pg.size(), pg.data(), u0g.data(), ug.data(),
                                                      prg.data(), tg.data(), true, ig.data());
    if (st == NSWE_ECUDA || st == NSWE_ENOMEM) return st;
    for (size_t a = 0; a < idx.size(); ++a)
      if (infos) infos[idx[a]] = ig[a];
    if (st != NSWE_OK && worst == NSWE_OK) worst = st;
  }
  return (nswe_status)worst;
}

}  // namespace nswe
