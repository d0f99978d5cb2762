// Allocation-free variant of the nested Newton multigrid solve.
//
// Some callers cannot call cudaMalloc: code that runs after another
// allocator (for example a framework's caching allocator) has reserved the
// device memory it is allowed to use, real-time loops that must not block on
// the implicit device synchronisation of cudaMalloc/cudaFree, or hosts that
// forbid allocation after start-up. nswe_newton_solve_noalloc serves them:
// it solves one problem with the same kernel as nswe_newton_solve, but its
// problem description and solver workspace live in one file-scope device
// array of fixed size (g_noalloc_scratch below), which every GPU that loads
// the library holds until the process exits. The caller passes the inputs
// and the output as device pointers.
//
// Host code must not take the array's name as a device address: on the host
// it is only a stand-in. The address is obtained once per device with
// cudaGetSymbolAddress, with that device current, by the first call of the
// entry point on that device; make that first call before any stream
// capture. Every call shares the array and leaves the last call's contents
// in it; calls whose work overlaps on the GPU (different streams, or several
// host threads) race on it and must be serialised by the caller. The address
// is kept for the life of the process; after cudaDeviceReset the array may
// move, so the entry point must not be used on that device again.
#include <cmath>
#include <cstring>
#include <mutex>

#include "nswe_internal.h"

using namespace nswe;

namespace {

// Workspace of a problem of up to NSWE_NOALLOC_MAX_CELLS cells: per level,
// face widths (N_l+1), U, R, dU (2 N_l each), J (20 N_l), Dinv (4 N_l),
// derived geometry (4 N_l + 2), each slot rounded to 32 doubles (below
// 35 * 2N + 7 * 32 * 16 over all levels), plus the Jacobian workspace of the
// finest level (34 N + 50) and the problem description and task (below
// 1024).
constexpr size_t kSlot = 32;
constexpr size_t kScratchDoubles =
    (35 * 2 + 34) * (size_t)NSWE_NOALLOC_MAX_CELLS + 7 * kSlot * NSWE_MAX_LEVELS + 2 * kSlot + 1024;

static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

size_t slot(size_t n) { return (n + kSlot - 1) / kSlot * kSlot; }

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double *g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on `device` (which must be current).
nswe_status scratch_address(int device, double **out) {
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_addr[device]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return NSWE_ECUDA;
    g_scratch_addr[device] = static_cast<double *>(p);
  }
  *out = g_scratch_addr[device];
  return NSWE_OK;
}

// Writes the problem description and its SolveTask record into the scratch array and
// gathers the face widths of every level from the finest ones.
__global__ void k_noalloc_setup(ProbDev P, SolveTask T, ProbDev *prob_slot, SolveTask *task_slot,
                                const double *sigma_face) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    *prob_slot = P;
    T.prob = prob_slot;
    *task_slot = T;
  }
  for (int l = 0; l < P.levels; ++l) {
    double *sf = const_cast<double *>(P.lev[l].sf);
    for (int f = threadIdx.x; f <= P.lev[l].N; f += blockDim.x) sf[f] = sigma_face[(size_t)f << l];
  }
}

}  // namespace

extern "C" nswe_status nswe_newton_solve_noalloc(int device, void *stream, int N, int levels, double x0,
                                                 double x1, double g, const double *sigma_face,
                                                 const double *gauss_geom, const nswe_bc1d *left,
                                                 const nswe_bc1d *right, const double *U0, double *U,
                                                 const nswe_params *params, nswe_info *info) {
  if (N > NSWE_NOALLOC_MAX_CELLS) return NSWE_EINVAL;  // larger than the fixed scratch array
  if (!sigma_face || !gauss_geom || !U0 || !U || !params || !left || !right) return NSWE_EINVAL;
  if (left->kind < NSWE_BC_DISCHARGE || left->kind > NSWE_BC_EXTRAP || right->kind < NSWE_BC_DISCHARGE ||
      right->kind > NSWE_BC_EXTRAP || !std::isfinite(left->h) || !std::isfinite(left->q) ||
      !std::isfinite(right->h) || !std::isfinite(right->q))
    return NSWE_EINVAL;
  if (levels < 1 || levels > NSWE_MAX_LEVELS || N < 4 || N % (1 << (levels - 1)) != 0) return NSWE_EINVAL;
  const int NL = N >> (levels - 1);
  if (NL < 4 || NL > kMaxCoarse) return NSWE_EINVAL;
  if (!(x1 > x0) || !(g > 0.0) || !std::isfinite(x0) || !std::isfinite(x1) || !std::isfinite(g))
    return NSWE_EINVAL;
  const nswe_params &p = *params;
  if (!(p.tau > 0.0 && p.tau <= 1.0) || !(p.alpha >= 0.0) || !(p.omega > 0.0 && p.omega < 2.0) ||
      !(p.tol > 0.0) || p.nu1 < 0 || p.nu2 < 0 || p.nu3 < 1 || p.n_max < 1 || p.nu1 > 1000 || p.nu2 > 1000 ||
      p.nu3 > 1000 || (p.jacobian != NSWE_JAC_SIMPLIFIED && p.jacobian != NSWE_JAC_FULL) ||
      (p.precision != NSWE_PREC_FP64 && p.precision != NSWE_PREC_MIXED))
    return NSWE_EINVAL;
  const int s0 = (p.nest_start >= 0 && p.nest_start < levels) ? p.nest_start : levels - 1;
  for (int l = 0; l <= s0; ++l)
    if (!(p.eps[l] > 0.0) || !std::isfinite(p.eps[l])) return NSWE_EINVAL;

  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev || device >= kMaxDevices)
    return NSWE_EINVAL;
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) return NSWE_ECUDA;
  if (prev != device && cudaSetDevice(device) != cudaSuccess) return NSWE_ECUDA;
  nswe_status st = NSWE_OK;
  double *base = nullptr;
  if ((st = scratch_address(device, &base)) == NSWE_OK) {
    // Carve the array: problem description and task first, then the levels.
    double *a = base;
    ProbDev *prob_slot = reinterpret_cast<ProbDev *>(a);
    a += slot((sizeof(ProbDev) + sizeof(double) - 1) / sizeof(double));
    SolveTask *task_slot = reinterpret_cast<SolveTask *>(a);
    a += slot((sizeof(SolveTask) + sizeof(double) - 1) / sizeof(double));
    ProbDev P;
    std::memset(&P, 0, sizeof(P));
    P.levels = levels;
    P.g = g;
    P.bl = left->kind;
    P.br = right->kind;
    P.blh = left->h;
    P.blq = left->q;
    P.brh = right->h;
    P.brq = right->q;
    size_t gq_off = 0;
    for (int l = 0; l < levels; ++l) {
      const size_t Nl = (size_t)(N >> l);
      LevelDev &Lv = P.lev[l];
      Lv.N = (int)Nl;
      Lv.dx = (x1 - x0) / (double)Nl;
      Lv.gq = gauss_geom + gq_off;  // the caller's array, read in place
      gq_off += 6 * Nl;
      Lv.sf = a;
      a += slot(Nl + 1);
      Lv.U = a;
      a += slot(2 * Nl);
      Lv.R = a;
      a += slot(2 * Nl);
      Lv.dU = a;
      a += slot(2 * Nl);
      Lv.J = a;
      a += slot(20 * Nl);
      Lv.Dinv = a;
      a += slot(4 * Nl);
      Lv.gd = a;
      a += slot(gd_doubles(Nl));
    }
    P.jw = a;
    a += slot(jw_doubles((size_t)N));
    if ((size_t)(a - base) > kScratchDoubles) {
      st = NSWE_EINVAL;  // cannot happen for N <= NSWE_NOALLOC_MAX_CELLS; kept as a guard
    } else {
      SolveTask T;
      T.prob = prob_slot;
      T.U0 = U0;
      T.U = U;
      T.info = info;
      T.prm = nullptr;
      T.derive = 0;
      T.done = nullptr;
      cudaStream_t s = (cudaStream_t)stream;
      k_noalloc_setup<<<1, kThreads, 0, s>>>(P, T, prob_slot, task_slot, sigma_face);
      if (cudaGetLastError() != cudaSuccess || launch_geom_derive(prob_slot, N, s) != cudaSuccess ||
          launch_solve(task_slot, 1, p, NL, s) != cudaSuccess)
        st = NSWE_ECUDA;
    }
  }
  if (prev != device) cudaSetDevice(prev);
  return st;
}
