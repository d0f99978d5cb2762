// Continuous-batching solve server for 1D problems.
//
// A request is one nested Newton-multigrid solve (Algorithm 3) of a 1D
// problem given by host arrays. The server keeps each admitted solve's
// problem description, geometry and Newton/multigrid workspace resident in
// one block of a device arena whose size the caller fixes, so a request is
// admitted only when its footprint fits (first come, first served). Admitted
// requests are launched together, one thread block each, on whichever of the
// server's streams is idle; launches on different streams run concurrently,
// so requests arriving while others are being solved start without waiting
// for them. Results come back through pinned host memory, with host
// timestamps of submission, admission, launch and completion.
//
// One scheduler thread per server issues every CUDA call of the server's 1D
// work; the public calls only exchange requests and results with it under a
// mutex.
//
// 2D requests go to a pool of worker threads instead, each with its own
// stream and context: a 2D Newton step is sequenced from the host, so one
// solve keeps one host thread. A worker takes the oldest 2D request once its
// footprint fits in the 2D budget beside the solves in flight, builds the
// problem, solves it and files the result with the same tickets.
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <iterator>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "nswe_internal.h"

using namespace nswe;

// ----------------------------------------------------------------------------
// First-fit arena over [0, size): offsets aligned to `align`, freed blocks
// coalesced with their free neighbours.
struct nswe_arena_s {
  size_t size = 0, align = 256, used = 0, peak = 0;
  std::map<size_t, size_t> free_blocks;  // offset -> length
  std::unordered_map<size_t, size_t> live;  // offset -> length

  bool alloc(size_t bytes, size_t *off) {
    if (bytes == 0) bytes = 1;
    const size_t need = (bytes + align - 1) / align * align;
    for (auto it = free_blocks.begin(); it != free_blocks.end(); ++it) {
      if (it->second < need) continue;
      const size_t o = it->first, len = it->second;
      free_blocks.erase(it);
      if (len > need) free_blocks[o + need] = len - need;
      live[o] = need;
      used += need;
      if (used > peak) peak = used;
      *off = o;
      return true;
    }
    return false;
  }
  bool release(size_t off) {
    auto it = live.find(off);
    if (it == live.end()) return false;
    size_t o = off, len = it->second;
    live.erase(it);
    used -= len;
    auto next = free_blocks.lower_bound(o);
    if (next != free_blocks.end() && o + len == next->first) {
      len += next->second;
      next = free_blocks.erase(next);
    }
    if (next != free_blocks.begin()) {
      auto prev = std::prev(next);
      if (prev->first + prev->second == o) {
        prev->second += len;
        return true;
      }
    }
    free_blocks[o] = len;
    return true;
  }
  size_t largest_free() const {
    size_t m = 0;
    for (const auto &b : free_blocks) m = b.second > m ? b.second : m;
    return m;
  }
};

namespace {

size_t rdup(size_t n, size_t a) { return (n + a - 1) / a * a; }
constexpr size_t kSlotBytes = 256;
size_t slot_bytes(size_t bytes) { return rdup(bytes, kSlotBytes); }

uint64_t now_ns() {
  return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

// Byte layout of one request. Device block: problem description,
// parameters, geometry and initial guess (the upload part, copied from a
// pinned mirror in one transfer), then the workspace. Host block (pinned,
// mapped into the device address space): the upload mirror, then the result
// part the solve kernel writes directly: record, solution, completion flag.
struct Layout {
  size_t prob, prm, geo, u0, work, jw;  // device byte offsets
  size_t up_bytes, dev_total;
  size_t info, uout, flag, host_total;  // host byte offsets (after the mirror)
  size_t geo_doubles;
};

Layout layout_1d(int N, int levels, int s0) {
  Layout L;
  size_t o = 0;
  L.prob = o;
  o += slot_bytes(sizeof(ProbDev));
  L.prm = o;
  o += slot_bytes(sizeof(nswe_params));
  L.geo = o;
  size_t geo = 0;
  for (int l = 0; l < levels; ++l) geo += rdup((size_t)(N >> l) + 1, 32) + rdup(6 * (size_t)(N >> l), 32);
  L.geo_doubles = geo;
  o += slot_bytes(geo * sizeof(double));
  L.u0 = o;
  o += slot_bytes(2 * (size_t)(N >> s0) * sizeof(double));
  L.up_bytes = o;
  L.work = o;
  for (int l = 0; l < levels; ++l) {
    const size_t Nl = (size_t)(N >> l);
    o += slot_bytes(2 * Nl * sizeof(double)) * 3 + slot_bytes(20 * Nl * sizeof(double)) +
         slot_bytes(4 * Nl * sizeof(double)) + slot_bytes(gd_doubles(Nl) * sizeof(double));
  }
  L.jw = o;
  o += slot_bytes(jw_doubles((size_t)N) * sizeof(double));
  L.dev_total = o;
  size_t h = L.up_bytes;
  L.info = h;
  h += slot_bytes(sizeof(nswe_info));
  L.uout = h;
  h += slot_bytes(2 * (size_t)N * sizeof(double));
  L.flag = h;
  h += slot_bytes(sizeof(int));
  L.host_total = h;
  return L;
}

struct Request {
  unsigned long long ticket = 0;
  int dim = 1;
  int N = 0, levels = 0, s0 = 0;
  // 2D: grid, domain, boundary kinds and states, footprint
  int Nx = 0, Ny = 0;
  double y0 = 0, y1 = 0;
  std::vector<int> kinds;
  double bcs[12] = {};
  size_t foot2d = 0;
  double x0 = 0, x1 = 0, g = 0;
  nswe_bc1d left{}, right{};
  nswe_params prm{};
  std::vector<double> sf, gq, u0;  // host copies made at submission
  Layout lay{};
  size_t dev_off = 0, host_off = 0;
  int stream = -1;
  nswe_server_times times{};
  nswe_info info{};
  int status = NSWE_OK;
  std::vector<double> U;  // result
};

// A launch in flight on one stream. Its requests are tracked in the server's
// running list only: a finished request may be taken (and deleted) by the
// caller before the launch's other solves end.
struct Batch {
  bool busy = false;
};

}  // namespace

struct nswe_server_s {
  int device = 0;
  nswe_server_config cfg{};
  // latency form (nswe_server_set_cluster): a 1D launch runs one problem per
  // cluster of cl_ctas CTAs when the 1D solves in flight, its own included,
  // are at most cl_max (cl_ctas 1: never)
  std::atomic<int> cl_ctas{1}, cl_max{0}, cl_team_cells{1024};
  char *dev_base = nullptr;
  char *host_base = nullptr;      // pinned, mapped
  char *host_base_dev = nullptr;  // its device address
  nswe_arena_s dev_arena, host_arena;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> events;
  std::vector<SolveTask *> task_dev;  // per stream [max_batch]
  std::vector<SolveTask *> task_host;  // pinned mirrors
  std::vector<Batch> batches;

  std::mutex mu;
  std::condition_variable cv;
  std::deque<Request *> submitted, waiting;
  std::unordered_map<unsigned long long, Request *> done;
  std::deque<unsigned long long> completed;
  unsigned long long next_ticket = 1;
  std::atomic<bool> stop{false};
  std::atomic<int> error{NSWE_OK};
  nswe_server_stats stats{};
  std::thread worker;

  std::vector<Request *> running;  // launched, not yet finished

  // 2D requests
  std::deque<Request *> waiting2d;
  size_t used2d = 0;  // footprints of the 2D solves in flight
  std::condition_variable cv2;
  std::vector<std::thread> workers2d;

  void run();
  void run2d();
  bool admit_and_launch(int s);
  bool finish_requests();
  bool release_stream(int s);
  void fill_upload(Request *r, char *h, char *d);
};

namespace {

// ProbDev of a request whose block starts at device address d.
ProbDev prob_of(const Request &r, char *d) {
  ProbDev P;
  std::memset(&P, 0, sizeof(P));
  P.levels = r.levels;
  P.g = r.g;
  P.bl = r.left.kind;
  P.br = r.right.kind;
  P.blh = r.left.h;
  P.blq = r.left.q;
  P.brh = r.right.h;
  P.brq = r.right.q;
  double *geo = reinterpret_cast<double *>(d + r.lay.geo);
  char *w = d + r.lay.work;
  for (int l = 0; l < r.levels; ++l) {
    const size_t Nl = (size_t)(r.N >> l);
    LevelDev &Lv = P.lev[l];
    Lv.N = (int)Nl;
    Lv.dx = (r.x1 - r.x0) / (double)Nl;
    Lv.sf = geo;
    geo += rdup(Nl + 1, 32);
  }
  for (int l = 0; l < r.levels; ++l) {
    const size_t Nl = (size_t)(r.N >> l);
    P.lev[l].gq = geo;
    geo += rdup(6 * Nl, 32);
  }
  for (int l = 0; l < r.levels; ++l) {
    const size_t Nl = (size_t)(r.N >> l);
    LevelDev &Lv = P.lev[l];
    auto take = [&](size_t doubles) {
      double *p = reinterpret_cast<double *>(w);
      w += slot_bytes(doubles * sizeof(double));
      return p;
    };
    Lv.U = take(2 * Nl);
    Lv.R = take(2 * Nl);
    Lv.dU = take(2 * Nl);
    Lv.J = take(20 * Nl);
    Lv.Dinv = take(4 * Nl);
    Lv.gd = take(gd_doubles(Nl));
  }
  P.jw = reinterpret_cast<double *>(d + r.lay.jw);
  return P;
}

}  // namespace

// Writes the upload part of request r into its pinned mirror h (device block
// at d).
void nswe_server_s::fill_upload(Request *r, char *h, char *d) {
  ProbDev P = prob_of(*r, d);
  std::memcpy(h + r->lay.prob, &P, sizeof(P));
  std::memcpy(h + r->lay.prm, &r->prm, sizeof(nswe_params));
  double *geo = reinterpret_cast<double *>(h + r->lay.geo);
  std::memset(geo, 0, r->lay.geo_doubles * sizeof(double));
  size_t off = 0;
  for (int l = 0; l < r->levels; ++l) {
    const int Nl = r->N >> l;
    for (int f = 0; f <= Nl; ++f) geo[off + f] = r->sf[(size_t)f << l];
    off += rdup((size_t)Nl + 1, 32);
  }
  size_t src = 0;
  for (int l = 0; l < r->levels; ++l) {
    const size_t Nl = (size_t)(r->N >> l);
    std::memcpy(geo + off, r->gq.data() + src, sizeof(double) * 6 * Nl);
    src += 6 * Nl;
    off += rdup(6 * Nl, 32);
  }
  std::memcpy(h + r->lay.u0, r->u0.data(), sizeof(double) * r->u0.size());
}

// Admits waiting requests (first come, first served, one precision per
// launch) and launches them on idle stream s. Returns true if it launched.
bool nswe_server_s::admit_and_launch(int s) {
  Batch &b = batches[s];
  std::vector<Request *> take;
  {
    std::lock_guard<std::mutex> lk(mu);
    if (waiting.empty()) return false;
    // Batching window: hold a launch that would not be full until its
    // oldest request has waited batch_window_s.
    if (cfg.batch_window_s > 0.0 && (int)waiting.size() < cfg.max_batch &&
        (double)(now_ns() - waiting.front()->times.t_submit_ns) < cfg.batch_window_s * 1e9)
      return false;
    while (!waiting.empty() && (int)take.size() < cfg.max_batch) {
      Request *r = waiting.front();
      if (!take.empty() && r->prm.precision != take[0]->prm.precision) break;
      size_t doff = 0, hoff = 0;
      if (!dev_arena.alloc(r->lay.dev_total, &doff)) break;
      if (!host_arena.alloc(r->lay.host_total, &hoff)) {
        dev_arena.release(doff);
        break;
      }
      r->dev_off = doff;
      r->host_off = hoff;
      r->times.t_admit_ns = now_ns();
      waiting.pop_front();
      take.push_back(r);
    }
    stats.device_bytes_used = dev_arena.used;
    stats.device_bytes_peak = dev_arena.peak;
    stats.waiting = (int)waiting.size();
  }
  if (take.empty()) return false;
  cudaStream_t st = streams[s];
  int max_coarse = 4, max_nb = 3;
  for (size_t i = 0; i < take.size(); ++i) {
    Request *r = take[i];
    char *d = dev_base + r->dev_off, *h = host_base + r->host_off;
    fill_upload(r, h, d);
    if (cudaMemcpyAsync(d, h, r->lay.up_bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) {
      error = NSWE_ECUDA;
      return false;
    }
    char *hd = host_base_dev + r->host_off;  // the host block as the device sees it
    *reinterpret_cast<volatile int *>(h + r->lay.flag) = 0;
    SolveTask &t = task_host[s][i];
    t.prob = reinterpret_cast<const ProbDev *>(d + r->lay.prob);
    t.U0 = reinterpret_cast<const double *>(d + r->lay.u0);
    t.U = reinterpret_cast<double *>(hd + r->lay.uout);
    t.info = reinterpret_cast<nswe_info *>(hd + r->lay.info);
    t.prm = reinterpret_cast<const nswe_params *>(d + r->lay.prm);
    t.derive = 1;
    t.done = reinterpret_cast<int *>(hd + r->lay.flag);
    r->stream = s;
    const int c = r->N >> (r->levels - 1);
    if (c > max_coarse) max_coarse = c;
    if (r->prm.jacobian == NSWE_JAC_FULL) max_nb = 5;
  }
  const int n = (int)take.size();
  nswe_params launch = take[0]->prm;
  const uint64_t tl = now_ns();
  const int ctas = cl_ctas.load();
  const bool cluster = ctas > 1 && (int)(running.size() + take.size()) <= cl_max.load();
  if (cudaMemcpyAsync(task_dev[s], task_host[s], sizeof(SolveTask) * n, cudaMemcpyHostToDevice, st) !=
          cudaSuccess ||
      (cluster ? launch_solve_cluster(task_dev[s], n, launch, max_coarse, max_nb, ctas, cl_team_cells.load(), st)
               : launch_solve_sized(task_dev[s], n, launch, max_coarse, max_nb,
                                    launch.precision == NSWE_PREC_MIXED ? kServerShapeMixed : kServerShapeFp64,
                                    st)) != cudaSuccess) {
    error = NSWE_ECUDA;
    return false;
  }
  for (Request *r : take) r->times.t_launch_ns = tl;
  if (cudaEventRecord(events[s], st) != cudaSuccess) {
    error = NSWE_ECUDA;
    return false;
  }
  running.insert(running.end(), take.begin(), take.end());
  b.busy = true;
  {
    std::lock_guard<std::mutex> lk(mu);
    stats.launches += 1;
    stats.running += n;
  }
  return true;
}

// Completes every running request whose solve has raised its flag: the
// record and the solution are already in its pinned block. Its device and
// host blocks return to the arenas at once (the solve no longer touches
// them), while the launch's other solves may still run.
bool nswe_server_s::finish_requests() {
  std::vector<Request *> fin;
  for (size_t i = 0; i < running.size();) {
    Request *r = running[i];
    const char *h = host_base + r->host_off;
    if (*reinterpret_cast<const volatile int *>(h + r->lay.flag) != 0) {
      fin.push_back(r);
      running[i] = running.back();
      running.pop_back();
    } else {
      ++i;
    }
  }
  if (fin.empty()) return false;
  // The flag was read before the data it publishes (weakly ordered hosts).
  std::atomic_thread_fence(std::memory_order_acquire);
  const uint64_t td = now_ns();
  std::lock_guard<std::mutex> lk(mu);
  for (Request *r : fin) {
    const char *h = host_base + r->host_off;
    std::memcpy(&r->info, h + r->lay.info, sizeof(nswe_info));
    r->status = r->info.status;
    r->U.resize(2 * (size_t)r->N);
    std::memcpy(r->U.data(), h + r->lay.uout, sizeof(double) * 2 * r->N);
    r->times.t_done_ns = td;
    dev_arena.release(r->dev_off);
    host_arena.release(r->host_off);
    done[r->ticket] = r;
    completed.push_back(r->ticket);
  }
  stats.running -= (int)fin.size();
  stats.completed += (int)fin.size();
  stats.device_bytes_used = dev_arena.used;
  cv.notify_all();
  return true;
}

// Frees stream s once its launch has ended; a solve of that launch without a
// raised flag by then means the launch failed.
bool nswe_server_s::release_stream(int s) {
  Batch &b = batches[s];
  if (!b.busy) return false;
  const cudaError_t q = cudaEventQuery(events[s]);
  if (q == cudaErrorNotReady) return false;
  if (q != cudaSuccess) {
    error = NSWE_ECUDA;
    return false;
  }
  finish_requests();
  for (Request *r : running)
    if (r->stream == s) error = NSWE_ECUDA;  // launch ended without this solve's flag
  b.busy = false;
  return true;
}

void nswe_server_s::run() {
  if (cudaSetDevice(device) != cudaSuccess) {
    error = NSWE_ECUDA;
    return;
  }
  while (!stop.load() && error.load() == NSWE_OK) {
    bool progress = false;
    {
      std::lock_guard<std::mutex> lk(mu);
      while (!submitted.empty()) {
        waiting.push_back(submitted.front());
        submitted.pop_front();
      }
    }
    progress |= finish_requests();
    for (int s = 0; s < (int)streams.size(); ++s) progress |= release_stream(s);
    for (int s = 0; s < (int)streams.size(); ++s)
      if (!batches[s].busy) progress |= admit_and_launch(s);
    if (!progress) {
      std::unique_lock<std::mutex> lk(mu);
      cv.wait_for(lk, std::chrono::microseconds(50), [&] { return stop.load() || !submitted.empty(); });
    }
  }
  // Let launched work finish before the streams go away.
  for (cudaStream_t st : streams) cudaStreamSynchronize(st);
}

extern "C" {

namespace {

// Builds request r's 2D problem on ctx (stream s), runs its nested solve and
// copies the result into r->U; the problem and the buffers are freed before
// returning. Returns the solve's status.
nswe_status solve2d_request(nswe_ctx ctx, cudaStream_t s, Request *r) {
  nswe_prob p = nullptr;
  nswe_status st = nswe_prob_create_2d(ctx, &p, r->Nx, r->Ny, r->levels, r->x0, r->x1, r->y0, r->y1, r->g,
                                       r->gq.data(), r->kinds.data(), r->bcs);
  if (st != NSWE_OK) return st;
  const size_t n = (size_t)r->Nx * r->Ny;
  double *dU0 = nullptr, *dU = nullptr;
  if (cudaMalloc(&dU0, sizeof(double) * r->u0.size()) != cudaSuccess ||
      cudaMalloc(&dU, sizeof(double) * 3 * n) != cudaSuccess)
    st = NSWE_ENOMEM;
  if (st == NSWE_OK &&
      cudaMemcpyAsync(dU0, r->u0.data(), sizeof(double) * r->u0.size(), cudaMemcpyHostToDevice, s) != cudaSuccess)
    st = NSWE_ECUDA;
  if (st == NSWE_OK) st = nswe_newton_solve(ctx, p, dU0, dU, &r->prm, &r->info);
  if (st != NSWE_EINVAL && st != NSWE_ENOMEM && st != NSWE_ECUDA) {  // a solve outcome: the state is valid
    r->U.resize(3 * n);
    if (cudaMemcpyAsync(r->U.data(), dU, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      st = NSWE_ECUDA;
  }
  cudaFree(dU0);
  cudaFree(dU);
  nswe_prob_destroy(p);
  return st;
}

}  // namespace

// One 2D worker (see the top of the file).
void nswe_server_s::run2d() {
  cudaStream_t s = nullptr;
  nswe_ctx ctx = nullptr;
  if (cudaSetDevice(device) != cudaSuccess || cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
      nswe_ctx_create(&ctx, device, s) != NSWE_OK) {
    int ok = NSWE_OK;
    error.compare_exchange_strong(ok, NSWE_ECUDA);
    cv.notify_all();
    if (s) cudaStreamDestroy(s);
    return;
  }
  for (;;) {
    Request *r = nullptr;
    {
      std::unique_lock<std::mutex> lk(mu);
      cv2.wait(lk, [&] {
        return stop.load() || error.load() != NSWE_OK ||
               (!waiting2d.empty() && used2d + waiting2d.front()->foot2d <= cfg.device_bytes_2d);
      });
      if (stop.load() || error.load() != NSWE_OK) break;
      r = waiting2d.front();
      waiting2d.pop_front();
      used2d += r->foot2d;
      stats.running += 1;
      r->times.t_admit_ns = now_ns();
    }
    cv2.notify_all();  // the next request may fit as well
    r->times.t_launch_ns = now_ns();
    const nswe_status st = solve2d_request(ctx, s, r);
    r->status = st;
    r->times.t_done_ns = now_ns();
    {
      std::lock_guard<std::mutex> lk(mu);
      used2d -= r->foot2d;
      stats.running -= 1;
      stats.completed += 1;
      if (st == NSWE_ECUDA || st == NSWE_ENOMEM) {
        int ok = NSWE_OK;
        error.compare_exchange_strong(ok, (int)st);
      }
      done[r->ticket] = r;
      completed.push_back(r->ticket);
    }
    cv.notify_all();
    cv2.notify_all();
  }
  nswe_ctx_destroy(ctx);
  cudaStreamDestroy(s);
}

nswe_status nswe_arena_create(nswe_arena *out, size_t bytes, size_t align) {
  if (!out || bytes == 0 || align == 0 || (align & (align - 1)) != 0) return NSWE_EINVAL;
  nswe_arena_s *a = new (std::nothrow) nswe_arena_s;
  if (!a) return NSWE_ENOMEM;
  a->size = bytes / align * align;
  a->align = align;
  if (a->size) a->free_blocks[0] = a->size;
  *out = a;
  return NSWE_OK;
}

nswe_status nswe_arena_alloc(nswe_arena a, size_t bytes, size_t *offset) {
  if (!a || !offset) return NSWE_EINVAL;
  return a->alloc(bytes, offset) ? NSWE_OK : NSWE_ENOMEM;
}

nswe_status nswe_arena_free(nswe_arena a, size_t offset) {
  if (!a) return NSWE_EINVAL;
  return a->release(offset) ? NSWE_OK : NSWE_EINVAL;
}

nswe_status nswe_arena_query(nswe_arena a, size_t *used, size_t *peak, size_t *largest_free) {
  if (!a) return NSWE_EINVAL;
  if (used) *used = a->used;
  if (peak) *peak = a->peak;
  if (largest_free) *largest_free = a->largest_free();
  return NSWE_OK;
}

nswe_status nswe_arena_destroy(nswe_arena a) {
  delete a;
  return NSWE_OK;
}

size_t nswe_server_footprint_1d(int N, int levels, int nest_start) {
  if (N < 4 || levels < 1 || levels > NSWE_MAX_LEVELS) return 0;
  const int s0 = (nest_start >= 0 && nest_start < levels) ? nest_start : levels - 1;
  return layout_1d(N, levels, s0).dev_total;
}

nswe_status nswe_server_create(nswe_server *out, int device, const nswe_server_config *cfg) {
  if (!out || !cfg || cfg->device_bytes < (1u << 20) || cfg->host_bytes < (1u << 20) || cfg->streams < 1 ||
      cfg->streams > 16 || cfg->max_batch < 1 || cfg->max_batch > 65536 || !(cfg->batch_window_s >= 0.0) ||
      !(cfg->batch_window_s <= 10.0))
    return NSWE_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return NSWE_EINVAL;
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess) return NSWE_ECUDA;
  nswe_server_s *sv = new (std::nothrow) nswe_server_s;
  if (!sv) return NSWE_ENOMEM;
  sv->device = device;
  sv->cfg = *cfg;
  nswe_status st = NSWE_OK;
  void *hd = nullptr;
  if (cudaMalloc(&sv->dev_base, cfg->device_bytes) != cudaSuccess ||
      cudaHostAlloc(&sv->host_base, cfg->host_bytes, cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess) {
    st = NSWE_ENOMEM;
  } else if (cudaHostGetDevicePointer(&hd, sv->host_base, 0) != cudaSuccess) {
    st = NSWE_ECUDA;
  } else {
    sv->host_base_dev = static_cast<char *>(hd);
    sv->dev_arena.size = cfg->device_bytes / kSlotBytes * kSlotBytes;
    sv->dev_arena.free_blocks[0] = sv->dev_arena.size;
    sv->host_arena.size = cfg->host_bytes / kSlotBytes * kSlotBytes;
    sv->host_arena.free_blocks[0] = sv->host_arena.size;
    sv->streams.resize(cfg->streams);
    sv->events.resize(cfg->streams);
    sv->task_dev.resize(cfg->streams, nullptr);
    sv->task_host.resize(cfg->streams, nullptr);
    sv->batches.resize(cfg->streams);
    for (int s = 0; s < cfg->streams && st == NSWE_OK; ++s) {
      if (cudaStreamCreateWithFlags(&sv->streams[s], cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&sv->events[s], cudaEventDisableTiming) != cudaSuccess ||
          cudaMalloc(&sv->task_dev[s], sizeof(SolveTask) * cfg->max_batch) != cudaSuccess ||
          cudaMallocHost(&sv->task_host[s], sizeof(SolveTask) * cfg->max_batch) != cudaSuccess)
        st = NSWE_ENOMEM;
    }
  }
  if (st != NSWE_OK) {
    nswe_server_destroy(sv);
    cudaSetDevice(prev);
    return st;
  }
  sv->worker = std::thread([sv] { sv->run(); });
  if (cfg->device_bytes_2d > 0)
    for (int w = 0; w < cfg->streams; ++w) sv->workers2d.emplace_back([sv] { sv->run2d(); });
  cudaSetDevice(prev);
  *out = sv;
  return NSWE_OK;
}

size_t nswe_server_footprint_2d(int Nx, int Ny, int levels, int nest_start) {
  if (levels < 1 || levels > NSWE_MAX_LEVELS || Nx < 4 || Ny < 4 || (long)Nx * Ny > (1L << 26)) return 0;
  if (Nx % (1 << (levels - 1)) || Ny % (1 << (levels - 1))) return 0;
  const int NLx = Nx >> (levels - 1), NLy = Ny >> (levels - 1);
  if (NLx < 4 || NLy < 4 || NLx * NLy > 512) return 0;
  const int s0 = (nest_start >= 0 && nest_start < levels) ? nest_start : levels - 1;
  const size_t n = (size_t)Nx * Ny, ns = (size_t)(Nx >> s0) * (Ny >> s0);
  return prob2d_device_bytes(Nx, Ny, levels) + sizeof(double) * 3 * (n + ns);
}

nswe_status nswe_server_submit_2d(nswe_server sv, int Nx, int Ny, int levels, double x0, double x1, double y0,
                                  double y1, double g, const double *gauss_geom, const int *bc_kind,
                                  const double *bc_state, const double *U0, const nswe_params *params,
                                  unsigned long long *ticket) {
  if (!sv || !gauss_geom || !bc_kind || !bc_state || !U0 || !params || !ticket) return NSWE_EINVAL;
  if (sv->cfg.device_bytes_2d == 0) return NSWE_EINVAL;
  if (sv->error.load() != NSWE_OK) return (nswe_status)sv->error.load();
  const size_t foot = nswe_server_footprint_2d(Nx, Ny, levels, params->nest_start);
  if (foot == 0) return NSWE_EINVAL;
  if (!(x1 > x0) || !(y1 > y0) || !(g > 0.0) || !std::isfinite(x0) || !std::isfinite(x1) || !std::isfinite(y0) ||
      !std::isfinite(y1) || !std::isfinite(g))
    return NSWE_EINVAL;
  const int s0 = (params->nest_start >= 0 && params->nest_start < levels) ? params->nest_start : levels - 1;
  nswe_status st = check_params_2d(params, levels, s0);
  if (st != NSWE_OK) return st;
  if (foot > sv->cfg.device_bytes_2d) return NSWE_ENOMEM;  // can never be admitted
  size_t nk = 0, ng = 0;
  for (int l = 0; l < levels; ++l) {
    nk += 2 * (size_t)((Nx >> l) + (Ny >> l));
    ng += 8 * (size_t)(Nx >> l) * (Ny >> l);
  }
  for (size_t i = 0; i < nk; ++i)
    if (bc_kind[i] < NSWE_BC2_REFLECT || bc_kind[i] > NSWE_BC2_DEPTH) return NSWE_EINVAL;
  for (int i = 0; i < 12; ++i)
    if (!std::isfinite(bc_state[i])) return NSWE_EINVAL;
  Request *r = new (std::nothrow) Request;
  if (!r) return NSWE_ENOMEM;
  r->dim = 2;
  r->Nx = Nx;
  r->Ny = Ny;
  r->levels = levels;
  r->s0 = s0;
  r->x0 = x0;
  r->x1 = x1;
  r->y0 = y0;
  r->y1 = y1;
  r->g = g;
  r->prm = *params;
  r->foot2d = foot;
  r->gq.assign(gauss_geom, gauss_geom + ng);
  r->kinds.assign(bc_kind, bc_kind + nk);
  std::memcpy(r->bcs, bc_state, sizeof(r->bcs));
  r->u0.assign(U0, U0 + 3 * (size_t)(Nx >> s0) * (Ny >> s0));
  for (double v : r->gq)
    if (!std::isfinite(v)) st = NSWE_EINVAL;
  for (double v : r->u0)
    if (!std::isfinite(v)) st = NSWE_EINVAL;
  if (st != NSWE_OK) {
    delete r;
    return st;
  }
  r->times.t_submit_ns = now_ns();
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    r->ticket = sv->next_ticket++;
    sv->waiting2d.push_back(r);
    sv->stats.submitted += 1;
  }
  sv->cv2.notify_all();
  *ticket = r->ticket;
  return NSWE_OK;
}

nswe_status nswe_server_submit_1d(nswe_server sv, int N, int levels, double x0, double x1, double g,
                                  const double *sigma_face, const double *gauss_geom, const nswe_bc1d *left,
                                  const nswe_bc1d *right, const double *U0, const nswe_params *params,
                                  unsigned long long *ticket) {
  if (!sv || !sigma_face || !gauss_geom || !left || !right || !U0 || !params || !ticket) return NSWE_EINVAL;
  if (sv->error.load() != NSWE_OK) return (nswe_status)sv->error.load();
  if (levels < 1 || levels > NSWE_MAX_LEVELS || N < 4 || N % (1 << (levels - 1)) != 0) return NSWE_EINVAL;
  const int NL = N >> (levels - 1);
  if (NL < 4 || NL > kMaxCoarse) return NSWE_EINVAL;
  if (!(x1 > x0) || !(g > 0.0) || !std::isfinite(x0) || !std::isfinite(x1) || !std::isfinite(g))
    return NSWE_EINVAL;
  if (left->kind < NSWE_BC_DISCHARGE || left->kind > NSWE_BC_EXTRAP || right->kind < NSWE_BC_DISCHARGE ||
      right->kind > NSWE_BC_EXTRAP)
    return NSWE_EINVAL;
  const int s0 = (params->nest_start >= 0 && params->nest_start < levels) ? params->nest_start : levels - 1;
  nswe_status st = check_params_1d(params, levels, s0);
  if (st != NSWE_OK) return st;
  Request *r = new (std::nothrow) Request;
  if (!r) return NSWE_ENOMEM;
  r->N = N;
  r->levels = levels;
  r->s0 = s0;
  r->x0 = x0;
  r->x1 = x1;
  r->g = g;
  r->left = *left;
  r->right = *right;
  r->prm = *params;
  r->lay = layout_1d(N, levels, s0);
  if (r->lay.dev_total > sv->dev_arena.size || r->lay.host_total > sv->host_arena.size) {
    delete r;
    return NSWE_ENOMEM;  // can never be admitted
  }
  size_t ngq = 0;
  for (int l = 0; l < levels; ++l) ngq += 6 * (size_t)(N >> l);
  r->sf.assign(sigma_face, sigma_face + N + 1);
  r->gq.assign(gauss_geom, gauss_geom + ngq);
  r->u0.assign(U0, U0 + 2 * (size_t)(N >> s0));
  for (double v : r->sf)
    if (!std::isfinite(v) || !(v > 0.0)) st = NSWE_EINVAL;
  for (double v : r->gq)
    if (!std::isfinite(v)) st = NSWE_EINVAL;
  if (st != NSWE_OK) {
    delete r;
    return st;
  }
  r->times.t_submit_ns = now_ns();
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    r->ticket = sv->next_ticket++;
    sv->submitted.push_back(r);
    sv->stats.submitted += 1;
  }
  sv->cv.notify_all();
  *ticket = r->ticket;
  return NSWE_OK;
}

nswe_status nswe_server_poll(nswe_server sv, unsigned long long *tickets, int max, int *count) {
  if (!sv || !count || max < 0 || (max > 0 && !tickets)) return NSWE_EINVAL;
  std::lock_guard<std::mutex> lk(sv->mu);
  int n = 0;
  while (n < max && !sv->completed.empty()) {
    tickets[n++] = sv->completed.front();
    sv->completed.pop_front();
  }
  *count = n;
  return (nswe_status)sv->error.load();
}

nswe_status nswe_server_wait(nswe_server sv, int min_completed, double timeout_s) {
  if (!sv || !(timeout_s >= 0.0)) return NSWE_EINVAL;
  std::unique_lock<std::mutex> lk(sv->mu);
  const bool ok = sv->cv.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] {
    return sv->error.load() != NSWE_OK || (int)sv->completed.size() >= min_completed;
  });
  if (sv->error.load() != NSWE_OK) return (nswe_status)sv->error.load();
  return ok ? NSWE_OK : NSWE_ETIMEOUT;
}

nswe_status nswe_server_take(nswe_server sv, unsigned long long ticket, double *U, nswe_info *info,
                             nswe_server_times *times) {
  if (!sv) return NSWE_EINVAL;
  Request *r = nullptr;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->done.find(ticket);
    if (it == sv->done.end()) return NSWE_EINVAL;
    r = it->second;
    sv->done.erase(it);
  }
  if (U) std::memcpy(U, r->U.data(), sizeof(double) * r->U.size());
  if (info) *info = r->info;
  if (times) *times = r->times;
  delete r;
  return NSWE_OK;
}

nswe_status nswe_server_set_cluster(nswe_server sv, int ctas, int max_in_flight, int team_cells) {
  if (!sv || ctas < 1 || ctas > kMaxClusterCtas || max_in_flight < 0 || team_cells < 1) return NSWE_EINVAL;
  sv->cl_team_cells = team_cells;
  sv->cl_max = max_in_flight;
  sv->cl_ctas = ctas;
  return NSWE_OK;
}

nswe_status nswe_server_query(nswe_server sv, nswe_server_stats *out) {
  if (!sv || !out) return NSWE_EINVAL;
  std::lock_guard<std::mutex> lk(sv->mu);
  *out = sv->stats;
  out->waiting = (int)(sv->waiting.size() + sv->submitted.size() + sv->waiting2d.size());
  return (nswe_status)sv->error.load();
}

nswe_status nswe_server_destroy(nswe_server sv) {
  if (!sv) return NSWE_EINVAL;
  {
    std::lock_guard<std::mutex> lk(sv->mu);  // a worker between its test and its wait sees stop
    sv->stop = true;
  }
  sv->cv.notify_all();
  sv->cv2.notify_all();
  if (sv->worker.joinable()) sv->worker.join();
  for (auto &t : sv->workers2d)  // each finishes the solve it holds
    if (t.joinable()) t.join();
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(sv->device);
  for (size_t s = 0; s < sv->streams.size(); ++s) {
    if (sv->streams[s]) cudaStreamSynchronize(sv->streams[s]);
    if (sv->events[s]) cudaEventDestroy(sv->events[s]);
    if (sv->streams[s]) cudaStreamDestroy(sv->streams[s]);
    if (sv->task_dev[s]) cudaFree(sv->task_dev[s]);
    if (sv->task_host[s]) cudaFreeHost(sv->task_host[s]);
  }
  if (sv->dev_base) cudaFree(sv->dev_base);
  if (sv->host_base) cudaFreeHost(sv->host_base);
  for (Request *r : sv->submitted) delete r;
  for (Request *r : sv->waiting) delete r;
  for (Request *r : sv->waiting2d) delete r;
  for (Request *r : sv->running) delete r;
  for (auto &kv : sv->done) delete kv.second;
  delete sv;
  if (prev >= 0) cudaSetDevice(prev);
  return NSWE_OK;
}

}  // extern "C"
