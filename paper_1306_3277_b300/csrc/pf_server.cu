// pf_server.cu -- continuous-batching likelihood server (pf_server_* of pf.h).
//
// A scheduler thread owns one CUDA stream and a table of slots.  Every
// iteration it
//   1. retires the filters that an earlier iteration reported finished (their
//      results were copied back asynchronously), freeing slot and memory;
//   2. admits queued requests (FIFO) while a slot is free and the request's
//      device bytes fit in the budget; their buffers come from a private,
//      stream-ordered memory pool, their y from a pinned staging arena;
//   3. launches, over the tiles of every admitted filter, the init kernel for
//      the new ones, then one propagate launch per model class and one
//      resample launch, so every running filter advances one observation;
//      the descriptor table and tile map are uploaded only when a slot
//      changed, and results are copied back only by iterations that launch
//      some filter's last observation or every RESULTS_EVERY-th one.
// With more than one branch (pf_server_configure), the running filters are
// dealt into that many groups of about equal work per step, and each group's
// launches of an iteration (init, propagate per model class, resample) run on
// a stream of their own, forked from and joined back into the scheduler's
// stream: one group's launches fill the SMs that another's leave idle (the
// tail of a wave, a class bound by the FP64 unit beside one bound by FP32).
// The same kernels and per-filter reduction order as pf_run are used, so a
// request's log-likelihood is bit-identical to pf_run of the same request.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "pf.h"
#include "pf_internal.h"
#include "pf_runtime.h"

using namespace pfb;

namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

struct Request {
  uint64_t ticket = 0;
  pf_model m{};
  int64_t P = 0;
  int32_t T = 0;
  double dt = 0.0;
  Shape sh;
  double theta[8] = {0};
  std::vector<double> y;
  uint64_t seed = 0;
  size_t bytes = 0;
  double t_submit = 0.0, t_done = 0.0;
  // while running
  int slot = -1;
  bool fresh = false;
  int32_t launched_steps = 0;  // observations launched so far
  std::vector<void*> bufs;
  FilterDev desc{};
  // result
  double ll = 0.0;
  int status = PF_OK;
};

constexpr size_t ARENA_HALF = size_t(16) << 20;  // pinned staging per iteration parity
constexpr int MAX_BRANCHES = 8;
constexpr int DEFAULT_BRANCHES = 4;

// Relative device time of one step of one tile of a request's model class
// (per-launch times at 2^20 particles, mixed precision: windkessel 76 us,
// Lorenz '96 N = 8 120 us, N = 40 425 us; FP64 Lorenz '96 about 4x its mixed
// form).  Only the balance of the branches depends on it.
double tile_cost(const Request* r) {
  if (r->m.kind == PF_WINDKESSEL || r->m.kind == PF_WINDKESSEL_EXP) return 75.0;
  double c = 100.0 + double(r->m.N) * double(r->m.substeps);
  if (r->m.kind == PF_LORENZ96_SDE) c *= 3.5;  // the normals of every substep
  return r->m.prec == PF_FP64 ? 4.0 * c : c;
}

}  // namespace

struct pf_server {
  size_t budget = 0;
  int max_slots = 0;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Request*> queue;
  std::unordered_map<uint64_t, Request*> finished;
  std::unordered_set<uint64_t> pending;  // tickets queued or running
  uint64_t next_ticket = 1;
  int64_t n_running = 0, n_completed = 0, n_iter = 0;
  bool stop = false;
  bool broken = false;  // a CUDA error ended the scheduler's work: requests fail with PF_ECUDA
  std::thread thr;
  std::atomic<int> branches{DEFAULT_BRANCHES};  // launch groups per iteration
  bool regroup = false;  // under mu: branches changed, rebuild the tile map
  // scheduler-owned
  cudaStream_t st = nullptr;
  cudaStream_t st_br[MAX_BRANCHES] = {};  // the branches' streams
  cudaEvent_t ev_fork = nullptr;          // forks the branches off st
  cudaEvent_t ev_join[MAX_BRANCHES] = {};
  cudaMemPool_t pool = nullptr;
  std::vector<Request*> slots;
  size_t used = 0;
  FilterDev* d_fds = nullptr;
  FilterDev* h_fds[2] = {nullptr, nullptr};
  int2* d_tmap = nullptr;
  int2* h_tmap[2] = {nullptr, nullptr};
  size_t tmap_cap = 0;
  double* d_res = nullptr;
  double* h_res[2] = {nullptr, nullptr};
  char* arena[2] = {nullptr, nullptr};
  cudaEvent_t ev[2] = {nullptr, nullptr};
  bool ev_live[2] = {false, false};
  std::vector<Request*> launched[2];  // requests in slots as of each in-flight iteration
  // the descriptor table and tile map on the device stay valid while no slot
  // is filled or freed and no new filter needs its initial draw
  bool map_dirty = true;
  struct Seg {
    int kind, N, prec;
    size_t off, n;
    int br;  // branch
  };
  struct Range {
    size_t off, n;
    int br;
  };
  std::vector<Seg> run_seg;    // the running filters' tile-map segments, by branch and class
  std::vector<Range> run_br;   // each branch's running tiles (contiguous in the tile map)
  size_t n_run = 0;
  int64_t iter = 0;
};

// Results are fetched (the results kernel and a copy back) only by iterations
// that launch some filter's last observation, and by every RESULTS_EVERY-th
// iteration, which finds the filters that degenerated early (their kernels
// are no-ops until then).
constexpr int RESULTS_EVERY = 32;

namespace {

bool alloc_request(pf_server* s, Request* r) {
  auto get = [&](size_t n) -> void* {
    if (n == 0) return nullptr;
    void* p = nullptr;
    if (injected_alloc_failure()) return nullptr;
    if (cudaMallocFromPoolAsync(&p, n, s->pool, s->st) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    r->bufs.push_back(p);
    return p;
  };
  const Shape& sh = r->sh;
  const size_t xs = size_t(r->m.N) * size_t(r->P) * sh.state_bytes;
  FilterDev& d = r->desc;
  memset(&d, 0, sizeof d);
  d.x[0] = get(xs);
  d.x[1] = get(xs);
  d.ctil = static_cast<double*>(get(size_t(r->P) * 8));
  if (sh.mode != MODE_ALWAYS) {
    d.ell = static_cast<double*>(get(size_t(r->P) * 8));
    d.lam = static_cast<double*>(get(size_t(r->P) * 8));
  }
  d.anc = static_cast<int32_t*>(get(size_t(r->P) * 4));
  double* flow = sh.nflow ? static_cast<double*>(get(size_t(sh.nflow) * 8)) : nullptr;
  d.tp = static_cast<TilePart*>(get(size_t(sh.ntiles) * sizeof(TilePart)));
  d.gp = static_cast<GroupPart*>(get(size_t(sh.ngroups) * sizeof(GroupPart)));
  d.ctl = static_cast<Ctl*>(get(sizeof(Ctl)));
  double* y = static_cast<double*>(get(r->y.size() * 8));
  const bool ok = d.x[0] && d.x[1] && d.ctil && d.anc && d.tp && d.gp && d.ctl && y &&
                  (sh.mode == MODE_ALWAYS || (d.ell && d.lam)) && (!sh.nflow || flow);
  if (!ok) return false;
  d.kind = r->m.kind;
  d.N = r->m.N;
  d.s = r->m.substeps;
  d.stride = l96_kind(r->m.kind) ? r->m.obs_stride : 1;
  d.prec = r->m.prec;
  d.Ny = sh.Ny;
  d.P = int32_t(r->P);
  d.T = r->T;
  d.ntiles = sh.ntiles;
  d.ngroups = sh.ngroups;
  d.mode = sh.mode;
  d.resampler = r->m.resampler;
  d.obs_every = r->m.obs_every > 1 ? r->m.obs_every : 1;
  d.obs_mask = sh.obs_mask;
  d.dt = r->dt;
  d.thr = r->m.ess_threshold;
  d.seed = r->seed;
  memcpy(d.theta, r->theta, sizeof d.theta);
  d.flow = flow;
  d.y = y;
  cudaMemsetAsync(d.gp, 0, size_t(sh.ngroups) * sizeof(GroupPart), s->st);
  cudaMemsetAsync(d.ctl, 0, sizeof(Ctl), s->st);
  if (flow) launch_flow(flow, sh.nflow, r->m.flow_peak, r->m.flow_period, r->dt, s->st);
  return true;
}

void free_request_buffers(pf_server* s, Request* r) {
  for (void* p : r->bufs) cudaFreeAsync(p, s->st);
  r->bufs.clear();
}

void finish(pf_server* s, Request* r) {
  r->t_done = now_s();
  std::lock_guard<std::mutex> lk(s->mu);
  s->finished[r->ticket] = r;
  s->pending.erase(r->ticket);
  s->n_completed += 1;
  s->n_running -= 1;
}

// End every request in a slot with status st (their buffers freed, stream-
// ordered), and forget the in-flight iterations' result lists.
void fail_running(pf_server* s, pf_status st) {
  for (int q = 0; q < 2; ++q) s->launched[q].clear();
  for (int k = 0; k < s->max_slots; ++k) {
    Request* r = s->slots[k];
    if (!r) continue;
    free_request_buffers(s, r);
    s->used -= r->bytes;
    s->slots[k] = nullptr;
    r->slot = -1;
    r->status = st;
    r->ll = 0.0;
    finish(s, r);
  }
  s->map_dirty = true;
}

// A CUDA error is sticky for the context: end the running and the queued
// requests with PF_ECUDA and take no more work (pf_server_submit refuses).
void break_server(pf_server* s) {
  cudaGetLastError();
  fail_running(s, PF_ECUDA);
  for (int q = 0; q < 2; ++q) s->ev_live[q] = false;
  std::lock_guard<std::mutex> lk(s->mu);
  s->broken = true;
  const double t = now_s();
  for (Request* r : s->queue) {
    r->status = PF_ECUDA;
    r->ll = 0.0;
    r->t_done = t;
    s->finished[r->ticket] = r;
    s->pending.erase(r->ticket);
    s->n_completed += 1;
  }
  s->queue.clear();
}

// Wait for the iteration that used this parity, then retire the filters it
// reported finished (degenerate, or past their last observation).  False if
// the wait reported a CUDA error (the server is then broken).
bool retire(pf_server* s, int parity) {
  if (!s->ev_live[parity]) return true;
  cudaError_t e = cudaEventSynchronize(s->ev[parity]);
  if (e == cudaSuccess && injected_wait_failure()) e = cudaErrorLaunchFailure;
  if (e != cudaSuccess) {
    break_server(s);
    return false;
  }
  s->ev_live[parity] = false;
  const double* res = s->h_res[parity];
  for (Request* r : s->launched[parity]) {
    const int k = r->slot;
    if (k < 0 || s->slots[k] != r) continue;
    const double ll = res[3 * k], stt = res[3 * k + 1], step = res[3 * k + 2];
    if (stt != 0.0 || step > double(r->T)) {
      r->ll = ll;
      r->status = stt != 0.0 ? PF_EDEGENERATE : PF_OK;
      free_request_buffers(s, r);
      s->used -= r->bytes;
      s->slots[k] = nullptr;
      r->slot = -1;
      s->map_dirty = true;
      finish(s, r);
    }
  }
  s->launched[parity].clear();
  return true;
}

// Room for ntm tile-map entries (twice that, to grow rarely) in both pinned
// staging copies and on the device; after the stream has drained.  On a
// failed allocation nothing is left allocated and false is returned.
bool grow_tile_map(pf_server* s, size_t ntm) {
  cudaStreamSynchronize(s->st);
  for (int q = 0; q < 2; ++q) {
    if (s->h_tmap[q]) cudaFreeHost(s->h_tmap[q]);
    s->h_tmap[q] = nullptr;
  }
  if (s->d_tmap) cudaFree(s->d_tmap);
  s->d_tmap = nullptr;
  s->tmap_cap = 0;
  bool ok = true;
  for (int q = 0; q < 2; ++q)
    ok = ok && cudaMallocHost((void**)&s->h_tmap[q], sizeof(int2) * ntm * 2) == cudaSuccess;
  ok = ok && cudaMalloc((void**)&s->d_tmap, sizeof(int2) * ntm * 2) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    for (int q = 0; q < 2; ++q) {
      if (s->h_tmap[q]) cudaFreeHost(s->h_tmap[q]);
      s->h_tmap[q] = nullptr;
    }
    if (s->d_tmap) cudaFree(s->d_tmap);
    s->d_tmap = nullptr;
    return false;
  }
  s->tmap_cap = ntm * 2;
  return true;
}

void scheduler(pf_server* s) {
  cudaSetDevice(s->device);
  int parity = 0;
  for (;;) {
    // the pinned buffers of this parity were last used two iterations ago
    if (!retire(s, parity)) continue;
    size_t arena_used = 0;
    std::vector<Request*> admitted;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      if (s->regroup) {
        s->map_dirty = true;
        s->regroup = false;
      }
      bool any_running = false;
      for (Request* r : s->slots) any_running = any_running || r;
      if (s->broken || (!any_running && s->queue.empty() && !s->ev_live[0] && !s->ev_live[1])) {
        if (s->stop) break;
        s->cv.wait_for(lk, std::chrono::milliseconds(2));
        continue;
      }
      while (!s->queue.empty()) {
        Request* r = s->queue.front();
        int free_slot = -1;
        for (int k = 0; k < s->max_slots; ++k)
          if (!s->slots[k]) {
            free_slot = k;
            break;
          }
        const size_t ybytes = (r->y.size() * 8 + 255) & ~size_t(255);
        if (free_slot < 0 || s->used + r->bytes > s->budget || arena_used + ybytes > ARENA_HALF)
          break;
        s->queue.pop_front();
        s->slots[free_slot] = r;
        r->slot = free_slot;
        s->used += r->bytes;
        arena_used += ybytes;
        s->n_running += 1;
        admitted.push_back(r);
      }
    }
    size_t aoff = 0;
    for (Request* r : admitted) {
      if (!alloc_request(s, r)) {
        free_request_buffers(s, r);
        s->used -= r->bytes;
        s->slots[r->slot] = nullptr;
        r->slot = -1;
        r->status = PF_ENOMEM;
        r->ll = 0.0;
        finish(s, r);
        continue;
      }
      char* stage = s->arena[parity] + aoff;
      memcpy(stage, r->y.data(), r->y.size() * 8);
      cudaMemcpyAsync(const_cast<double*>(r->desc.y), stage, r->y.size() * 8,
                      cudaMemcpyHostToDevice, s->st);
      aoff += (r->y.size() * 8 + 255) & ~size_t(255);
      r->fresh = true;
    }
    if (!admitted.empty()) s->map_dirty = true;
    std::vector<pf_server::Seg> new_seg;
    if (s->map_dirty) {
      // descriptors and tile map of this iteration:
      // [running tiles by branch, then class | new tiles by branch, then class]
      FilterDev* hf = s->h_fds[parity];
      const int nb = std::min(std::max(s->branches.load(), 1), MAX_BRANCHES);
      // deal the filters into the branches, longest per-step work first, each
      // to the branch with the least work so far
      std::vector<std::pair<double, int>> order;
      for (int k = 0; k < s->max_slots; ++k) {
        Request* r = s->slots[k];
        if (!r) {
          memset(&hf[k], 0, sizeof(FilterDev));
          continue;
        }
        hf[k] = r->desc;
        order.push_back({-tile_cost(r) * r->sh.ntiles, k});
      }
      std::sort(order.begin(), order.end());
      std::vector<double> load(nb, 0.0);
      typedef std::map<std::tuple<int, int, int>, std::vector<int2>> ClassTiles;
      std::vector<ClassTiles> run_cls(nb), new_cls(nb);
      for (const auto& o : order) {
        const int k = o.second;
        Request* r = s->slots[k];
        const int b = int(std::min_element(load.begin(), load.end()) - load.begin());
        load[b] -= o.first;
        auto key = std::make_tuple(r->m.kind, r->m.N, r->m.prec);
        for (int t = 0; t < r->sh.ntiles; ++t) {
          run_cls[b][key].push_back(make_int2(k, t));
          if (r->fresh) new_cls[b][key].push_back(make_int2(k, t));
        }
      }
      size_t ntm = 0;
      for (int b = 0; b < nb; ++b) {
        for (auto& kv : run_cls[b]) ntm += kv.second.size();
        for (auto& kv : new_cls[b]) ntm += kv.second.size();
      }
      if (ntm == 0) {  // nothing running: drain the other parity and wait for work
        retire(s, parity ^ 1);
        continue;
      }
      if (ntm > s->tmap_cap && !grow_tile_map(s, ntm)) {
        // no room for the map: the stream has drained, so retire what the
        // other parity's iteration finished and end the rest with PF_ENOMEM
        if (retire(s, parity ^ 1)) fail_running(s, PF_ENOMEM);
        continue;
      }
      int2* tm = s->h_tmap[parity];
      s->run_seg.clear();
      s->run_br.clear();
      size_t off = 0;
      for (int b = 0; b < nb; ++b) {
        const size_t b0 = off;
        for (auto& kv : run_cls[b]) {
          memcpy(tm + off, kv.second.data(), kv.second.size() * sizeof(int2));
          s->run_seg.push_back({std::get<0>(kv.first), std::get<1>(kv.first),
                                std::get<2>(kv.first), off, kv.second.size(), b});
          off += kv.second.size();
        }
        if (off > b0) s->run_br.push_back({b0, off - b0, b});
      }
      s->n_run = off;
      for (int b = 0; b < nb; ++b)
        for (auto& kv : new_cls[b]) {
          memcpy(tm + off, kv.second.data(), kv.second.size() * sizeof(int2));
          new_seg.push_back({std::get<0>(kv.first), std::get<1>(kv.first), std::get<2>(kv.first),
                             off, kv.second.size(), b});
          off += kv.second.size();
        }
      cudaMemcpyAsync(s->d_fds, hf, sizeof(FilterDev) * s->max_slots, cudaMemcpyHostToDevice,
                      s->st);
      cudaMemcpyAsync(s->d_tmap, tm, sizeof(int2) * off, cudaMemcpyHostToDevice, s->st);
      // the next iteration keeps this map unless the new filters (whose init
      // tiles are in it) or a slot change make it stale
      s->map_dirty = !new_seg.empty();
    }
    if (s->run_br.size() <= 1) {
      for (const pf_server::Seg& g : new_seg)
        launch_init(g.kind, g.N, g.prec, s->d_fds, s->d_tmap + g.off, int(g.n), s->st);
      for (const pf_server::Seg& g : s->run_seg)
        launch_propagate(g.kind, g.N, g.prec, s->d_fds, s->d_tmap + g.off, int(g.n), s->st);
      launch_resample(s->d_fds, s->d_tmap, int(s->n_run), s->st);
    } else {
      cudaEventRecord(s->ev_fork, s->st);
      for (size_t q = 0; q < s->run_br.size(); ++q) {
        cudaStream_t sb = s->st_br[q];
        const int b = s->run_br[q].br;
        cudaStreamWaitEvent(sb, s->ev_fork, 0);
        for (const pf_server::Seg& g : new_seg)
          if (g.br == b)
            launch_init(g.kind, g.N, g.prec, s->d_fds, s->d_tmap + g.off, int(g.n), sb);
        for (const pf_server::Seg& g : s->run_seg)
          if (g.br == b)
            launch_propagate(g.kind, g.N, g.prec, s->d_fds, s->d_tmap + g.off, int(g.n), sb);
        launch_resample(s->d_fds, s->d_tmap + s->run_br[q].off, int(s->run_br[q].n), sb);
        cudaEventRecord(s->ev_join[q], sb);
        cudaStreamWaitEvent(s->st, s->ev_join[q], 0);
      }
    }
    bool fetch = s->iter % RESULTS_EVERY == 0;
    for (Request* r : s->slots)
      if (r && ++r->launched_steps >= r->T) fetch = true;
    if (fetch) {
      double* dres = s->d_res + size_t(parity) * 3 * s->max_slots;
      launch_results(s->d_fds, s->max_slots, dres, s->st);
      cudaMemcpyAsync(s->h_res[parity], dres, sizeof(double) * 3 * s->max_slots,
                      cudaMemcpyDeviceToHost, s->st);
    }
    cudaEventRecord(s->ev[parity], s->st);  // also guards this parity's staging buffers
    if (cudaGetLastError() != cudaSuccess) {  // a launch or copy of this iteration failed
      break_server(s);
      continue;
    }
    s->ev_live[parity] = true;
    s->iter += 1;
    for (Request* r : s->slots)
      if (r) {
        if (fetch) s->launched[parity].push_back(r);  // retire() reads their results
        r->fresh = false;
      }
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->n_iter += 1;
    }
    parity ^= 1;
  }
}

}  // namespace

extern "C" pf_status pf_server_create(size_t device_mem_budget, int32_t max_slots,
                                      pf_server** out) {
  if (!out || max_slots < 1 || max_slots > 4096 || device_mem_budget == 0)
    return fail(PF_EINVAL, "pf_server_create: bad arguments");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return fail(PF_ECUDA, "no CUDA device");
  }
  pf_server* s = new pf_server();
  s->budget = device_mem_budget;
  s->max_slots = max_slots;
  s->slots.assign(max_slots, nullptr);
  cudaGetDevice(&s->device);
  cudaMemPoolProps props;
  memset(&props, 0, sizeof props);
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = s->device;
  cudaError_t e = cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMemPoolCreate(&s->pool, &props);
  if (e == cudaSuccess) {
    uint64_t thr = UINT64_MAX;
    e = cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  if (e == cudaSuccess) e = cudaMalloc((void**)&s->d_fds, sizeof(FilterDev) * max_slots);
  if (e == cudaSuccess) e = cudaMalloc((void**)&s->d_res, sizeof(double) * 6 * max_slots);
  for (int q = 0; q < 2 && e == cudaSuccess; ++q) {
    e = cudaMallocHost((void**)&s->h_fds[q], sizeof(FilterDev) * max_slots);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&s->h_res[q], sizeof(double) * 3 * max_slots);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&s->arena[q], ARENA_HALF);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev[q], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_fork, cudaEventDisableTiming);
  for (int b = 0; b < MAX_BRANCHES && e == cudaSuccess; ++b) {
    e = cudaStreamCreateWithFlags(&s->st_br[b], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_join[b], cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    pf_server_destroy(s);
    return fail(PF_ECUDA, "server set-up: %s", cudaGetErrorString(e));
  }
  s->thr = std::thread(scheduler, s);
  *out = s;
  return PF_OK;
}

extern "C" pf_status pf_server_submit(pf_server* s, const pf_model* m, int64_t P, int32_t T,
                                      double dt, const double* theta, const double* y,
                                      uint64_t seed, uint64_t* ticket) {
  if (!s || !theta || !y || !ticket) return fail(PF_EINVAL, "pf_server_submit: NULL argument");
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->broken) return fail(PF_ECUDA, "the server stopped after a CUDA error");
  }
  Shape sh;
  pf_status st = check_shape(m, P, T, dt, &sh);
  if (st != PF_OK) return st;
  if (m->resampler == PF_RESAMPLE_MULTINOMIAL)
    return fail(PF_EINVAL, "the server does not take the multinomial resampler");
  const size_t need = pf_device_bytes(m, P, T, 0) + 256 * 16;
  if (need > s->budget || size_t(T) * sh.Ny * 8 > ARENA_HALF)
    return fail(PF_ENOMEM, "request needs %zu bytes, budget is %zu", need, s->budget);
  Request* r = new Request();
  r->m = *m;
  r->P = P;
  r->T = T;
  r->dt = dt;
  r->sh = sh;
  memcpy(r->theta, theta, sizeof(double) * pf_theta_size(m->kind));
  r->y.assign(y, y + size_t(T) * sh.Ny);
  r->seed = seed;
  r->bytes = need;
  r->t_submit = now_s();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    r->ticket = s->next_ticket++;
    s->pending.insert(r->ticket);
    s->queue.push_back(r);
  }
  s->cv.notify_one();
  *ticket = r->ticket;
  return PF_OK;
}

extern "C" pf_status pf_server_poll(pf_server* s, uint64_t ticket, double* loglik,
                                    double* latency_s) {
  if (!s) return fail(PF_EINVAL, "server is NULL");
  Request* r = nullptr;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->finished.find(ticket);
    if (it == s->finished.end()) {
      if (s->pending.count(ticket)) return PF_EBUSY;
      return fail(PF_EINVAL, "ticket %llu is unknown or was already collected",
                  (unsigned long long)ticket);
    }
    r = it->second;
    s->finished.erase(it);
  }
  if (loglik) *loglik = r->ll;
  if (latency_s) *latency_s = r->t_done - r->t_submit;
  const pf_status st = pf_status(r->status);
  delete r;
  return st;
}

extern "C" pf_status pf_server_configure(pf_server* s, int32_t branches) {
  if (!s) return fail(PF_EINVAL, "server is NULL");
  if (branches < 1 || branches > MAX_BRANCHES)
    return fail(PF_EINVAL, "pf_server_configure: branches must be 1..%d", MAX_BRANCHES);
  s->branches.store(branches);
  std::lock_guard<std::mutex> lk(s->mu);
  s->regroup = true;
  return PF_OK;
}

extern "C" pf_status pf_server_stats(pf_server* s, int64_t* queued, int64_t* running,
                                     int64_t* completed, int64_t* iterations) {
  if (!s) return fail(PF_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> lk(s->mu);
  if (queued) *queued = int64_t(s->queue.size());
  if (running) *running = s->n_running;
  if (completed) *completed = s->n_completed;
  if (iterations) *iterations = s->n_iter;
  return PF_OK;
}

extern "C" pf_status pf_server_destroy(pf_server* s) {
  if (!s) return PF_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    for (Request* r : s->queue) delete r;
    s->queue.clear();
  }
  s->cv.notify_all();
  if (s->thr.joinable()) s->thr.join();
  if (s->st) cudaStreamSynchronize(s->st);
  for (Request* r : s->slots)
    if (r) {
      free_request_buffers(s, r);
      delete r;
    }
  for (auto& kv : s->finished) delete kv.second;
  if (s->st) cudaStreamSynchronize(s->st);
  if (s->d_fds) cudaFree(s->d_fds);
  if (s->d_tmap) cudaFree(s->d_tmap);
  if (s->d_res) cudaFree(s->d_res);
  for (int q = 0; q < 2; ++q) {
    if (s->h_fds[q]) cudaFreeHost(s->h_fds[q]);
    if (s->h_tmap[q]) cudaFreeHost(s->h_tmap[q]);
    if (s->h_res[q]) cudaFreeHost(s->h_res[q]);
    if (s->arena[q]) cudaFreeHost(s->arena[q]);
    if (s->ev[q]) cudaEventDestroy(s->ev[q]);
  }
  for (int b = 0; b < MAX_BRANCHES; ++b) {
    if (s->st_br[b]) cudaStreamDestroy(s->st_br[b]);
    if (s->ev_join[b]) cudaEventDestroy(s->ev_join[b]);
  }
  if (s->ev_fork) cudaEventDestroy(s->ev_fork);
  if (s->pool) cudaMemPoolDestroy(s->pool);
  if (s->st) cudaStreamDestroy(s->st);
  delete s;
  return PF_OK;
}
