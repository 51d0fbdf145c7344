// pf_api.cu -- host runtime behind the C ABI of include/pf.h: filter
// creation, launch plans (descriptor tables, tile maps and one captured CUDA
// graph per plan), single and batched runs.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "pf.h"
#include "pf_internal.h"
#include "pf_runtime.h"

using namespace pfb;

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string g_err;

pf_status pfb::fail(pf_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

extern "C" const char* pf_last_error(void) { return g_err.c_str(); }

// ---------------------------------------------------------------------------
// host-side fault injection: the k-th next device allocation of a filter or a
// served request fails as if the device were out of memory
// ---------------------------------------------------------------------------
static std::atomic<int> g_fail_alloc_countdown{0};

bool pfb::injected_alloc_failure() {
  int k = g_fail_alloc_countdown.load();
  while (k > 0) {
    if (g_fail_alloc_countdown.compare_exchange_weak(k, k - 1)) return k == 1;
  }
  return false;
}

extern "C" pf_status pf_debug_fail_allocation(int32_t k) {
  if (k < 0) return fail(PF_EINVAL, "k = %d < 0", k);
  g_fail_alloc_countdown.store(k);
  return PF_OK;
}

// ... and the k-th next wait of a server's scheduler for one of its iterations
// reports a CUDA error, as a failed kernel would
static std::atomic<int> g_persist_unfilled{0};  // plans count one slot nothing fills

extern "C" pf_status pf_debug_persist_wait_limit(double seconds) {
  if (!(seconds > 0.0 && seconds <= 60.0))
    return fail(PF_EINVAL, "the wait limit must be in (0, 60] seconds");
  const cudaError_t e = set_persist_wait_limit(static_cast<unsigned long long>(seconds * 1e9));
  if (e != cudaSuccess) return fail(PF_ECUDA, "wait limit: %s", cudaGetErrorString(e));
  return PF_OK;
}

extern "C" pf_status pf_debug_persist_unfilled_slot(int32_t on) {
  if (on != 0 && on != 1) return fail(PF_EINVAL, "on must be 0 or 1");
  g_persist_unfilled.store(on);
  return PF_OK;
}

static std::atomic<int> g_fail_wait_countdown{0};

bool pfb::injected_wait_failure() {
  int k = g_fail_wait_countdown.load();
  while (k > 0) {
    if (g_fail_wait_countdown.compare_exchange_weak(k, k - 1)) return k == 1;
  }
  return false;
}

extern "C" pf_status pf_debug_fail_server_wait(int32_t k) {
  if (k < 0) return fail(PF_EINVAL, "k = %d < 0", k);
  g_fail_wait_countdown.store(k);
  return PF_OK;
}

#define CK(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) return fail(PF_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

// ---------------------------------------------------------------------------
// shapes
// ---------------------------------------------------------------------------
extern "C" int32_t pf_theta_size(int32_t kind) {
  return wk_kind(kind) ? 7 : l96_kind(kind) ? 5 : 0;
}

pf_status pfb::check_shape(const pf_model* m, int64_t P, int32_t T, double dt, Shape* sh) {
  if (!m) return fail(PF_EINVAL, "model is NULL");
  if (m->resampler < PF_RESAMPLE_SYSTEMATIC || m->resampler > PF_RESAMPLE_MULTINOMIAL)
    return fail(PF_EINVAL, "unknown resampler %d", m->resampler);
  if (!supported(m->kind, m->N, m->prec))
    return fail(PF_EINVAL, "unsupported model: kind %d, N %d, precision %d", m->kind, m->N,
                m->prec);
  if (P < 1 || P > MAX_P) return fail(PF_EINVAL, "P = %lld outside [1, 2^24]", (long long)P);
  if (T < 1) return fail(PF_EINVAL, "T = %d must be >= 1", T);
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(PF_EINVAL, "dt must be finite and > 0");
  if (m->substeps < 1) return fail(PF_EINVAL, "substeps must be >= 1");
  if (!(m->ess_threshold >= 0.0) || !std::isfinite(m->ess_threshold))
    return fail(PF_EINVAL, "ess_threshold must be finite and >= 0");
  if (m->obs_every < 0 || m->obs_count < 0)
    return fail(PF_EINVAL, "obs_every and obs_count must be >= 0");
  int Ny = 1;
  uint64_t mask = 1;
  if (l96_kind(m->kind)) {
    if (m->obs_stride < 1) return fail(PF_EINVAL, "obs_stride must be >= 1");
    Ny = (m->N + m->obs_stride - 1) / m->obs_stride;
    if (m->obs_count > 0 && m->obs_count < Ny) Ny = m->obs_count;
    mask = 0;
    for (int n = 0, k = 0; n < m->N && k < Ny; n += m->obs_stride, ++k) mask |= (1ull << n);
  } else {
    if (!(m->flow_period > 0.0) || !std::isfinite(m->flow_period) || !std::isfinite(m->flow_peak))
      return fail(PF_EINVAL, "flow_period must be finite and > 0, flow_peak finite");
  }
  if (double(T) * double(m->substeps) > 2.0e9) return fail(PF_EINVAL, "T * substeps too large");
  sh->Ny = Ny;
  sh->obs_mask = mask;
  sh->ntiles = int((P + TILE - 1) / TILE);
  sh->ngroups = (sh->ntiles + GROUP - 1) / GROUP;
  sh->mode = m->ess_threshold >= 1.0 ? MODE_ALWAYS : (m->ess_threshold == 0.0 ? MODE_NEVER
                                                                              : MODE_ADAPTIVE);
  sh->state_bytes = size_t(m->prec == PF_FP64 ? 8 : 4);
  sh->nflow = wk_kind(m->kind) ? int64_t(T) * m->substeps + 1 : 0;
  return PF_OK;
}

// A small FP64 windkessel filter draws its normals ahead, in one launch over the
// whole GPU at the start of a run, instead of on the FP64 unit of the few SMs
// its tiles occupy: entries of that table (0 when the filter does not).
static constexpr int64_t kNoiseMaxP = int64_t(1) << 14;
static constexpr int64_t kNoiseMaxEntries = int64_t(8) << 20;  // 64 MiB of doubles
static int64_t noise_entries(const pf_model* m, int64_t P, int32_t T) {
  if (!wk_kind(m->kind) || m->prec != PF_FP64 || P > kNoiseMaxP) return 0;
  const int64_t n = int64_t(T) * m->substeps * P;
  return n <= kNoiseMaxEntries ? n : 0;
}

static size_t bytes_for(const pf_model* m, const Shape& sh, int64_t P, int32_t T, int hist) {
  size_t b = 2 * size_t(m->N) * size_t(P) * sh.state_bytes;
  b += size_t(P) * 8;                                     // ctil
  if (sh.mode != MODE_ALWAYS) b += 2 * size_t(P) * 8;     // ell, lam
  b += size_t(P) * 4;                                     // anc
  if (hist) b += size_t(T) * size_t(P) * 4;               // history
  b += size_t(sh.nflow) * 8;                              // flow
  b += size_t(noise_entries(m, P, T)) * 8;                 // FP64 normals drawn ahead
  b += size_t(sh.ntiles) * sizeof(TilePart) + size_t(sh.ngroups) * sizeof(GroupPart);
  b += sizeof(Ctl);
  b += size_t(T) * size_t(sh.Ny) * 8;                     // observations (plan side)
  if (m->resampler == PF_RESAMPLE_MULTINOMIAL)             // spacing sums, tile offsets
    b += size_t(P) * 8 + (size_t(sh.ntiles) + 1) * 8;
  return b;
}

extern "C" size_t pf_device_bytes(const pf_model* m, int64_t P, int32_t T, int32_t history) {
  Shape sh;
  // dt does not change the size
  if (check_shape(m, P, T, 1.0, &sh) != PF_OK) return 0;
  return bytes_for(m, sh, P, T, history);
}

// ---------------------------------------------------------------------------
// filters
// ---------------------------------------------------------------------------
static void free_filter_buffers(pf_filter* f) {
  void* ptrs[] = {f->x[0], f->x[1], f->ctil, f->ell, f->lam, f->anc, f->hist,
                  f->flow, f->tp, f->gp, f->ctl, f->path, f->path_idx, f->mn_t, f->mn_part,
                  f->znoise};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (f->h_res) cudaFreeHost(f->h_res);
  if (f->own) cudaStreamDestroy(f->own);
}

extern "C" pf_status pf_create(const pf_model* m, int64_t P, int32_t T, double dt,
                               pf_filter** out) {
  if (!out) return fail(PF_EINVAL, "out is NULL");
  Shape sh;
  pf_status st = check_shape(m, P, T, dt, &sh);
  if (st != PF_OK) return st;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return fail(PF_ECUDA, "no CUDA device");
  }
  pf_filter* f = new pf_filter();
  f->m = *m;
  f->P = P;
  f->T = T;
  f->dt = dt;
  f->sh = sh;
  cudaGetDevice(&f->device);
  auto alloc = [&](void** p, size_t n) -> bool {
    if (n == 0) return true;
    if (injected_alloc_failure()) return false;
    return cudaMalloc(p, n) == cudaSuccess;
  };
  bool ok = cudaStreamCreateWithFlags(&f->own, cudaStreamNonBlocking) == cudaSuccess;
  const size_t xs = size_t(m->N) * size_t(P) * sh.state_bytes;
  ok = ok && alloc(&f->x[0], xs) && alloc(&f->x[1], xs);
  ok = ok && alloc((void**)&f->ctil, size_t(P) * 8);
  if (sh.mode != MODE_ALWAYS)
    ok = ok && alloc((void**)&f->ell, size_t(P) * 8) && alloc((void**)&f->lam, size_t(P) * 8);
  ok = ok && alloc((void**)&f->anc, size_t(P) * 4);
  ok = ok && alloc((void**)&f->flow, size_t(sh.nflow) * 8);
  ok = ok && alloc((void**)&f->znoise, size_t(noise_entries(m, P, T)) * 8);
  ok = ok && alloc((void**)&f->tp, size_t(sh.ntiles) * sizeof(TilePart));
  ok = ok && alloc((void**)&f->gp, size_t(sh.ngroups) * sizeof(GroupPart));
  ok = ok && alloc((void**)&f->ctl, sizeof(Ctl));
  if (m->resampler == PF_RESAMPLE_MULTINOMIAL)
    ok = ok && alloc((void**)&f->mn_t, size_t(P) * 8) &&
         alloc((void**)&f->mn_part, (size_t(sh.ntiles) + 1) * 8);
  ok = ok && cudaMallocHost((void**)&f->h_res, 64) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    free_filter_buffers(f);
    delete f;
    return fail(PF_ENOMEM, "device allocation failed for P = %lld, T = %d", (long long)P, T);
  }
  cudaError_t e = cudaMemsetAsync(f->gp, 0, size_t(sh.ngroups) * sizeof(GroupPart), f->own);
  if (e == cudaSuccess) e = cudaMemsetAsync(f->ctl, 0, sizeof(Ctl), f->own);
  if (e == cudaSuccess && sh.nflow > 0)
    e = launch_flow(f->flow, sh.nflow, m->flow_peak, m->flow_period, dt, f->own);
  if (e == cudaSuccess) e = cudaStreamSynchronize(f->own);
  if (e != cudaSuccess) {
    free_filter_buffers(f);
    delete f;
    return fail(PF_ECUDA, "filter set-up: %s", cudaGetErrorString(e));
  }
  FilterDev& d = f->desc;
  memset(&d, 0, sizeof d);
  d.kind = m->kind;
  d.N = m->N;
  d.s = m->substeps;
  d.stride = l96_kind(m->kind) ? m->obs_stride : 1;
  d.prec = m->prec;
  d.Ny = sh.Ny;
  d.P = int32_t(P);
  d.T = T;
  d.ntiles = sh.ntiles;
  d.ngroups = sh.ngroups;
  d.hist = 0;
  d.mode = sh.mode;
  d.resampler = m->resampler;
  d.obs_every = m->obs_every > 1 ? m->obs_every : 1;
  d.obs_mask = sh.obs_mask;
  d.dt = dt;
  d.thr = m->ess_threshold;
  d.x[0] = f->x[0];
  d.x[1] = f->x[1];
  d.ctil = f->ctil;
  d.ell = f->ell;
  d.lam = f->lam;
  d.anc = f->anc;
  d.flow = f->flow;
  d.tp = f->tp;
  d.gp = f->gp;
  d.ctl = f->ctl;
  d.mn_t = f->mn_t;
  d.mn_part = f->mn_part;
  d.znoise = f->znoise;
  f->bytes = bytes_for(m, sh, P, T, 0);
  *out = f;
  return PF_OK;
}

// ---------------------------------------------------------------------------
// plans
// ---------------------------------------------------------------------------
static std::mutex g_plan_mu;
static std::map<std::vector<pf_filter*>, Plan*> g_plans;  // cached batch plans
// per filter list: its launch shape (cluster bound, branches, resample grid)
// four launch chains: a batch that is not autotuned keeps the SMs busier than
// with one chain (the 256-filter benchmark batch 36.9 against 44.2 ms), and a
// single filter is one chain anyway
static const pf_batch_shape kDefaultShape = {0, 4, 8, 0, 1};
static std::map<std::vector<pf_filter*>, pf_batch_shape> g_shapes;

static void destroy_plan(Plan* p) {
  if (!p) return;
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->st) cudaStreamSynchronize(p->st);
  if (p->st2) cudaStreamSynchronize(p->st2);
  void* dptrs[] = {p->d_fds, p->d_tmap, p->d_ycat, p->d_res, p->d_cta, p->d_pq, p->d_slots,
                   p->d_slots_init};
  for (void* q : dptrs)
    if (q) cudaFree(q);
  void* hptrs[] = {p->h_fds, p->h_ycat, p->h_res, p->h_perr};
  for (void* q : hptrs)
    if (q) cudaFreeHost(q);
  if (p->ev_staged) cudaEventDestroy(p->ev_staged);
  if (p->ev_done) cudaEventDestroy(p->ev_done);
  if (p->ev_fork) cudaEventDestroy(p->ev_fork);
  if (p->ev_join) cudaEventDestroy(p->ev_join);
  if (p->ev_fork_br) cudaEventDestroy(p->ev_fork_br);
  for (Branch& b : p->branches) {
    if (b.st) cudaStreamSynchronize(b.st);
    if (b.ev_join) cudaEventDestroy(b.ev_join);
    if (b.st) cudaStreamDestroy(b.st);
  }
  if (p->st2) cudaStreamDestroy(p->st2);
  if (p->st) cudaStreamDestroy(p->st);
  delete p;
}

// Steps first..last of one branch on st (the initial draw of its filters when
// init).
template <typename Hook>
static cudaError_t enqueue_branch(Plan* p, const Branch& b, int first, int last,
                                  cudaStream_t st, Profiler* prof, Hook&& hook, bool init) {
  cudaError_t le = cudaSuccess;
  auto timed = [&](int kind, auto&& launch) {
    if (prof) prof->begin(kind, st);
    const cudaError_t r = launch();
    if (prof) prof->end(st);
    return r;
  };
  const int2* tall = p->d_tmap + b.all_offset;
  for (size_t q = 0; q < b.noise.size() && le == cudaSuccess; ++q) {
    const pf_filter* f = p->filters[b.noise[q]];
    le = launch_noise(p->d_fds, b.noise[q], std::max(first, 1), std::min(last, f->T), int(f->P),
                      f->m.substeps, st);
  }
  if (init) {
    for (size_t c = 0; c < b.classes.size() && le == cudaSuccess; ++c) {
      const PlanClass& pc = b.classes[c];
      le = timed(PROF_INIT, [&] {
        return launch_init(pc.kind, pc.N, pc.prec, p->d_fds, p->d_tmap + pc.offset, pc.ntiles,
                           st);
      });
    }
    if (le == cudaSuccess) le = hook(0);
  }
  for (int i = first; i <= std::min(last, b.maxT) && le == cudaSuccess; ++i) {
    for (size_t c = 0; c < b.classes.size() && le == cudaSuccess; ++c) {
      const PlanClass& pc = b.classes[c];
      if (b.cnt_cls[c][i] == 0) continue;
      le = timed(PROF_PROPAGATE, [&] {
        return launch_propagate_sub(pc.kind, pc.N, pc.prec, pc.sub, p->d_fds,
                                    p->d_tmap + pc.offset, b.cnt_cls[c][i], st);
      });
    }
    if (le == cudaSuccess) le = hook(i);
    if (le == cudaSuccess && b.has_mn && b.cnt_all[i + 1] > 0)
      le = timed(PROF_RESAMPLE,
                 [&] { return launch_mn_scan(p->d_fds, tall, b.cnt_all[i + 1], p->nf, st); });
    if (le == cudaSuccess && b.cnt_all[i + 1] > 0)
      le = timed(PROF_RESAMPLE, [&] {
        return launch_resample(p->d_fds, tall, b.cnt_all[i + 1], st,
                               p->shape.resample_blocks_per_sm);
      });
  }
  return le;
}

// The launch sequence of steps first..last of a plan: the initial draw when
// `init` (normally first == 1), then for every step of every branch one
// propagate launch per class and one resample launch (only over the branch's
// filters that are still running), then the results gather.  Branches after
// the first are forked off st with an event and joined back before the
// results (with a profiler, or a single branch, everything runs on st, one
// launch after the other).  hook(i) is called after the propagate launches of
// step i (and hook(0) after init), to enqueue work that reads x(t_i); it is
// only used with single-filter plans.  With a profiler, every launch is
// bracketed by CUDA events on the same stream.
static cudaError_t no_hook(int) { return cudaSuccess; }

template <typename Hook>
static cudaError_t enqueue_steps(Plan* p, int first, int last, cudaStream_t st, Profiler* prof,
                                 Hook&& hook, bool init, bool results = true) {
  cudaError_t le = cudaSuccess;
  const size_t nb = p->branches.size();
  if (nb <= 1 || prof) {
    for (size_t b = 0; b < nb && le == cudaSuccess; ++b)
      le = enqueue_branch(p, p->branches[b], first, last, st, prof, hook, init);
  } else {
    le = cudaEventRecord(p->ev_fork_br, st);
    for (size_t b = 1; b < nb && le == cudaSuccess; ++b) {
      const Branch& br = p->branches[b];
      le = cudaStreamWaitEvent(br.st, p->ev_fork_br, 0);
      if (le == cudaSuccess) le = enqueue_branch(p, br, first, last, br.st, nullptr, hook, init);
      if (le == cudaSuccess) le = cudaEventRecord(br.ev_join, br.st);
    }
    if (le == cudaSuccess) le = enqueue_branch(p, p->branches[0], first, last, st, nullptr, hook, init);
    for (size_t b = 1; b < nb && le == cudaSuccess; ++b)
      le = cudaStreamWaitEvent(st, p->branches[b].ev_join, 0);
  }
  if (le == cudaSuccess && results) {
    if (prof) prof->begin(PROF_RESULTS, st);
    le = launch_results(p->d_fds, p->nf, p->d_res, st);
    if (prof) prof->end(st);
  }
  return le;
}

// The tiled filters' whole run: the per-step chains, or the persistent launch
// (the queue reset to the plan's first items, the initial draw per class, one
// k_persist launch), then the results gather when `results`.
static cudaError_t enqueue_tiled_run(Plan* p, cudaStream_t st, Profiler* prof, bool results) {
  if (p->persist_set == 0) return enqueue_steps(p, 1, p->maxT, st, prof, no_hook, true, results);
  // every level's first items, the rest of the slots empty
  cudaError_t le = cudaMemcpyAsync(p->d_slots, p->d_slots_init,
                                   sizeof(unsigned long long) * p->persist_total,
                                   cudaMemcpyDeviceToDevice, st);
  if (le == cudaSuccess)  // the run's header; err_any is kept
    le = cudaMemcpyAsync(p->d_pq, p->d_pq_init, offsetof(PersistQueue, err_any),
                         cudaMemcpyDeviceToDevice, st);
  for (size_t b = 0; b < p->branches.size() && le == cudaSuccess; ++b) {
    for (const PlanClass& pc : p->branches[b].classes) {
      if (prof) prof->begin(PROF_INIT, st);
      le = launch_init(pc.kind, pc.N, pc.prec, p->d_fds, p->d_tmap + pc.offset, pc.ntiles, st);
      if (prof) prof->end(st);
      if (le != cudaSuccess) break;
    }
  }
  if (le == cudaSuccess) {
    if (prof) prof->begin(PROF_PROPAGATE, st);
    le = launch_persist(p->persist_set, p->d_fds, p->d_pq, p->d_slots, p->persist_kt,
                        p->shape.persistent_blocks_per_sm, st);
    if (prof) prof->end(st);
  }
  if (le == cudaSuccess && results) {
    if (prof) prof->begin(PROF_RESULTS, st);
    le = launch_results(p->d_fds, p->nf, p->d_res, st);
    if (prof) prof->end(st);
  }
  return le;
}

// The launch sequence of one whole run of a plan.  The cluster filters run on
// a side branch (their own stream, forked and joined with events, so a
// captured graph holds two parallel branches) next to the tiled steps of the
// others; with a profiler everything runs on st, one launch after the other.
static cudaError_t enqueue_run(Plan* p, cudaStream_t st, Profiler* prof) {
  if (p->cta_total == 0) return enqueue_tiled_run(p, st, prof, true);
  cudaStream_t side = prof ? st : p->st2;
  cudaError_t le = cudaSuccess;
  // the cluster filters' FP64 normals, drawn ahead before the fork
  for (size_t q = 0; q < p->cta_noise.size() && le == cudaSuccess; ++q) {
    const pf_filter* f = p->filters[p->cta_noise[q]];
    le = launch_noise(p->d_fds, p->cta_noise[q], 1, f->T, int(f->P), f->m.substeps, st);
  }
  if (!prof && le == cudaSuccess) {
    le = cudaEventRecord(p->ev_fork, st);
    if (le == cudaSuccess) le = cudaStreamWaitEvent(side, p->ev_fork, 0);
  }
  for (size_t c = 0; c < p->cta_classes.size() && le == cudaSuccess; ++c) {
    const PlanClass& pc = p->cta_classes[c];
    if (prof) prof->begin(PROF_PROPAGATE, st);
    le = launch_filter_cluster(pc.kind, pc.N, pc.prec, p->d_fds, p->d_cta + pc.offset,
                               pc.ntiles, p->cta_cluster[c], side);
    if (prof) prof->end(st);
  }
  if (le == cudaSuccess && !prof) le = cudaEventRecord(p->ev_join, side);
  if (le == cudaSuccess) le = enqueue_tiled_run(p, st, prof, false);
  if (le == cudaSuccess && !prof) le = cudaStreamWaitEvent(st, p->ev_join, 0);
  if (le == cudaSuccess) {
    if (prof) prof->begin(PROF_RESULTS, st);
    le = launch_results(p->d_fds, p->nf, p->d_res, st);
    if (prof) prof->end(st);
  }
  return le;
}

cudaError_t pfb::enqueue_plan_steps(Plan* p, int first, int last, bool init, cudaStream_t st) {
  if (p->cta_total > 0) return cudaErrorNotSupported;  // cluster filters run whole runs only
  return enqueue_steps(p, first, last, st, nullptr, no_hook, init);
}

// Tile maps sorted by T descending so that the filters still running at step
// i own a prefix of every map.
// A filter runs whole on a thread-block cluster when the plan allows it for
// its particle count, its tiles fit one cluster (one CTA per tile) and its
// resampling is not multinomial (the spacing scan is a separate set of
// launches).
static bool cta_eligible(const pf_filter* f, int64_t cta_max_p) {
  return cta_max_p > 0 && f->P <= cta_max_p && f->sh.ntiles <= MAX_CLUSTER_TILES &&
         f->m.resampler != PF_RESAMPLE_MULTINOMIAL;
}

pf_status pfb::build_plan(const std::vector<pf_filter*>& fl, Plan** out,
                          const pf_batch_shape& shape) {
  Plan* p = new Plan();
  p->filters = fl;
  p->shape = shape;
  const int64_t cta_max_p = shape.cta_max_particles;
  const int nf = int(fl.size());
  std::vector<int> order(nf);
  for (int k = 0; k < nf; ++k) order[k] = k;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return fl[a]->T > fl[b]->T; });
  size_t ytot = 0;
  p->yoff.resize(nf);
  for (int k = 0; k < nf; ++k) {
    p->yoff[k] = ytot;
    ytot += size_t(fl[k]->T) * size_t(fl[k]->sh.Ny);
  }
  // the cluster filters, per class and cluster size (= their tile count), the
  // longest runs first (clusters start in the order the hardware hands them out)
  std::map<std::tuple<int, int, int, int>, std::vector<int>> cta_lists;
  for (int k = 0; k < nf; ++k)
    if (cta_eligible(fl[k], cta_max_p))
      cta_lists[std::make_tuple(fl[k]->m.kind, fl[k]->m.N, fl[k]->m.prec, fl[k]->sh.ntiles)]
          .push_back(k);
  std::vector<int> cta_all;
  for (auto& kv : cta_lists) {
    std::vector<int>& v = kv.second;
    std::stable_sort(v.begin(), v.end(), [&](int a, int b) { return fl[a]->T > fl[b]->T; });
    p->cta_classes.push_back({std::get<0>(kv.first), std::get<1>(kv.first),
                              std::get<2>(kv.first), int(cta_all.size()), int(v.size())});
    p->cta_cluster.push_back(std::get<3>(kv.first));
    cta_all.insert(cta_all.end(), v.begin(), v.end());
  }
  // drawn-ahead normals serve a filter that runs alone (latency-bound); a batch
  // fills the GPU anyway, and would redraw every filter's table per launch sequence
  p->use_noise = nf == 1;
  for (int k : cta_all)
    if (fl[k]->znoise && p->use_noise) p->cta_noise.push_back(k);
  p->cta_total = int(cta_all.size());
  // the tiled filters, longest runs first, dealt in turn into the branches
  std::vector<int> tiled;
  for (int k : order)
    if (!cta_eligible(fl[k], cta_max_p)) tiled.push_back(k);
  for (pf_filter* f : fl) p->has_mn = p->has_mn || f->m.resampler == PF_RESAMPLE_MULTINOMIAL;
  // the multinomial spacing kernels walk every filter of the plan: one branch
  int nbr = p->has_mn ? 1 : std::max(1, std::min<int>(shape.branches, int(tiled.size())));
  std::vector<std::vector<int>> members(nbr);
  for (size_t r = 0; r < tiled.size(); ++r) members[r % nbr].push_back(tiled[r]);
  // one device array: every tiled filter's tiles (sorted by T), then per
  // branch its tiles and each of its classes' tiles (all sorted by T)
  std::vector<int2> tm;
  for (int k : tiled)
    for (int t = 0; t < fl[k]->sh.ntiles; ++t) tm.push_back(make_int2(k, t));
  p->ntiles_all = int(tm.size());
  // per-step counts: entries of a T-sorted list with T >= i
  auto counts = [](const std::vector<int>& Ts, int maxT, std::vector<int>& cnt) {
    cnt.assign(maxT + 2, 0);
    for (int i = 1; i <= maxT + 1; ++i) {
      int n = 0;
      while (n < int(Ts.size()) && Ts[n] >= i) ++n;
      cnt[i] = n;
    }
  };
  int maxT = 0;
  p->branches.resize(nbr);
  for (int bi = 0; bi < nbr; ++bi) {
    Branch& br = p->branches[bi];
    std::map<std::tuple<int, int, int>, int> cls_index;
    std::vector<std::vector<int2>> cls_tiles;
    std::vector<std::vector<int>> cls_T;
    std::vector<int> all_T;
    br.all_offset = int(tm.size());
    for (int k : members[bi]) {
      pf_filter* f = fl[k];
      auto key = std::make_tuple(f->m.kind, f->m.N, f->m.prec);
      auto it = cls_index.find(key);
      int c;
      if (it == cls_index.end()) {
        c = int(cls_tiles.size());
        cls_index[key] = c;
        cls_tiles.emplace_back();
        cls_T.emplace_back();
        br.classes.push_back({f->m.kind, f->m.N, f->m.prec, 0, 0});
      } else {
        c = it->second;
      }
      for (int t = 0; t < f->sh.ntiles; ++t) {
        cls_tiles[c].push_back(make_int2(k, t));
        cls_T[c].push_back(f->T);
        tm.push_back(make_int2(k, t));
        all_T.push_back(f->T);
      }
      br.maxT = std::max(br.maxT, f->T);
      br.has_mn = br.has_mn || f->m.resampler == PF_RESAMPLE_MULTINOMIAL;
      if (f->znoise && p->use_noise) br.noise.push_back(k);
    }
    for (size_t c = 0; c < cls_tiles.size(); ++c) {
      br.classes[c].offset = int(tm.size());
      br.classes[c].ntiles = int(cls_tiles[c].size());
      tm.insert(tm.end(), cls_tiles[c].begin(), cls_tiles[c].end());
    }
    // a plan whose tiles (all of its tiled filters', which the branches run
    // at once) would leave SMs idle spreads each FP64 tile's propagation over
    // several blocks (k_propagate_sub)
    for (PlanClass& pc : br.classes)
      pc.sub = propagate_sub(pc.kind, pc.N, pc.prec, p->ntiles_all);
    counts(all_T, br.maxT, br.cnt_all);
    br.cnt_cls.resize(cls_tiles.size());
    for (size_t c = 0; c < cls_tiles.size(); ++c) counts(cls_T[c], br.maxT, br.cnt_cls[c]);
    maxT = std::max(maxT, br.maxT);
  }
  p->nf = nf;
  p->maxT = maxT;
  // the persistent launch: every tiled filter of a class the kernel is
  // compiled for (in one of its class sets), none resampled multinomially
  std::vector<unsigned long long> persist_init;  // the slot array every run starts from
  PersistQueue pq0{};                             // and its queue header
  if (shape.persistent_blocks_per_sm > 0 && !tiled.empty()) {
    int set = 0;
    bool ok = true;
    for (int k : tiled) {
      const int bit = persist_class_bit(fl[k]->m.kind, fl[k]->m.N, fl[k]->m.prec);
      ok = ok && bit != 0 && fl[k]->m.resampler != PF_RESAMPLE_MULTINOMIAL;
      set |= bit;
    }
    if (ok && persist_set_supported(set)) {
      const int kt = shape.tiles_per_item;
      int tmax = 1;
      for (int k : tiled) tmax = std::max(tmax, fl[k]->T);
      // the items of every level over the whole run, and each level's first
      // ones (the longest runs first within a level)
      unsigned long long cnt[PERSIST_LEVELS] = {};
      std::vector<unsigned long long> first[PERSIST_LEVELS];
      for (int k : tiled) {
        const int nt = fl[k]->sh.ntiles, T = fl[k]->T;
        const int nP = (nt + kt - 1) / kt;              // propagate items per step
        const int nR = (nt + RS_CHUNK - 1) / RS_CHUNK;  // resample items per step
        const int l0 = persist_level(T, tmax);
        if (nt <= kt) {  // the whole run on the CTA that takes its first item
          cnt[l0] += 1;
          first[l0].push_back(persist_item(k, PHASE_PROP, 0));
        } else {  // every phase through the queue: propagate at 1..T, resample at 1..T-1
          for (int i = 1; i <= T; ++i) cnt[persist_level(T - i + 1, tmax)] += nP;
          for (int i = 1; i < T; ++i) cnt[persist_level(T - i, tmax)] += nR;
          for (int q = 0; q < nP; ++q) first[l0].push_back(persist_item(k, PHASE_PROP, q));
        }
      }
      // fault injection for tests: one slot more than the filters fill, in
      // the level of the longest runs' first items (its wait runs out)
      if (g_persist_unfilled.load() != 0) cnt[persist_level(tmax, tmax)] += 1;
      unsigned long long base = 0;
      for (int l = 0; l < PERSIST_LEVELS; ++l) {
        PersistLevel& L = pq0.lv[l];
        L.head = 0;
        L.tail = first[l].size();
        L.total = cnt[l];
        L.base = base;
        L.cap = cnt[l];
        persist_init.resize(base + cnt[l], 0ull);
        std::copy(first[l].begin(), first[l].end(), persist_init.begin() + base);
        base += cnt[l];
      }
      pq0.maxT = tmax;
      p->persist_set = set;
      p->persist_kt = kt;
      p->persist_total = base;
    }
  }

  cudaError_t e = cudaStreamCreateWithFlags(&p->st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_staged, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_done, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMalloc((void**)&p->d_fds, sizeof(FilterDev) * nf);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&p->h_fds, sizeof(FilterDev) * nf);
  if (e == cudaSuccess) e = cudaMalloc((void**)&p->d_tmap, sizeof(int2) * std::max<size_t>(tm.size(), 1));
  if (e == cudaSuccess) e = cudaMalloc((void**)&p->d_ycat, sizeof(double) * std::max<size_t>(ytot, 1));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&p->h_ycat, sizeof(double) * std::max<size_t>(ytot, 1));
  if (e == cudaSuccess) e = cudaMalloc((void**)&p->d_res, sizeof(double) * 3 * nf);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&p->h_res, sizeof(double) * 3 * nf);
  if (e == cudaSuccess && p->cta_total > 0) {
    e = cudaStreamCreateWithFlags(&p->st2, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc((void**)&p->d_cta, sizeof(int) * cta_all.size());
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(p->d_cta, cta_all.data(), sizeof(int) * cta_all.size(),
                          cudaMemcpyHostToDevice, p->st);
  }
  if (e == cudaSuccess && p->branches.size() > 1) {
    e = cudaEventCreateWithFlags(&p->ev_fork_br, cudaEventDisableTiming);
    for (size_t b = 1; b < p->branches.size() && e == cudaSuccess; ++b) {
      e = cudaStreamCreateWithFlags(&p->branches[b].st, cudaStreamNonBlocking);
      if (e == cudaSuccess)
        e = cudaEventCreateWithFlags(&p->branches[b].ev_join, cudaEventDisableTiming);
    }
  }
  if (e == cudaSuccess && !tm.empty())
    e = cudaMemcpyAsync(p->d_tmap, tm.data(), sizeof(int2) * tm.size(), cudaMemcpyHostToDevice,
                        p->st);
  if (e == cudaSuccess && p->persist_set != 0) {
    e = cudaMalloc((void**)&p->d_pq, 2 * sizeof(PersistQueue));
    if (e == cudaSuccess) {
      p->d_pq_init = p->d_pq + 1;
      e = cudaMalloc((void**)&p->d_slots, sizeof(unsigned long long) * p->persist_total);
    }
    if (e == cudaSuccess)
      e = cudaMalloc((void**)&p->d_slots_init, sizeof(unsigned long long) * p->persist_total);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&p->h_perr, sizeof(int));
    if (e == cudaSuccess) {
      *p->h_perr = 0;
      e = cudaMemcpyAsync(p->d_pq, &pq0, sizeof(PersistQueue), cudaMemcpyHostToDevice, p->st);
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(p->d_pq_init, &pq0, sizeof(PersistQueue), cudaMemcpyHostToDevice, p->st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(p->d_slots_init, persist_init.data(),
                          sizeof(unsigned long long) * p->persist_total, cudaMemcpyHostToDevice,
                          p->st);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->st);
  if (e != cudaSuccess) {
    destroy_plan(p);
    return fail(e == cudaErrorMemoryAllocation ? PF_ENOMEM : PF_ECUDA, "plan set-up: %s",
                cudaGetErrorString(e));
  }
  for (int k = 0; k < nf; ++k) {
    p->h_fds[k] = fl[k]->desc;
    if (!p->use_noise) p->h_fds[k].znoise = nullptr;
    p->h_fds[k].y = p->d_ycat + p->yoff[k];
  }
  // capture the whole run: init, then T x (propagate per class, resample)
  cudaGraph_t g = nullptr;
  e = cudaStreamBeginCapture(p->st, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    const cudaError_t le = enqueue_run(p, p->st, nullptr);
    e = cudaStreamEndCapture(p->st, &g);
    if (e == cudaSuccess) e = le;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&p->exec, g, 0);
  if (g) cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    cudaGetLastError();
    destroy_plan(p);
    return fail(PF_ECUDA, "graph capture: %s", cudaGetErrorString(e));
  }
  *out = p;
  return PF_OK;
}

static bool is_device_ptr(const void* ptr) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Stage theta, seed and y of every filter of the plan on st (descriptors and
// host observations through pinned copies, device inputs device to device).
pf_status pfb::stage_plan(Plan* p, const double* const* theta, const double* const* y,
                          const uint64_t* seeds, const int32_t* hist_on, cudaStream_t st) {
  CK(cudaEventSynchronize(p->ev_staged));  // pinned staging of the previous run consumed
  std::vector<int> dev_theta, dev_y;
  for (int k = 0; k < p->nf; ++k) {
    pf_filter* f = p->filters[k];
    FilterDev& d = p->h_fds[k];
    d = f->desc;
    d.y = p->d_ycat + p->yoff[k];
    if (!p->use_noise) d.znoise = nullptr;
    d.seed = seeds[k];
    if (hist_on && hist_on[k]) {
      d.hist = 1;
      d.anc = f->hist;
    }
    const int nth = pf_theta_size(f->m.kind);
    if (!theta[k] || !y[k]) return fail(PF_EINVAL, "theta / y of filter %d is NULL", k);
    if (is_device_ptr(theta[k])) dev_theta.push_back(k);
    else memcpy(d.theta, theta[k], sizeof(double) * nth);
    const size_t ny = size_t(f->T) * size_t(f->sh.Ny);
    if (is_device_ptr(y[k])) dev_y.push_back(k);
    else memcpy(p->h_ycat + p->yoff[k], y[k], sizeof(double) * ny);
  }
  CK(cudaMemcpyAsync(p->d_fds, p->h_fds, sizeof(FilterDev) * p->nf, cudaMemcpyHostToDevice, st));
  size_t ytot = 0;
  for (int k = 0; k < p->nf; ++k) ytot += size_t(p->filters[k]->T) * p->filters[k]->sh.Ny;
  if (dev_y.size() < size_t(p->nf))
    CK(cudaMemcpyAsync(p->d_ycat, p->h_ycat, sizeof(double) * ytot, cudaMemcpyHostToDevice, st));
  for (int k : dev_y) {
    const size_t ny = size_t(p->filters[k]->T) * p->filters[k]->sh.Ny;
    CK(cudaMemcpyAsync(p->d_ycat + p->yoff[k], y[k], sizeof(double) * ny,
                       cudaMemcpyDeviceToDevice, st));
  }
  for (int k : dev_theta) {
    const int nth = pf_theta_size(p->filters[k]->m.kind);
    CK(cudaMemcpyAsync(p->d_fds[k].theta, theta[k], sizeof(double) * nth,
                       cudaMemcpyDeviceToDevice, st));
  }
  CK(cudaEventRecord(p->ev_staged, st));
  return PF_OK;
}

// Stage the inputs of every filter of the plan and launch its graph on st.
pf_status pfb::run_plan(Plan* p, const double* const* theta, const double* const* y,
                        const uint64_t* seeds, const int32_t* hist_on, cudaStream_t st,
                        Profiler* prof) {
  pf_status ps = stage_plan(p, theta, y, seeds, hist_on, st);
  if (ps != PF_OK) return ps;
  if (prof) CK(enqueue_run(p, st, prof));
  else CK(cudaGraphLaunch(p->exec, st));
  CK(cudaMemcpyAsync(p->h_res, p->d_res, sizeof(double) * 3 * p->nf, cudaMemcpyDeviceToHost, st));
  if (p->persist_set != 0)
    CK(cudaMemcpyAsync(p->h_perr, &p->d_pq->err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaEventRecord(p->ev_done, st));
  return PF_OK;
}

// After a run of the plan has completed: the persistent launch's failure, if
// any, as a status (PF_OK otherwise).
pf_status pfb::persist_status(const Plan* p, int err) {
  if (p->persist_set == 0 || err == 0) return PF_OK;
  if (err == 1) return fail(PF_ETIMEOUT, "persistent batch launch: a wait for a work item ran out");
  return fail(PF_ECUDA, "persistent batch launch: inconsistent work queue (code %d)", err);
}

// ---------------------------------------------------------------------------
// single filter
// ---------------------------------------------------------------------------
extern "C" pf_status pf_run(pf_filter* f, const double* theta, const double* y, uint64_t seed,
                            double* loglik, void* final_particles, int32_t* ancestors,
                            uint32_t flags, void* cuda_stream) {
  if (!f) return fail(PF_EINVAL, "filter is NULL");
  if (!theta || !y || !loglik) return fail(PF_EINVAL, "theta, y and loglik are required");
  if (flags & ~PF_FLAG_ASYNC) return fail(PF_EINVAL, "unknown flags 0x%x", flags);
  const bool async = (flags & PF_FLAG_ASYNC) != 0;
  if (async) {
    if (!is_device_ptr(loglik) || (final_particles && !is_device_ptr(final_particles)) ||
        (ancestors && !is_device_ptr(ancestors)))
      return fail(PF_EINVAL, "PF_FLAG_ASYNC needs device output pointers");
  }
  cudaStream_t st = cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : f->own;
  if (ancestors && !f->hist) {
    if (cudaMalloc((void**)&f->hist, size_t(f->T) * size_t(f->P) * 4) != cudaSuccess) {
      cudaGetLastError();
      f->hist = nullptr;
      return fail(PF_ENOMEM, "ancestor history of %lld bytes",
                  (long long)(size_t(f->T) * size_t(f->P) * 4));
    }
  }
  if (!f->wplan) {
    // a filter of at most MAX_CLUSTER_TILES tiles runs whole on one
    // thread-block cluster (no per-step launches); others take the tiled path
    std::vector<pf_filter*> one{f};
    pf_batch_shape shape = kDefaultShape;
    if (cta_eligible(f, f->P)) shape.cta_max_particles = f->P;
    pf_status ps = build_plan(one, &f->wplan, shape);
    if (ps != PF_OK) return ps;
  }
  Plan* p = f->wplan;
  f->last = p;
  const int32_t hist_on = ancestors ? 1 : 0;
  f->range_pos = -1;
  pf_status ps = run_plan(p, &theta, &y, &seed, &hist_on, st, f->prof);
  if (ps != PF_OK) return ps;
  const int64_t P = f->P;
  if (final_particles)
    CK(cudaMemcpyAsync(final_particles, f->x[f->T & 1], size_t(f->m.N) * P * f->sh.state_bytes,
                       cudaMemcpyDefault, st));
  if (ancestors)
    CK(cudaMemcpyAsync(ancestors, f->hist, size_t(f->T) * P * 4, cudaMemcpyDefault, st));
  if (async) {
    CK(cudaMemcpyAsync(loglik, p->d_res, sizeof(double), cudaMemcpyDeviceToDevice, st));
    CK(cudaEventRecord(p->ev_done, st));
    f->pending = true;
    return PF_OK;
  }
  CK(cudaEventRecord(p->ev_done, st));
  CK(cudaEventSynchronize(p->ev_done));
  const double ll = p->h_res[0];
  const int status = int(p->h_res[1]);
  if (is_device_ptr(loglik)) CK(cudaMemcpy(loglik, &ll, sizeof(double), cudaMemcpyHostToDevice));
  else *loglik = ll;
  return status == ST_OK ? PF_OK : PF_EDEGENERATE;
}

// ---------------------------------------------------------------------------
// interval continuation and single-path sampling (Algorithm 2 over t_{r:s})
// ---------------------------------------------------------------------------
static pf_status ensure_history(pf_filter* f) {
  if (f->hist) return PF_OK;
  if (cudaMalloc((void**)&f->hist, size_t(f->T) * size_t(f->P) * 4) != cudaSuccess) {
    cudaGetLastError();
    f->hist = nullptr;
    return fail(PF_ENOMEM, "ancestor history of %lld bytes",
                (long long)(size_t(f->T) * size_t(f->P) * 4));
  }
  return PF_OK;
}

static pf_status ensure_plan(pf_filter* f) {
  if (f->plan) return PF_OK;
  std::vector<pf_filter*> one{f};
  return build_plan(one, &f->plan, kDefaultShape);
}

extern "C" pf_status pf_run_range(pf_filter* f, const double* theta, const double* y,
                                  uint64_t seed, int32_t r, int32_t s, double* loglik,
                                  void* particles, void* cuda_stream) {
  if (!f) return fail(PF_EINVAL, "filter is NULL");
  if (!y || !loglik) return fail(PF_EINVAL, "y and loglik are required");
  if (r < 0 || s <= r || s > f->T)
    return fail(PF_EINVAL, "range (%d, %d] is not inside (0, %d]", r, s, f->T);
  if (r == 0 && !theta) return fail(PF_EINVAL, "theta is required when r = 0");
  if (r > 0 && r != f->range_pos)
    return fail(PF_EINVAL, "the filter does not stand at t_%d (continue from its last s, or "
                "start again at r = 0)", r);
  pf_status ps = ensure_plan(f);
  if (ps != PF_OK) return ps;
  Plan* p = f->plan;
  f->last = p;
  cudaStream_t st = cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : f->own;
  f->range_pos = -1;
  CK(cudaEventSynchronize(p->ev_staged));
  if (r == 0) {
    FilterDev& d = p->h_fds[0];
    d = f->desc;
    d.y = p->d_ycat;
    d.seed = seed;
    const int nth = pf_theta_size(f->m.kind);
    const bool dev_theta = is_device_ptr(theta);
    if (!dev_theta) memcpy(d.theta, theta, sizeof(double) * nth);
    CK(cudaMemcpyAsync(p->d_fds, p->h_fds, sizeof(FilterDev), cudaMemcpyHostToDevice, st));
    if (dev_theta)
      CK(cudaMemcpyAsync(p->d_fds[0].theta, theta, sizeof(double) * nth,
                         cudaMemcpyDeviceToDevice, st));
  } else {
    p->h_fds[0].seed = seed;  // the key of this interval's steps
    CK(cudaMemcpyAsync(&p->d_fds[0].seed, &p->h_fds[0].seed, sizeof(uint64_t),
                       cudaMemcpyHostToDevice, st));
  }
  const size_t off = size_t(r) * f->sh.Ny;
  const size_t ny = size_t(s - r) * f->sh.Ny;
  if (is_device_ptr(y)) {
    CK(cudaMemcpyAsync(p->d_ycat + off, y, sizeof(double) * ny, cudaMemcpyDeviceToDevice, st));
  } else {
    memcpy(p->h_ycat + off, y, sizeof(double) * ny);
    CK(cudaMemcpyAsync(p->d_ycat + off, p->h_ycat + off, sizeof(double) * ny,
                       cudaMemcpyHostToDevice, st));
  }
  CK(cudaEventRecord(p->ev_staged, st));
  CK(enqueue_steps(p, r + 1, s, st, f->prof, no_hook, r == 0));
  CK(cudaMemcpyAsync(p->h_res, p->d_res, sizeof(double) * 3, cudaMemcpyDeviceToHost, st));
  if (particles)
    CK(cudaMemcpyAsync(particles, f->x[s & 1], size_t(f->m.N) * f->P * f->sh.state_bytes,
                       cudaMemcpyDefault, st));
  CK(cudaEventRecord(p->ev_done, st));
  CK(cudaEventSynchronize(p->ev_done));
  f->range_pos = s;
  const double ll = p->h_res[0];
  if (is_device_ptr(loglik)) CK(cudaMemcpy(loglik, &ll, sizeof(double), cudaMemcpyHostToDevice));
  else *loglik = ll;
  return int(p->h_res[1]) == ST_OK ? PF_OK : PF_EDEGENERATE;
}

extern "C" pf_status pf_sample_path(pf_filter* f, const double* theta, const double* y,
                                    uint64_t seed, double* loglik, double* path,
                                    int32_t* path_index, void* cuda_stream) {
  if (!f) return fail(PF_EINVAL, "filter is NULL");
  if (!theta || !y || !loglik || !path) return fail(PF_EINVAL, "theta, y, loglik and path are required");
  pf_status ps = ensure_history(f);
  if (ps == PF_OK) ps = ensure_plan(f);
  if (ps != PF_OK) return ps;
  const int T = f->T, N = f->m.N;
  if (!f->path) {
    if (cudaMalloc((void**)&f->path, sizeof(double) * size_t(T + 1) * N) != cudaSuccess ||
        cudaMalloc((void**)&f->path_idx, sizeof(int32_t) * size_t(T + 1)) != cudaSuccess) {
      cudaGetLastError();
      return fail(PF_ENOMEM, "path buffers");
    }
  }
  Plan* p = f->plan;
  f->last = p;
  cudaStream_t st = cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : f->own;
  f->range_pos = -1;
  // pass 1: the filter with its ancestor history, then the pick and the trace
  const int32_t hist_on = 1;
  ps = run_plan(p, &theta, &y, &seed, &hist_on, st, nullptr);
  if (ps != PF_OK) return ps;
  CK(cudaMemsetAsync(f->path_idx + T, 0x7f, sizeof(int32_t), st));
  CK(launch_path_pick(p->d_fds, f->sh.ntiles, f->path_idx + T, st));
  CK(launch_path_trace(p->d_fds, f->path_idx, st));
  // pass 2: the same run again (same descriptor, so bit-identical states),
  // copying x(t_i) of particle b_i after each propagate
  const int prec = f->m.prec;
  const int P = int(f->P);
  CK(enqueue_steps(
      p, 1, T, st, nullptr,
      [&](int i) { return launch_path_copy(f->x[i & 1], prec, N, P, f->path_idx, i, f->path, st); },
      true));
  CK(cudaMemcpyAsync(path, f->path, sizeof(double) * size_t(T + 1) * N, cudaMemcpyDefault, st));
  if (path_index)
    CK(cudaMemcpyAsync(path_index, f->path_idx, sizeof(int32_t) * size_t(T + 1),
                       cudaMemcpyDefault, st));
  CK(cudaEventRecord(p->ev_done, st));
  CK(cudaEventSynchronize(p->ev_done));
  const double ll = p->h_res[0];
  if (is_device_ptr(loglik)) CK(cudaMemcpy(loglik, &ll, sizeof(double), cudaMemcpyHostToDevice));
  else *loglik = ll;
  return int(p->h_res[1]) == ST_OK ? PF_OK : PF_EDEGENERATE;
}

// ---------------------------------------------------------------------------
// teacher-forced step (diagnostic)
// ---------------------------------------------------------------------------
extern "C" pf_status pf_debug_step(pf_filter* f, const double* theta, const double* y,
                                   uint64_t seed, int32_t i, const void* x_prev,
                                   const int32_t* anc, void* x_out, double* incr,
                                   int32_t* anc_next) {
  if (!f) return fail(PF_EINVAL, "filter is NULL");
  if (!theta || !y || !x_prev) return fail(PF_EINVAL, "theta, y and x_prev are required");
  if (i < 1 || i > f->T) return fail(PF_EINVAL, "step %d is not in [1, %d]", i, f->T);
  pf_status ps = ensure_plan(f);
  if (ps != PF_OK) return ps;
  Plan* p = f->plan;
  f->last = p;
  cudaStream_t st = f->own;
  f->range_pos = -1;
  CK(cudaEventSynchronize(p->ev_staged));
  FilterDev& d = p->h_fds[0];
  d = f->desc;
  d.y = p->d_ycat;
  d.seed = seed;
  const int nth = pf_theta_size(f->m.kind);
  const bool dev_theta = is_device_ptr(theta);
  if (!dev_theta) memcpy(d.theta, theta, sizeof(double) * nth);
  CK(cudaMemcpyAsync(p->d_fds, p->h_fds, sizeof(FilterDev), cudaMemcpyHostToDevice, st));
  if (dev_theta)
    CK(cudaMemcpyAsync(p->d_fds[0].theta, theta, sizeof(double) * nth, cudaMemcpyDeviceToDevice,
                       st));
  const size_t ny = size_t(f->T) * f->sh.Ny;
  if (is_device_ptr(y)) {
    CK(cudaMemcpyAsync(p->d_ycat, y, sizeof(double) * ny, cudaMemcpyDeviceToDevice, st));
  } else {
    memcpy(p->h_ycat, y, sizeof(double) * ny);
    CK(cudaMemcpyAsync(p->d_ycat, p->h_ycat, sizeof(double) * ny, cudaMemcpyHostToDevice, st));
  }
  CK(cudaEventRecord(p->ev_staged, st));
  const size_t xs = size_t(f->m.N) * size_t(f->P) * f->sh.state_bytes;
  CK(cudaMemcpyAsync(f->x[(i - 1) & 1], x_prev, xs, cudaMemcpyDefault, st));
  if (anc) CK(cudaMemcpyAsync(f->anc, anc, size_t(f->P) * 4, cudaMemcpyDefault, st));
  CK(launch_debug_ctl(p->d_fds, i, anc ? 0 : 1, st));
  // step i's propagate and resample launches, as in a run
  CK(enqueue_plan_steps(p, i, i, false, st));
  if (anc_next && i < f->T) {
    CK(launch_next_ancestors(p->d_fds, f->sh.ntiles, f->anc, st));
    CK(cudaMemcpyAsync(anc_next, f->anc, size_t(f->P) * 4, cudaMemcpyDefault, st));
  }
  CK(cudaMemcpyAsync(p->h_res, p->d_res, sizeof(double) * 3, cudaMemcpyDeviceToHost, st));
  if (x_out) CK(cudaMemcpyAsync(x_out, f->x[i & 1], xs, cudaMemcpyDefault, st));
  CK(cudaEventRecord(p->ev_done, st));
  CK(cudaEventSynchronize(p->ev_done));
  const double ll = p->h_res[0];
  if (incr) {
    if (is_device_ptr(incr)) CK(cudaMemcpy(incr, &ll, sizeof(double), cudaMemcpyHostToDevice));
    else *incr = ll;
  }
  // the filter now stands at t_i; a continuation resumes from here
  f->range_pos = int(p->h_res[1]) == ST_OK ? i : -1;
  return int(p->h_res[1]) == ST_OK ? PF_OK : PF_EDEGENERATE;
}

extern "C" pf_status pf_wait(pf_filter* f) {
  if (!f) return fail(PF_EINVAL, "filter is NULL");
  if (!f->last) return PF_OK;
  CK(cudaEventSynchronize(f->last->ev_done));
  f->pending = false;
  return int(f->last->h_res[1]) == ST_OK ? PF_OK : PF_EDEGENERATE;
}

extern "C" pf_status pf_destroy(pf_filter* f) {
  if (!f) return PF_OK;
  // the filter's own work only: an asynchronous run ends with its plan's
  // ev_done, set-up work runs on f->own, and destroy_plan drains the streams
  // of every plan the filter is part of (the batched forms are synchronous)
  if (f->plan && f->plan->ev_done) cudaEventSynchronize(f->plan->ev_done);
  if (f->wplan && f->wplan->ev_done) cudaEventSynchronize(f->wplan->ev_done);
  if (f->own) cudaStreamSynchronize(f->own);
  {
    std::lock_guard<std::mutex> lk(g_plan_mu);
    for (auto it = g_plans.begin(); it != g_plans.end();) {
      if (std::find(it->first.begin(), it->first.end(), f) != it->first.end()) {
        destroy_plan(it->second);
        it = g_plans.erase(it);
      } else {
        ++it;
      }
    }
    for (auto it = g_shapes.begin(); it != g_shapes.end();) {
      if (std::find(it->first.begin(), it->first.end(), f) != it->first.end())
        it = g_shapes.erase(it);
      else
        ++it;
    }
  }
  destroy_plan(f->plan);
  destroy_plan(f->wplan);
  free_filter_buffers(f);
  delete f->prof;
  delete f;
  return PF_OK;
}

// ---------------------------------------------------------------------------
// batched
// ---------------------------------------------------------------------------
// The cached launch plan of a filter list (built on first use; at most eight
// are kept, the oldest evicted).  The filters must be distinct.
pf_status pfb::batch_plan(const std::vector<pf_filter*>& key, Plan** out) {
  pf_batch_shape shape = kDefaultShape;
  {
    std::lock_guard<std::mutex> lk(g_plan_mu);
    auto it = g_plans.find(key);
    if (it != g_plans.end()) {
      *out = it->second;
      return PF_OK;
    }
    auto c = g_shapes.find(key);
    if (c != g_shapes.end()) shape = c->second;
  }
  Plan* p = nullptr;
  pf_status ps = build_plan(key, &p, shape);
  if (ps != PF_OK) return ps;
  std::lock_guard<std::mutex> lk(g_plan_mu);
  if (g_plans.size() >= 8) {
    destroy_plan(g_plans.begin()->second);
    g_plans.erase(g_plans.begin());
  }
  g_plans[key] = p;
  *out = p;
  return PF_OK;
}

extern "C" pf_status pf_batch_run(int32_t nfilt, pf_filter* const* f, const double* const* theta,
                                  const double* const* y, const uint64_t* seeds, double* logliks,
                                  int32_t* per_filter_status, void* cuda_stream) {
  if (nfilt < 1 || !f || !theta || !y || !seeds || !logliks || !per_filter_status)
    return fail(PF_EINVAL, "pf_batch_run: bad arguments");
  std::vector<pf_filter*> key(f, f + nfilt);
  for (int k = 0; k < nfilt; ++k)
    if (!key[k]) return fail(PF_EINVAL, "filter %d is NULL", k);
  {
    std::vector<pf_filter*> sorted(key);
    std::sort(sorted.begin(), sorted.end());
    if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end())
      return fail(PF_EINVAL, "a filter appears twice in the batch");
  }
  Plan* p = nullptr;
  pf_status bs = batch_plan(key, &p);
  if (bs != PF_OK) return bs;
  cudaStream_t st = cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : p->st;
  for (int k = 0; k < nfilt; ++k) key[k]->range_pos = -1;
  pf_status ps = run_plan(p, theta, y, seeds, nullptr, st, nullptr);
  if (ps != PF_OK) return ps;
  CK(cudaEventSynchronize(p->ev_done));
  if (p->persist_set != 0) {
    ps = persist_status(p, *p->h_perr);
    if (ps != PF_OK) return ps;
  }
  for (int k = 0; k < nfilt; ++k) {
    logliks[k] = p->h_res[3 * k];
    per_filter_status[k] = int(p->h_res[3 * k + 1]) == ST_OK ? PF_OK : PF_EDEGENERATE;
  }
  return PF_OK;
}

static pf_status batch_key(int32_t nfilt, pf_filter* const* f, std::vector<pf_filter*>* key) {
  if (nfilt < 1 || !f) return fail(PF_EINVAL, "empty filter list");
  key->assign(f, f + nfilt);
  for (int k = 0; k < nfilt; ++k)
    if (!(*key)[k]) return fail(PF_EINVAL, "filter %d is NULL", k);
  std::vector<pf_filter*> sorted(*key);
  std::sort(sorted.begin(), sorted.end());
  if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end())
    return fail(PF_EINVAL, "a filter appears twice in the batch");
  return PF_OK;
}

static bool same_shape(const pf_batch_shape& a, const pf_batch_shape& b) {
  return a.cta_max_particles == b.cta_max_particles && a.branches == b.branches &&
         a.resample_blocks_per_sm == b.resample_blocks_per_sm &&
         a.persistent_blocks_per_sm == b.persistent_blocks_per_sm &&
         a.tiles_per_item == b.tiles_per_item;
}

extern "C" pf_status pf_batch_set_shape(int32_t nfilt, pf_filter* const* f,
                                        const pf_batch_shape* shape) {
  std::vector<pf_filter*> key;
  pf_status ps = batch_key(nfilt, f, &key);
  if (ps != PF_OK) return ps;
  if (!shape) return fail(PF_EINVAL, "shape is NULL");
  if (shape->cta_max_particles < 0) return fail(PF_EINVAL, "cta_max_particles must be >= 0");
  if (shape->branches < 1) return fail(PF_EINVAL, "branches must be >= 1");
  if (shape->resample_blocks_per_sm < 1 || shape->resample_blocks_per_sm > 8)
    return fail(PF_EINVAL, "resample_blocks_per_sm must be in 1..8");
  if (shape->persistent_blocks_per_sm < 0 || shape->persistent_blocks_per_sm > 8)
    return fail(PF_EINVAL, "persistent_blocks_per_sm must be in 0..8");
  const int kt = shape->tiles_per_item;
  if (kt != 1 && kt != 2 && kt != 4 && kt != 8)
    return fail(PF_EINVAL, "tiles_per_item must be 1, 2, 4 or 8");
  std::lock_guard<std::mutex> lk(g_plan_mu);
  g_shapes[key] = *shape;
  auto it = g_plans.find(key);
  if (it != g_plans.end() && !same_shape(it->second->shape, *shape)) {
    destroy_plan(it->second);  // rebuilt with the new shape on its next use
    g_plans.erase(it);
  }
  return PF_OK;
}

extern "C" pf_status pf_batch_get_shape(int32_t nfilt, pf_filter* const* f,
                                        pf_batch_shape* shape) {
  std::vector<pf_filter*> key;
  pf_status ps = batch_key(nfilt, f, &key);
  if (ps != PF_OK) return ps;
  if (!shape) return fail(PF_EINVAL, "shape is NULL");
  std::lock_guard<std::mutex> lk(g_plan_mu);
  auto it = g_shapes.find(key);
  *shape = it != g_shapes.end() ? it->second : kDefaultShape;
  return PF_OK;
}

extern "C" pf_status pf_batch_configure(int32_t nfilt, pf_filter* const* f,
                                        int64_t cta_max_particles) {
  pf_batch_shape shape = kDefaultShape;
  pf_status ps = pf_batch_get_shape(nfilt, f, &shape);
  if (ps != PF_OK) return ps;
  shape.cta_max_particles = cta_max_particles;
  return pf_batch_set_shape(nfilt, f, &shape);
}

// Host-clock time of the list's batch run with the given shape: one untimed
// run (plan and graph), then the mean of two timed ones.
static pf_status time_shape(int32_t nfilt, pf_filter* const* f, const double* const* theta,
                            const double* const* y, const uint64_t* seeds,
                            const pf_batch_shape& shape, double* ms) {
  std::vector<double> ll(nfilt > 0 ? nfilt : 1);
  std::vector<int32_t> st(nfilt > 0 ? nfilt : 1);
  pf_status ps = pf_batch_set_shape(nfilt, f, &shape);
  if (ps != PF_OK) return ps;
  double acc = 0.0;
  for (int rep = 0; rep < 3; ++rep) {
    const auto t0 = std::chrono::steady_clock::now();
    ps = pf_batch_run(nfilt, f, theta, y, seeds, ll.data(), st.data(), nullptr);
    if (ps != PF_OK) return ps;
    const auto t1 = std::chrono::steady_clock::now();
    if (rep > 0) acc += std::chrono::duration<double, std::milli>(t1 - t0).count();
  }
  *ms = acc / 2.0;
  return PF_OK;
}

extern "C" pf_status pf_batch_autotune(int32_t nfilt, pf_filter* const* f,
                                       const double* const* theta, const double* const* y,
                                       const uint64_t* seeds, int64_t* chosen) {
  static const int64_t cta_bounds[] = {0, 256, 512, 1024, 2048};
  static const int32_t branch_counts[] = {1, 2, 4, 8, 16};
  static const int32_t rs_grids[] = {2, 4, 8};
  static const int32_t persist_bps[] = {2, 3, 4};
  static const int32_t tiles_items[] = {1, 2, 4};
  pf_batch_shape best = kDefaultShape;
  double best_ms = 0.0;
  pf_status ps = time_shape(nfilt, f, theta, y, seeds, best, &best_ms);
  if (ps != PF_OK) return ps;
  // one field at a time, from the default; the persistent launch's CTAs per
  // SM and tiles per item jointly (its best shape needs both)
  for (int field = 0; field < 4; ++field) {
    const pf_batch_shape base = best;
    std::vector<pf_batch_shape> cands;
    pf_batch_shape c = base;
    if (field == 0) {
      for (int64_t b : cta_bounds) {
        c.cta_max_particles = b;
        cands.push_back(c);
      }
    } else if (field == 1) {
      for (int32_t b : branch_counts) {
        c.branches = b;
        cands.push_back(c);
      }
    } else if (field == 2) {
      for (int32_t g : rs_grids) {
        c.resample_blocks_per_sm = g;
        cands.push_back(c);
      }
    } else {
      c.persistent_blocks_per_sm = 0;
      c.tiles_per_item = 1;
      cands.push_back(c);
      for (int32_t b : persist_bps)
        for (int32_t k : tiles_items) {
          c.persistent_blocks_per_sm = b;
          c.tiles_per_item = k;
          cands.push_back(c);
        }
    }
    for (const pf_batch_shape& cand : cands) {
      if (same_shape(cand, base)) continue;
      double ms = 0.0;
      ps = time_shape(nfilt, f, theta, y, seeds, cand, &ms);
      if (ps != PF_OK) return ps;
      if (ms < best_ms) {
        best_ms = ms;
        best = cand;
      }
    }
  }
  ps = pf_batch_set_shape(nfilt, f, &best);
  if (ps == PF_OK && chosen) *chosen = best.cta_max_particles;
  return ps;
}

// ---------------------------------------------------------------------------
// diagnostics
// ---------------------------------------------------------------------------
extern "C" pf_status pf_profile_enable(pf_filter* f, int32_t on) {
  if (!f) return fail(PF_EINVAL, "filter is NULL");
  if (on && !f->prof) f->prof = new Profiler();
  if (!on) {
    delete f->prof;
    f->prof = nullptr;
  }
  return PF_OK;
}

extern "C" pf_status pf_profile_read(pf_filter* f, double* ms, int64_t* launches) {
  if (!f || !f->prof) return fail(PF_EINVAL, "profiling is not enabled on this filter");
  return f->prof->read(ms, launches);
}
