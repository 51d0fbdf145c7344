// pf_runtime.h -- host runtime objects shared by pf_api.cu and pf_server.cu.
#pragma once
#include <cstdint>
#include <vector>

#include "pf.h"
#include "pf_internal.h"

namespace pfb {

struct Shape {
  int Ny = 1;
  uint64_t obs_mask = 1;
  int ntiles = 0, ngroups = 0, mode = MODE_ALWAYS;
  size_t state_bytes = 8;
  int64_t nflow = 0;
};

struct PlanClass {
  int kind, N, prec;
  int offset;   // first entry of the class's tiles in Plan::d_tmap
  int ntiles;
  int sub = 1;  // propagate blocks per tile (k_propagate_sub; a filter running alone)
};

struct Plan;

enum { PROF_INIT = 0, PROF_PROPAGATE = 1, PROF_RESAMPLE = 2, PROF_RESULTS = 3, PROF_KINDS = 4 };

// Per-launch CUDA-event timing of direct (non-graph) runs, summed per kernel kind.
struct Profiler {
  struct Pair {
    int kind;
    cudaEvent_t a, b;
  };
  std::vector<cudaEvent_t> pool;
  std::vector<Pair> pairs;
  size_t next = 0;
  cudaEvent_t take() {
    if (next == pool.size()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      pool.push_back(e);
    }
    return pool[next++];
  }
  void begin(int kind, cudaStream_t st) {
    Pair pr{kind, take(), nullptr};
    cudaEventRecord(pr.a, st);
    pairs.push_back(pr);
  }
  void end(cudaStream_t st) {
    pairs.back().b = take();
    cudaEventRecord(pairs.back().b, st);
  }
  pf_status read(double* ms, int64_t* launches) {
    double acc[PROF_KINDS] = {0, 0, 0, 0};
    int64_t cnt[PROF_KINDS] = {0, 0, 0, 0};
    for (const Pair& pr : pairs) {
      if (cudaEventSynchronize(pr.b) != cudaSuccess) return PF_ECUDA;
      float t = 0.f;
      cudaEventElapsedTime(&t, pr.a, pr.b);
      acc[pr.kind] += t;
      cnt[pr.kind] += 1;
    }
    for (int k = 0; k < PROF_KINDS; ++k) {
      if (ms) ms[k] = acc[k];
      if (launches) launches[k] = cnt[k];
    }
    pairs.clear();
    next = 0;
    return PF_OK;
  }
  ~Profiler() {
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
  }
};

}  // namespace pfb

struct pf_filter {
  pf_model m{};
  int64_t P = 0;
  int32_t T = 0;
  double dt = 0.0;
  int device = 0;
  pfb::Shape sh;
  cudaStream_t own = nullptr;
  void* x[2] = {nullptr, nullptr};
  double* ctil = nullptr;
  double* ell = nullptr;
  double* lam = nullptr;
  int32_t* anc = nullptr;
  int32_t* hist = nullptr;
  double* mn_t = nullptr;        // multinomial resampling: spacing sums [P]
  double* mn_part = nullptr;     // multinomial resampling: tile offsets [ntiles + 1]
  double* path = nullptr;        // [T+1][N] sampled path (pf_sample_path)
  int32_t* path_idx = nullptr;   // [T+1] its particle indices
  double* flow = nullptr;
  double* znoise = nullptr;      // FP64 windkessel: normals drawn ahead [T * s][P] (small filters)
  pfb::TilePart* tp = nullptr;
  pfb::GroupPart* gp = nullptr;
  pfb::Ctl* ctl = nullptr;
  double* h_res = nullptr;
  pfb::FilterDev desc{};
  pfb::Plan* plan = nullptr;      // tiled single-filter plan: intervals, paths, debug steps
  pfb::Plan* wplan = nullptr;     // whole runs (pf_run): the cluster path for a small filter
  pfb::Plan* last = nullptr;      // the plan of the last pf_run (pf_wait)
  pfb::Profiler* prof = nullptr;
  bool pending = false;
  int32_t range_pos = -1;        // t_s reached by the last pf_run_range, else -1
  size_t bytes = 0;
};

namespace pfb {

// One independent chain of per-step launches over some of a plan's tiled
// filters: its tile maps (sorted by T, descending) and per-step tile counts.
// The branches of a plan run concurrently, each at its own pace (branch 0 on
// the launching stream, the others on their own streams, forked and joined
// with events, so a captured graph holds them as parallel branches).
struct Branch {
  std::vector<PlanClass> classes;           // offset / ntiles into Plan::d_tmap
  std::vector<int> noise;                   // filters whose FP64 normals are drawn ahead
  int all_offset = 0;                       // the branch's all-tiles map in Plan::d_tmap
  int maxT = 0;
  bool has_mn = false;                      // some filter resamples multinomially
  std::vector<int> cnt_all;                 // [i]: tiles of the branch's filters with T >= i
  std::vector<std::vector<int>> cnt_cls;    // per class
  cudaStream_t st = nullptr;                // branches 1..: their own stream
  cudaEvent_t ev_join = nullptr;
};

// A launch plan: descriptors of its filters, tile maps and one instantiated
// CUDA graph covering the whole run.
struct Plan {
  std::vector<pf_filter*> filters;
  int nf = 0, maxT = 0, ntiles_all = 0;     // d_tmap[0, ntiles_all): every tiled filter's tiles
  bool has_mn = false;                      // some filter resamples multinomially
  bool use_noise = false;                   // single filter: FP64 normals drawn ahead
  pf_batch_shape shape{0, 1, 8};            // the launch shape the plan was built for
  std::vector<Branch> branches;
  cudaEvent_t ev_fork_br = nullptr;         // forks the branches off the launching stream
  std::vector<size_t> yoff;                 // offset of each filter's y in d_ycat
  FilterDev* d_fds = nullptr;
  FilterDev* h_fds = nullptr;               // pinned
  int2* d_tmap = nullptr;
  double* d_ycat = nullptr;
  double* h_ycat = nullptr;                 // pinned
  double* d_res = nullptr;
  double* h_res = nullptr;                  // pinned
  cudaStream_t st = nullptr;
  cudaEvent_t ev_staged = nullptr, ev_done = nullptr;
  cudaGraphExec_t exec = nullptr;
  // cluster path: filters with at most cta_max_p particles (0: none) and at
  // most MAX_CLUSTER_TILES tiles run whole, one thread-block cluster each, on
  // a side branch of the graph
  int cta_total = 0;
  std::vector<PlanClass> cta_classes;       // offset / ntiles = first / count in d_cta
  std::vector<int> cta_cluster;             // cluster size (= tiles) of each of those
  std::vector<int> cta_noise;               // cluster filters whose FP64 normals are drawn ahead
  int* d_cta = nullptr;                     // filter indices, per class
  cudaStream_t st2 = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // persistent launch (k_persist) of the tiled filters, when the shape asks
  // for it and the plan qualifies: the class set of the kernel (0: the
  // per-step chains), tiles per item, the queue and its slots, the slot array
  // every run starts from (each level's first items, the rest empty) and the
  // queue header every run starts from
  int persist_set = 0;
  int persist_kt = 1;
  unsigned long long persist_total = 0;
  PersistQueue* d_pq = nullptr;
  PersistQueue* d_pq_init = nullptr;
  unsigned long long* d_slots = nullptr;
  unsigned long long* d_slots_init = nullptr;
  int* h_perr = nullptr;                    // pinned: the run's queue error
};

pf_status fail(pf_status st, const char* fmt, ...);
// Host-side fault injection (pf_debug_fail_allocation): true for the one
// device allocation of a filter or a served request chosen to fail.
bool injected_alloc_failure();
// ... (pf_debug_fail_server_wait): true for the one wait of a server's
// scheduler chosen to report a CUDA error.
bool injected_wait_failure();
pf_status check_shape(const pf_model* m, int64_t P, int32_t T, double dt, Shape* sh);
pf_status build_plan(const std::vector<pf_filter*>& fl, Plan** out, const pf_batch_shape& shape);
pf_status stage_plan(Plan* p, const double* const* theta, const double* const* y,
                     const uint64_t* seeds, const int32_t* hist_on, cudaStream_t st);
pf_status run_plan(Plan* p, const double* const* theta, const double* const* y,
                   const uint64_t* seeds, const int32_t* hist_on, cudaStream_t st,
                   Profiler* prof);
pf_status batch_plan(const std::vector<pf_filter*>& key, Plan** out);
// After a run of the plan has completed: err (the run's queue error word, read
// back by run_plan into h_perr) as a status, PF_OK without a persistent launch.
pf_status persist_status(const Plan* p, int err);
// Direct launches of steps first..last of a plan (with the initial draw when
// init), then the results gather; no staging, no graph.
cudaError_t enqueue_plan_steps(Plan* p, int first, int last, bool init, cudaStream_t st);

}  // namespace pfb
