// pf_internal.h -- host-side launchers shared by the runtime translation units.
#pragma once
#include <cuda_runtime.h>

#include "pf_dev.cuh"

namespace pfb {

// The invariant-violation counters of a checked build (CHK_KINDS of them),
// copied to out and zeroed (diagnostic).
cudaError_t read_checks(unsigned long long* out);
// The propagate kernels' weight exponential on n device values (diagnostic).
cudaError_t launch_weight_exp(const double* d, double* w, int64_t n, cudaStream_t st);
cudaError_t launch_tile_prefix(const double* w, double* prefix, double* total, int64_t n,
                               cudaStream_t st);
cudaError_t launch_log_sum(const double* s, double* y, int64_t n, cudaStream_t st);

bool supported(int kind, int N, int prec);
cudaError_t launch_init(int kind, int N, int prec, const FilterDev* fds, const int2* tmap,
                        int nblocks, cudaStream_t st);
cudaError_t launch_propagate(int kind, int N, int prec, const FilterDev* fds, const int2* tmap,
                             int nblocks, cudaStream_t st);
// The sub-tile propagate launch (k_propagate_sub): propagate_sub gives the
// blocks per tile (1, 2 or 4) for tiles of this class in a plan of ntiles
// tiles in all; launch_propagate_sub launches with it (sub = 1:
// launch_propagate).  Same results as launch_propagate.
int propagate_sub(int kind, int N, int prec, int ntiles);
cudaError_t launch_propagate_sub(int kind, int N, int prec, int sub, const FilterDev* fds,
                                 const int2* tmap, int ntiles, cudaStream_t st);
// resample kernel over the listed tiles, its grid at most blocks_per_sm (1..8)
// blocks per SM
cudaError_t launch_resample(const FilterDev* fds, const int2* tmap, int nblocks, cudaStream_t st,
                            int blocks_per_sm = 8);
// the FP64 windkessel normals of filter fds[k] (P particles, s substeps) for
// steps first..last drawn ahead into its table
cudaError_t launch_noise(const FilterDev* fds, int k, int first, int last, int P, int s,
                         cudaStream_t st);
// the control block of fds[0] set to propagate to t_step from a loaded state,
// ancestors from the array (anc_identity 0) or the identity (diagnostic)
cudaError_t launch_debug_ctl(const FilterDev* fds, int step, int anc_identity, cudaStream_t st);
// the ancestors the next propagation of fds[0] takes, into out [P] (diagnostic)
cudaError_t launch_next_ancestors(const FilterDev* fds, int ntiles, int32_t* out,
                                  cudaStream_t st);
// one thread-block cluster of cluster_size CTAs per listed filter runs its
// whole run (initial draw and all steps); the filters have at most
// cluster_size tiles
cudaError_t launch_filter_cluster(int kind, int N, int prec, const FilterDev* fds,
                                  const int* list, int nfilters, int cluster_size,
                                  cudaStream_t st);
// The batched form's persistent launch (k_persist): the model-class bit of
// the persistent kernel for (kind, N, prec), 0 when it has none; whether a set
// of class bits has a compiled kernel; the launch over queue q (kt tiles per
// item, a power of two up to MAX_CLUSTER_TILES; blocks_per_sm CTAs per SM,
// capped at the kernel's occupancy).
int persist_class_bit(int kind, int N, int prec);
// The persistent kernel's wait limit in global-timer ns (current device).
cudaError_t set_persist_wait_limit(unsigned long long ns);
bool persist_set_supported(int set);
cudaError_t launch_persist(int set, const FilterDev* fds, PersistQueue* q,
                           unsigned long long* slots, int kt, int blocks_per_sm,
                           cudaStream_t st);
cudaError_t launch_flow(double* flow, int64_t n, double peak, double period, double dt,
                        cudaStream_t st);
cudaError_t launch_results(const FilterDev* fds, int nf, double* out, cudaStream_t st);
cudaError_t launch_mn_scan(const FilterDev* fds, const int2* tmap, int ntiles, int nf,
                           cudaStream_t st);
cudaError_t launch_path_pick(const FilterDev* fds, int ntiles, int32_t* pick, cudaStream_t st);
cudaError_t launch_path_trace(const FilterDev* fds, int32_t* idx, cudaStream_t st);
cudaError_t launch_path_copy(const void* x, int prec, int N, int P, const int32_t* idx, int i,
                             double* path, cudaStream_t st);

}  // namespace pfb
