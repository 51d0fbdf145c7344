// pf_noalloc.cu -- pf_run_noalloc: one filter run that allocates no memory.
//
// Some callers cannot allocate device memory at the point where they need a
// likelihood: code that runs while a caller-owned memory pool or arena holds
// the whole device budget, code inside a framework that forbids allocation
// on its hot path (allocation can synchronise the device or fail under
// fragmentation), or real-time loops that must not touch the allocator at
// all.  For them this entry point runs the same kernels as pf_run, with every
// internal buffer (descriptor, tile map, particle state, weights, ancestors,
// partial sums, control block) carved out of one file-scope device array of
// fixed size, g_noalloc_scratch, kept until the process exits.
//
// The array belongs to this file's device module, which CUDA loads on a
// device lazily: the first call on each device loads it there, and that load
// is what reserves the array's device memory.  So a caller should make one
// call on every device it uses at set-up, before its own pool takes the
// device budget and before any stream capture.
//
// The host never dereferences the array's name: on the host that name is
// only a stand-in, so every call looks up the array's device address on the
// current device with cudaGetSymbolAddress (cheap once the module is loaded,
// and never stale after a device reset) and hands only that address to the
// kernels.
#include <cstring>

#include "pf.h"
#include "pf_internal.h"
#include "pf_runtime.h"

using namespace pfb;

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[PF_NOALLOC_SCRATCH_BYTES];


// Copy the descriptor (by value) and theta (device pointer) into the scratch
// descriptor, and write the single-filter tile map (0, t).
__global__ void k_noalloc_setup(FilterDev desc, const double* __restrict__ theta, int ntheta,
                                FilterDev* __restrict__ d_desc, int2* __restrict__ tmap,
                                int ntiles) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k == 0) {
    for (int c = 0; c < ntheta; ++c) desc.theta[c] = theta[c];
    *d_desc = desc;
  }
  if (k < ntiles) tmap[k] = make_int2(0, k);
}

// Copy the run's log-likelihood and status to the caller's outputs.
__global__ void k_noalloc_out(const FilterDev* __restrict__ d_desc, double* __restrict__ loglik,
                              int32_t* __restrict__ status) {
  const Ctl* c = d_desc->ctl;
  *loglik = __ldcg(&c->ll);
  if (status) *status = __ldcg(&c->status) == ST_OK ? PF_OK : PF_EDEGENERATE;
}

pf_status scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return fail(PF_ECUDA, "pf_run_noalloc: no current CUDA device");
  }
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p) {
    cudaGetLastError();
    return fail(PF_ECUDA, "pf_run_noalloc: cudaGetSymbolAddress on device %d: %s", dev,
                cudaGetErrorString(e));
  }
  *out = p;
  return PF_OK;
}

// True when ptr is memory the current device's kernels can address (device or
// managed memory).  cudaPointerGetAttributes allocates nothing; a host array
// passed by mistake is refused here instead of faulting in a kernel.
bool device_addressable(const void* ptr) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Bump allocator over the scratch array (256-byte aligned regions).
struct Carve {
  char* base;
  size_t off = 0;
  template <typename T>
  T* take(size_t bytes) {
    T* p = reinterpret_cast<T*>(base + off);
    off += (bytes + 255) & ~size_t(255);
    return p;
  }
};

size_t layout_bytes(const pf_model* m, const Shape& sh, int64_t P) {
  Carve c{nullptr};
  const size_t xs = size_t(m->N) * size_t(P) * sh.state_bytes;
  c.take<FilterDev>(sizeof(FilterDev));
  c.take<int2>(sizeof(int2) * size_t(sh.ntiles));
  c.take<char>(xs);
  c.take<char>(xs);
  c.take<double>(8 * size_t(P));
  if (sh.mode != MODE_ALWAYS) {
    c.take<double>(8 * size_t(P));
    c.take<double>(8 * size_t(P));
  }
  c.take<int32_t>(4 * size_t(P));
  c.take<double>(8 * size_t(sh.nflow));
  c.take<TilePart>(sizeof(TilePart) * size_t(sh.ntiles));
  c.take<GroupPart>(sizeof(GroupPart) * size_t(sh.ngroups));
  c.take<Ctl>(sizeof(Ctl));
  return c.off;
}

}  // namespace

extern "C" pf_status pf_run_noalloc(const pf_model* m, int64_t P, int32_t T, double dt,
                                    const double* theta, const double* y, uint64_t seed,
                                    double* loglik, int32_t* status, void* final_particles,
                                    void* cuda_stream) {
  Shape sh;
  pf_status st = check_shape(m, P, T, dt, &sh);
  if (st != PF_OK) return st;
  if (m->resampler == PF_RESAMPLE_MULTINOMIAL)
    return fail(PF_EINVAL, "pf_run_noalloc does not take the multinomial resampler");
  if (!theta || !y || !loglik) return fail(PF_EINVAL, "pf_run_noalloc: theta, y, loglik required");
  {
    const void* ptrs[] = {theta, y, loglik, status, final_particles};
    const char* names[] = {"theta", "y", "loglik", "status", "final_particles"};
    for (int k = 0; k < 5; ++k)
      if (ptrs[k] && !device_addressable(ptrs[k]))
        return fail(PF_EINVAL, "pf_run_noalloc: %s is not device memory of the current device",
                    names[k]);
  }
  const size_t need = layout_bytes(m, sh, P);
  if (need > size_t(PF_NOALLOC_SCRATCH_BYTES))
    return fail(PF_EINVAL,
                "pf_run_noalloc: this filter needs %zu bytes of scratch, the fixed array holds %zu "
                "(use pf_create/pf_run for larger filters)",
                need, size_t(PF_NOALLOC_SCRATCH_BYTES));
  void* scratch = nullptr;
  st = scratch_address(&scratch);
  if (st != PF_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);

  Carve c{static_cast<char*>(scratch)};
  const size_t xs = size_t(m->N) * size_t(P) * sh.state_bytes;
  FilterDev* d_desc = c.take<FilterDev>(sizeof(FilterDev));
  int2* tmap = c.take<int2>(sizeof(int2) * size_t(sh.ntiles));
  FilterDev d;
  memset(&d, 0, sizeof d);
  d.x[0] = c.take<char>(xs);
  d.x[1] = c.take<char>(xs);
  d.ctil = c.take<double>(8 * size_t(P));
  if (sh.mode != MODE_ALWAYS) {
    d.ell = c.take<double>(8 * size_t(P));
    d.lam = c.take<double>(8 * size_t(P));
  }
  d.anc = c.take<int32_t>(4 * size_t(P));
  double* flow = c.take<double>(8 * size_t(sh.nflow));
  d.tp = c.take<TilePart>(sizeof(TilePart) * size_t(sh.ntiles));
  d.gp = c.take<GroupPart>(sizeof(GroupPart) * size_t(sh.ngroups));
  d.ctl = c.take<Ctl>(sizeof(Ctl));
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
  d.seed = seed;
  d.dt = dt;
  d.thr = m->ess_threshold;
  d.y = y;
  d.flow = sh.nflow ? flow : nullptr;

  // The array keeps the previous call's contents: zero the group tickets and
  // the control block before this run (the init kernel also resets them).
  cudaError_t e = cudaMemsetAsync(d.gp, 0, sizeof(GroupPart) * size_t(sh.ngroups), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(d.ctl, 0, sizeof(Ctl), s);
  if (e == cudaSuccess) {
    const int nb = (sh.ntiles + 255) / 256;
    k_noalloc_setup<<<nb, 256, 0, s>>>(d, theta, pf_theta_size(m->kind), d_desc, tmap,
                                       sh.ntiles);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && sh.nflow)
    e = launch_flow(flow, sh.nflow, m->flow_peak, m->flow_period, dt, s);
  if (e == cudaSuccess) e = launch_init(m->kind, m->N, m->prec, d_desc, tmap, sh.ntiles, s);
  for (int i = 1; i <= T && e == cudaSuccess; ++i) {
    e = launch_propagate(m->kind, m->N, m->prec, d_desc, tmap, sh.ntiles, s);
    if (e == cudaSuccess && i < T) e = launch_resample(d_desc, tmap, sh.ntiles, s);
  }
  if (e == cudaSuccess) {
    k_noalloc_out<<<1, 1, 0, s>>>(d_desc, loglik, status);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && final_particles)
    e = cudaMemcpyAsync(final_particles, d.x[T & 1], xs, cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return fail(PF_ECUDA, "pf_run_noalloc: %s", cudaGetErrorString(e));
  return PF_OK;
}
