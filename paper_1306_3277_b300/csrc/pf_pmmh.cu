// pf_pmmh.cu -- marginal Metropolis-Hastings chains over the parameters
// (Algorithm 3, acceptance rule Eq. mh, Sec. 3.1.3) with particle-filter
// likelihood estimates: the pseudo-marginal sampler.
//
// One iteration of all chains is three enqueued steps on one stream:
//   k_pmmh_propose   one thread per chain: theta' ~ q(.|theta), written into
//                    the chain's filter descriptor with a fresh filter key;
//   the batch plan's CUDA graph: every chain's filter over y(t_1..t_T);
//   k_pmmh_accept    one thread per chain: alpha ~ U(0, 1], accept iff
//                    alpha <= l' p(theta') q(theta|theta') / (l p(theta) q(theta'|theta)),
//                    evaluated in log space; the chain state and the sample
//                    row of the iteration are written on the device.
// The host never waits inside the loop.
//
// Random numbers (Philox key = the sampler's seed, counter (chain c,
// iteration i, (5 << 16) | block, 0)): block 0 the acceptance uniform in
// (0, 1] (words 1:0); block 1 the filter key (words 1:0 low, 3:2 high);
// block 16 + 64 d + a draw a of component d -- the first Box-Muller normal of
// the block for the truncated gaussian (attempts a = 0..63, the first inside
// the bounds is taken, none inside keeps the current value), or the unit
// exponential -log u, u in (0, 1] from words 1:0, for the inverse gamma of
// integer shape k (terms a = 0..k-1; Gamma(k, 1) is their sum).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "pf_params.cuh"
#include "pf_runtime.h"

namespace pfb {
namespace {

struct Chains {
  double* theta;    // [nc][MAX_THETA] current parameters
  double* ll;       // [nc] log-likelihood estimate at theta
  double* lp;       // [nc] log prior at theta
  double* theta_p;  // [nc][MAX_THETA] proposal
  double* lp_p;     // [nc] log prior at the proposal
  double* lqr;      // [nc] log q(theta|theta') - log q(theta'|theta)
  int32_t* acc;     // [nc] accepted moves
};

__device__ uint64_t filter_key(uint64_t seed, uint32_t c, uint32_t i) {
  return philox_key(seed, c, i, PURPOSE_PMMH, 1u);
}

__global__ void k_pmmh_start(Spec sp, FilterDev* __restrict__ fds, int nc, Chains ch,
                             uint64_t seed) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  double* tp = ch.theta_p + size_t(c) * MAX_THETA;
  for (int d = 0; d < sp.nth; ++d) fds[c].theta[d] = tp[d];
  ch.lp_p[c] = log_prior(sp, tp);
  ch.lqr[c] = 0.0;
  ch.acc[c] = 0;
  fds[c].seed = filter_key(seed, uint32_t(c), 0u);
}

__global__ void k_pmmh_propose(Spec sp, FilterDev* __restrict__ fds, int nc, Chains ch,
                               uint64_t seed, int it) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  double* out = ch.theta_p + size_t(c) * MAX_THETA;
  const double lqr = propose(sp, ch.theta + size_t(c) * MAX_THETA, seed, uint32_t(c), uint32_t(it),
                             PURPOSE_PMMH, out);
  for (int d = 0; d < sp.nth; ++d) fds[c].theta[d] = out[d];
  ch.lp_p[c] = log_prior(sp, out);
  ch.lqr[c] = lqr;
  fds[c].seed = filter_key(seed, uint32_t(c), uint32_t(it));
}

__global__ void k_pmmh_accept(Spec sp, const FilterDev* __restrict__ fds, int nc, Chains ch,
                              uint64_t seed, int it, double* __restrict__ samples_row,
                              double* __restrict__ ll_row) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  const Ctl* ctl = fds[c].ctl;
  const double llp = ldcg(&ctl->status) == ST_OK ? ldcg(&ctl->ll) : -INFINITY;
  bool accept = true;
  if (it > 0) {
    const double lpp = ch.lp_p[c];
    const uint4 w = rng_block(seed, uint32_t(c), uint32_t(it), PURPOSE_PMMH, 0u);
    const double log_alpha = log_pos(u53_open_closed(w.x, w.y));
    const double ratio = (llp + lpp + ch.lqr[c]) - (ch.ll[c] + ch.lp[c]);
    accept = lpp > -INFINITY && log_alpha <= ratio;
  }
  double* th = ch.theta + size_t(c) * MAX_THETA;
  if (accept) {
    const double* tp = ch.theta_p + size_t(c) * MAX_THETA;
    for (int d = 0; d < sp.nth; ++d) th[d] = tp[d];
    ch.ll[c] = llp;
    ch.lp[c] = ch.lp_p[c];
    if (it > 0) ch.acc[c] += 1;
  }
  for (int d = 0; d < sp.nth; ++d) samples_row[size_t(c) * sp.nth + d] = th[d];
  ll_row[c] = ch.ll[c];
}

}  // namespace
}  // namespace pfb

using namespace pfb;

#define CKP(x)                                                                        \
  do {                                                                                \
    cudaError_t e_ = (x);                                                             \
    if (e_ != cudaSuccess) {                                                          \
      cudaGetLastError();                                                             \
      ps = fail(PF_ECUDA, "%s: %s", #x, cudaGetErrorString(e_));                     \
      goto done;                                                                      \
    }                                                                                 \
  } while (0)

extern "C" pf_status pf_pmmh_run(int32_t nc, pf_filter* const* f, const double* y,
                                 const pf_param* spec, const double* theta0, int32_t niter,
                                 uint64_t seed, double* samples, double* logliks,
                                 int32_t* accepted, void* cuda_stream) {
  if (nc < 1 || !f || !y || !spec || !theta0 || niter < 0 || !samples || !logliks)
    return fail(PF_EINVAL, "pf_pmmh_run: bad arguments");
  std::vector<pf_filter*> key(f, f + nc);
  for (int c = 0; c < nc; ++c) {
    if (!key[c]) return fail(PF_EINVAL, "filter %d is NULL", c);
    if (key[c]->m.kind != key[0]->m.kind || key[c]->T != key[0]->T ||
        key[c]->sh.Ny != key[0]->sh.Ny)
      return fail(PF_EINVAL, "chain %d: every filter needs the same model kind, T and Ny", c);
  }
  {
    std::vector<pf_filter*> sorted(key);
    std::sort(sorted.begin(), sorted.end());
    if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end())
      return fail(PF_EINVAL, "a filter serves two chains");
  }
  const int nth = pf_theta_size(key[0]->m.kind);
  pf_status ps = check_spec(spec, nth);
  if (ps != PF_OK) return ps;
  Plan* p = nullptr;
  ps = batch_plan(key, &p);
  if (ps != PF_OK) return ps;
  cudaStream_t st = cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : p->st;
  for (pf_filter* fl : key) fl->range_pos = -1;

  Spec sp;
  memset(&sp, 0, sizeof sp);
  memcpy(sp.p, spec, sizeof(pf_param) * nth);
  sp.nth = nth;
  std::vector<const double*> th(nc), ys(nc, y);
  for (int c = 0; c < nc; ++c) th[c] = theta0 + size_t(c) * nth;
  std::vector<uint64_t> seeds(nc, 0);
  std::vector<double> th_pad(size_t(nc) * MAX_THETA, 0.0);
  for (int c = 0; c < nc; ++c) memcpy(&th_pad[size_t(c) * MAX_THETA], th[c], sizeof(double) * nth);

  Chains ch{};
  void* block = nullptr;
  double* d_samples = nullptr;
  double* d_ll = nullptr;
  const size_t n_samples = size_t(niter + 1) * nc * nth;
  const size_t n_ll = size_t(niter + 1) * nc;
  const int threads = 128, blocks = (nc + threads - 1) / threads;
  ps = stage_plan(p, th.data(), ys.data(), seeds.data(), nullptr, st);
  if (ps != PF_OK) return ps;
  {
    const size_t per = size_t(nc) * (2 * MAX_THETA + 4) * sizeof(double) + size_t(nc) * 4;
    CKP(cudaMalloc(&block, per + (n_samples + n_ll) * sizeof(double)));
    double* q = static_cast<double*>(block);
    ch.theta = q; q += size_t(nc) * MAX_THETA;
    ch.theta_p = q; q += size_t(nc) * MAX_THETA;
    ch.ll = q; q += nc;
    ch.lp = q; q += nc;
    ch.lp_p = q; q += nc;
    ch.lqr = q; q += nc;
    d_samples = q; q += n_samples;
    d_ll = q; q += n_ll;
    ch.acc = reinterpret_cast<int32_t*>(q);
  }
  CKP(cudaMemcpyAsync(ch.theta_p, th_pad.data(), th_pad.size() * sizeof(double),
                      cudaMemcpyHostToDevice, st));
  if (p->persist_set != 0)  // failures of this call's persistent launches, checked at the end
    CKP(cudaMemsetAsync(&p->d_pq->err_any, 0, sizeof(int), st));
  k_pmmh_start<<<blocks, threads, 0, st>>>(sp, p->d_fds, nc, ch, seed);
  CKP(cudaGetLastError());
  CKP(cudaGraphLaunch(p->exec, st));
  k_pmmh_accept<<<blocks, threads, 0, st>>>(sp, p->d_fds, nc, ch, seed, 0, d_samples, d_ll);
  CKP(cudaGetLastError());
  for (int it = 1; it <= niter; ++it) {
    k_pmmh_propose<<<blocks, threads, 0, st>>>(sp, p->d_fds, nc, ch, seed, it);
    CKP(cudaGetLastError());
    CKP(cudaGraphLaunch(p->exec, st));
    k_pmmh_accept<<<blocks, threads, 0, st>>>(sp, p->d_fds, nc, ch, seed, it,
                                              d_samples + size_t(it) * nc * nth,
                                              d_ll + size_t(it) * nc);
    CKP(cudaGetLastError());
  }
  CKP(cudaMemcpyAsync(samples, d_samples, n_samples * sizeof(double), cudaMemcpyDefault, st));
  CKP(cudaMemcpyAsync(logliks, d_ll, n_ll * sizeof(double), cudaMemcpyDefault, st));
  if (accepted)
    CKP(cudaMemcpyAsync(accepted, ch.acc, size_t(nc) * sizeof(int32_t), cudaMemcpyDefault, st));
  if (p->persist_set != 0)
    CKP(cudaMemcpyAsync(p->h_perr, &p->d_pq->err_any, sizeof(int), cudaMemcpyDeviceToHost, st));
  CKP(cudaStreamSynchronize(st));
  if (p->persist_set != 0) ps = persist_status(p, *p->h_perr);
done:
  if (block) {
    cudaStreamSynchronize(st);
    cudaFree(block);
  }
  return ps;
}
