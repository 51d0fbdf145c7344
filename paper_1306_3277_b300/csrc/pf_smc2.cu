// pf_smc2.cu -- SMC^2 over the model parameters (Algorithm 4, Sec. 3.1.4):
// P_theta parameter particles, each owning a resident particle filter of P
// state particles; all filters of a population advance in shared launches.
//
// Two populations of filters, A (current) and B (rejuvenation).  Step i:
//   k_smc2_select    a^j ~ Multinomial(v(t_{i-1})) (one block, FP64 scan);
//   k_smc2_propose   theta' ~ q(.|theta^{a^j}) into B_j's descriptor;
//   B's plan         B_j := Filter(theta', t_{0:i-1}) (initial draw + i-1 steps);
//   k_smc2_accept    the rule of Eq. mh against l^{a^j}(t_{i-1});
//   k_smc2_copy      a rejected j takes the state of A_{a^j} (particles,
//                    ancestors, carried weights, control block) into B_j;
//   swap A and B;
//   k_smc2_keys      a fresh Philox key per filter for the continuation;
//   A's plan         every filter over t_{i-1:i} (one propagate + resample);
//   k_smc2_weights   v^j(t_i) = l^j(t_i) / l^j(t_{i-1}) and the evidence
//                    increment log mean_j v^j(t_i).
// The host only enqueues; nothing waits until the end.
//
// Random numbers (key = the sampler's seed, counter (j, i, (6 << 16) | block, 0)):
// block 0 the multinomial uniform in [0, 1); block 1 the key of B_j's run;
// block 2 the key of the continuation (step 0: of A_j's initial draw);
// block 3 the acceptance uniform in (0, 1]; blocks 16 + 64 d + a the prior
// draw (step 0) or the proposal (step i) of component d.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "pf_params.cuh"
#include "pf_runtime.h"

namespace pfb {
namespace {

constexpr int SEL_THREADS = 1024;

struct Base {
  double v[MAX_THETA];
};

struct Pop {
  double* theta;  // [nt][MAX_THETA]
  double* lp;     // [nt] log prior
  double* ll;     // [nt] log l^j(t_i), the filter's accumulated log-likelihood
};

__device__ double block_max_1024(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  v = l < (blockDim.x >> 5) ? red[l] : -INFINITY;
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Inclusive scan of one value per thread over the block (warp scans, then the
// warp totals in order); *total receives the block total.
__device__ double block_scan_1024(double v, double* red, double* total) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  for (int o = 1; o < 32; o <<= 1) {
    const double n = __shfl_up_sync(0xffffffffu, v, o);
    if (l >= o) v += n;
  }
  __syncthreads();
  if (l == 31) red[w] = v;
  __syncthreads();
  if (w == 0) {
    double t = l < (blockDim.x >> 5) ? red[l] : 0.0;
    for (int o = 1; o < 32; o <<= 1) {
      const double n = __shfl_up_sync(0xffffffffu, t, o);
      if (l >= o) t += n;
    }
    red[l] = t;  // inclusive prefix of the warp totals
  }
  __syncthreads();
  const double off = w > 0 ? red[w - 1] : 0.0;
  *total = red[(blockDim.x >> 5) - 1];
  return v + off;
}

__global__ void k_smc2_init(Spec sp, Base base, FilterDev* __restrict__ fds, int nt, Pop cur,
                            double* __restrict__ logv, uint64_t seed) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nt) return;
  double* th = cur.theta + size_t(j) * MAX_THETA;
  prior_draw(sp, base.v, seed, uint32_t(j), PURPOSE_SMC2, th);
  for (int d = 0; d < sp.nth; ++d) fds[j].theta[d] = th[d];
  cur.lp[j] = log_prior(sp, th);
  cur.ll[j] = 0.0;
  logv[j] = 0.0;
  fds[j].seed = philox_key(seed, uint32_t(j), 0u, PURPOSE_SMC2, 2u);
}

// Multinomial ancestors from the theta-weights: a^j = the first k whose
// cumulative weight C_k exceeds u_j C_{nt-1}.  One block; each thread scans a
// contiguous chunk, the chunks are combined by a block scan.
__global__ void __launch_bounds__(SEL_THREADS) k_smc2_select(int nt, const double* __restrict__ logv,
                                                             double* __restrict__ C,
                                                             int32_t* __restrict__ anc,
                                                             int32_t* __restrict__ status,
                                                             uint64_t seed, int i) {
  __shared__ double red[32];
  const int tid = threadIdx.x;
  double m = -INFINITY;
  for (int j = tid; j < nt; j += SEL_THREADS) m = fmax(m, logv[j]);
  const double M = block_max_1024(m, red);
  const int chunk = (nt + SEL_THREADS - 1) / SEL_THREADS;
  const int lo = min(nt, tid * chunk), hi = min(nt, lo + chunk);
  double s = 0.0;
  for (int k = lo; k < hi; ++k) s += M == -INFINITY ? 0.0 : exp(logv[k] - M);
  double tot;  // the scan's total; the search uses C[nt-1], accumulated like every C_k
  const double incl = block_scan_1024(s, red, &tot);
  (void)tot;
  double run = incl - s;
  for (int k = lo; k < hi; ++k) {
    run += M == -INFINITY ? 0.0 : exp(logv[k] - M);
    C[k] = run;
  }
  __syncthreads();
  const double total = C[nt - 1];
  if (!(total > 0.0)) {
    if (tid == 0) *status = ST_DEGENERATE;
    for (int j = tid; j < nt; j += SEL_THREADS) anc[j] = j;
    return;
  }
  for (int j = tid; j < nt; j += SEL_THREADS) {
    const uint4 w = rng_block(seed, uint32_t(j), uint32_t(i), PURPOSE_SMC2, 0u);
    const double tau = u53_closed_open(w.x, w.y) * total;
    int a = 0, b = nt;
    while (a < b) {
      const int mid = a + (b - a) / 2;
      if (C[mid] > tau) b = mid;
      else a = mid + 1;
    }
    anc[j] = min(a, nt - 1);
  }
}

__global__ void k_smc2_propose(Spec sp, FilterDev* __restrict__ fdsB, int nt, Pop cur,
                               const int32_t* __restrict__ anc, double* __restrict__ theta_p,
                               double* __restrict__ lp_p, double* __restrict__ lqr,
                               uint64_t seed, int i) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nt) return;
  const int a = anc[j];
  double* out = theta_p + size_t(j) * MAX_THETA;
  lqr[j] = propose(sp, cur.theta + size_t(a) * MAX_THETA, seed, uint32_t(j), uint32_t(i),
                   PURPOSE_SMC2, out);
  lp_p[j] = log_prior(sp, out);
  for (int d = 0; d < sp.nth; ++d) fdsB[j].theta[d] = out[d];
  fdsB[j].seed = philox_key(seed, uint32_t(j), uint32_t(i), PURPOSE_SMC2, 1u);
}

__global__ void k_smc2_accept(Spec sp, FilterDev* __restrict__ fdsB, int nt, Pop cur, Pop nxt,
                              const int32_t* __restrict__ anc, const double* __restrict__ theta_p,
                              const double* __restrict__ lp_p, const double* __restrict__ lqr,
                              int32_t* __restrict__ from, int32_t* __restrict__ acc_i,
                              uint64_t seed, int i) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nt) return;
  const Ctl* ctl = fdsB[j].ctl;
  const double llp = ldcg(&ctl->status) == ST_OK ? ldcg(&ctl->ll) : -INFINITY;
  const int a = anc[j];
  const uint4 w = rng_block(seed, uint32_t(j), uint32_t(i), PURPOSE_SMC2, 3u);
  const double log_alpha = log_pos(u53_open_closed(w.x, w.y));
  const double ratio = (llp + lp_p[j] + lqr[j]) - (cur.ll[a] + cur.lp[a]);
  const bool accept = lp_p[j] > -INFINITY && log_alpha <= ratio;
  double* th = nxt.theta + size_t(j) * MAX_THETA;
  if (accept) {
    for (int d = 0; d < MAX_THETA; ++d) th[d] = theta_p[size_t(j) * MAX_THETA + d];
    nxt.lp[j] = lp_p[j];
    nxt.ll[j] = llp;
    from[j] = -1;
    atomicAdd(acc_i, 1);
  } else {
    const double* ta = cur.theta + size_t(a) * MAX_THETA;
    for (int d = 0; d < MAX_THETA; ++d) th[d] = ta[d];
    for (int d = 0; d < sp.nth; ++d) fdsB[j].theta[d] = ta[d];
    nxt.lp[j] = cur.lp[a];
    nxt.ll[j] = cur.ll[a];
    from[j] = a;
  }
}

// B_j := the state of A_{from[j]} at t_{i-1} for every rejected j: state
// particles x(t_{i-1}), the ancestor row of the next propagation, the carried
// log-weights and the control block.  One block per tile of B.
__global__ void __launch_bounds__(TILE) k_smc2_copy(const FilterDev* __restrict__ fdsA,
                                                    const FilterDev* __restrict__ fdsB,
                                                    const int2* __restrict__ tmap,
                                                    const int32_t* __restrict__ from, int par) {
  const int2 ft = tmap[blockIdx.x];
  const int a = from[ft.x];
  if (a < 0) return;
  const FilterDev& s = fdsA[a];
  const FilterDev& d = fdsB[ft.x];
  const int P = d.P;
  const int p = ft.y * TILE + threadIdx.x;
  if (p < P) {
    if (d.prec == PREC_MIXED) {
      const float* xs = static_cast<const float*>(s.x[par]);
      float* xd = static_cast<float*>(d.x[par]);
      for (int n = 0; n < d.N; ++n) xd[size_t(n) * P + p] = xs[size_t(n) * P + p];
    } else {
      const double* xs = static_cast<const double*>(s.x[par]);
      double* xd = static_cast<double*>(d.x[par]);
      for (int n = 0; n < d.N; ++n) xd[size_t(n) * P + p] = xs[size_t(n) * P + p];
    }
    d.anc[p] = s.anc[p];
    if (d.mode != MODE_ALWAYS) d.lam[p] = s.lam[p];
  }
  if (ft.y == 0 && threadIdx.x == 0) *d.ctl = *s.ctl;
}

__global__ void k_smc2_keys(FilterDev* __restrict__ fds, int nt, uint64_t seed, int i) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nt) return;
  fds[j].seed = philox_key(seed, uint32_t(j), uint32_t(i), PURPOSE_SMC2, 2u);
}

// v^j(t_i) from the continued filters and the evidence increment log mean v.
__global__ void __launch_bounds__(SEL_THREADS) k_smc2_weights(const FilterDev* __restrict__ fds,
                                                              int nt, double* __restrict__ ll,
                                                              double* __restrict__ logv,
                                                              double* __restrict__ incr) {
  __shared__ double red[32];
  const int tid = threadIdx.x;
  double m = -INFINITY;
  for (int j = tid; j < nt; j += SEL_THREADS) {
    const Ctl* c = fds[j].ctl;
    const double lnew = ldcg(&c->status) == ST_OK ? ldcg(&c->ll) : -INFINITY;
    double lv = lnew - ll[j];
    if (lv != lv) lv = -INFINITY;
    logv[j] = lv;
    ll[j] = lnew;
    m = fmax(m, lv);
  }
  const double M = block_max_1024(m, red);
  double s = 0.0;
  for (int j = tid; j < nt; j += SEL_THREADS) s += M == -INFINITY ? 0.0 : exp(logv[j] - M);
  double tot;
  block_scan_1024(s, red, &tot);
  if (tid == 0) *incr = M + log(tot) - log(double(nt));
}

}  // namespace
}  // namespace pfb

using namespace pfb;

#define CKS(x)                                                                        \
  do {                                                                                \
    cudaError_t e_ = (x);                                                             \
    if (e_ != cudaSuccess) {                                                          \
      cudaGetLastError();                                                             \
      ps = fail(PF_ECUDA, "%s: %s", #x, cudaGetErrorString(e_));                     \
      goto done;                                                                      \
    }                                                                                 \
  } while (0)

extern "C" pf_status pf_smc2_run(const pf_model* m, int64_t P, int32_t T, double dt,
                                 const double* y, int32_t ntheta, const pf_param* spec,
                                 const double* theta_base, uint64_t seed, double* theta_out,
                                 double* logw_out, double* log_evidence, double* evidence_incr,
                                 int32_t* accepted, void* cuda_stream) {
  if (!m || !y || !spec || !theta_base || !theta_out || !logw_out || !log_evidence)
    return fail(PF_EINVAL, "pf_smc2_run: bad arguments");
  if (ntheta < 1 || ntheta > (1 << 16))
    return fail(PF_EINVAL, "ntheta = %d is outside [1, 65536]", ntheta);
  const int nth = pf_theta_size(m->kind);
  if (nth == 0) return fail(PF_EINVAL, "unknown model kind %d", m->kind);
  pf_status ps = check_spec(spec, nth);
  if (ps != PF_OK) return ps;
  for (int d = 0; d < nth; ++d) {
    const pf_param& p = spec[d];
    if ((p.prior == PF_PRIOR_GAMMA || p.prior == PF_PRIOR_INV_GAMMA) &&
        !(p.a >= 1.0 && p.a <= 64.0 && p.a == std::floor(p.a)))
      return fail(PF_EINVAL, "theta[%d]: SMC^2 draws gamma priors with integer shapes 1..64", d);
  }
  std::vector<pf_filter*> fl(2 * size_t(ntheta), nullptr);
  for (size_t k = 0; k < fl.size(); ++k) {
    ps = pf_create(m, P, T, dt, &fl[k]);
    if (ps != PF_OK) {
      for (pf_filter* f : fl)
        if (f) pf_destroy(f);
      return ps;
    }
  }
  std::vector<pf_filter*> la(fl.begin(), fl.begin() + ntheta), lb(fl.begin() + ntheta, fl.end());
  Plan *pa = nullptr, *pb = nullptr;
  void* block = nullptr;
  cudaStream_t st = nullptr;
  Spec sp;
  Base base;
  Pop cur{}, nxt{};
  double *logv = nullptr, *C = nullptr, *theta_p = nullptr, *lp_p = nullptr, *lqr = nullptr,
         *incr = nullptr;
  int32_t *anc = nullptr, *from = nullptr, *acc = nullptr, *status = nullptr;
  std::vector<double> h_theta, h_incr(T);
  std::vector<int32_t> h_acc(T);
  int32_t h_status = ST_OK;
  const int threads = 128, blocks = (ntheta + threads - 1) / threads;
  memset(&sp, 0, sizeof sp);
  memcpy(sp.p, spec, sizeof(pf_param) * nth);
  sp.nth = nth;
  memset(&base, 0, sizeof base);
  memcpy(base.v, theta_base, sizeof(double) * nth);
  ps = batch_plan(la, &pa);
  if (ps == PF_OK) ps = batch_plan(lb, &pb);
  if (ps != PF_OK) goto done;
  st = cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : pa->st;
  {
    std::vector<const double*> th(ntheta, theta_base), ys(ntheta, y);
    std::vector<uint64_t> seeds(ntheta, 0);
    ps = stage_plan(pa, th.data(), ys.data(), seeds.data(), nullptr, st);
    if (ps == PF_OK) ps = stage_plan(pb, th.data(), ys.data(), seeds.data(), nullptr, st);
    if (ps != PF_OK) goto done;
  }
  {
    const size_t nt = size_t(ntheta);
    const size_t nd = 3 * nt * MAX_THETA + 4 * nt + 3 * nt + nt + nt + size_t(T);
    const size_t ni = 2 * nt + size_t(T) + 1;
    CKS(cudaMalloc(&block, nd * sizeof(double) + ni * sizeof(int32_t)));
    double* q = static_cast<double*>(block);
    cur.theta = q; q += nt * MAX_THETA;
    nxt.theta = q; q += nt * MAX_THETA;
    theta_p = q; q += nt * MAX_THETA;
    cur.lp = q; q += nt;
    cur.ll = q; q += nt;
    nxt.lp = q; q += nt;
    nxt.ll = q; q += nt;
    logv = q; q += nt;
    C = q; q += nt;
    lp_p = q; q += nt;
    lqr = q; q += nt;
    q += nt;  // spare
    incr = q; q += T;
    int32_t* r = reinterpret_cast<int32_t*>(q);
    anc = r; r += nt;
    from = r; r += nt;
    acc = r; r += T;
    status = r;
  }
  CKS(cudaMemsetAsync(acc, 0, sizeof(int32_t) * (size_t(T) + 1), st));  // acc[T], status
  k_smc2_init<<<blocks, threads, 0, st>>>(sp, base, pa->d_fds, ntheta, cur, logv, seed);
  CKS(cudaGetLastError());
  CKS(enqueue_plan_steps(pa, 1, 0, true, st));  // x^j(t_0) of every parameter particle
  for (int i = 1; i <= T; ++i) {
    k_smc2_select<<<1, SEL_THREADS, 0, st>>>(ntheta, logv, C, anc, status, seed, i);
    CKS(cudaGetLastError());
    k_smc2_propose<<<blocks, threads, 0, st>>>(sp, pb->d_fds, ntheta, cur, anc, theta_p, lp_p,
                                               lqr, seed, i);
    CKS(cudaGetLastError());
    CKS(enqueue_plan_steps(pb, 1, i - 1, true, st));
    k_smc2_accept<<<blocks, threads, 0, st>>>(sp, pb->d_fds, ntheta, cur, nxt, anc, theta_p, lp_p,
                                              lqr, from, acc + (i - 1), seed, i);
    CKS(cudaGetLastError());
    k_smc2_copy<<<pb->ntiles_all, TILE, 0, st>>>(pa->d_fds, pb->d_fds, pb->d_tmap, from,
                                                 (i - 1) & 1);
    CKS(cudaGetLastError());
    std::swap(pa, pb);
    std::swap(cur, nxt);
    k_smc2_keys<<<blocks, threads, 0, st>>>(pa->d_fds, ntheta, seed, i);
    CKS(cudaGetLastError());
    CKS(enqueue_plan_steps(pa, i, i, false, st));
    k_smc2_weights<<<1, SEL_THREADS, 0, st>>>(pa->d_fds, ntheta, cur.ll, logv, incr + (i - 1));
    CKS(cudaGetLastError());
  }
  h_theta.resize(size_t(ntheta) * MAX_THETA);
  CKS(cudaMemcpyAsync(h_theta.data(), cur.theta, h_theta.size() * sizeof(double),
                      cudaMemcpyDeviceToHost, st));
  CKS(cudaMemcpyAsync(h_incr.data(), incr, sizeof(double) * T, cudaMemcpyDeviceToHost, st));
  CKS(cudaMemcpyAsync(h_acc.data(), acc, sizeof(int32_t) * T, cudaMemcpyDeviceToHost, st));
  CKS(cudaMemcpyAsync(&h_status, status, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  CKS(cudaMemcpyAsync(logw_out, logv, sizeof(double) * ntheta, cudaMemcpyDefault, st));
  CKS(cudaStreamSynchronize(st));
  {
    std::vector<double> packed(size_t(ntheta) * nth);
    for (int j = 0; j < ntheta; ++j)
      memcpy(&packed[size_t(j) * nth], &h_theta[size_t(j) * MAX_THETA], sizeof(double) * nth);
    CKS(cudaMemcpy(theta_out, packed.data(), packed.size() * sizeof(double), cudaMemcpyDefault));
    double lz = 0.0;
    for (int i = 0; i < T; ++i) lz += h_incr[i];
    if (h_status != ST_OK) lz = -INFINITY;
    CKS(cudaMemcpy(log_evidence, &lz, sizeof(double), cudaMemcpyDefault));
    if (evidence_incr)
      CKS(cudaMemcpy(evidence_incr, h_incr.data(), sizeof(double) * T, cudaMemcpyDefault));
    if (accepted)
      CKS(cudaMemcpy(accepted, h_acc.data(), sizeof(int32_t) * T, cudaMemcpyDefault));
  }
  ps = h_status == ST_OK ? PF_OK : PF_EDEGENERATE;
done:
  if (st) cudaStreamSynchronize(st);
  if (block) cudaFree(block);
  for (pf_filter* f : fl)
    if (f) pf_destroy(f);
  return ps;
}
