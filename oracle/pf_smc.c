/*
 * pf_smc.c -- the oracle's samplers built on the particle filter: marginal
 * Metropolis-Hastings (Algorithm 3, Eq. mh, Sec. 3.1.3) and SMC^2
 * (Algorithm 4, Sec. 3.1.4).
 *
 * TEST INFRASTRUCTURE ONLY (see pf_oracle.h).  Plain FP64 C, one chain after
 * the other, each step in the order the algorithm states it.
 *
 * Random numbers: Philox key = the sampler's seed, counter (chain j,
 * iteration i, (purpose 5 << 16) | block, 0):
 *   block 0     acceptance uniform alpha in (0, 1] (words 1:0);
 *   block 1     Philox key of the filter run of (j, i) (words 1:0 low, 3:2 high);
 *   block 16 + 64 d + a   draw a of parameter d: the first Box-Muller normal
 *               of the block (truncated gaussian, attempts a = 0..63), or the
 *               exponential -log u, u in (0, 1] from words 1:0 (inverse
 *               gamma with integer shape, terms a = 0..shape-1).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "pf_oracle.h"

#define OR_MAX_THETA 8
#define OR_TG_ATTEMPTS 64

static int32_t or_theta_size(int32_t kind) { return OR_IS_WK(kind) ? 7 : 5; }

/* Standard normal CDF. */
static double or_Phi(double x) { return 0.5 * erfc(-x * M_SQRT1_2); }

/* log of the mass a N(mu, sd^2) puts on [lo, hi] (the truncated gaussian's normaliser). */
static double or_tg_log_mass(double mu, double sd, double lo, double hi) {
  const double up = isinf(hi) ? 1.0 : or_Phi((hi - mu) / sd);
  const double dn = isinf(lo) ? 0.0 : or_Phi((lo - mu) / sd);
  return log(up - dn);
}

/* Log prior density (Sec. 2.1 parameter blocks), summed over components. */
double or_log_prior(const or_param *spec, int32_t nth, const double *th) {
  double lp = 0.0;
  int32_t d;
  for (d = 0; d < nth; ++d) {
    const or_param *p = spec + d;
    const double x = th[d];
    switch (p->prior) {
      case OR_PRIOR_UNIFORM:
        if (!(x >= p->a && x <= p->b)) return -INFINITY;
        lp += -log(p->b - p->a);
        break;
      case OR_PRIOR_GAUSSIAN: {
        const double z = (x - p->a) / p->b;
        lp += -0.5 * z * z - log(p->b) - 0.5 * log(2.0 * M_PI);
        break;
      }
      case OR_PRIOR_GAMMA:
        if (!(x > 0.0)) return -INFINITY;
        lp += (p->a - 1.0) * log(x) - x / p->b - lgamma(p->a) - p->a * log(p->b);
        break;
      case OR_PRIOR_INV_GAMMA:
        if (!(x > 0.0)) return -INFINITY;
        lp += p->a * log(p->b) - lgamma(p->a) - (p->a + 1.0) * log(x) - p->b / x;
        break;
      default:
        break;
    }
  }
  return lp;
}

/* log density of the inverse gamma IG(shape, scale) at x */
static double or_ig_logpdf(double x, double shape, double scale) {
  return shape * log(scale) - lgamma(shape) - (shape + 1.0) * log(x) - scale / x;
}

static double or_propose_p(const or_param *spec, int32_t nth, const double *th, uint64_t seed,
                           uint32_t j, uint32_t i, uint32_t purpose, double *out);

double or_propose(const or_param *spec, int32_t nth, const double *th, uint64_t seed, uint32_t j,
                  uint32_t i, double *out) {
  return or_propose_p(spec, nth, th, seed, j, i, OR_PURPOSE_PMMH, out);
}

static double or_propose_p(const or_param *spec, int32_t nth, const double *th, uint64_t seed,
                           uint32_t j, uint32_t i, uint32_t purpose, double *out) {
  double lqr = 0.0;
  int32_t d;
  for (d = 0; d < nth; ++d) {
    const or_param *p = spec + d;
    const double x = th[d];
    out[d] = x;
    if (p->proposal == OR_PROPOSE_TRUNC_GAUSSIAN) {
      int32_t a;
      for (a = 0; a < OR_TG_ATTEMPTS; ++a) {
        const uint32_t blk = 16u + 64u * (uint32_t)d + (uint32_t)a;
        const double z = or_normal64(seed, j, i, purpose, 2u * blk);
        const double xn = fma(p->c, z, x);
        if (xn >= p->d && xn <= p->e) {
          out[d] = xn;
          break;
        }
      }
      /* the gaussian kernel is symmetric: only the normalisers remain */
      lqr += or_tg_log_mass(x, p->c, p->d, p->e) - or_tg_log_mass(out[d], p->c, p->d, p->e);
    } else if (p->proposal == OR_PROPOSE_INV_GAMMA) {
      const int32_t k = (int32_t)p->c;
      double sum = 0.0;
      int32_t a;
      for (a = 0; a < k; ++a) {
        uint32_t w[4];
        or_block(seed, j, i, purpose, 16u + 64u * (uint32_t)d + (uint32_t)a, w);
        sum += -or_log(or_u53_open_zero(w[0], w[1]));
      }
      /* Gamma(k, 1) = sum of k unit exponentials; IG(k, s) = s / Gamma(k, 1) */
      out[d] = (p->d * x) / sum;
      lqr += or_ig_logpdf(x, p->c, p->d * out[d]) - or_ig_logpdf(out[d], p->c, p->d * x);
    }
  }
  return lqr;
}

static uint64_t or_filter_key(uint64_t seed, uint32_t j, uint32_t i) {
  uint32_t w[4];
  or_block(seed, j, i, OR_PURPOSE_PMMH, 1u, w);
  return ((uint64_t)w[1] << 32) | (uint64_t)w[0];
}

/* Likelihood of theta: particle filter (Algorithm 2), the exact Kalman
 * filter (Algorithm 1, windkessel only) or none (prior-only chains). */
static double or_loglik(const or_model *m, const double *y, int64_t P, int32_t T, int32_t lik,
                        const double *th, uint64_t key, int32_t nthreads, int *near) {
  double ll = 0.0;
  *near = 0;
  if (lik == OR_LIK_NONE) return 0.0;
  if (lik == OR_LIK_KALMAN) return or_kalman_windkessel(m, th, y, T);
  {
    double *diag = (double *)malloc(sizeof(double) * 8 * (size_t)T);
    int32_t st = or_pf_run(m, th, y, key, P, T, nthreads, &ll, NULL, NULL, diag);
    int32_t i;
    if (st == OR_OK) {
      for (i = 0; i < T; ++i)
        if (diag[8 * i + 7] > 0.0) *near = 1;
    } else {
      ll = -INFINITY;
    }
    free(diag);
  }
  return ll;
}

int32_t or_pmmh(const or_model *m, const double *y, int64_t P, int32_t T, int32_t lik,
                int32_t nchains, const or_param *spec, const double *theta0, int32_t niter,
                uint64_t seed, int32_t nthreads, double *samples, double *logliks,
                int32_t *accepted, int32_t *near) {
  const int32_t nth = or_theta_size(m->kind);
  int32_t c, i;
  if (nchains < 1 || niter < 0 || P < 1 || T < 1) return OR_EINVAL;
  if (lik == OR_LIK_KALMAN && !OR_IS_WK(m->kind)) return OR_EINVAL;
  for (c = 0; c < nchains; ++c) {
    double th[OR_MAX_THETA], thp[OR_MAX_THETA];
    double ll, lp;
    int nr;
    memcpy(th, theta0 + (int64_t)c * nth, sizeof(double) * (size_t)nth);
    lp = or_log_prior(spec, nth, th);
    ll = or_loglik(m, y, P, T, lik, th, or_filter_key(seed, (uint32_t)c, 0u), nthreads, &nr);
    accepted[c] = 0;
    memcpy(samples + (int64_t)c * nth, th, sizeof(double) * (size_t)nth);
    logliks[c] = ll;
    near[c] = nr;
    for (i = 1; i <= niter; ++i) {
      const int64_t row = (int64_t)i * nchains + c;
      uint32_t w[4];
      double lqr, lpp, llp = -INFINITY, log_alpha, ratio;
      int accept = 0, nrp = 0;
      /* propose */
      lqr = or_propose(spec, nth, th, seed, (uint32_t)c, (uint32_t)i, thp);
      lpp = or_log_prior(spec, nth, thp);
      /* likelihood of the proposal (skipped outside the prior's support) */
      if (lpp > -INFINITY)
        llp = or_loglik(m, y, P, T, lik, thp, or_filter_key(seed, (uint32_t)c, (uint32_t)i),
                        nthreads, &nrp);
      /* alpha ~ U(0, 1]; accept iff alpha <= the Metropolis-Hastings ratio */
      or_block(seed, (uint32_t)c, (uint32_t)i, OR_PURPOSE_PMMH, 0u, w);
      log_alpha = or_log(or_u53_open_zero(w[0], w[1]));
      ratio = (llp + lpp + lqr) - (ll + lp);
      accept = lpp > -INFINITY && log_alpha <= ratio;
      near[row] = nrp || (lpp > -INFINITY &&
                          fabs(log_alpha - ratio) <= 1e-9 * (1.0 + fabs(llp) + fabs(ll)));
      if (accept) {
        memcpy(th, thp, sizeof(double) * (size_t)nth);
        ll = llp;
        lp = lpp;
        accepted[c] += 1;
      }
      memcpy(samples + row * nth, th, sizeof(double) * (size_t)nth);
      logliks[row] = ll;
    }
  }
  return OR_OK;
}

/* ======================================================================
 * SMC^2 (Algorithm 4).  P_theta parameter particles, each with its own
 * bootstrap filter of P state particles.  For i = 1..T:
 *   a^j ~ Multinomial(v(t_{i-1}))                      (theta resampling)
 *   theta' ~ q(.|theta^{a^j}); l' = Filter(theta', t_{0:i-1}); accept with
 *     the rule of Eq. mh against l^{a^j}(t_{i-1})        (rejuvenation)
 *   v^j(t_i) = Filter(theta^j, t_{i-1:i}) likelihood increment,
 *   l^j(t_i) = l^j(t_{i-1}) v^j(t_i).
 * log evidence = sum_i log( (1/P_theta) sum_j v^j(t_i) ).
 *
 * A parameter particle's filter is a resident filter that is started, copied
 * (on rejection, from its ancestor) and continued one observation at a time
 * with a new Philox key per call.  The oracle represents it by its key
 * schedule (sched[0] the initial draw's key, sched[i] the key of step i, as
 * in or_pf_run_sched) and re-runs it from t_0 whenever it needs it.
 *
 * Random numbers (key = the sampler's seed, counter (j, i, (6 << 16) | block, 0)):
 *   block 0  multinomial uniform of particle j at step i, [0, 1) (words 1:0);
 *   block 1  key of the rejuvenation filter run of (j, i);
 *   block 2  key of the continuation of (j, i) over t_{i-1:i} (i = 0: the
 *            initial filter of particle j);
 *   block 3  acceptance uniform in (0, 1];
 *   block 16 + 64 d + a  draws of component d: step 0 the prior draw, step
 *            i >= 1 the proposal (as in or_pmmh).
 * Likelihood modes: OR_LIK_PF (the filter above) or OR_LIK_KALMAN (exact
 * increments of the windkessel's Kalman filter, which makes the sampler
 * IBIS with the same moves; used to pin the parameter-level steps).
 * ==================================================================== */

/* Prior draw of every component (integer shapes for gamma / inverse gamma). */
static int or_prior_draw(const or_param *spec, int32_t nth, const double *base, uint64_t seed,
                         uint32_t j, double *out) {
  int32_t d;
  for (d = 0; d < nth; ++d) {
    const or_param *p = spec + d;
    const uint32_t blk = 16u + 64u * (uint32_t)d;
    uint32_t w[4];
    switch (p->prior) {
      case OR_PRIOR_UNIFORM:
        or_block(seed, j, 0u, OR_PURPOSE_SMC2, blk, w);
        out[d] = fma(p->b - p->a, or_u53_half_open(w[0], w[1]), p->a);
        break;
      case OR_PRIOR_GAUSSIAN:
        out[d] = fma(p->b, or_normal64(seed, j, 0u, OR_PURPOSE_SMC2, 2u * blk), p->a);
        break;
      case OR_PRIOR_GAMMA:
      case OR_PRIOR_INV_GAMMA: {
        const int32_t k = (int32_t)p->a;
        double sum = 0.0;
        int32_t a;
        if ((double)k != p->a || k < 1 || k > 64) return 0;
        for (a = 0; a < k; ++a) {
          or_block(seed, j, 0u, OR_PURPOSE_SMC2, blk + (uint32_t)a, w);
          sum += -or_log(or_u53_open_zero(w[0], w[1]));
        }
        out[d] = p->prior == OR_PRIOR_GAMMA ? p->b * sum : p->b / sum;
        break;
      }
      default:
        out[d] = base[d];
    }
  }
  return 1;
}

static uint64_t or_smc2_key(uint64_t seed, uint32_t j, uint32_t i, uint32_t blk) {
  uint32_t w[4];
  or_block(seed, j, i, OR_PURPOSE_SMC2, blk, w);
  return ((uint64_t)w[1] << 32) | (uint64_t)w[0];
}

/* log-likelihood of y(t_1..t_n) of a filter with key schedule sched[0..n]. */
static double or_sched_loglik(const or_model *m, const double *th, const double *y, int64_t P,
                              int32_t n, const uint64_t *sched, int32_t lik, int32_t nthreads,
                              int *near) {
  double ll = 0.0;
  *near = 0;
  if (n == 0) return 0.0;
  if (lik == OR_LIK_KALMAN) return or_kalman_windkessel(m, th, y, n);
  {
    double *diag = (double *)malloc(sizeof(double) * 8 * (size_t)n);
    int32_t st = or_pf_run_sched(m, th, y, 0, sched, P, n, nthreads, &ll, NULL, NULL, diag, NULL,
                                 NULL);
    int32_t i;
    if (st == OR_OK) {
      for (i = 0; i + 1 < n; ++i) /* the last step's targets are never drawn */
        if (diag[8 * i + 7] > 0.0) *near = 1;
    } else {
      ll = -INFINITY;
    }
    free(diag);
  }
  return ll;
}

int32_t or_smc2(const or_model *m, const double *y, int64_t P, int32_t T, int32_t lik,
                int32_t ntheta, const or_param *spec, const double *base, uint64_t seed,
                int32_t nthreads, double *theta_out, double *logv_out, double *log_evidence,
                double *incr, int32_t *accepted, int32_t *near) {
  const int32_t nth = or_theta_size(m->kind);
  const int64_t S = T + 1;
  double *th = NULL, *thn = NULL, *lp = NULL, *lpn = NULL, *ll = NULL, *lln = NULL, *logv = NULL;
  double *C = NULL;
  uint64_t *sch = NULL, *schn = NULL;
  int32_t j, i, status = OR_OK;
  double logZ = 0.0;
  if (ntheta < 1 || P < 1 || T < 1) return OR_EINVAL;
  if (lik == OR_LIK_KALMAN && !OR_IS_WK(m->kind)) return OR_EINVAL;
  th = (double *)malloc(sizeof(double) * (size_t)ntheta * OR_MAX_THETA);
  thn = (double *)malloc(sizeof(double) * (size_t)ntheta * OR_MAX_THETA);
  lp = (double *)malloc(sizeof(double) * (size_t)ntheta);
  lpn = (double *)malloc(sizeof(double) * (size_t)ntheta);
  ll = (double *)malloc(sizeof(double) * (size_t)ntheta);
  lln = (double *)malloc(sizeof(double) * (size_t)ntheta);
  logv = (double *)malloc(sizeof(double) * (size_t)ntheta);
  C = (double *)malloc(sizeof(double) * (size_t)ntheta);
  sch = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(ntheta * S));
  schn = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(ntheta * S));

  /* initialise: theta^j ~ p(theta), v^j = 1/P_theta, l^j = 1, x^j(t_0) drawn
   * by the particle's initial filter (key block 2 of step 0) */
  for (j = 0; j < ntheta; ++j) {
    if (!or_prior_draw(spec, nth, base, seed, (uint32_t)j, th + (int64_t)j * OR_MAX_THETA)) {
      status = OR_EINVAL;
      goto out;
    }
    lp[j] = or_log_prior(spec, nth, th + (int64_t)j * OR_MAX_THETA);
    ll[j] = 0.0;
    logv[j] = 0.0;
    sch[(int64_t)j * S] = or_smc2_key(seed, (uint32_t)j, 0u, 2u);
  }
  for (i = 1; i <= T; ++i) {
    double M = -INFINITY, sum = 0.0, comp = 0.0, tot;
    int nr = 0;
    accepted[i - 1] = 0;
    /* cumulative theta-weights (compensated) for the multinomial draws */
    for (j = 0; j < ntheta; ++j)
      if (logv[j] > M) M = logv[j];
    for (j = 0; j < ntheta; ++j) {
      const double w = (M == -INFINITY) ? 0.0 : exp(logv[j] - M);
      const double t = sum + w;
      comp += (fabs(sum) >= fabs(w)) ? (sum - t) + w : (w - t) + sum;
      sum = t;
      C[j] = sum + comp;
    }
    tot = C[ntheta - 1];
    if (!(tot > 0.0)) {
      status = OR_EDEGENERATE;
      goto out;
    }
    for (j = 0; j < ntheta; ++j) {
      uint32_t w[4];
      double tau, thp[OR_MAX_THETA], lqr, lpp, llp = -INFINITY, log_alpha, ratio;
      int32_t a = 0, lo = 0, hi = ntheta, k, acc;
      int nrp = 0;
      /* a^j: the first k with C_k > u tot */
      or_block(seed, (uint32_t)j, (uint32_t)i, OR_PURPOSE_SMC2, 0u, w);
      tau = or_u53_half_open(w[0], w[1]) * tot;
      while (lo < hi) {
        const int32_t mid = lo + (hi - lo) / 2;
        if (C[mid] > tau) hi = mid;
        else lo = mid + 1;
      }
      a = lo < ntheta ? lo : ntheta - 1;
      for (k = 0; k < ntheta; ++k)
        if (fabs(C[k] - tau) <= 1e-12 * tot) nr = 1;
      /* rejuvenate: propose, run the proposal's filter over t_{0:i-1}, accept or reject */
      lqr = or_propose_p(spec, nth, th + (int64_t)a * OR_MAX_THETA, seed, (uint32_t)j,
                         (uint32_t)i, OR_PURPOSE_SMC2, thp);
      lpp = or_log_prior(spec, nth, thp);
      {
        uint64_t *sp = schn + (int64_t)j * S;
        const uint64_t kb = or_smc2_key(seed, (uint32_t)j, (uint32_t)i, 1u);
        int32_t q;
        for (q = 0; q < i; ++q) sp[q] = kb;
        if (lpp > -INFINITY) llp = or_sched_loglik(m, thp, y, P, i - 1, sp, lik, nthreads, &nrp);
      }
      or_block(seed, (uint32_t)j, (uint32_t)i, OR_PURPOSE_SMC2, 3u, w);
      log_alpha = or_log(or_u53_open_zero(w[0], w[1]));
      ratio = (llp + lpp + lqr) - (ll[a] + lp[a]);
      acc = lpp > -INFINITY && log_alpha <= ratio;
      if (nrp || (lpp > -INFINITY &&
                  fabs(log_alpha - ratio) <= 1e-9 * (1.0 + fabs(llp) + fabs(ll[a]))))
        nr = 1;
      if (acc) {
        memcpy(thn + (int64_t)j * OR_MAX_THETA, thp, sizeof(double) * OR_MAX_THETA);
        lpn[j] = lpp;
        lln[j] = llp;
        accepted[i - 1] += 1;
      } else {
        memcpy(thn + (int64_t)j * OR_MAX_THETA, th + (int64_t)a * OR_MAX_THETA,
               sizeof(double) * OR_MAX_THETA);
        memcpy(schn + (int64_t)j * S, sch + (int64_t)a * S, sizeof(uint64_t) * (size_t)i);
        lpn[j] = lp[a];
        lln[j] = ll[a];
      }
    }
    { /* the new population replaces the old one */
      double *t;
      uint64_t *u;
      t = th; th = thn; thn = t;
      t = lp; lp = lpn; lpn = t;
      t = ll; ll = lln; lln = t;
      u = sch; sch = schn; schn = u;
    }
    /* continue every particle's filter over t_{i-1:i} with a new key */
    M = -INFINITY;
    for (j = 0; j < ntheta; ++j) {
      uint64_t *sp = sch + (int64_t)j * S;
      double lnew;
      int nrp = 0;
      sp[i] = or_smc2_key(seed, (uint32_t)j, (uint32_t)i, 2u);
      lnew = or_sched_loglik(m, th + (int64_t)j * OR_MAX_THETA, y, P, i, sp, lik, nthreads, &nrp);
      if (nrp) nr = 1;
      logv[j] = lnew - ll[j];
      if (logv[j] != logv[j]) logv[j] = -INFINITY;
      ll[j] = lnew;
      if (logv[j] > M) M = logv[j];
    }
    /* evidence increment: log of the mean theta-weight */
    sum = 0.0;
    comp = 0.0;
    for (j = 0; j < ntheta; ++j) {
      const double w = (M == -INFINITY) ? 0.0 : exp(logv[j] - M);
      const double t = sum + w;
      comp += (fabs(sum) >= fabs(w)) ? (sum - t) + w : (w - t) + sum;
      sum = t;
    }
    incr[i - 1] = M + log(sum + comp) - log((double)ntheta);
    logZ += incr[i - 1];
    near[i - 1] = nr;
  }
  for (j = 0; j < ntheta; ++j) {
    memcpy(theta_out + (int64_t)j * nth, th + (int64_t)j * OR_MAX_THETA, sizeof(double) * (size_t)nth);
    logv_out[j] = logv[j];
  }
  *log_evidence = logZ;
out:
  free(th); free(thn); free(lp); free(lpn); free(ll); free(lln); free(logv); free(C);
  free(sch); free(schn);
  return status;
}
