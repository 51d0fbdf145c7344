/*
 * pf_smc.c -- the oracle's samplers built on the particle filter: marginal
 * Metropolis-Hastings (Algorithm 3, Eq. mh, Sec. 3.1.3).
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

static int32_t or_theta_size(int32_t kind) { return kind == OR_WINDKESSEL ? 7 : 5; }

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

double or_propose(const or_param *spec, int32_t nth, const double *th, uint64_t seed, uint32_t j,
                  uint32_t i, double *out) {
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
        const double z = or_normal64(seed, j, i, OR_PURPOSE_PMMH, 2u * blk);
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
        or_block(seed, j, i, OR_PURPOSE_PMMH, 16u + 64u * (uint32_t)d + (uint32_t)a, w);
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
  if (lik == OR_LIK_KALMAN && m->kind != OR_WINDKESSEL) return OR_EINVAL;
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
