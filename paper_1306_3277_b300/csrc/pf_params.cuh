// pf_params.cuh -- priors and proposals over the model parameters theta
// (the parameter and proposal_parameter blocks of the paper's model listings,
// Sec. 2.1), shared by the marginal Metropolis-Hastings (Algorithm 3) and
// SMC^2 (Algorithm 4) samplers.  Device code plus the host-side spec check.
#pragma once
#include <cmath>

#include "pf_runtime.h"

namespace pfb {

constexpr int MAX_THETA = 8;
constexpr int TG_ATTEMPTS = 64;
constexpr uint32_t PURPOSE_PMMH = 5;  // Philox purposes of the two samplers
constexpr uint32_t PURPOSE_SMC2 = 6;

struct Spec {
  pf_param p[MAX_THETA];
  int nth;
};

__device__ inline double log_prior(const Spec& sp, const double* th) {
  double lp = 0.0;
  for (int d = 0; d < sp.nth; ++d) {
    const pf_param& p = sp.p[d];
    const double x = th[d];
    switch (p.prior) {
      case PF_PRIOR_UNIFORM:
        if (!(x >= p.a && x <= p.b)) return -INFINITY;
        lp += -log(p.b - p.a);
        break;
      case PF_PRIOR_GAUSSIAN: {
        const double z = (x - p.a) / p.b;
        lp += -0.5 * z * z - log(p.b) - 0.5 * log(2.0 * 3.141592653589793);
        break;
      }
      case PF_PRIOR_GAMMA:
        if (!(x > 0.0)) return -INFINITY;
        lp += (p.a - 1.0) * log(x) - x / p.b - lgamma(p.a) - p.a * log(p.b);
        break;
      case PF_PRIOR_INV_GAMMA:
        if (!(x > 0.0)) return -INFINITY;
        lp += p.a * log(p.b) - lgamma(p.a) - (p.a + 1.0) * log(x) - p.b / x;
        break;
      default:
        break;
    }
  }
  return lp;
}

// log of the probability N(mu, sd^2) gives to [lo, hi]
__device__ inline double tg_log_mass(double mu, double sd, double lo, double hi) {
  const double up = isinf(hi) ? 1.0 : 0.5 * erfc(-(hi - mu) / sd * 0.7071067811865476);
  const double dn = isinf(lo) ? 0.0 : 0.5 * erfc(-(lo - mu) / sd * 0.7071067811865476);
  return log(up - dn);
}

__device__ inline double ig_logpdf(double x, double shape, double scale) {
  return shape * log(scale) - lgamma(shape) - (shape + 1.0) * log(x) - scale / x;
}

// A 64-bit Philox key from the block (j, i, purpose, blk): words 1:0 low, 3:2 high.
__device__ __forceinline__ uint64_t philox_key(uint64_t seed, uint32_t j, uint32_t i,
                                               uint32_t purpose, uint32_t blk) {
  const uint4 w = rng_block(seed, j, i, purpose, blk);
  return (uint64_t(w.y) << 32) | uint64_t(w.x);
}

// One proposal theta' ~ q(.|theta) of stream (j, i, purpose): the truncated
// gaussian takes the first of 64 attempts (blocks 16 + 64 d + a) that lands
// inside its bounds (none: theta_d unchanged); the inverse gamma of integer
// shape k is scale / Gamma(k, 1), Gamma(k, 1) the sum of k unit exponentials
// -log u (blocks 16 + 64 d + a, a < k).  Returns log q(theta|theta') -
// log q(theta'|theta).
__device__ inline double propose(const Spec& sp, const double* th, uint64_t seed, uint32_t j,
                          uint32_t i, uint32_t purpose, double* out) {
  double lqr = 0.0;
  for (int d = 0; d < sp.nth; ++d) {
    const pf_param& p = sp.p[d];
    const double x = th[d];
    double xn = x;
    if (p.proposal == PF_PROPOSE_TRUNC_GAUSSIAN) {
      for (int a = 0; a < TG_ATTEMPTS; ++a) {
        const uint4 w = rng_block(seed, j, i, purpose, 16u + 64u * uint32_t(d) + uint32_t(a));
        double z0, z1;
        normal_pair64(w, &z0, &z1);
        const double v = fma(p.c, z0, x);
        if (v >= p.d && v <= p.e) {
          xn = v;
          break;
        }
      }
      lqr += tg_log_mass(x, p.c, p.d, p.e) - tg_log_mass(xn, p.c, p.d, p.e);
    } else if (p.proposal == PF_PROPOSE_INV_GAMMA) {
      const int k = int(p.c);
      double sum = 0.0;
      for (int a = 0; a < k; ++a) {
        const uint4 w = rng_block(seed, j, i, purpose, 16u + 64u * uint32_t(d) + uint32_t(a));
        sum = sum + -log_pos(u53_open_closed(w.x, w.y));
      }
      xn = (p.d * x) / sum;
      lqr += ig_logpdf(x, p.c, p.d * xn) - ig_logpdf(xn, p.c, p.d * x);
    }
    out[d] = xn;
  }
  return lqr;
}

// A draw from the prior of stream (j, 0, purpose), blocks 16 + 64 d + a:
// uniform a + (b - a) u (u in [0, 1) from words 1:0), gaussian a + b z (the
// first Box-Muller normal), gamma b G and inverse gamma b / G with G the sum
// of `a` (an integer) unit exponentials; fixed components come from base.
__device__ inline void prior_draw(const Spec& sp, const double* base, uint64_t seed, uint32_t j,
                           uint32_t purpose, double* out) {
  for (int d = 0; d < sp.nth; ++d) {
    const pf_param& p = sp.p[d];
    const uint32_t blk = 16u + 64u * uint32_t(d);
    switch (p.prior) {
      case PF_PRIOR_UNIFORM: {
        const uint4 w = rng_block(seed, j, 0u, purpose, blk);
        out[d] = fma(p.b - p.a, u53_closed_open(w.x, w.y), p.a);
        break;
      }
      case PF_PRIOR_GAUSSIAN: {
        double z0, z1;
        normal_pair64(rng_block(seed, j, 0u, purpose, blk), &z0, &z1);
        out[d] = fma(p.b, z0, p.a);
        break;
      }
      case PF_PRIOR_GAMMA:
      case PF_PRIOR_INV_GAMMA: {
        const int k = int(p.a);
        double sum = 0.0;
        for (int a = 0; a < k; ++a) {
          const uint4 w = rng_block(seed, j, 0u, purpose, blk + uint32_t(a));
          sum = sum + -log_pos(u53_open_closed(w.x, w.y));
        }
        out[d] = p.prior == PF_PRIOR_GAMMA ? p.b * sum : p.b / sum;
        break;
      }
      default:
        out[d] = base[d];
    }
  }
}

inline pf_status check_spec(const pf_param* spec, int nth) {
  for (int d = 0; d < nth; ++d) {
    const pf_param& p = spec[d];
    bool ok = true;
    switch (p.prior) {
      case PF_PRIOR_FIXED: break;
      case PF_PRIOR_UNIFORM: ok = p.a < p.b; break;
      case PF_PRIOR_GAUSSIAN: ok = p.b > 0.0; break;
      case PF_PRIOR_GAMMA:
      case PF_PRIOR_INV_GAMMA: ok = p.a > 0.0 && p.b > 0.0; break;
      default: ok = false;
    }
    if (!ok) return fail(PF_EINVAL, "prior of theta[%d]: bad kind or parameters", d);
    switch (p.proposal) {
      case PF_PROPOSE_FIXED: break;
      case PF_PROPOSE_TRUNC_GAUSSIAN: ok = p.c > 0.0 && p.d < p.e; break;
      case PF_PROPOSE_INV_GAMMA:
        ok = p.c >= 1.0 && p.c <= 64.0 && p.c == std::floor(p.c) && p.d > 0.0;
        break;
      default: ok = false;
    }
    if (!ok) return fail(PF_EINVAL, "proposal of theta[%d]: bad kind or parameters", d);
  }
  return PF_OK;
}


}  // namespace pfb
