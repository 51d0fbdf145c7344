/*
 * pf_oracle.c -- plain CPU oracle of the bootstrap particle filter
 * (arXiv 1306.3277, Algorithm 2, Sec. 3.1.2) with systematic resampling
 * (Sec. 3.3, Kitagawa 1996) and an ESS test.
 *
 * TEST INFRASTRUCTURE ONLY: called by the tests, the smoke check and the
 * CPU-baseline leg of the benchmark, never by the product path.  It shares no
 * code with the CUDA implementation.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -fPIC -shared (oracle/build.py).
 * -ffp-contract=off matters: every fused multiply-add below is an explicit
 * fma()/fmaf() call, every other operation is rounded on its own.
 *
 * Readings of the paper that this file takes (all listed in the design notes):
 *  - windkessel transition: Euler step x + dt (F/C - x/(RC)) + N(0, q) per
 *    substep, F(t_{k}) held over [t_k, t_k + dt); observation N(x + Z F(t_i), r)
 *    (Sec. 2.1.1 gives an exact-exponential form with noise on the flow; the
 *    Euler form is the workload's);
 *  - second argument of N(.,.) is a variance;
 *  - flow F(t) = peak sin(2 pi t / period) on the first half period, else 0;
 *  - Lorenz '96: classic RK4 of Eq. (lorenz96-ode), additive N(0, q) noise on
 *    every component once per observation interval;
 *  - first propagation uses identity ancestors (all initial weights equal);
 *  - no resampling after the final observation;
 *  - the constant -Ny/2 log(2 pi r) of the Gaussian observation density is
 *    added to each likelihood increment, not to the particle log-weights;
 *  - the particle log-weight is -(1/2) rss / r, rss the residual sum of
 *    squares (fma-accumulated over the observed components in index order);
 *  - systematic target j sits at (j + u) S / P and takes the first particle
 *    whose cumulative weight C_k exceeds it (Sec. 3.3).
 */
#include "pf_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ======================================================================
 * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
 * easy as 1, 2, 3", SC'11): 10 rounds of a 4x32-bit bijection keyed by a
 * 2x32-bit key; the key is bumped by the Weyl constants between rounds.
 * ==================================================================== */
#define OR_PHILOX_M0 0xD2511F53u
#define OR_PHILOX_M1 0xCD9E8D57u
#define OR_PHILOX_W0 0x9E3779B9u
#define OR_PHILOX_W1 0xBB67AE85u

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  int round;
  for (round = 0; round < 10; ++round) {
    uint64_t prod0, prod1;
    uint32_t y0, y1, y2, y3;
    if (round > 0) {
      k0 += OR_PHILOX_W0;
      k1 += OR_PHILOX_W1;
    }
    prod0 = (uint64_t)OR_PHILOX_M0 * (uint64_t)x0;
    prod1 = (uint64_t)OR_PHILOX_M1 * (uint64_t)x2;
    y0 = (uint32_t)(prod1 >> 32) ^ x1 ^ k0;
    y1 = (uint32_t)prod1;
    y2 = (uint32_t)(prod0 >> 32) ^ x3 ^ k1;
    y3 = (uint32_t)prod0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Counter layout: (particle j, time index i, (purpose << 16) | block, 0);
 * key = (low, high) 32-bit halves of the 64-bit seed. */
void or_block(uint64_t seed, uint32_t j, uint32_t i, uint32_t purpose, uint32_t blk,
                     uint32_t w[4]) {
  uint32_t ctr[4], key[2];
  ctr[0] = j;
  ctr[1] = i;
  ctr[2] = (purpose << 16) | blk;
  ctr[3] = 0u;
  key[0] = (uint32_t)(seed & 0xffffffffu);
  key[1] = (uint32_t)(seed >> 32);
  or_philox4x32_10(ctr, key, w);
}

/* 53-bit uniforms from the 64-bit word (hi:lo). */
double or_u53_half_open(uint32_t lo, uint32_t hi) { /* [0, 1) */
  uint64_t v = ((((uint64_t)hi) << 32) | (uint64_t)lo) >> 11;
  return (double)v * 0x1.0p-53;
}
double or_u53_open_zero(uint32_t lo, uint32_t hi) { /* (0, 1] */
  uint64_t v = ((((uint64_t)hi) << 32) | (uint64_t)lo) >> 11;
  return (double)(v + 1u) * 0x1.0p-53;
}

/* ======================================================================
 * Own natural logarithm (FP64).  Reduction x = m 2^e with m in [1/sqrt2,
 * sqrt2), then log m = 2 atanh(f), f = (m-1)/(m+1), by its odd power series
 * 2 (f + f^3/3 + f^5/5 + ...) truncated after the f^23 term (|f| <= 0.1716,
 * truncation error below 2^-60 relative), and log x = e ln2 + log m with ln2
 * split into two doubles.  Valid for positive finite normal x.
 * ==================================================================== */
static const double OR_LN2_HI = 0x1.62e42fefa39efp-1;
static const double OR_LN2_LO = 0x1.abc9e3b39803fp-56;
static const double OR_SQRT1_2 = 0x1.6a09e667f3bcdp-1;

double or_log(double x) {
  int e;
  double m, f, t, s, p, r, de;
  if (x == 0.0) return -INFINITY;
  m = frexp(x, &e); /* x = m 2^e, m in [0.5, 1) */
  if (m < OR_SQRT1_2) {
    m = m + m;
    e = e - 1;
  }
  f = (m - 1.0) / (m + 1.0);
  t = f + f;
  s = f * f;
  p = 1.0 / 23.0;
  p = fma(p, s, 1.0 / 21.0);
  p = fma(p, s, 1.0 / 19.0);
  p = fma(p, s, 1.0 / 17.0);
  p = fma(p, s, 1.0 / 15.0);
  p = fma(p, s, 1.0 / 13.0);
  p = fma(p, s, 1.0 / 11.0);
  p = fma(p, s, 1.0 / 9.0);
  p = fma(p, s, 1.0 / 7.0);
  p = fma(p, s, 1.0 / 5.0);
  p = fma(p, s, 1.0 / 3.0);
  r = fma(t * s, p, t);
  de = (double)e;
  return fma(de, OR_LN2_HI, fma(de, OR_LN2_LO, r));
}

/* ======================================================================
 * Own exponential (FP64), Cody and Waite's reduction: k = rint(x / ln2),
 * r = x - k ln2 with ln2 in two parts (two fmas), |r| <= ln2 / 2; e^r by its
 * Taylor series to r^14 (truncation below 2^-63 relative), then
 * e^x = e^r 2^k.  +inf above 709.78, 0 below -745.14, NaN passes through.
 * Used where the state depends on an exponential (the exact windkessel),
 * so that both implementations compute it bit for bit alike.
 * ==================================================================== */
double or_exp(double x) {
  double k, r, p;
  if (x != x) return x;
  if (x > 709.782712893384) return INFINITY;
  if (x < -745.1332191019412) return 0.0;
  k = rint(x * 0x1.71547652b82fep+0);
  r = fma(-k, OR_LN2_HI, x);
  r = fma(-k, OR_LN2_LO, r);
  p = 1.0 / 87178291200.0;
  p = fma(p, r, 1.0 / 6227020800.0);
  p = fma(p, r, 1.0 / 479001600.0);
  p = fma(p, r, 1.0 / 39916800.0);
  p = fma(p, r, 1.0 / 3628800.0);
  p = fma(p, r, 1.0 / 362880.0);
  p = fma(p, r, 1.0 / 40320.0);
  p = fma(p, r, 1.0 / 5040.0);
  p = fma(p, r, 1.0 / 720.0);
  p = fma(p, r, 1.0 / 120.0);
  p = fma(p, r, 1.0 / 24.0);
  p = fma(p, r, 1.0 / 6.0);
  p = fma(p, r, 0.5);
  p = fma(p, r, 1.0);
  p = fma(p, r, 1.0);
  return ldexp(p, (int)k);
}

/* ======================================================================
 * Own sin(2 pi u), cos(2 pi u) for u in [0, 1) (FP64).  Quarter-turn
 * reduction q = rint(4u), r = 4u - q in [-1/2, 1/2] (exact), x = r pi/2 with
 * pi/2 split in two doubles, then the Taylor series of sin to x^19 and of cos
 * to x^20 (|x| <= pi/4, truncation below 2^-60), then the quadrant rotation.
 * ==================================================================== */
static const double OR_PIO2_HI = 0x1.921fb54442d18p+0;
static const double OR_PIO2_LO = 0x1.1a62633145c07p-54;

void or_sincos2pi(double u, double *sn, double *cs) {
  double v = 4.0 * u;
  double q = rint(v);
  double r = v - q;
  double x = fma(r, OR_PIO2_HI, r * OR_PIO2_LO);
  double s = x * x;
  double ps, pc, sx, cx;
  int quadrant;
  ps = -1.0 / 121645100408832000.0;          /* -1/19! */
  ps = fma(ps, s, 1.0 / 355687428096000.0);  /*  1/17! */
  ps = fma(ps, s, -1.0 / 1307674368000.0);   /* -1/15! */
  ps = fma(ps, s, 1.0 / 6227020800.0);       /*  1/13! */
  ps = fma(ps, s, -1.0 / 39916800.0);        /* -1/11! */
  ps = fma(ps, s, 1.0 / 362880.0);           /*  1/9!  */
  ps = fma(ps, s, -1.0 / 5040.0);            /* -1/7!  */
  ps = fma(ps, s, 1.0 / 120.0);              /*  1/5!  */
  ps = fma(ps, s, -1.0 / 6.0);               /* -1/3!  */
  sx = fma(x * s, ps, x);
  pc = 1.0 / 2432902008176640000.0;          /*  1/20! */
  pc = fma(pc, s, -1.0 / 6402373705728000.0);/* -1/18! */
  pc = fma(pc, s, 1.0 / 20922789888000.0);   /*  1/16! */
  pc = fma(pc, s, -1.0 / 87178291200.0);     /* -1/14! */
  pc = fma(pc, s, 1.0 / 479001600.0);        /*  1/12! */
  pc = fma(pc, s, -1.0 / 3628800.0);         /* -1/10! */
  pc = fma(pc, s, 1.0 / 40320.0);            /*  1/8!  */
  pc = fma(pc, s, -1.0 / 720.0);             /* -1/6!  */
  pc = fma(pc, s, 1.0 / 24.0);               /*  1/4!  */
  pc = fma(pc, s, -0.5);                     /* -1/2!  */
  cx = fma(s, pc, 1.0);
  quadrant = ((int)q) & 3;
  if (quadrant == 0) { *sn = sx; *cs = cx; }
  else if (quadrant == 1) { *sn = cx; *cs = -sx; }
  else if (quadrant == 2) { *sn = -sx; *cs = -cx; }
  else { *sn = -cx; *cs = sx; }
}

/* FP32 counterparts, same method, series cut where FP32 no longer sees them. */
static const float OR_LN2F_HI = 0x1.62e430p-1f;
static const float OR_LN2F_LO = -0x1.05c610p-29f;
static const float OR_SQRT1_2F = 0x1.6a09e6p-1f;
static const float OR_PIO2F_HI = 0x1.921fb6p+0f;
static const float OR_PIO2F_LO = -0x1.777a5cp-25f;

float or_logf(float x) {
  int e;
  float m, f, t, s, p, r, de;
  if (x == 0.0f) return -INFINITY;
  m = frexpf(x, &e);
  if (m < OR_SQRT1_2F) {
    m = m + m;
    e = e - 1;
  }
  f = (m - 1.0f) / (m + 1.0f);
  t = f + f;
  s = f * f;
  p = 1.0f / 11.0f;
  p = fmaf(p, s, 1.0f / 9.0f);
  p = fmaf(p, s, 1.0f / 7.0f);
  p = fmaf(p, s, 1.0f / 5.0f);
  p = fmaf(p, s, 1.0f / 3.0f);
  r = fmaf(t * s, p, t);
  de = (float)e;
  return fmaf(de, OR_LN2F_HI, fmaf(de, OR_LN2F_LO, r));
}

void or_sincos2pif(float u, float *sn, float *cs) {
  float v = 4.0f * u;
  float q = rintf(v);
  float r = v - q;
  float x = fmaf(r, OR_PIO2F_HI, r * OR_PIO2F_LO);
  float s = x * x;
  float ps, pc, sx, cx;
  int quadrant;
  ps = -1.0f / 39916800.0f;             /* -1/11! */
  ps = fmaf(ps, s, 1.0f / 362880.0f);   /*  1/9!  */
  ps = fmaf(ps, s, -1.0f / 5040.0f);    /* -1/7!  */
  ps = fmaf(ps, s, 1.0f / 120.0f);      /*  1/5!  */
  ps = fmaf(ps, s, -1.0f / 6.0f);       /* -1/3!  */
  sx = fmaf(x * s, ps, x);
  pc = 1.0f / 479001600.0f;             /*  1/12! */
  pc = fmaf(pc, s, -1.0f / 3628800.0f); /* -1/10! */
  pc = fmaf(pc, s, 1.0f / 40320.0f);    /*  1/8!  */
  pc = fmaf(pc, s, -1.0f / 720.0f);     /* -1/6!  */
  pc = fmaf(pc, s, 1.0f / 24.0f);       /*  1/4!  */
  pc = fmaf(pc, s, -0.5f);              /* -1/2!  */
  cx = fmaf(s, pc, 1.0f);
  quadrant = ((int)q) & 3;
  if (quadrant == 0) { *sn = sx; *cs = cx; }
  else if (quadrant == 1) { *sn = cx; *cs = -sx; }
  else if (quadrant == 2) { *sn = -sx; *cs = -cx; }
  else { *sn = -cx; *cs = sx; }
}

/* ======================================================================
 * Normals by Box-Muller (z0 = sqrt(-2 ln u1) cos 2 pi u2,
 * z1 = sqrt(-2 ln u1) sin 2 pi u2).
 * FP64: one Philox block gives u1 in (0,1] from words (w1:w0) and u2 in
 *       [0,1) from (w3:w2): one pair, normals 2b, 2b+1 of the stream.
 * FP32: one block gives two pairs, (w0, w1) and (w2, w3), each u1 =
 *       ((w >> 8) + 1) 2^-24 in (0,1], u2 = (w >> 8) 2^-24 in [0,1):
 *       normals 4b .. 4b+3 of the stream.
 * ==================================================================== */
double or_normal64(uint64_t seed, uint32_t j, uint32_t i, uint32_t purpose, uint32_t q) {
  uint32_t w[4];
  double u1, u2, rad, sn, cs;
  or_block(seed, j, i, purpose, q >> 1, w);
  u1 = or_u53_open_zero(w[0], w[1]);
  u2 = or_u53_half_open(w[2], w[3]);
  rad = sqrt(-2.0 * or_log(u1));
  or_sincos2pi(u2, &sn, &cs);
  return (q & 1u) ? rad * sn : rad * cs;
}

float or_normal32(uint64_t seed, uint32_t j, uint32_t i, uint32_t purpose, uint32_t q) {
  uint32_t w[4], wa, wb;
  float u1, u2, rad, sn, cs;
  or_block(seed, j, i, purpose, q >> 2, w);
  if ((q >> 1) & 1u) { wa = w[2]; wb = w[3]; }
  else { wa = w[0]; wb = w[1]; }
  u1 = (float)((wa >> 8) + 1u) * 0x1.0p-24f;
  u2 = (float)(wb >> 8) * 0x1.0p-24f;
  rad = sqrtf(-2.0f * or_logf(u1));
  or_sincos2pif(u2, &sn, &cs);
  return (q & 1u) ? rad * sn : rad * cs;
}

/* Bulk form for statistical tests: out[j nq + q] = normal q of stream (j, i, purpose). */
void or_fill_normals(uint64_t seed, int32_t prec, uint32_t i, uint32_t purpose, uint32_t nj,
                     uint32_t nq, double *out) {
  uint32_t j, q;
  for (j = 0; j < nj; ++j)
    for (q = 0; q < nq; ++q)
      out[(size_t)j * nq + q] = prec == OR_MIXED ? (double)or_normal32(seed, j, i, purpose, q)
                                                 : or_normal64(seed, j, i, purpose, q);
}

/* One uniform in [0,1) per resampling step i: block (0, i, RESAMPLE, 0). */
double or_resample_uniform(uint64_t seed, uint32_t i) {
  uint32_t w[4];
  or_block(seed, 0u, i, OR_PURPOSE_RESAMPLE, 0u, w);
  return or_u53_half_open(w[0], w[1]);
}

/* ======================================================================
 * Windkessel input F(t_k), t_k = k dt (Eq. flow, read as a half sine of
 * the given peak and period), held constant over [t_k, t_k + dt).
 * ==================================================================== */
void or_flow_table(double peak, double period, double dt, int64_t n, double *out) {
  int64_t k;
  for (k = 0; k < n; ++k) {
    double t = (double)k * dt;
    double ph = t / period;
    double fr = ph - floor(ph);
    if (fr < 0.5) {
      double sn, cs;
      or_sincos2pi(fr, &sn, &cs);
      out[k] = peak * sn;
    } else {
      out[k] = 0.0;
    }
  }
}

/* ======================================================================
 * Lorenz '96 (Eq. lorenz96-ode): dx_n/dt = (x_{n+1} - x_{n-2}) x_{n-1} - x_n + F,
 * cyclic indices, evaluated as fma(x_{n+1} - x_{n-2}, x_{n-1}, F - x_n).
 * Classic RK4 (Sec. 2.1.2) with the combination accumulated as
 * x + h/6 k1 + h/3 k2 + h/3 k3 + h/6 k4 by successive fmas.
 * ==================================================================== */
static void or_l96_rhs(const double *xs, double *k, int32_t N, double F) {
  int32_t n;
  for (n = 0; n < N; ++n) {
    double xp1 = xs[(n + 1) % N];
    double xm1 = xs[(n + N - 1) % N];
    double xm2 = xs[(n + N - 2) % N];
    k[n] = fma(xp1 - xm2, xm1, F - xs[n]);
  }
}

static void or_l96_rk4_step(double *x, int32_t N, double F, double dt, double *k, double *xs,
                            double *acc) {
  double h2 = 0.5 * dt, h3 = dt / 3.0, h6 = dt / 6.0;
  int32_t n;
  or_l96_rhs(x, k, N, F);
  for (n = 0; n < N; ++n) { acc[n] = fma(h6, k[n], x[n]); xs[n] = fma(h2, k[n], x[n]); }
  or_l96_rhs(xs, k, N, F);
  for (n = 0; n < N; ++n) { acc[n] = fma(h3, k[n], acc[n]); xs[n] = fma(h2, k[n], x[n]); }
  or_l96_rhs(xs, k, N, F);
  for (n = 0; n < N; ++n) { acc[n] = fma(h3, k[n], acc[n]); xs[n] = fma(dt, k[n], x[n]); }
  or_l96_rhs(xs, k, N, F);
  for (n = 0; n < N; ++n) x[n] = fma(h6, k[n], acc[n]);
}

void or_l96_rk4(double *x, int32_t N, double F, double dt, int32_t nsteps) {
  double *buf = (double *)malloc(sizeof(double) * 3 * (size_t)N);
  int32_t s;
  for (s = 0; s < nsteps; ++s) or_l96_rk4_step(x, N, F, dt, buf, buf + N, buf + 2 * N);
  free(buf);
}

static void or_l96_rhsf(const float *xs, float *k, int32_t N, float F) {
  int32_t n;
  for (n = 0; n < N; ++n) {
    float xp1 = xs[(n + 1) % N];
    float xm1 = xs[(n + N - 1) % N];
    float xm2 = xs[(n + N - 2) % N];
    k[n] = fmaf(xp1 - xm2, xm1, F - xs[n]);
  }
}

static void or_l96_rk4_stepf(float *x, int32_t N, float F, float dt, float *k, float *xs,
                             float *acc) {
  float h2 = 0.5f * dt, h3 = dt / 3.0f, h6 = dt / 6.0f;
  int32_t n;
  or_l96_rhsf(x, k, N, F);
  for (n = 0; n < N; ++n) { acc[n] = fmaf(h6, k[n], x[n]); xs[n] = fmaf(h2, k[n], x[n]); }
  or_l96_rhsf(xs, k, N, F);
  for (n = 0; n < N; ++n) { acc[n] = fmaf(h3, k[n], acc[n]); xs[n] = fmaf(h2, k[n], x[n]); }
  or_l96_rhsf(xs, k, N, F);
  for (n = 0; n < N; ++n) { acc[n] = fmaf(h3, k[n], acc[n]); xs[n] = fmaf(dt, k[n], x[n]); }
  or_l96_rhsf(xs, k, N, F);
  for (n = 0; n < N; ++n) x[n] = fmaf(h6, k[n], acc[n]);
}

void or_l96_rk4f(float *x, int32_t N, float F, float dt, int32_t nsteps) {
  float *buf = (float *)malloc(sizeof(float) * 3 * (size_t)N);
  int32_t s;
  for (s = 0; s < nsteps; ++s) or_l96_rk4_stepf(x, N, F, dt, buf, buf + N, buf + 2 * N);
  free(buf);
}

/* The same RK4 step with a per-component forcing Fv[n] in place of F (the
 * stochastic form: F plus the substep's Wiener increment over its length). */
static void or_l96_rhs_v(const double *xs, double *k, int32_t N, const double *Fv) {
  int32_t n;
  for (n = 0; n < N; ++n) {
    double xp1 = xs[(n + 1) % N];
    double xm1 = xs[(n + N - 1) % N];
    double xm2 = xs[(n + N - 2) % N];
    k[n] = fma(xp1 - xm2, xm1, Fv[n] - xs[n]);
  }
}

static void or_l96_rk4_step_v(double *x, int32_t N, const double *Fv, double dt, double *k,
                              double *xs, double *acc) {
  double h2 = 0.5 * dt, h3 = dt / 3.0, h6 = dt / 6.0;
  int32_t n;
  or_l96_rhs_v(x, k, N, Fv);
  for (n = 0; n < N; ++n) { acc[n] = fma(h6, k[n], x[n]); xs[n] = fma(h2, k[n], x[n]); }
  or_l96_rhs_v(xs, k, N, Fv);
  for (n = 0; n < N; ++n) { acc[n] = fma(h3, k[n], acc[n]); xs[n] = fma(h2, k[n], x[n]); }
  or_l96_rhs_v(xs, k, N, Fv);
  for (n = 0; n < N; ++n) { acc[n] = fma(h3, k[n], acc[n]); xs[n] = fma(dt, k[n], x[n]); }
  or_l96_rhs_v(xs, k, N, Fv);
  for (n = 0; n < N; ++n) x[n] = fma(h6, k[n], acc[n]);
}

static void or_l96_rhs_vf(const float *xs, float *k, int32_t N, const float *Fv) {
  int32_t n;
  for (n = 0; n < N; ++n) {
    float xp1 = xs[(n + 1) % N];
    float xm1 = xs[(n + N - 1) % N];
    float xm2 = xs[(n + N - 2) % N];
    k[n] = fmaf(xp1 - xm2, xm1, Fv[n] - xs[n]);
  }
}

static void or_l96_rk4_step_vf(float *x, int32_t N, const float *Fv, float dt, float *k,
                               float *xs, float *acc) {
  float h2 = 0.5f * dt, h3 = dt / 3.0f, h6 = dt / 6.0f;
  int32_t n;
  or_l96_rhs_vf(x, k, N, Fv);
  for (n = 0; n < N; ++n) { acc[n] = fmaf(h6, k[n], x[n]); xs[n] = fmaf(h2, k[n], x[n]); }
  or_l96_rhs_vf(xs, k, N, Fv);
  for (n = 0; n < N; ++n) { acc[n] = fmaf(h3, k[n], acc[n]); xs[n] = fmaf(h2, k[n], x[n]); }
  or_l96_rhs_vf(xs, k, N, Fv);
  for (n = 0; n < N; ++n) { acc[n] = fmaf(h3, k[n], acc[n]); xs[n] = fmaf(dt, k[n], x[n]); }
  or_l96_rhs_vf(xs, k, N, Fv);
  for (n = 0; n < N; ++n) x[n] = fmaf(h6, k[n], acc[n]);
}

/* ======================================================================
 * Scalar Kalman filter (Algorithm 1 reduced to one dimension) for the
 * Euler windkessel: x_{k+1} = a x_k + b_k + N(0, q), a = 1 - dt/(RC),
 * b_k = dt F_k / C; y_i = x_{i s} + Z F_{i s} + N(0, r); x_0 ~ N(m0, s0^2).
 * Returns log p(y_{1:T} | theta) (the likelihood line of Algorithm 1).
 * ==================================================================== */
double or_kalman_windkessel(const or_model *m, const double *th, const double *y, int32_t T) {
  const double R = th[0], C = th[1], Z = th[2], q = th[3], r = th[4], m0 = th[5], s0 = th[6];
  const int32_t s = m->substeps;
  const double dt = m->dt;
  const int64_t nflow = (int64_t)T * s + 1;
  double *F = (double *)malloc(sizeof(double) * (size_t)nflow);
  /* Euler form: a = 1 - dt/(RC), input dt F/C, noise q; exact form (the
   * paper's transition): a = exp(-dt/(RC)), input R(1-a) F, and the flow
   * noise N(0, (dt sqrt(q))^2) scaled by R(1-a) */
  const int exact = m->kind == OR_WINDKESSEL_EXP;
  double a = exact ? exp(-dt / (R * C)) : 1.0 - dt / (R * C);
  const double bin = exact ? R * (1.0 - a) : dt / C;
  const double qv = exact ? bin * bin * dt * dt * q : q;
  double mu = m0, V = s0 * s0, ll = 0.0;
  int32_t i, mm;
  or_flow_table(m->flow_peak, m->flow_period, dt, nflow, F);
  for (i = 1; i <= T; ++i) {
    double nu, Sv, d, K;
    for (mm = 0; mm < s; ++mm) {
      int64_t k = (int64_t)(i - 1) * s + mm;
      mu = exact ? a * mu + bin * F[k] : a * mu + dt * F[k] / C;
      V = a * a * V + qv;
    }
    if (m->obs_every > 1 && i % m->obs_every != 0) continue; /* no observation at t_i */
    nu = mu + Z * F[(int64_t)i * s];
    Sv = V + r;
    d = y[i - 1] - nu;
    ll += -0.5 * log(2.0 * M_PI * Sv) - 0.5 * d * d / Sv;
    K = V / Sv;
    mu = mu + K * d;
    V = V * r / Sv;
  }
  free(F);
  return ll;
}

/* ======================================================================
 * Log-sum-exp pieces (the likelihood line of Algorithm 2 in log space):
 * M = max ell, w = exp(ell - M), S = sum w, Q = sum w^2, both by Neumaier's
 * compensated summation so that S is close to the correctly rounded sum.
 * ==================================================================== */
static void or_neumaier_add(double *sum, double *comp, double v) {
  double t = *sum + v;
  if (fabs(*sum) >= fabs(v)) *comp += (*sum - t) + v;
  else *comp += (v - t) + *sum;
  *sum = t;
}

void or_lse(const double *ell, int64_t P, double *Mo, double *So, double *Qo) {
  double M = -INFINITY, s = 0.0, sc = 0.0, q = 0.0, qc = 0.0;
  int64_t j;
  for (j = 0; j < P; ++j)
    if (ell[j] > M) M = ell[j];
  if (M == -INFINITY) { *Mo = M; *So = 0.0; *Qo = 0.0; return; }
  for (j = 0; j < P; ++j) {
    double w = exp(ell[j] - M);
    or_neumaier_add(&s, &sc, w);
    or_neumaier_add(&q, &qc, w * w);
  }
  *Mo = M; *So = s + sc; *Qo = q + qc;
}

/* ======================================================================
 * Systematic resampling (Sec. 3.3): cumulative weights C_k (compensated
 * inclusive prefix of w = exp(ell - M)), total S = C_{P-1}, one uniform u.
 * Target j (j = 0..P-1) sits at tau_j = (j + u) S / P and takes the first
 * particle whose cumulative weight exceeds it: a_j = min{k : C_k > tau_j},
 * clamped to P-1.  Ancestors come out sorted.  A target within 1e-12 S of
 * C_k or C_{k-1} counts as near (another rounding of the same comparison
 * may decide it the other way).
 * ==================================================================== */
static int64_t or_systematic_from_w(const double *w, int64_t P, double u, int32_t *anc,
                                    double *Cbuf) {
  double sum = 0.0, comp = 0.0, S;
  int64_t j, k, near = 0;
  for (k = 0; k < P; ++k) {
    or_neumaier_add(&sum, &comp, w[k]);
    Cbuf[k] = sum + comp;
  }
  S = Cbuf[P - 1];
  for (j = 0; j < P; ++j) {
    const double tau = ((double)j + u) * S / (double)P;
    int64_t lo = 0, hi = P; /* first k in [lo, hi) with C_k > tau */
    while (lo < hi) {
      int64_t mid = lo + (hi - lo) / 2;
      if (Cbuf[mid] > tau) hi = mid;
      else lo = mid + 1;
    }
    k = lo < P ? lo : P - 1;
    anc[j] = (int32_t)k;
    if (fabs(tau - Cbuf[k]) <= 1e-12 * S || (k > 0 && fabs(tau - Cbuf[k - 1]) <= 1e-12 * S))
      ++near;
  }
  return near;
}

/* ======================================================================
 * Stratified and multinomial resampling (Sec. 3.3; Algorithm 2 draws the
 * ancestors from a multinomial).  Both compare targets tau_j with the
 * cumulative weights C_k (compensated) and give a_j = min{k : C_k > tau_j},
 * clamped to P-1; targets increase with j, so ancestors come out sorted.
 *   stratified:  tau_j = (j + u_j) S / P, u_j in [0, 1) from Philox block
 *                (j, i, RESAMPLE, 1), words 1:0.
 *   multinomial: P + 1 unit exponentials e_l = -log v_l (own log), v_l in
 *                (0, 1] the 53-bit uniform of words 1:0 of block
 *                (l, i, RESAMPLE, 2); partial sums G_m = e_0 + .. + e_m
 *                (compensated); tau_j = (G_j / G_P) S.  (G_0, .., G_{P-1}) /
 *                G_P are the order statistics of P independent uniforms, so
 *                the offspring counts are Multinomial(P, w / S).
 * A target within 1e-12 S of C_k or C_{k-1} counts as near.
 * ==================================================================== */
static int64_t or_resample_other(const double *w, int64_t P, int32_t kind, uint64_t seed,
                                 uint32_t i, int32_t *anc, double *Cbuf) {
  double sum = 0.0, comp = 0.0, S, GP = 1.0;
  double *G = NULL;
  int64_t j, k, near = 0;
  for (k = 0; k < P; ++k) {
    or_neumaier_add(&sum, &comp, w[k]);
    Cbuf[k] = sum + comp;
  }
  S = Cbuf[P - 1];
  if (kind == OR_RESAMPLE_MULTINOMIAL) {
    double gs = 0.0, gc = 0.0;
    uint32_t wd[4];
    G = (double *)malloc(sizeof(double) * (size_t)P);
    for (j = 0; j <= P; ++j) {
      or_block(seed, (uint32_t)j, i, OR_PURPOSE_RESAMPLE, 2u, wd);
      or_neumaier_add(&gs, &gc, -or_log(or_u53_open_zero(wd[0], wd[1])));
      if (j < P) G[j] = gs + gc;
    }
    GP = gs + gc;
  }
  for (j = 0; j < P; ++j) {
    double tau;
    int64_t lo = 0, hi = P;
    if (kind == OR_RESAMPLE_STRATIFIED) {
      uint32_t wd[4];
      or_block(seed, (uint32_t)j, i, OR_PURPOSE_RESAMPLE, 1u, wd);
      tau = ((double)j + or_u53_half_open(wd[0], wd[1])) * S / (double)P;
    } else {
      tau = (G[j] / GP) * S;
    }
    while (lo < hi) {
      int64_t mid = lo + (hi - lo) / 2;
      if (Cbuf[mid] > tau) hi = mid;
      else lo = mid + 1;
    }
    k = lo < P ? lo : P - 1;
    anc[j] = (int32_t)k;
    if (fabs(tau - Cbuf[k]) <= 1e-12 * S || (k > 0 && fabs(tau - Cbuf[k - 1]) <= 1e-12 * S))
      ++near;
  }
  free(G);
  return near;
}

int64_t or_resample(const double *ell, int64_t P, int32_t kind, uint64_t seed, uint32_t i,
                    int32_t *anc) {
  double M, S, Q;
  double *w = (double *)malloc(sizeof(double) * (size_t)P);
  double *C = (double *)malloc(sizeof(double) * (size_t)P);
  int64_t j, near;
  or_lse(ell, P, &M, &S, &Q);
  for (j = 0; j < P; ++j) w[j] = exp(ell[j] - M);
  if (kind == OR_RESAMPLE_SYSTEMATIC)
    near = or_systematic_from_w(w, P, or_resample_uniform(seed, i), anc, C);
  else
    near = or_resample_other(w, P, kind, seed, i, anc, C);
  free(w);
  free(C);
  return near;
}

int64_t or_systematic(const double *ell, int64_t P, double u, int32_t *anc) {
  double M, S, Q;
  double *w = (double *)malloc(sizeof(double) * (size_t)P);
  double *C = (double *)malloc(sizeof(double) * (size_t)P);
  int64_t j, near;
  or_lse(ell, P, &M, &S, &Q);
  for (j = 0; j < P; ++j) w[j] = exp(ell[j] - M);
  near = or_systematic_from_w(w, P, u, anc, C);
  free(w);
  free(C);
  return near;
}

/* ======================================================================
 * Propagation and weighting of one particle (Algorithm 2, propagate and
 * weight lines).  xin / xout: the particle's N components.
 * ==================================================================== */
typedef struct {
  const or_model *m;
  const double *th;
  const double *flow;
  uint64_t seed;
  int32_t Ny;
  double r;
} or_ctx;

/* FP64 path. */
static double or_prop_weight64(const or_ctx *cx, uint32_t j, int32_t i, double *x, double *tmp,
                               const double *yi) {
  const or_model *m = cx->m;
  const int32_t N = m->N, s = m->substeps;
  double acc = 0.0;
  int32_t n, mm;
  if (m->kind == OR_WINDKESSEL) {
    const double R = cx->th[0], C = cx->th[1], Z = cx->th[2], sq = sqrt(cx->th[3]);
    double xv = x[0], h, d;
    for (mm = 0; mm < s; ++mm) {
      double Fk = cx->flow[(int64_t)(i - 1) * s + mm];
      double drift = Fk / C - xv / (R * C);
      double z = or_normal64(cx->seed, j, (uint32_t)i, OR_PURPOSE_PROP, (uint32_t)mm);  /* normal number mm */
      xv = fma(m->dt, drift, xv);
      xv = fma(sq, z, xv);
    }
    x[0] = xv;
    h = fma(Z, cx->flow[(int64_t)i * s], xv);
    d = yi[0] - h;
    acc = fma(d, d, acc);
  } else if (m->kind == OR_WINDKESSEL_EXP) {
    /* the paper's transition: x <- a x + R (1 - a) (F_k + xi), a = exp(-dt/(RC)),
     * xi ~ N(0, (dt sqrt(sigma2))^2), normal number mm of stream (j, i, PROP) */
    const double R = cx->th[0], C = cx->th[1], Z = cx->th[2];
    const double a = or_exp(-(m->dt / (R * C)));
    const double b = R * (1.0 - a);
    const double sd = m->dt * sqrt(cx->th[3]);
    double xv = x[0], h, d;
    for (mm = 0; mm < s; ++mm) {
      double Fk = cx->flow[(int64_t)(i - 1) * s + mm];
      double z = or_normal64(cx->seed, j, (uint32_t)i, OR_PURPOSE_PROP, (uint32_t)mm);
      xv = fma(a, xv, b * fma(sd, z, Fk));
    }
    x[0] = xv;
    h = fma(Z, cx->flow[(int64_t)i * s], xv);
    d = yi[0] - h;
    acc = fma(d, d, acc);
  } else if (m->kind == OR_LORENZ96_SDE) {
    /* the paper's form: RK4 substep mm with forcing F + sqrt(sigma2) dW_n / dt,
     * dW_n = sqrt(dt) z, z = normal number mm N + n of stream (j, i, PROP) */
    const double F = cx->th[0], sw = sqrt(cx->th[1] / m->dt);
    double Fv[256];
    for (mm = 0; mm < s; ++mm) {
      for (n = 0; n < N; ++n) {
        double z = or_normal64(cx->seed, j, (uint32_t)i, OR_PURPOSE_PROP, (uint32_t)(mm * N + n));
        Fv[n] = fma(sw, z, F);
      }
      or_l96_rk4_step_v(x, N, Fv, m->dt, tmp, tmp + N, tmp + 2 * N);
    }
    for (n = 0; n < N && n / m->obs_stride < cx->Ny; n += m->obs_stride) {
      double d = yi[n / m->obs_stride] - x[n];
      acc = fma(d, d, acc);
    }
  } else {
    const double F = cx->th[0], sx = sqrt(cx->th[1]);
    for (mm = 0; mm < s; ++mm) or_l96_rk4_step(x, N, F, m->dt, tmp, tmp + N, tmp + 2 * N);
    for (n = 0; n < N; ++n) {
      double z = or_normal64(cx->seed, j, (uint32_t)i, OR_PURPOSE_PROP, (uint32_t)n);
      x[n] = fma(sx, z, x[n]);
    }
    for (n = 0; n < N && n / m->obs_stride < cx->Ny; n += m->obs_stride) {
      double d = yi[n / m->obs_stride] - x[n];
      acc = fma(d, d, acc);
    }
  }
  return -0.5 * acc / cx->r;
}

/* Mixed path: FP32 state, RK4/Euler and noise; FP64 residuals and weight. */
static double or_prop_weight32(const or_ctx *cx, uint32_t j, int32_t i, float *x, float *tmp,
                               const double *yi) {
  const or_model *m = cx->m;
  const int32_t N = m->N, s = m->substeps;
  const float dtf = (float)m->dt;
  double acc = 0.0;
  int32_t n, mm;
  if (m->kind == OR_WINDKESSEL) {
    const float R = (float)cx->th[0], C = (float)cx->th[1];
    const float sq = sqrtf((float)cx->th[3]);
    const double Z = cx->th[2];
    float xv = x[0];
    double h, d;
    for (mm = 0; mm < s; ++mm) {
      float Fk = (float)cx->flow[(int64_t)(i - 1) * s + mm];
      float drift = Fk / C - xv / (R * C);
      float z = or_normal32(cx->seed, j, (uint32_t)i, OR_PURPOSE_PROP, (uint32_t)mm);  /* normal number mm */
      xv = fmaf(dtf, drift, xv);
      xv = fmaf(sq, z, xv);
    }
    x[0] = xv;
    h = fma(Z, cx->flow[(int64_t)i * s], (double)xv);
    d = yi[0] - h;
    acc = fma(d, d, acc);
  } else if (m->kind == OR_WINDKESSEL_EXP) {
    /* a, R (1 - a) and dt sqrt(sigma2) in FP64 (own exp), rounded to FP32 */
    const double R = cx->th[0], C = cx->th[1], Z = cx->th[2];
    const double a64 = or_exp(-(m->dt / (R * C)));
    const float a = (float)a64, b = (float)(R * (1.0 - a64));
    const float sd = (float)(m->dt * sqrt(cx->th[3]));
    float xv = x[0];
    double h, d;
    for (mm = 0; mm < s; ++mm) {
      float Fk = (float)cx->flow[(int64_t)(i - 1) * s + mm];
      float z = or_normal32(cx->seed, j, (uint32_t)i, OR_PURPOSE_PROP, (uint32_t)mm);
      xv = fmaf(a, xv, b * fmaf(sd, z, Fk));
    }
    x[0] = xv;
    h = fma(Z, cx->flow[(int64_t)i * s], (double)xv);
    d = yi[0] - h;
    acc = fma(d, d, acc);
  } else if (m->kind == OR_LORENZ96_SDE) {
    const float F = (float)cx->th[0], sw = sqrtf((float)cx->th[1] / dtf);
    float Fv[256];
    for (mm = 0; mm < s; ++mm) {
      for (n = 0; n < N; ++n) {
        float z = or_normal32(cx->seed, j, (uint32_t)i, OR_PURPOSE_PROP, (uint32_t)(mm * N + n));
        Fv[n] = fmaf(sw, z, F);
      }
      or_l96_rk4_step_vf(x, N, Fv, dtf, tmp, tmp + N, tmp + 2 * N);
    }
    for (n = 0; n < N && n / m->obs_stride < cx->Ny; n += m->obs_stride) {
      double d = yi[n / m->obs_stride] - (double)x[n];
      acc = fma(d, d, acc);
    }
  } else {
    const float F = (float)cx->th[0], sx = sqrtf((float)cx->th[1]);
    for (mm = 0; mm < s; ++mm) or_l96_rk4_stepf(x, N, F, dtf, tmp, tmp + N, tmp + 2 * N);
    for (n = 0; n < N; ++n) {
      float z = or_normal32(cx->seed, j, (uint32_t)i, OR_PURPOSE_PROP, (uint32_t)n);
      x[n] = fmaf(sx, z, x[n]);
    }
    for (n = 0; n < N && n / m->obs_stride < cx->Ny; n += m->obs_stride) {
      double d = yi[n / m->obs_stride] - (double)x[n];
      acc = fma(d, d, acc);
    }
  }
  return -0.5 * acc / cx->r;
}

/* ======================================================================
 * The filter (Algorithm 2 with r = 0, s = T).
 *   init:  x_n^j(t0) = m0 + s0 z (normal number n of stream (j, 0, INIT));
 *          windkessel substep mm of interval i uses normal number mm of
 *          stream (j, i, PROP); Lorenz '96 component n uses normal number n.
 *   carry: lam_j (log-weights carried from the last step) with
 *          L = log sum_j exp(lam_j); after resampling lam = 0, L = log P.
 *   step i: ell_j = lam_j + logw_j (non-finite -> -inf); M, S, Q;
 *          increment = (M + log S) - L + c_obs, c_obs = -Ny/2 log(2 pi r);
 *          ESS = S^2 / Q; if i < T and (thr >= 1 or ESS < thr P): systematic
 *          resampling with u = resample uniform of step i, lam = 0, L = log P;
 *          else (i < T): identity ancestors, lam_j = ell_j - M, L = log S.
 *   anc row i-1 holds the ancestors used to propagate into t_i (row 0 is the
 *   identity).
 * ==================================================================== */
int32_t or_pf_run(const or_model *m, const double *th, const double *y, uint64_t seed, int64_t P,
                  int32_t T, int32_t nthreads, double *loglik, double *xfinal, int32_t *anc,
                  double *diag) {
  return or_pf_run_ex(m, th, y, seed, P, T, nthreads, loglik, xfinal, anc, diag, NULL, NULL);
}

/* As or_pf_run, plus optionally the whole state history xhist [T+1][N][P]
 * (row i = x(t_i), row 0 the initial draw) and the final log-weights
 * ellT [P] (ell at t_T, including carried weights). */
int32_t or_pf_run_ex(const or_model *m, const double *th, const double *y, uint64_t seed,
                     int64_t P, int32_t T, int32_t nthreads, double *loglik, double *xfinal,
                     int32_t *anc, double *diag, double *xhist, double *ellT) {
  return or_pf_run_sched(m, th, y, seed, NULL, P, T, nthreads, loglik, xfinal, anc, diag, xhist,
                         ellT);
}

/* As or_pf_run_ex with a seed schedule: when sched is not NULL, the initial
 * draw uses the Philox key sched[0] and step i (its propagation, weights and
 * the resampling after it) uses sched[i], i = 1..T; this is the run that
 * advancing a filter interval by interval with a new key per interval
 * gives.  With sched NULL every draw uses seed. */
/* The state of one filter between observations: the particles x(t_{i-1})
 * (array a; b receives x(t_i)), the ancestors that propagate into t_i
 * (identity or acur), the carried log-weights lam with their normaliser L,
 * and the likelihood so far. */
typedef struct {
  const or_model *m;
  or_ctx cx;
  int64_t P;
  int32_t T, N, every, mixed;
  double c_obs;
  double *xa, *xb;   /* FP64 state, SoA [N][P] */
  float *fa, *fb;    /* FP32 state, SoA [N][P] */
  double *ell, *lam, *w, *Cbuf;
  int32_t *acur;
  double ll, L;
  int lam_zero, anc_identity;
} or_state;

/* Observation i (the loop body of Algorithm 2): propagate every particle from
 * its ancestor and weight it; then, at an observed step, the log-sum-exp,
 * the likelihood increment, the ESS test and the resampling (or the carry of
 * the weights).  dg[8] receives (M, S, Q, ESS, resampled, u, increment, near
 * targets).  Returns OR_OK, or OR_EDEGENERATE (ll set to -inf). */
static int32_t or_step(or_state *r, int32_t i, const double *yi, double *dg) {
  const int64_t P = r->P;
  const int32_t N = r->N;
  const int observed = (i % r->every) == 0;
  double M, S, Q, ess, incr, u = 0.0;
  int resample;
  int64_t j, near = 0;
  /* propagate and weight every particle from its ancestor */
#pragma omp parallel
  {
    double xloc[4 * 256];
    float floc[4 * 256];
#pragma omp for schedule(static)
    for (j = 0; j < P; ++j) {
      int64_t a = r->anc_identity ? j : (int64_t)r->acur[j];
      int32_t n;
      double lw, e;
      if (r->mixed) {
        for (n = 0; n < N; ++n) floc[n] = r->fa[(int64_t)n * P + a];
        lw = or_prop_weight32(&r->cx, (uint32_t)j, i, floc, floc + N, yi);
        for (n = 0; n < N; ++n) r->fb[(int64_t)n * P + j] = floc[n];
      } else {
        for (n = 0; n < N; ++n) xloc[n] = r->xa[(int64_t)n * P + a];
        lw = or_prop_weight64(&r->cx, (uint32_t)j, i, xloc, xloc + N, yi);
        for (n = 0; n < N; ++n) r->xb[(int64_t)n * P + j] = xloc[n];
      }
      if (!observed) lw = 0.0;
      e = r->lam_zero ? lw : r->lam[j] + lw;
      if (e != e) e = -INFINITY;
      r->ell[j] = e;
    }
  }
  if (r->mixed) { float *t = r->fa; r->fa = r->fb; r->fb = t; }
  else { double *t = r->xa; r->xa = r->xb; r->xb = t; }
  if (!observed) {
    /* a step without an observation only propagates: no weight, no
     * likelihood term, no resampling, carried weights unchanged */
    r->anc_identity = 1;
    if (dg) dg[0] = dg[1] = dg[2] = dg[3] = dg[4] = dg[5] = dg[6] = dg[7] = 0.0;
    return OR_OK;
  }
  or_lse(r->ell, P, &M, &S, &Q);
  if (!(M > -INFINITY) || !(S > 0.0) || M == INFINITY) {
    r->ll = -INFINITY;
    if (dg) {
      dg[0] = M; dg[1] = S; dg[2] = Q; dg[3] = 0.0; dg[4] = 0.0; dg[5] = 0.0;
      dg[6] = -INFINITY; dg[7] = 0.0;
    }
    return OR_EDEGENERATE;
  }
  incr = ((M + log(S)) - r->L) + r->c_obs;
  r->ll += incr;
  ess = (S * S) / Q;
  resample = (i < r->T) && (r->m->ess_threshold >= 1.0 || ess < r->m->ess_threshold * (double)P);
  if (resample) {
    for (j = 0; j < P; ++j) r->w[j] = exp(r->ell[j] - M);
    if (r->m->resampler == OR_RESAMPLE_SYSTEMATIC) {
      u = or_resample_uniform(r->cx.seed, (uint32_t)i);
      near = or_systematic_from_w(r->w, P, u, r->acur, r->Cbuf);
    } else {
      near = or_resample_other(r->w, P, r->m->resampler, r->cx.seed, (uint32_t)i, r->acur,
                               r->Cbuf);
    }
    r->anc_identity = 0;
    r->lam_zero = 1;
    r->L = log((double)P);
  } else if (i < r->T) {
    for (j = 0; j < P; ++j) r->lam[j] = r->ell[j] - M;
    r->anc_identity = 1;
    r->lam_zero = 0;
    r->L = log(S);
  }
  if (dg) {
    dg[0] = M; dg[1] = S; dg[2] = Q; dg[3] = ess; dg[4] = resample ? 1.0 : 0.0;
    dg[5] = u; dg[6] = incr; dg[7] = (double)near;
  }
  return OR_OK;
}

/* Shape checks, buffers and constants of a filter state (x0 not drawn). */
static int32_t or_state_open(or_state *r, const or_model *m, const double *th, uint64_t seed,
                             int64_t P, int32_t T, int32_t nthreads) {
  const int32_t N = m->N, s = m->substeps;
  const int32_t stride = OR_IS_L96(m->kind) ? m->obs_stride : 1;
  const int32_t Nys = OR_IS_L96(m->kind) ? (N + stride - 1) / stride : 1;
  const int32_t Ny = (OR_IS_L96(m->kind) && m->obs_count > 0 && m->obs_count < Nys)
                         ? m->obs_count : Nys;
  const double rv = OR_IS_L96(m->kind) ? th[2] : th[4];
  double *flow = NULL;
  memset(r, 0, sizeof *r);
  if (P <= 0 || T <= 0 || N <= 0 || s <= 0) return OR_EINVAL;
  if (m->kind < OR_WINDKESSEL || m->kind > OR_LORENZ96_SDE) return OR_EINVAL;
  if (OR_IS_WK(m->kind) && N != 1) return OR_EINVAL;
  if (OR_IS_L96(m->kind) && (N < 4 || N > 256 || stride <= 0)) return OR_EINVAL;
  if (m->resampler < OR_RESAMPLE_SYSTEMATIC || m->resampler > OR_RESAMPLE_MULTINOMIAL)
    return OR_EINVAL;
  if (m->obs_every < 0 || m->obs_count < 0) return OR_EINVAL;
#ifdef _OPENMP
  /* 0 means every core this process may run on; set either way, so that an
     earlier call's count does not carry over */
  omp_set_num_threads(nthreads > 0 ? nthreads : omp_get_num_procs());
#else
  (void)nthreads;
#endif
  if (OR_IS_WK(m->kind)) {
    flow = (double *)malloc(sizeof(double) * (size_t)((int64_t)T * s + 1));
    or_flow_table(m->flow_peak, m->flow_period, m->dt, (int64_t)T * s + 1, flow);
  }
  r->m = m;
  r->P = P;
  r->T = T;
  r->N = N;
  r->every = m->obs_every > 1 ? m->obs_every : 1;
  r->mixed = (m->prec == OR_MIXED);
  r->c_obs = -0.5 * (double)Ny * log(2.0 * M_PI * rv);
  if (r->mixed) {
    r->fa = (float *)malloc(sizeof(float) * (size_t)(N * P));
    r->fb = (float *)malloc(sizeof(float) * (size_t)(N * P));
  } else {
    r->xa = (double *)malloc(sizeof(double) * (size_t)(N * P));
    r->xb = (double *)malloc(sizeof(double) * (size_t)(N * P));
  }
  r->ell = (double *)malloc(sizeof(double) * (size_t)P);
  r->lam = (double *)malloc(sizeof(double) * (size_t)P);
  r->w = (double *)malloc(sizeof(double) * (size_t)P);
  r->Cbuf = (double *)malloc(sizeof(double) * (size_t)P);
  r->acur = (int32_t *)malloc(sizeof(int32_t) * (size_t)P);
  r->cx.m = m;
  r->cx.th = th;
  r->cx.flow = flow;
  r->cx.seed = seed;
  r->cx.Ny = Ny;
  r->cx.r = rv;
  r->ll = 0.0;
  r->L = log((double)P);
  r->lam_zero = 1;
  r->anc_identity = 1;
  return OR_OK;
}

static void or_state_close(or_state *r) {
  free((void *)r->cx.flow);
  free(r->xa); free(r->xb); free(r->fa); free(r->fb);
  free(r->ell); free(r->lam); free(r->w); free(r->Cbuf); free(r->acur);
}

/* Particle j's component n of the current state, as a double. */
static double or_state_x(const or_state *r, int64_t k) {
  return r->mixed ? (double)r->fa[k] : r->xa[k];
}

int32_t or_pf_run_sched(const or_model *m, const double *th, const double *y, uint64_t seed,
                        const uint64_t *sched, int64_t P, int32_t T, int32_t nthreads,
                        double *loglik, double *xfinal, int32_t *anc, double *diag,
                        double *xhist, double *ellT) {
  const double m0 = OR_IS_L96(m->kind) ? th[3] : th[5];
  const double s0 = OR_IS_L96(m->kind) ? th[4] : th[6];
  or_state r;
  int32_t i, status = OR_OK;
  int64_t j;
  int32_t st = or_state_open(&r, m, th, sched ? sched[0] : seed, P, T, nthreads);
  if (st != OR_OK) {
    or_state_close(&r);
    return st;
  }
  {
    const int32_t N = r.N;
    const uint64_t key0 = r.cx.seed;
    /* initialisation (Algorithm 2, init lines) */
#pragma omp parallel for schedule(static)
    for (j = 0; j < P; ++j) {
      int32_t n;
      for (n = 0; n < N; ++n) {
        if (r.mixed) {
          float z = or_normal32(key0, (uint32_t)j, 0u, OR_PURPOSE_INIT, (uint32_t)n);
          r.fa[(int64_t)n * P + j] = fmaf((float)s0, z, (float)m0);
        } else {
          double z = or_normal64(key0, (uint32_t)j, 0u, OR_PURPOSE_INIT, (uint32_t)n);
          r.xa[(int64_t)n * P + j] = fma(s0, z, m0);
        }
      }
    }
  }
  if (xhist) {
    for (j = 0; j < (int64_t)r.N * P; ++j) xhist[j] = or_state_x(&r, j);
  }
  for (i = 1; i <= T; ++i) {
    if (sched) r.cx.seed = sched[i];
    if (anc) {
      for (j = 0; j < P; ++j)
        anc[(int64_t)(i - 1) * P + j] = r.anc_identity ? (int32_t)j : r.acur[j];
    }
    status = or_step(&r, i, y + (int64_t)(i - 1) * r.cx.Ny,
                     diag ? diag + (int64_t)(i - 1) * 8 : NULL);
    if (xhist) {
      double *xr = xhist + (int64_t)i * r.N * P;
      for (j = 0; j < (int64_t)r.N * P; ++j) xr[j] = or_state_x(&r, j);
    }
    if (ellT && i == T) memcpy(ellT, r.ell, sizeof(double) * (size_t)P);
    if (status != OR_OK) break;
  }
  *loglik = r.ll;
  if (xfinal && status == OR_OK) {
    for (j = 0; j < (int64_t)r.N * P; ++j) xfinal[j] = or_state_x(&r, j);
  }
  or_state_close(&r);
  return status;
}

/* Teacher-forced step: observation i of Algorithm 2 from a given state --
 * x(t_{i-1}) in x_prev [N][P] (values of the state precision), the ancestors
 * a(t_i) in anc [P] (NULL: identity), carried log-weights zero (as after a
 * resampling) -- by the same step function the whole run uses.  Outputs
 * x(t_i) in x_next [N][P], the likelihood increment in *incr, the ancestors
 * of step i + 1 in anc_next [P] (the identity when step i carried its
 * weights; untouched for i = T) and the step's diagnostics in diag[8]. */
int32_t or_pf_step(const or_model *m, const double *th, const double *y, uint64_t seed,
                   int64_t P, int32_t T, int32_t i, int32_t nthreads, const double *x_prev,
                   const int32_t *anc, double *x_next, double *incr, int32_t *anc_next,
                   double *diag) {
  or_state r;
  int64_t j;
  int32_t st;
  if (i < 1 || i > T) return OR_EINVAL;
  st = or_state_open(&r, m, th, seed, P, T, nthreads);
  if (st != OR_OK) {
    or_state_close(&r);
    return st;
  }
  for (j = 0; j < (int64_t)r.N * P; ++j) {
    if (r.mixed) r.fa[j] = (float)x_prev[j];
    else r.xa[j] = x_prev[j];
  }
  if (anc) {
    memcpy(r.acur, anc, sizeof(int32_t) * (size_t)P);
    r.anc_identity = 0;
  }
  st = or_step(&r, i, y + (int64_t)(i - 1) * r.cx.Ny, diag);
  if (incr) *incr = r.ll;
  if (x_next) {
    for (j = 0; j < (int64_t)r.N * P; ++j) x_next[j] = or_state_x(&r, j);
  }
  if (anc_next && st == OR_OK && i < T) {
    for (j = 0; j < P; ++j) anc_next[j] = r.anc_identity ? (int32_t)j : r.acur[j];
  }
  or_state_close(&r);
  return st;
}

/* ======================================================================
 * Single state path (the last lines of Algorithm 2): draw one particle j
 * from the final weights, j = min{k : C_k > v S} with v the path uniform of
 * the run (block (0, T + 1, PATH, 0), 53 bits), C_k the compensated prefix
 * of exp(ell_T - M) and S = C_{P-1}; then follow the ancestors back:
 * b_T = j, b_{i-1} = a(t_i)[b_i], and return x(t_i) of particle b_i.
 * path [T+1][N], idx [T+1].  Returns the filter's status.
 * ==================================================================== */
int32_t or_sample_path(const or_model *m, const double *th, const double *y, uint64_t seed,
                       int64_t P, int32_t T, int32_t nthreads, double *loglik, double *path,
                       int32_t *idx) {
  const int32_t N = m->N;
  double *xhist = (double *)malloc(sizeof(double) * (size_t)(T + 1) * (size_t)N * (size_t)P);
  int32_t *anc = (int32_t *)malloc(sizeof(int32_t) * (size_t)T * (size_t)P);
  double *ellT = (double *)malloc(sizeof(double) * (size_t)P);
  double *C = (double *)malloc(sizeof(double) * (size_t)P);
  int32_t status = or_pf_run_ex(m, th, y, seed, P, T, nthreads, loglik, NULL, anc, NULL, xhist,
                                ellT);
  if (status == OR_OK) {
    double M = -INFINITY, sum = 0.0, comp = 0.0, v, vS;
    int64_t k, j, lo, hi;
    int32_t i, n;
    uint32_t w[4];
    for (k = 0; k < P; ++k)
      if (ellT[k] > M) M = ellT[k];
    for (k = 0; k < P; ++k) {
      or_neumaier_add(&sum, &comp, exp(ellT[k] - M));
      C[k] = sum + comp;
    }
    or_block(seed, 0u, (uint32_t)(T + 1), OR_PURPOSE_PATH, 0u, w);
    v = or_u53_half_open(w[0], w[1]);
    vS = v * C[P - 1];
    lo = 0;
    hi = P;
    while (lo < hi) {
      int64_t mid = lo + (hi - lo) / 2;
      if (C[mid] > vS) hi = mid;
      else lo = mid + 1;
    }
    j = lo < P ? lo : P - 1;
    for (i = T; i >= 0; --i) {
      idx[i] = (int32_t)j;
      for (n = 0; n < N; ++n) path[(int64_t)i * N + n] = xhist[((int64_t)i * N + n) * P + j];
      if (i > 0) j = anc[(int64_t)(i - 1) * P + j];
    }
  }
  free(xhist); free(anc); free(ellT); free(C);
  return status;
}
