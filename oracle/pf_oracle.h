/*
 * pf_oracle.h -- plain, slow CPU oracle for the bootstrap particle filter of
 * Murray, "Bayesian State-Space Modelling on High-Performance Hardware Using
 * LibBi" (arXiv 1306.3277), Algorithm 2 (Sec. 3.1.2), with systematic
 * resampling (Sec. 3.3) and an effective-sample-size test.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may include, link or
 * call this library: only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark do.  It shares no code with the CUDA implementation.
 *
 * Every arithmetic convention (operation order, explicit fma, own log and
 * sincos for Box-Muller, Philox counter layout) is stated next to the code
 * that implements it, so that the CUDA side can be written independently to
 * the same definitions and compared bit for bit.
 *
 * Every function here is pinned by a -m "not gpu" test against something
 * other than itself (published known answers, libm, closed forms, a Kalman
 * filter, brute-force enumeration); the list is in oracle/__init__.py.
 */
#ifndef PF_ORACLE_H
#define PF_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Model kinds: the windkessel with Euler substeps and additive state noise,
 * Lorenz '96 with additive noise once per observation, and the paper-exact
 * forms of both: the windkessel's exponential decay with noise on the flow,
 * and Lorenz '96 with a Wiener increment inside every RK4 substep. */
enum { OR_WINDKESSEL = 0, OR_LORENZ96 = 1, OR_WINDKESSEL_EXP = 2, OR_LORENZ96_SDE = 3 };
#define OR_IS_WK(kind) ((kind) == OR_WINDKESSEL || (kind) == OR_WINDKESSEL_EXP)
#define OR_IS_L96(kind) ((kind) == OR_LORENZ96 || (kind) == OR_LORENZ96_SDE)
enum { OR_FP64 = 0, OR_MIXED = 1 };
enum { OR_OK = 0, OR_EINVAL = 1, OR_EDEGENERATE = 4 };
enum { OR_RESAMPLE_SYSTEMATIC = 0, OR_RESAMPLE_STRATIFIED = 1, OR_RESAMPLE_MULTINOMIAL = 2 };
/* Philox counter word 2 carries (purpose << 16) | block index. */
enum { OR_PURPOSE_INIT = 1, OR_PURPOSE_PROP = 2, OR_PURPOSE_RESAMPLE = 3, OR_PURPOSE_PATH = 4,
       OR_PURPOSE_PMMH = 5, OR_PURPOSE_SMC2 = 6 };

typedef struct {
  int32_t kind;          /* OR_WINDKESSEL or OR_LORENZ96 */
  int32_t N;             /* state dimension (1 for the windkessel) */
  int32_t substeps;      /* Euler / RK4 substeps per observation interval */
  int32_t obs_stride;    /* Lorenz '96: components n with n % obs_stride == 0 are observed */
  int32_t prec;          /* OR_FP64 or OR_MIXED (FP32 state and noise, FP64 weights) */
  int32_t resampler;     /* OR_RESAMPLE_SYSTEMATIC / _STRATIFIED / _MULTINOMIAL */
  double dt;             /* substep length */
  double ess_threshold;  /* >= 1: resample every step; else resample iff ESS < thr * P */
  double flow_peak;      /* windkessel input F(t): peak of the half sine */
  double flow_period;    /* windkessel input F(t): period */
  int32_t obs_every;     /* 0 or 1: every step observed; k: only steps i with i % k == 0 */
  int32_t obs_count;     /* Lorenz '96: 0 = every strided component; else the first
                            obs_count of them (sparse observations) */
} or_model;

/* --- random numbers ---------------------------------------------------- */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* Philox block of counter (j, i, (purpose << 16) | blk, 0), key = seed halves */
void or_block(uint64_t seed, uint32_t j, uint32_t i, uint32_t purpose, uint32_t blk,
              uint32_t w[4]);
/* 53-bit uniforms from the 64-bit word (hi:lo): [0, 1) and (0, 1] */
double or_u53_half_open(uint32_t lo, uint32_t hi);
double or_u53_open_zero(uint32_t lo, uint32_t hi);
/* normal number q of the stream (j, i, purpose), FP64 (2 normals per block) */
double or_normal64(uint64_t seed, uint32_t j, uint32_t i, uint32_t purpose, uint32_t q);
/* normal number q of the stream (j, i, purpose), FP32 (4 normals per block) */
float or_normal32(uint64_t seed, uint32_t j, uint32_t i, uint32_t purpose, uint32_t q);
double or_resample_uniform(uint64_t seed, uint32_t i);
void or_fill_normals(uint64_t seed, int32_t prec, uint32_t i, uint32_t purpose, uint32_t nj,
                     uint32_t nq, double *out);

/* --- project-written elementary functions ----------------------------- */
double or_log(double x);
double or_exp(double x);
void or_sincos2pi(double u, double *s, double *c);
float or_logf(float x);
void or_sincos2pif(float u, float *s, float *c);

/* --- model pieces ------------------------------------------------------- */
void or_flow_table(double peak, double period, double dt, int64_t n, double *out);
/* deterministic Lorenz '96 RK4, nsteps steps of dt, in place (FP64) */
void or_l96_rk4(double *x, int32_t N, double F, double dt, int32_t nsteps);
void or_l96_rk4f(float *x, int32_t N, float F, float dt, int32_t nsteps);
/* scalar Kalman filter for the Euler-discretised windkessel */
double or_kalman_windkessel(const or_model *m, const double *theta, const double *y, int32_t T);

/* --- resampling pieces -------------------------------------------------- */
void or_lse(const double *ell, int64_t P, double *M, double *S, double *Q);
/* systematic resampling from log-weights; returns the number of
 * near-boundary targets (|E_k - j| <= 1e-12 P, E_k = C_k P / S - u) */
int64_t or_systematic(const double *ell, int64_t P, double u, int32_t *anc);
/* resampling of step i with any of the three schemes (systematic uses the
 * uniform of or_resample_uniform); returns the near-boundary count */
int64_t or_resample(const double *ell, int64_t P, int32_t kind, uint64_t seed, uint32_t i,
                    int32_t *anc);

/* --- the filter --------------------------------------------------------- */
/* diag, if not NULL, receives per step i (row i-1) 8 doubles:
 * M, S, Q, ESS, resampled (0/1), u, log-likelihood increment, near-boundary count */
int32_t or_pf_run(const or_model *m, const double *theta, const double *y, uint64_t seed,
                  int64_t P, int32_t T, int32_t nthreads, double *loglik,
                  double *xfinal, int32_t *anc, double *diag);

int32_t or_pf_run_ex(const or_model *m, const double *theta, const double *y, uint64_t seed,
                     int64_t P, int32_t T, int32_t nthreads, double *loglik, double *xfinal,
                     int32_t *anc, double *diag, double *xhist, double *ellT);
int32_t or_pf_run_sched(const or_model *m, const double *theta, const double *y, uint64_t seed,
                        const uint64_t *sched, int64_t P, int32_t T, int32_t nthreads,
                        double *loglik, double *xfinal, int32_t *anc, double *diag,
                        double *xhist, double *ellT);
/* teacher-forced step i from x(t_{i-1}) = x_prev [N][P] and a(t_i) = anc [P]
 * (NULL: identity), carried log-weights zero: x_next [N][P] = x(t_i), *incr =
 * log Z_i, anc_next [P] = a(t_{i+1}) (i < T), diag [8] as above */
int32_t or_pf_step(const or_model *m, const double *theta, const double *y, uint64_t seed,
                   int64_t P, int32_t T, int32_t i, int32_t nthreads, const double *x_prev,
                   const int32_t *anc, double *x_next, double *incr, int32_t *anc_next,
                   double *diag);
/* one state path by ancestry (end of Algorithm 2); path [T+1][N], idx [T+1] */
int32_t or_sample_path(const or_model *m, const double *theta, const double *y, uint64_t seed,
                       int64_t P, int32_t T, int32_t nthreads, double *loglik, double *path,
                       int32_t *idx);

/* --- marginal Metropolis-Hastings (Algorithm 3, Eq. mh) ---------------- */
enum { OR_PRIOR_FIXED = 0, OR_PRIOR_UNIFORM = 1, OR_PRIOR_GAUSSIAN = 2, OR_PRIOR_GAMMA = 3,
       OR_PRIOR_INV_GAMMA = 4 };
enum { OR_PROPOSE_FIXED = 0, OR_PROPOSE_TRUNC_GAUSSIAN = 1, OR_PROPOSE_INV_GAMMA = 2 };
enum { OR_LIK_PF = 0, OR_LIK_KALMAN = 1, OR_LIK_NONE = 2 };

typedef struct {
  int32_t prior;      /* OR_PRIOR_*: uniform (a, b); gaussian (mean a, sd b);
                         gamma (shape a, scale b); inverse gamma (shape a, scale b) */
  int32_t proposal;   /* OR_PROPOSE_*: truncated gaussian around the current value
                         (sd c, bounds [d, e]); inverse gamma (integer shape c,
                         scale d * current value) */
  double a, b, c, d, e;
} or_param;

double or_log_prior(const or_param *spec, int32_t nth, const double *theta);
/* One proposal theta' ~ q(. | theta) of chain j at iteration i (Philox key
 * seed); returns log q(theta | theta') - log q(theta' | theta). */
double or_propose(const or_param *spec, int32_t nth, const double *theta, uint64_t seed,
                  uint32_t j, uint32_t i, double *theta_new);
/* nchains independent chains of niter iterations; samples [niter+1][nchains][nth],
 * logliks [niter+1][nchains], accepted [nchains], near [niter+1][nchains]. */
int32_t or_pmmh(const or_model *m, const double *y, int64_t P, int32_t T, int32_t lik,
                int32_t nchains, const or_param *spec, const double *theta0, int32_t niter,
                uint64_t seed, int32_t nthreads, double *samples, double *logliks,
                int32_t *accepted, int32_t *near);

/* --- SMC^2 (Algorithm 4) ---------------------------------------------- */
/* ntheta parameter particles; base supplies the components whose prior is
 * OR_PRIOR_FIXED.  Outputs: theta_out [ntheta][nth], logv_out [ntheta] (the
 * last step's log theta-weights), log_evidence, incr [T] (per-step log
 * evidence increments), accepted [T] (rejuvenation moves accepted), near [T]. */
int32_t or_smc2(const or_model *m, const double *y, int64_t P, int32_t T, int32_t lik,
                int32_t ntheta, const or_param *spec, const double *base, uint64_t seed,
                int32_t nthreads, double *theta_out, double *logv_out, double *log_evidence,
                double *incr, int32_t *accepted, int32_t *near);

#ifdef __cplusplus
}
#endif
#endif
