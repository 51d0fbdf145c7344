/*
 * pf.h -- C ABI of the B300 (sm_103a) bootstrap particle filter.
 *
 * The operation is the bootstrap particle filter of Murray, "Bayesian
 * State-Space Modelling on High-Performance Hardware Using LibBi"
 * (arXiv 1306.3277), Algorithm 2 (Sec. 3.1.2): for given parameters theta it
 * returns an estimate of the log marginal likelihood log p(y(t_1:T) | theta)
 * (the likelihood line of Algorithm 2, accumulated in log space), the final
 * particle cloud and the ancestor indices.  Resampling is systematic
 * (Sec. 3.3, one uniform per step, sorted ancestors) and is skipped on steps
 * whose effective sample size is at or above ess_threshold * P.
 *
 * Models (Sec. 2.1):
 *   PF_WINDKESSEL (Sec. 2.1.1), N = 1, theta = (R, C, Z, q, r, m0, s0):
 *     per substep x <- x + dt (F(t_k)/C - x/(R C)) + N(0, q), F held over
 *     [t_k, t_k + dt); observation y_i ~ N(x + Z F(t_i), r); x0 ~ N(m0, s0^2).
 *     F(t) = flow_peak sin(2 pi t / flow_period) on the first half of each
 *     period, else 0 (Eq. flow read as a half sine).
 *   PF_LORENZ96 (Sec. 2.1.2, Eq. lorenz96-ode), N in {4, 8, 12, 16, 20, 24,
 *     32, 40}, theta = (F, q, r, m0, s0): `substeps` classic RK4 steps of dt,
 *     then x_n += N(0, q) for every n; observation y ~ N(x_n, r) for every
 *     n with n % obs_stride == 0 (Ny = ceil(N / obs_stride));
 *     x0_n ~ N(m0, s0^2).
 *   Observation i is at t_i = i * substeps * dt, i = 1..T.
 *
 * Precision: PF_FP64 computes everything in FP64.  PF_MIXED keeps the state,
 * the integrator and the process noise in FP32 and the observation
 * log-weights, log-sum-exp, cumulative-weight scan and likelihood in FP64.
 * In both, the weight exponential exp(ell - M) is evaluated on the FP32 unit
 * in double-float arithmetic to about 2^-52 relative (pf_weight_exp).  A
 * tile's cumulative weights are, for the windkessel and Lorenz '96 with
 * N <= 12, exact sums in 2^-55 fixed point, each rounded once to FP64
 * (pf_weight_prefix), and for Lorenz '96 with N >= 16 sums in a fixed tree of
 * FP64 additions (a few ulp).
 *
 * Random numbers: Philox4x32-10 keyed by the 64-bit seed, counter
 * (particle, step, purpose << 16 | block, 0), Box-Muller normals.  A run is a
 * pure function of (filter configuration, theta, y, seed): the same call on
 * any B300 returns the same bits, alone or inside a batch.
 *
 * Errors: every entry point returns a pf_status; on anything but PF_OK (and
 * PF_EDEGENERATE, see pf_run) outputs are left untouched, and
 * pf_last_error() returns a message for the calling thread.  Calls on one
 * pf_filter must not overlap; different filters may be used from different
 * host threads.
 */
#ifndef PF_B300_H
#define PF_B300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PF_OK = 0,
  PF_EINVAL = 1,       /* bad argument (message in pf_last_error)            */
  PF_ENOMEM = 2,       /* device allocation failed / over the memory budget  */
  PF_ECUDA = 3,        /* a CUDA runtime call failed                         */
  PF_EDEGENERATE = 4,  /* every particle weight was zero or not a number     */
  PF_ETIMEOUT = 5,     /* a bounded wait ran out (the persistent batch launch) */
  PF_EBUSY = 6         /* result not ready / no capacity right now           */
} pf_status;

/* Model kinds (Sec. 2.1).  theta layouts:
 *   PF_WINDKESSEL, PF_WINDKESSEL_EXP: (R, C, Z, q, r, m0, s0)
 *   PF_LORENZ96, PF_LORENZ96_SDE:     (F, q, r, m0, s0)
 * r is the observation variance, (m0, s0) the initial mean and standard
 * deviation.  PF_WINDKESSEL takes Euler substeps x += dt (F/C - x/(RC)) plus
 * N(0, q) per substep; PF_WINDKESSEL_EXP is the paper's transition
 * x <- a x + R (1 - a) (F + xi), a = exp(-dt/(RC)), xi ~ N(0, (dt sqrt(q))^2)
 * (q the flow-noise variance sigma2).  PF_LORENZ96 adds N(0, q) to every
 * component once per observation after the RK4 substeps; PF_LORENZ96_SDE is
 * the paper's form, each RK4 substep of length dt carrying the forcing
 * F + sqrt(q) dW_n / dt with dW_n ~ N(0, dt) held over the substep. */
typedef enum {
  PF_WINDKESSEL = 0,
  PF_LORENZ96 = 1,
  PF_WINDKESSEL_EXP = 2,
  PF_LORENZ96_SDE = 3
} pf_model_kind;
typedef enum { PF_FP64 = 0, PF_MIXED = 1 } pf_precision;
/* Resampling scheme (Sec. 3.3; Algorithm 2 writes the multinomial draw).  All
 * three give sorted ancestors: target j sits at (j + u) S / P with one u per
 * step (systematic), at (j + u_j) S / P with one u_j per target (stratified),
 * or at the j-th order statistic of P uniforms, built from P + 1 exponential
 * spacings (multinomial).  The multinomial scheme adds one scan of the
 * spacings per step; the request server and pf_run_noalloc do not take it. */
typedef enum {
  PF_RESAMPLE_SYSTEMATIC = 0,
  PF_RESAMPLE_STRATIFIED = 1,
  PF_RESAMPLE_MULTINOMIAL = 2
} pf_resampler;

typedef struct {
  int32_t kind;          /* pf_model_kind                                       */
  int32_t N;             /* state dimension: 1 (windkessel) or a supported L96 N */
  int32_t substeps;      /* integrator substeps per observation interval, >= 1  */
  int32_t obs_stride;    /* Lorenz '96: observe n % obs_stride == 0, >= 1        */
  int32_t prec;          /* pf_precision                                        */
  int32_t resampler;     /* pf_resampler (0: systematic)                          */
  double ess_threshold;  /* >= 1: resample after every observation but the last;
                            in (0, 1): resample iff ESS < ess_threshold * P;
                            0: never resample                                  */
  double flow_peak;      /* windkessel input: peak of the half-sine flow        */
  double flow_period;    /* windkessel input: period of the flow, > 0           */
  int32_t obs_every;     /* 0 or 1: every step is observed; k > 1: only steps i
                            with i % k == 0 (sparse observations: the other
                            steps only propagate; their rows of y are unused) */
  int32_t obs_count;     /* Lorenz '96: 0 = every strided component observed;
                            else only the first obs_count of them (Ny)       */
} pf_model;

typedef struct pf_filter pf_filter;

/* Number of theta entries for a model kind (7 windkessel, 5 Lorenz '96), or 0. */
int32_t pf_theta_size(int32_t kind);

/* Create a filter for P particles (1 <= P <= 2^24) and T observations (T >= 1)
 * with substep dt > 0, on the current CUDA device.  Allocates every device
 * buffer the run needs (state double buffer, weights, ancestors, partials);
 * the library owns them until pf_destroy.  *out is set only on PF_OK. */
pf_status pf_create(const pf_model* m, int64_t P, int32_t T, double dt, pf_filter** out);

/* Bytes of device memory a filter of this shape holds (ancestor history
 * included when `history` is non-zero); 0 on invalid arguments. */
size_t pf_device_bytes(const pf_model* m, int64_t P, int32_t T, int32_t history);

#define PF_FLAG_ASYNC 1u  /* enqueue only: do not wait for the stream; outputs must be
                             device pointers, read the status later with pf_wait */

/* Run the filter over y(t_1..t_T) (Algorithm 2 with r = 0, s = T).
 *   theta            [pf_theta_size(kind)] doubles, host or device memory.
 *   y                [T][Ny] doubles, row i-1 = y(t_i), host or device memory.
 *   seed             64-bit Philox key.
 *   loglik           out: 1 double, log of the likelihood estimate, host or device.
 *   final_particles  out or NULL: [N][P] (component-major) x(t_T), in the
 *                    state precision (double for PF_FP64, float for PF_MIXED).
 *   ancestors        out or NULL: [T][P] int32, row i-1 = a(t_i), the ancestor
 *                    indices used to propagate into t_i (row 0 is the identity;
 *                    rows of steps that did not resample are the identity).
 *   flags            0 or PF_FLAG_ASYNC.
 *   cuda_stream      cudaStream_t to run on, or NULL for the filter's own stream.
 * All work runs on the GPU as one CUDA-graph launch; the inputs are copied to
 * the filter's buffers first, so they may be reused when the call returns
 * (host inputs) or when the stream passes this point (device inputs).
 * Returns PF_EDEGENERATE (and loglik = -inf) if at some step every weight was
 * zero or not a number; the other outputs are then undefined. */
pf_status pf_run(pf_filter* f, const double* theta, const double* y, uint64_t seed,
                 double* loglik, void* final_particles, int32_t* ancestors, uint32_t flags,
                 void* cuda_stream);

/* Algorithm 2 over an interval t_{r:s}: advance the filter from t_r to t_s.
 * r = 0 starts a new run (initial draw from theta); r > 0 must be the s of
 * the previous pf_run_range call on this filter, with no other run of it
 * (pf_run, pf_batch_run, pf_sample_path) in between, else PF_EINVAL.
 * Resampling after step i happens only for i < T, so splitting (0, T] into
 * consecutive intervals gives the same bits as one pf_run.
 *   theta      used when r = 0 (may be NULL when r > 0), host or device.
 *   y          [s-r][Ny] doubles: y(t_{r+1}) .. y(t_s), host or device, so
 *              observations can arrive interval by interval.
 *   seed       Philox key of this interval's steps (and of the initial draw
 *              when r = 0); the same key in every interval reproduces pf_run,
 *              a new key continues the filter with fresh randomness.
 *   loglik     out: log of the likelihood estimate of y(t_1..t_s).
 *   particles  out or NULL: [N][P] x(t_s) in the state precision.
 * Synchronous on cuda_stream (NULL: the filter's own stream).  Returns
 * PF_EDEGENERATE (loglik = -inf) once a step has degenerated. */
pf_status pf_run_range(pf_filter* f, const double* theta, const double* y, uint64_t seed,
                       int32_t r, int32_t s, double* loglik, void* particles, void* cuda_stream);

/* One state path drawn from the filter's approximation of the smoothing
 * distribution p(x(t_0..t_T) | y(t_1..t_T)) (end of Algorithm 2): particle
 * b_T is drawn from the final normalised weights with the Philox uniform of
 * block (0, T+1, purpose 4, 0) as the first k with C_k (P / S) > v P, and
 * b_{i-1} = a(t_i)[b_i] follows the ancestor history back to t_0.
 *   theta, y, seed  as for pf_run; loglik as for pf_run.
 *   path        out: [T+1][N] doubles, row i = x(t_i) of particle b_i, host or device.
 *   path_index  out or NULL: [T+1] int32, b_0 .. b_T.
 * Runs the filter twice (the second run regenerates the states it copies
 * from) and holds a [T][P] int32 ancestor history on the device.
 * Synchronous.  On PF_EDEGENERATE the path is NaN and the indices -1. */
pf_status pf_sample_path(pf_filter* f, const double* theta, const double* y, uint64_t seed,
                         double* loglik, double* path, int32_t* path_index, void* cuda_stream);

/* After a PF_FLAG_ASYNC run: wait for the filter's last run and return its
 * status (PF_OK or PF_EDEGENERATE). */
pf_status pf_wait(pf_filter* f);

/* Wait for the filter's own pending work (an asynchronous run; other work on
 * the device is not waited for), then free its device buffers and every
 * cached batch plan that lists it.  f = NULL does nothing.  Always PF_OK. */
pf_status pf_destroy(pf_filter* f);

/* Message describing the last error on this host thread ("" if none). */
const char* pf_last_error(void);

/* Many independent filters in one launch sequence (PMCMC proposals, SMC^2
 * parameter particles).  Filter k runs exactly as pf_run(f[k], theta[k],
 * y[k], seeds[k], ...) would, bit for bit; the filters may differ in model,
 * P, T and precision.  Pointers in theta[k], y[k] may be host or device
 * memory; logliks and per_filter_status are host arrays of nfilt entries.
 * The launch plan (tile map, CUDA graph) is cached for a repeated filter list.
 * Returns PF_OK if every filter ran (per-filter outcomes in
 * per_filter_status), else the first error; PF_ETIMEOUT if a CTA of the
 * persistent launch (pf_batch_shape) waited more than 4 s for a work item
 * (the results are then not valid). */
pf_status pf_batch_run(int32_t nfilt, pf_filter* const* f, const double* const* theta,
                       const double* const* y, const uint64_t* seeds, double* logliks,
                       int32_t* per_filter_status, void* cuda_stream);

/* The batched form's split of a filter list between its two paths (a batched
 * run of Algorithm 2 per filter either way): filters with at most
 * cta_max_particles particles (and at most 2048, not resampled
 * multinomially) run whole, each on one thread-block cluster (one CTA per
 * tile of 256 particles, cluster barriers between the phases of a step), on a
 * side branch of the plan's CUDA graph -- no per-step launches or grid-wide
 * hand-offs -- while the others take the tiled per-step launches.  Both paths
 * compute every filter with the same functions in the same order, so results
 * are bit-identical whatever the split.  0 (the default) sends every filter
 * to the tiled path.  Applies to pf_batch_run and pf_pmmh_run on this exact
 * filter list (f: nfilt filters of the caller, the list's order matters); a
 * cached plan for the list is rebuilt on its next use.  Host-only, no device
 * work.  PF_EINVAL for nfilt <= 0, a NULL list or filter, a filter listed
 * twice, or cta_max_particles < 0. */
pf_status pf_batch_configure(int32_t nfilt, pf_filter* const* f, int64_t cta_max_particles);

/* The whole launch shape of a batch.  No field changes any result: every
 * filter is computed by the same functions in the same order whatever the
 * shape; only how the filters share the GPU changes. */
typedef struct {
  int64_t cta_max_particles;      /* the cluster path's bound, as pf_batch_configure (0: none)    */
  int32_t branches;               /* >= 1: the tiled filters, longest runs first, are dealt in turn
                                     into this many independent chains of per-step launches; the
                                     chains run concurrently as parallel branches of the plan's
                                     CUDA graph, each at its own pace, and meet only at the end of
                                     the run (capped at the number of tiled filters; one chain
                                     when some filter resamples multinomially)                  */
  int32_t resample_blocks_per_sm; /* blocks per SM in the resample kernel's grid, 1..8            */
  int32_t persistent_blocks_per_sm; /* 0: the tiled filters run as the chains above.  1..8: they
                                     run in one persistent launch instead, this many CTAs per SM
                                     (capped at the kernel's occupancy): the CTAs take (filter,
                                     phase, tiles) work items from a device queue, and the CTA that
                                     finishes a filter's step or resampling queues the filter's next
                                     phase, so no filter waits for another.  Used when every tiled
                                     filter is a windkessel or a Lorenz '96 N = 8 filter of one
                                     precision, none resampled multinomially; otherwise ignored  */
  int32_t tiles_per_item;         /* persistent launch: tiles of 256 particles per work item, 1, 2,
                                     4 or 8; a filter of at most this many tiles runs whole on the
                                     CTA that takes its first item                               */
} pf_batch_shape;

/* Set / read the launch shape used for this exact filter list (as
 * pf_batch_configure: host-only; a cached plan is rebuilt on its next use).
 * The default shape is {0, 4, 8, 0, 1}.  PF_EINVAL for a bad list (as
 * pf_batch_configure), a NULL shape, cta_max_particles < 0, branches < 1,
 * resample_blocks_per_sm or persistent_blocks_per_sm outside 1..8 and 0..8,
 * or tiles_per_item not 1, 2, 4 or 8. */
pf_status pf_batch_set_shape(int32_t nfilt, pf_filter* const* f, const pf_batch_shape* shape);
pf_status pf_batch_get_shape(int32_t nfilt, pf_filter* const* f, pf_batch_shape* shape);

/* Autotuner of the launch shape: runs the batch (inputs as for pf_batch_run,
 * on the default stream, synchronously), one untimed and two timed runs per
 * candidate on the host clock, searching one field at a time from the
 * default: the cluster bound (0, 256, 512, 1024, 2048 particles), then the
 * number of branches (1, 2, 4, 8, 16), then the resample grid (2, 4, 8 blocks
 * per SM), then the persistent launch: off, or CTAs per SM (2, 3, 4) jointly
 * with tiles per item (1, 2, 4).  It keeps the fastest shape for the filter
 * list (as
 * pf_batch_set_shape would; pf_batch_get_shape reads it back) and returns its
 * cluster bound in *chosen (may be NULL).  The filters' results are those of
 * their last run, identical for every shape.  Errors: those of
 * pf_batch_set_shape and pf_batch_run, returned as soon as one occurs. */
pf_status pf_batch_autotune(int32_t nfilt, pf_filter* const* f, const double* const* theta,
                            const double* const* y, const uint64_t* seeds, int64_t* chosen);

/* ---- marginal Metropolis-Hastings over the parameters (Algorithm 3) ------ */

typedef enum {
  PF_PRIOR_FIXED = 0,      /* not sampled: contributes nothing                     */
  PF_PRIOR_UNIFORM = 1,    /* uniform on [a, b]                                    */
  PF_PRIOR_GAUSSIAN = 2,   /* gaussian, mean a, standard deviation b              */
  PF_PRIOR_GAMMA = 3,      /* gamma, shape a, scale b                              */
  PF_PRIOR_INV_GAMMA = 4   /* inverse gamma, shape a, scale b                      */
} pf_prior_kind;

typedef enum {
  PF_PROPOSE_FIXED = 0,           /* the component keeps its value                */
  PF_PROPOSE_TRUNC_GAUSSIAN = 1,  /* N(current, c^2) truncated to [d, e] (d, e may
                                     be -/+ infinity)                              */
  PF_PROPOSE_INV_GAMMA = 2        /* inverse gamma, integer shape c in [1, 64],
                                     scale d * current value                        */
} pf_proposal_kind;

/* Prior and proposal of one component of theta (the parameter and
 * proposal_parameter blocks of the paper's model listings). */
typedef struct {
  int32_t prior;      /* pf_prior_kind    */
  int32_t proposal;   /* pf_proposal_kind */
  double a, b;        /* prior parameters */
  double c, d, e;     /* proposal parameters */
} pf_param;

/* nchains independent marginal Metropolis-Hastings chains (Algorithm 3, the
 * acceptance rule of Eq. mh) whose likelihoods are particle-filter estimates
 * (the pseudo-marginal sampler).  Chain c runs its filter f[c] (all filters
 * of one model kind and T; P, precision and resampling may differ); every
 * iteration proposes theta' for all chains on the GPU, runs all nchains
 * filters as one batched launch sequence, and accepts or rejects on the GPU,
 * so the host only enqueues.
 *   y        [T][Ny] doubles, host or device, shared by the chains.
 *   spec     [pf_theta_size(kind)] priors / proposals, host.
 *   theta0   [nchains][pf_theta_size(kind)] starting points, host.
 *   niter    iterations after the starting point (>= 0).
 *   seed     Philox key of the proposals, acceptance uniforms and filter keys:
 *            counter (c, i, (5 << 16) | block, 0) -- block 0: uniform alpha in
 *            (0, 1]; block 1: the filter's key; block 16 + 64 d + a: draw a of
 *            component d (a Box-Muller normal, or the exponential -log u).
 *   samples  out: [niter+1][nchains][pf_theta_size(kind)] doubles, host or device.
 *   logliks  out: [niter+1][nchains] log-likelihood estimates of the samples.
 *   accepted out or NULL: [nchains] int32 accepted-move counts.
 * A proposal outside the prior's support or whose filter degenerates is
 * rejected.  Synchronous on cuda_stream (NULL: the plan's stream). */
pf_status pf_pmmh_run(int32_t nchains, pf_filter* const* f, const double* y,
                      const pf_param* spec, const double* theta0, int32_t niter, uint64_t seed,
                      double* samples, double* logliks, int32_t* accepted, void* cuda_stream);

/* SMC^2 over the parameters (Algorithm 4): ntheta parameter particles drawn
 * from the prior, each with its own filter of P particles (model m, T, dt);
 * for every observation i: multinomial resampling of the parameter particles
 * on their weights, one Metropolis-Hastings move per particle (Eq. mh, its
 * likelihood from a fresh filter over t_{0:i-1}; a rejected move keeps a
 * copy of the ancestor's filter), then every filter continues over
 * t_{i-1:i} and its likelihood increment is the particle's new weight.
 *   y            [T][Ny] doubles, host or device.
 *   spec         [pf_theta_size(kind)] priors / proposals, host; gamma and
 *                inverse-gamma priors need integer shapes 1..64 (drawn as
 *                sums of unit exponentials).
 *   theta_base   [pf_theta_size(kind)] values of the PF_PRIOR_FIXED components.
 *   seed         Philox key; counter (j, i, (6 << 16) | block, 0): block 0 the
 *                multinomial uniform, 1 the rejuvenation filter's key, 2 the
 *                continuation's key (step 0: the initial filter's), 3 the
 *                acceptance uniform, 16 + 64 d + a the prior draw (step 0) or
 *                proposal (step i) of component d.
 *   theta_out    out: [ntheta][pf_theta_size(kind)] the particles at t_T.
 *   logw_out     out: [ntheta] their log-weights log v^j(t_T).
 *   log_evidence out: sum_i log((1/ntheta) sum_j v^j(t_i)), the log of the
 *                marginal-likelihood estimate.
 *   evidence_incr out or NULL: [T] the per-observation terms of that sum.
 *   accepted     out or NULL: [T] moves accepted at each observation.
 * Outputs may be host or device memory.  Allocates 2 * ntheta filters for the
 * call (the rejuvenation population and the current one).  Synchronous;
 * PF_EDEGENERATE if every parameter particle's weight vanished. */
pf_status pf_smc2_run(const pf_model* m, int64_t P, int32_t T, double dt, const double* y,
                      int32_t ntheta, const pf_param* spec, const double* theta_base,
                      uint64_t seed, double* theta_out, double* logw_out, double* log_evidence,
                      double* evidence_incr, int32_t* accepted, void* cuda_stream);

/* Continuous-batching request server.  Requests (model, P, T, dt, theta, y,
 * seed) are queued on submit; a scheduler thread admits them when the device
 * memory budget and a slot allow, advances every admitted filter one
 * observation per iteration in shared launches, and retires finished ones, so
 * requests that arrive while others run join the next iteration.  Results are
 * bit-identical to pf_run of the same request. */
typedef struct pf_server pf_server;
pf_status pf_server_create(size_t device_mem_budget, int32_t max_slots, pf_server** out);
/* Queue a request; theta and y are copied.  PF_ENOMEM if the request alone
 * exceeds the budget, PF_EINVAL on bad arguments, PF_ECUDA once a CUDA error
 * has stopped the server. */
pf_status pf_server_submit(pf_server* s, const pf_model* m, int64_t P, int32_t T, double dt,
                           const double* theta, const double* y, uint64_t seed,
                           uint64_t* ticket);
/* PF_EBUSY while the request is queued or running; otherwise its final status,
 * with loglik and latency (seconds from submit to completion) filled in:
 * PF_OK, PF_EDEGENERATE, PF_ENOMEM (its buffers could not be allocated), or
 * PF_ECUDA (a CUDA error stopped the server; it then refuses new requests).
 * A finished ticket can be collected once: polling it again, or polling a
 * ticket this server never issued, gives PF_EINVAL. */
pf_status pf_server_poll(pf_server* s, uint64_t ticket, double* loglik, double* latency_s);
/* Launch groups per scheduler iteration, 1..8 (default 4, the best measured
 * on a mixed serving workload).  With b > 1 the running filters are dealt into
 * b groups of about equal work per step (longest first, each to the
 * least-loaded group) and each group's launches of an iteration run on a
 * stream of their own, forked from the scheduler's stream and joined back
 * before the iteration's results; with b = 1 every launch runs on one stream.
 * Results do not depend on b.  Takes effect at the next iteration; PF_EINVAL
 * outside 1..8. */
pf_status pf_server_configure(pf_server* s, int32_t branches);
/* Counters: queued, running, completed requests and scheduler iterations. */
pf_status pf_server_stats(pf_server* s, int64_t* queued, int64_t* running, int64_t* completed,
                          int64_t* iterations);
pf_status pf_server_destroy(pf_server* s);

/* ---- allocation-free run (no counterpart in the paper) ------------------- */

/* Size of the fixed device array pf_run_noalloc works in: 32 MiB.  The array
 * is reserved on a device by the first pf_run_noalloc call there (CUDA loads
 * the module that holds it lazily, on first use) and kept until the process
 * exits. */
#define PF_NOALLOC_SCRATCH_BYTES (32u << 20)

/* One run of the filter, exactly as pf_create + pf_run + pf_destroy would give
 * (same kernels, same bits), for callers that cannot allocate device memory
 * where they need a likelihood: code running while its own pool or arena
 * holds the device budget, frameworks that forbid allocation on the hot path
 * (an allocation may synchronise the device or fail under fragmentation), or
 * real-time loops that must not enter the allocator.  It calls no
 * cudaMalloc, cudaFree or other allocating routine: every internal buffer is
 * carved out of one fixed array of PF_NOALLOC_SCRATCH_BYTES.  The first call
 * on a device loads the array there (that load takes its 32 MiB of device
 * memory): make it at set-up, before the caller's own pool takes the device
 * budget and before any stream capture.
 *   m, P, T, dt   as for pf_create; a filter whose buffers do not fit in the
 *                 array is rejected with PF_EINVAL and a message giving the
 *                 bytes it needs (use pf_create/pf_run for it).
 *   theta         device pointer, pf_theta_size(kind) doubles.
 *   y             device pointer, [T][Ny] doubles (read during the run).
 *   seed          as for pf_run.
 *   loglik        device pointer, 1 double (out).
 *   status        device pointer or NULL: 1 int32 (out), PF_OK or PF_EDEGENERATE.
 *   final_particles device pointer or NULL: [N][P] in the state precision.
 *   cuda_stream   stream to enqueue on (NULL: the legacy default stream).
 * The call only enqueues work; outputs are valid once the stream reaches it.
 * Every call on a device shares the one array, which keeps the previous
 * call's contents (the run clears what must start at zero): calls that
 * overlap on the GPU (different streams, or several host threads) race and
 * must be serialised by the caller.  Every call looks up the array's device
 * address on the current device (so a device reset does not leave a stale
 * one).  theta, y, loglik, status and final_particles must be device (or
 * managed) memory of the current device: a host pointer is refused with
 * PF_EINVAL before anything is enqueued. */
pf_status pf_run_noalloc(const pf_model* m, int64_t P, int32_t T, double dt,
                         const double* theta, const double* y, uint64_t seed, double* loglik,
                         int32_t* status, void* final_particles, void* cuda_stream);

/* ---- diagnostics (no counterpart in the paper) -------------------------- */

/* Teacher-forced step: observation i (1 <= i <= T) of Algorithm 2's loop --
 * propagate, weight, log-sum-exp and likelihood increment, ESS test and the
 * resampling after it -- run by the same launches as step i of pf_run (the
 * propagate kernel, then the resample kernel), but from a state given from
 * outside, so that each step can be checked on its own against a reference
 * fed the same state.
 *   theta, y, seed  as for pf_run (y: all T rows; row i-1 is used).
 *   x_prev         x(t_{i-1}), [N][P] in the filter's state precision, HOST
 *                  or device.
 *   anc            a(t_i), [P] int32, HOST or device: the ancestors that
 *                  propagate into t_i; NULL: the identity.  The carried
 *                  log-weights start at zero, as after a resampling.
 *   x_out          x(t_i), [N][P] (or NULL).
 *   incr           the likelihood increment log Z_i of step i (or NULL).
 *   anc_next       [P] int32 (or NULL): the ancestors step i + 1 takes from
 *                  step i's resampling, as the resample kernel wrote them (the
 *                  identity when step i carried its weights); untouched for
 *                  i = T or a degenerate step.
 * Synchronous; returns PF_OK, PF_EDEGENERATE (a degenerate step) or an error.
 * The filter is left standing at t_i: pf_run_range(f, ..., i, s) continues
 * from it. */
pf_status pf_debug_step(pf_filter* f, const double* theta, const double* y, uint64_t seed,
                        int32_t i, const void* x_prev, const int32_t* anc, void* x_out,
                        double* incr, int32_t* anc_next);

/* Profiling mode: while enabled, pf_run launches the filter's kernels one by
 * one instead of as one CUDA graph and brackets every launch with CUDA events
 * on the run's stream.  Results are unchanged. */
pf_status pf_profile_enable(pf_filter* f, int32_t on);
/* Summed device time (ms) and launch counts of the runs since the last read,
 * per kernel kind: [0] init, [1] propagate+weight, [2] resample, [3] results.
 * Waits for those runs to finish. */
pf_status pf_profile_read(pf_filter* f, double* ms, int64_t* launches);

/* Measured dense fused-multiply-add throughput of the current GPU, in flop/s
 * (2 per FMA): prec PF_FP64, PF_MIXED (FP32) or 2 (FP32 pairs through the
 * packed f32x2 instruction, 4 flop per instruction).  Runs a few ~40 ms
 * kernels; *ms receives the duration of the best one. */
pf_status pf_measure_fma_peak(int32_t prec, double* flops_per_s, double* ms);

/* The exponential that the propagate kernels apply to the log-weights relative
 * to their tile maximum (Algorithm 2, weight and normalisation lines:
 * w = exp(ell - M), d = ell - M <= 0), evaluated on the device for n given
 * arguments: w[i] = e^{d[i]}.  A diagnostic that lets a test compare the
 * kernels' exponential (a table-driven method on the FP32 unit with two FP64
 * operations, relative error about 2^-52 for -700 < d <= 0) with a correctly
 * rounded one.  d and w are HOST arrays of n doubles owned by the caller
 * (they may not overlap); n = 0 does nothing.  Synchronous, on the current
 * device; allocates 16 n bytes of device memory for the call.  PF_EINVAL for
 * n < 0, n > 2^28 or a NULL array with n > 0; PF_ECUDA on a CUDA error. */
pf_status pf_weight_exp(const double* d, double* w, int64_t n);

/* The propagate kernels' in-tile cumulative weights (Algorithm 2's resampling
 * needs the prefix sums of the weights, Sec. 3.3), evaluated on the device
 * for given weights: per tile of 256 consecutive weights, prefix[j] = the sum
 * of the tile's weights up to j and totals[t] = the tile's sum, as the
 * windkessel and Lorenz '96 N <= 12 kernels compute them: each weight rounded
 * to an integer multiple of 2^-55 (nearest, ties to even), those summed
 * exactly in 64-bit integers, each sum rounded once to the nearest double;
 * this lets a test compare them with exact rational sums.
 * w, prefix: HOST arrays of n doubles; totals: HOST array of ceil(n / 256)
 * doubles; all owned by the caller and not overlapping; n = 0 does nothing.
 * Synchronous, on the current device; allocates device memory for the call.
 * PF_EINVAL for n < 0, n > 2^28, a NULL array with n > 0 or a weight outside
 * [0, 1] (the kernels' weights are exp(ell - M_tile) <= 1); PF_ECUDA on a
 * CUDA error. */
pf_status pf_weight_prefix(const double* w, double* prefix, double* totals, int64_t n);

/* The step combine's logarithm of the weight sum (Algorithm 2, likelihood
 * line: log Z_i = M + log S - log P with S = sum_j e^(ell_j - M) >= 1),
 * evaluated on the device for n given arguments: y[i] = log s[i].  A
 * diagnostic that lets a test compare the kernels' logarithm (an FP32
 * logarithm refined by one Newton step in FP64 with the weight exponential,
 * absolute error a few units of 2^-53 for 1 <= s <= 2^120; the library
 * logarithm elsewhere) with correctly rounded values.  s and y are HOST arrays
 * of n doubles owned by the caller (they may not overlap); n = 0 does nothing.
 * Synchronous, on the current device; allocates 16 n bytes of device memory
 * for the call.  PF_EINVAL for n < 0, n > 2^28 or a NULL array with n > 0;
 * PF_ECUDA on a CUDA error. */
pf_status pf_weight_sum_log(const double* s, double* y, int64_t n);

/* Host-side fault injection for tests: the k-th next device allocation made
 * for a filter (pf_create) or for a request the server admits fails as if
 * the device were out of memory -- once; k = 0 disarms.  pf_create then
 * returns PF_ENOMEM having freed what it had allocated, and the request is
 * finished with PF_ENOMEM (pf_server_poll) while the server goes on.  The
 * countdown is process-wide and shared by all threads.  PF_EINVAL for
 * k < 0. */
pf_status pf_debug_fail_allocation(int32_t k);

/* Host-side fault injection for tests: the k-th next wait of a server's
 * scheduler for one of its iterations (any server of the process) reports a
 * CUDA error, as a failed kernel would -- once; k = 0 disarms.  That server
 * then ends its running and queued requests with PF_ECUDA (pf_server_poll)
 * and refuses new ones (pf_server_submit returns PF_ECUDA); pf_server_destroy
 * still releases it.  The GPU itself is not touched.  PF_EINVAL for k < 0. */
pf_status pf_debug_fail_server_wait(int32_t k);

/* Failure detection of the batched form's persistent launch, for tests.
 * pf_debug_persist_wait_limit sets how long (seconds, > 0; 4 at load) a CTA
 * of any later persistent launch waits for a work item before it gives up:
 * the launch then ends with PF_ETIMEOUT from pf_batch_run, every kernel
 * having returned (no fault; the context stays usable).  It is set on the
 * current device, synchronously; PF_EINVAL for seconds <= 0 or > 60,
 * PF_ECUDA on a CUDA error.  pf_debug_persist_unfilled_slot(1) makes every
 * persistent plan built afterwards count one slot more than its filters fill
 * (a slot nothing ever fills: its wait runs out); 0 disarms.  Process-wide,
 * host-side; PF_EINVAL for values other than 0 and 1.  Neither has a
 * counterpart in the paper. */
pf_status pf_debug_persist_wait_limit(double seconds);
pf_status pf_debug_persist_unfilled_slot(int32_t on);

/* Invariant counters of a checked build of this library (compiled with
 * PF_CHECKED=1: libpf_b300_checked.so), the sanitizer substitute: the kernels
 * count, instead of assuming, violations of the path's invariants.
 *   counts[0]  ancestors read outside [0, P) (replaced by the particle's own
 *              index, so every access stays in bounds)
 *   counts[1]  particles whose propagated state is not finite
 *   counts[2]  in-tile cumulative weights that are negative or NaN, weights
 *              above 1, and in-tile cumulative weights that decrease (at all
 *              for the exact fixed-point sums, by more than 2^-49 relative for
 *              the FP64 tree, whose rounding stays below it)
 *   counts[3]  offspring ranges that end before they start or leave [0, P]
 * counts: host array of 4, owned by the caller, receives the counts since the
 * last call (then zeroed); *checked (may be NULL) receives 1 in a checked
 * build, 0 otherwise (whose counts are always 0).  Synchronous on the current
 * device.  PF_EINVAL for NULL counts; PF_ECUDA on a CUDA error. */
pf_status pf_debug_check_counts(uint64_t* counts, int32_t* checked);

#ifdef __cplusplus
}
#endif
#endif /* PF_B300_H */
