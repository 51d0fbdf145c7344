"""CPU oracle of the bootstrap particle filter (arXiv 1306.3277, Algorithm 2).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product path (``paper_1306_3277_b300``) never does, and the two
share no code: the oracle is plain C (``pf_oracle.c``) compiled with gcc,
the product is CUDA.

What each function follows, and what pins it (tests in ``tests/test_oracle_*``):

========================  =======================================  ==========================================
function                  follows                                   pinned by
========================  =======================================  ==========================================
philox4x32_10             Salmon et al. SC'11 (Philox4x32-10)       published known-answer vectors
                                                                    (tests/golden/philox4x32_10_kat.txt)
log / logf                atanh series of log (own)                libm log, <= 2 ulp; exact special values
exp                       Cody-Waite reduction + Taylor (own)      libm exp, <= 2 ulp; special values
sincos2pi / sincos2pif    quarter-turn reduction + Taylor (own)    libm sin/cos, exact quadrant points
normal64 / normal32       Box-Muller                               moments, Kolmogorov-Smirnov vs scipy
flow_table                Eq. (flow) read as a half sine           closed form with numpy.sin
l96_rk4 / l96_rk4f        Eq. (lorenz96-ode), classic RK4          fixed point, shift equivariance, energy
                                                                    decay exp(-2t) at F=0, 4th-order
                                                                    convergence, scipy solve_ivp
kalman_windkessel         Algorithm 1 (scalar)                     brute-force joint Gaussian (scipy)
lse                       Algorithm 2 likelihood line, log space   equal / one-hot weights, shift invariance,
                                                                    math.fsum
systematic                Sec. 3.3 systematic resampling           integer weights (exact), brute-force
                                                                    offspring enumeration on P <= 8
resample (stratified,     Sec. 3.3 / Algorithm 2 multinomial       exact rational targets from the
 multinomial)             (sorted: exponential spacings)           published Philox stream; offspring
                                                                    mean, variance, range over seeds
pf_run                    Algorithm 2                              Kalman likelihood (exact special case
                                                                    and convergence over P), closed-form
                                                                    deterministic Lorenz '96 likelihood
pf_run_sched              Algorithm 2 over t_{r:s} intervals,      constant schedule = pf_run; per-step
                          one Philox key per step                  keys still converge to the Kalman value
sample_path               Algorithm 2 ancestry trace (end)         exact rational pick, noiseless closed
                                                                    form, joint-Gaussian smoothing moments
log_prior / propose       Sec. 2.1 parameter / proposal blocks     scipy logpdf, KS of the draws, scipy
                                                                    Hastings correction
pmmh                      Algorithm 3, Eq. (mh)                    prior-only chains sample the prior;
                                                                    Kalman-likelihood chains match a grid
                                                                    posterior
smc2                      Algorithm 4                              exact-likelihood (Kalman) runs match
                                                                    quadrature evidence and posterior;
                                                                    filter runs keep the evidence
========================  =======================================  ==========================================
"""
import ctypes
import os

import numpy as np

from . import build as _build

WINDKESSEL = 0
LORENZ96 = 1
WINDKESSEL_EXP = 2
LORENZ96_SDE = 3
FP64 = 0
MIXED = 1
PURPOSE_INIT = 1
PURPOSE_PROP = 2
PURPOSE_RESAMPLE = 3
PURPOSE_PATH = 4
PURPOSE_PMMH = 5
PURPOSE_SMC2 = 6
OK = 0
RESAMPLE_SYSTEMATIC, RESAMPLE_STRATIFIED, RESAMPLE_MULTINOMIAL = range(3)
EINVAL = 1
EDEGENERATE = 4


class Model(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32),
        ("N", ctypes.c_int32),
        ("substeps", ctypes.c_int32),
        ("obs_stride", ctypes.c_int32),
        ("prec", ctypes.c_int32),
        ("resampler", ctypes.c_int32),
        ("dt", ctypes.c_double),
        ("ess_threshold", ctypes.c_double),
        ("flow_peak", ctypes.c_double),
        ("flow_period", ctypes.c_double),
        ("obs_every", ctypes.c_int32),
        ("obs_count", ctypes.c_int32),
    ]


_lib = None
_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.POINTER(ctypes.c_float)
_ip = ctypes.POINTER(ctypes.c_int32)
_up = ctypes.POINTER(ctypes.c_uint32)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.or_philox4x32_10.argtypes = [_up, _up, _up]
        L.or_normal64.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                  ctypes.c_uint32]
        L.or_normal64.restype = ctypes.c_double
        L.or_normal32.argtypes = L.or_normal64.argtypes
        L.or_normal32.restype = ctypes.c_float
        L.or_resample_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint32]
        L.or_resample_uniform.restype = ctypes.c_double
        L.or_fill_normals.argtypes = [ctypes.c_uint64, ctypes.c_int32, ctypes.c_uint32,
                                      ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, _dp]
        L.or_log.argtypes = [ctypes.c_double]
        L.or_log.restype = ctypes.c_double
        L.or_logf.argtypes = [ctypes.c_float]
        L.or_logf.restype = ctypes.c_float
        L.or_sincos2pi.argtypes = [ctypes.c_double, _dp, _dp]
        L.or_sincos2pif.argtypes = [ctypes.c_float, _fp, _fp]
        L.or_flow_table.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int64,
                                    _dp]
        L.or_l96_rk4.argtypes = [_dp, ctypes.c_int32, ctypes.c_double, ctypes.c_double, ctypes.c_int32]
        L.or_l96_rk4f.argtypes = [_fp, ctypes.c_int32, ctypes.c_float, ctypes.c_float, ctypes.c_int32]
        L.or_kalman_windkessel.argtypes = [ctypes.POINTER(Model), _dp, _dp, ctypes.c_int32]
        L.or_kalman_windkessel.restype = ctypes.c_double
        L.or_lse.argtypes = [_dp, ctypes.c_int64, _dp, _dp, _dp]
        L.or_systematic.argtypes = [_dp, ctypes.c_int64, ctypes.c_double, _ip]
        L.or_systematic.restype = ctypes.c_int64
        L.or_exp.argtypes = [ctypes.c_double]
        L.or_exp.restype = ctypes.c_double
        L.or_resample.argtypes = [_dp, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64,
                                  ctypes.c_uint32, _ip]
        L.or_resample.restype = ctypes.c_int64
        L.or_pf_run.argtypes = [ctypes.POINTER(Model), _dp, _dp, ctypes.c_uint64, ctypes.c_int64,
                                ctypes.c_int32, ctypes.c_int32, _dp, _dp, _ip, _dp]
        L.or_pf_run.restype = ctypes.c_int32
        L.or_pf_run_ex.argtypes = L.or_pf_run.argtypes + [_dp, _dp]
        L.or_pf_run_ex.restype = ctypes.c_int32
        L.or_pf_run_sched.argtypes = [ctypes.POINTER(Model), _dp, _dp, ctypes.c_uint64,
                                      ctypes.POINTER(ctypes.c_uint64), ctypes.c_int64,
                                      ctypes.c_int32, ctypes.c_int32, _dp, _dp, _ip, _dp, _dp, _dp]
        L.or_pf_run_sched.restype = ctypes.c_int32
        L.or_pmmh.argtypes = [ctypes.POINTER(Model), _dp, ctypes.c_int64, ctypes.c_int32,
                              ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(Param), _dp,
                              ctypes.c_int32, ctypes.c_uint64, ctypes.c_int32, _dp, _dp, _ip, _ip]
        L.or_pmmh.restype = ctypes.c_int32
        L.or_log_prior.argtypes = [ctypes.POINTER(Param), ctypes.c_int32, _dp]
        L.or_log_prior.restype = ctypes.c_double
        L.or_propose.argtypes = [ctypes.POINTER(Param), ctypes.c_int32, _dp, ctypes.c_uint64,
                                 ctypes.c_uint32, ctypes.c_uint32, _dp]
        L.or_propose.restype = ctypes.c_double
        L.or_smc2.argtypes = [ctypes.POINTER(Model), _dp, ctypes.c_int64, ctypes.c_int32,
                              ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(Param), _dp,
                              ctypes.c_uint64, ctypes.c_int32, _dp, _dp, _dp, _dp, _ip, _ip]
        L.or_smc2.restype = ctypes.c_int32
        L.or_pf_step.argtypes = [ctypes.POINTER(Model), _dp, _dp, ctypes.c_uint64, ctypes.c_int64,
                                 ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _dp, _ip, _dp,
                                 _dp, _ip, _dp]
        L.or_pf_step.restype = ctypes.c_int32
        L.or_sample_path.argtypes = [ctypes.POINTER(Model), _dp, _dp, ctypes.c_uint64,
                                     ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, _dp, _dp, _ip]
        L.or_sample_path.restype = ctypes.c_int32
        _lib = L
    return _lib


def _ptr(a, t):
    return a.ctypes.data_as(t)


def model(kind, N=1, substeps=1, obs_stride=1, prec=FP64, dt=0.01, ess_threshold=1.0,
          flow_peak=400.0, flow_period=1.0, resampler=0, obs_every=0, obs_count=0):
    return Model(kind, N, substeps, obs_stride, prec, resampler, dt, ess_threshold, flow_peak,
                 flow_period, obs_every, obs_count)


def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    lib().or_philox4x32_10(_ptr(c, _up), _ptr(k, _up), _ptr(o, _up))
    return o


def normal64(seed, j, i, purpose, q):
    return lib().or_normal64(seed, j, i, purpose, q)


def normal32(seed, j, i, purpose, q):
    return lib().or_normal32(seed, j, i, purpose, q)


def fill_normals(seed, prec, i, purpose, nj, nq):
    out = np.zeros((nj, nq), dtype=np.float64)
    lib().or_fill_normals(seed, prec, i, purpose, nj, nq, _ptr(out, _dp))
    return out


def resample_uniform(seed, i):
    return lib().or_resample_uniform(seed, i)


def log(x):
    return lib().or_log(float(x))


def exp(x):
    return lib().or_exp(x)


def logf(x):
    return lib().or_logf(float(np.float32(x)))


def sincos2pi(u):
    s = ctypes.c_double()
    c = ctypes.c_double()
    lib().or_sincos2pi(float(u), ctypes.byref(s), ctypes.byref(c))
    return s.value, c.value


def sincos2pif(u):
    s = ctypes.c_float()
    c = ctypes.c_float()
    lib().or_sincos2pif(float(np.float32(u)), ctypes.byref(s), ctypes.byref(c))
    return np.float32(s.value), np.float32(c.value)


def flow_table(peak, period, dt, n):
    out = np.zeros(n, dtype=np.float64)
    lib().or_flow_table(peak, period, dt, n, _ptr(out, _dp))
    return out


def l96_rk4(x, F, dt, nsteps):
    x = np.array(x, dtype=np.float64)
    lib().or_l96_rk4(_ptr(x, _dp), len(x), F, dt, nsteps)
    return x


def l96_rk4f(x, F, dt, nsteps):
    x = np.array(x, dtype=np.float32)
    lib().or_l96_rk4f(_ptr(x, _fp), len(x), float(np.float32(F)), float(np.float32(dt)), nsteps)
    return x


def kalman_windkessel(m, theta, y):
    th = np.ascontiguousarray(theta, dtype=np.float64)
    yy = np.ascontiguousarray(y, dtype=np.float64).ravel()
    return lib().or_kalman_windkessel(ctypes.byref(m), _ptr(th, _dp), _ptr(yy, _dp), len(yy))


def lse(ell):
    e = np.ascontiguousarray(ell, dtype=np.float64)
    M, S, Q = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    lib().or_lse(_ptr(e, _dp), len(e), ctypes.byref(M), ctypes.byref(S), ctypes.byref(Q))
    return M.value, S.value, Q.value


def systematic(ell, u):
    e = np.ascontiguousarray(ell, dtype=np.float64)
    anc = np.zeros(len(e), dtype=np.int32)
    near = lib().or_systematic(_ptr(e, _dp), len(e), float(u), _ptr(anc, _ip))
    return anc, int(near)


def resample(ell, kind, seed, i):
    """Ancestors of resampling step i (systematic, stratified or multinomial)
    from log-weights ell; returns (ancestors, near-boundary count)."""
    e = np.ascontiguousarray(ell, dtype=np.float64)
    anc = np.zeros(len(e), dtype=np.int32)
    near = lib().or_resample(_ptr(e, _dp), len(e), kind, seed, i, _ptr(anc, _ip))
    return anc, int(near)


def pf_run(m, theta, y, seed, P, T, nthreads=0, want_x=True, want_anc=True, want_diag=True):
    """Run the filter; returns dict(status, loglik, x [N][P], anc [T][P], diag [T][8])."""
    th = np.ascontiguousarray(theta, dtype=np.float64)
    yy = np.ascontiguousarray(y, dtype=np.float64)
    ll = ctypes.c_double()
    x = np.zeros((m.N, P), dtype=np.float64) if want_x else None
    anc = np.zeros((T, P), dtype=np.int32) if want_anc else None
    diag = np.zeros((T, 8), dtype=np.float64) if want_diag else None
    st = lib().or_pf_run(ctypes.byref(m), _ptr(th, _dp), _ptr(yy, _dp), seed, P, T, nthreads,
                         ctypes.byref(ll),
                         _ptr(x, _dp) if x is not None else None,
                         _ptr(anc, _ip) if anc is not None else None,
                         _ptr(diag, _dp) if diag is not None else None)
    return dict(status=st, loglik=ll.value, x=x, anc=anc, diag=diag)


def pf_run_ex(m, theta, y, seed, P, T, nthreads=0):
    """Filter run with the whole state history [T+1][N][P] and final log-weights [P]."""
    th = np.ascontiguousarray(theta, dtype=np.float64)
    yy = np.ascontiguousarray(y, dtype=np.float64)
    ll = ctypes.c_double()
    xh = np.zeros((T + 1, m.N, P), dtype=np.float64)
    ellT = np.zeros(P, dtype=np.float64)
    anc = np.zeros((T, P), dtype=np.int32)
    st = lib().or_pf_run_ex(ctypes.byref(m), _ptr(th, _dp), _ptr(yy, _dp), seed, P, T, nthreads,
                            ctypes.byref(ll), None, _ptr(anc, _ip), None, _ptr(xh, _dp),
                            _ptr(ellT, _dp))
    return dict(status=st, loglik=ll.value, xhist=xh, ellT=ellT, anc=anc)


def pf_step(m, theta, y, seed, P, T, i, x_prev, anc=None, nthreads=0):
    """Teacher-forced step i from x(t_{i-1}) [N][P] and a(t_i) [P] (None:
    identity): dict(status, incr, x [N][P], anc_next [P] or None, diag [8])."""
    th = np.ascontiguousarray(theta, dtype=np.float64)
    yy = np.ascontiguousarray(y, dtype=np.float64)
    xp = np.ascontiguousarray(x_prev, dtype=np.float64)
    a = None if anc is None else np.ascontiguousarray(anc, dtype=np.int32)
    x = np.zeros((m.N, P), dtype=np.float64)
    inc = ctypes.c_double()
    nxt = np.zeros(P, dtype=np.int32) if i < T else None
    dg = np.zeros(8, dtype=np.float64)
    st = lib().or_pf_step(ctypes.byref(m), _ptr(th, _dp), _ptr(yy, _dp), seed, P, T, i, nthreads,
                          _ptr(xp, _dp), None if a is None else _ptr(a, _ip), _ptr(x, _dp),
                          ctypes.byref(inc), None if nxt is None else _ptr(nxt, _ip),
                          _ptr(dg, _dp))
    return dict(status=st, incr=inc.value, x=x, anc_next=nxt, diag=dg)


def sample_path(m, theta, y, seed, P, T, nthreads=0):
    """One state path by ancestry: (status, loglik, path [T+1][N], idx [T+1])."""
    th = np.ascontiguousarray(theta, dtype=np.float64)
    yy = np.ascontiguousarray(y, dtype=np.float64)
    ll = ctypes.c_double()
    path = np.zeros((T + 1, m.N), dtype=np.float64)
    idx = np.zeros(T + 1, dtype=np.int32)
    st = lib().or_sample_path(ctypes.byref(m), _ptr(th, _dp), _ptr(yy, _dp), seed, P, T, nthreads,
                              ctypes.byref(ll), _ptr(path, _dp), _ptr(idx, _ip))
    return st, ll.value, path, idx


def pf_run_sched(m, theta, y, sched, P, T, nthreads=0, want_xhist=False):
    """Filter run with a seed schedule sched[0..T] (initial draw, then one key
    per step): loglik, final state, ancestors, diagnostics, optional history."""
    th = np.ascontiguousarray(theta, dtype=np.float64)
    yy = np.ascontiguousarray(y, dtype=np.float64)
    sc = np.ascontiguousarray(sched, dtype=np.uint64)
    assert len(sc) == T + 1
    ll = ctypes.c_double()
    x = np.zeros((m.N, P), dtype=np.float64)
    anc = np.zeros((T, P), dtype=np.int32)
    diag = np.zeros((T, 8), dtype=np.float64)
    xh = np.zeros((T + 1, m.N, P), dtype=np.float64) if want_xhist else None
    st = lib().or_pf_run_sched(ctypes.byref(m), _ptr(th, _dp), _ptr(yy, _dp), 0,
                               sc.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), P, T, nthreads,
                               ctypes.byref(ll), _ptr(x, _dp), _ptr(anc, _ip), _ptr(diag, _dp),
                               None if xh is None else _ptr(xh, _dp), None)
    return dict(status=st, loglik=ll.value, x=x, anc=anc, diag=diag, xhist=xh)


# ---- marginal Metropolis-Hastings (Algorithm 3) ---------------------------
PRIOR_FIXED, PRIOR_UNIFORM, PRIOR_GAUSSIAN, PRIOR_GAMMA, PRIOR_INV_GAMMA = range(5)
PROPOSE_FIXED, PROPOSE_TRUNC_GAUSSIAN, PROPOSE_INV_GAMMA = range(3)
LIK_PF, LIK_KALMAN, LIK_NONE = range(3)


class Param(ctypes.Structure):
    _fields_ = [("prior", ctypes.c_int32), ("proposal", ctypes.c_int32), ("a", ctypes.c_double),
                ("b", ctypes.c_double), ("c", ctypes.c_double), ("d", ctypes.c_double),
                ("e", ctypes.c_double)]


def params(spec):
    """spec: list of (prior, proposal, a, b, c, d, e) tuples -> ctypes array."""
    arr = (Param * len(spec))()
    for k, t in enumerate(spec):
        t = tuple(t) + (0.0,) * (7 - len(t))
        arr[k] = Param(int(t[0]), int(t[1]), *[float(v) for v in t[2:7]])
    return arr


def log_prior(spec, theta):
    th = np.ascontiguousarray(theta, dtype=np.float64)
    sp = params(spec)
    return lib().or_log_prior(sp, len(th), _ptr(th, _dp))


def propose(spec, theta, seed, j, i):
    """(theta', log q(theta|theta') - log q(theta'|theta)) of chain j at iteration i."""
    th = np.ascontiguousarray(theta, dtype=np.float64)
    out = np.zeros_like(th)
    sp = params(spec)
    lqr = lib().or_propose(sp, len(th), _ptr(th, _dp), seed, j, i, _ptr(out, _dp))
    return out, lqr


def pmmh(m, y, P, T, lik, spec, theta0, niter, seed, nthreads=0):
    """Chains of Algorithm 3: samples [niter+1][nchains][nth], logliks
    [niter+1][nchains], accepted [nchains], near [niter+1][nchains]."""
    th0 = np.ascontiguousarray(theta0, dtype=np.float64)
    nc, nth = th0.shape
    yy = np.ascontiguousarray(y, dtype=np.float64)
    sp = params(spec)
    samples = np.zeros((niter + 1, nc, nth))
    lls = np.zeros((niter + 1, nc))
    acc = np.zeros(nc, dtype=np.int32)
    near = np.zeros((niter + 1, nc), dtype=np.int32)
    st = lib().or_pmmh(ctypes.byref(m), _ptr(yy, _dp), P, T, lik, nc, sp, _ptr(th0, _dp), niter,
                       seed, nthreads, _ptr(samples, _dp), _ptr(lls, _dp), _ptr(acc, _ip),
                       _ptr(near, _ip))
    return dict(status=st, samples=samples, logliks=lls, accepted=acc, near=near)


def smc2(m, y, P, T, lik, ntheta, spec, base, seed, nthreads=0):
    """SMC^2 (Algorithm 4): final theta-particles, their log-weights, the log
    evidence and its per-step increments, accepted moves and near flags."""
    nth = 7 if m.kind in (WINDKESSEL, WINDKESSEL_EXP) else 5
    yy = np.ascontiguousarray(y, dtype=np.float64)
    b = np.ascontiguousarray(base, dtype=np.float64)
    sp = params(spec)
    th = np.zeros((ntheta, nth))
    logv = np.zeros(ntheta)
    lz = ctypes.c_double()
    incr = np.zeros(T)
    acc = np.zeros(T, dtype=np.int32)
    near = np.zeros(T, dtype=np.int32)
    st = lib().or_smc2(ctypes.byref(m), _ptr(yy, _dp), P, T, lik, ntheta, sp, _ptr(b, _dp), seed,
                       nthreads, _ptr(th, _dp), _ptr(logv, _dp), ctypes.byref(lz), _ptr(incr, _dp),
                       _ptr(acc, _ip), _ptr(near, _ip))
    return dict(status=st, theta=th, logv=logv, log_evidence=lz.value, incr=incr, accepted=acc,
                near=near)
