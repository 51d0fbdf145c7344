"""Pins of the oracle's whole filter (Algorithm 2): the exact Kalman
likelihood of the linear-Gaussian windkessel (a special case where the filter
is exact, and convergence over P), the closed-form likelihood of a
deterministic Lorenz '96 trajectory, degenerate inputs, and invariances."""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W


def _om(w, prec=None, thr=None):
    return O.model(w.kind, N=w.N, substeps=w.substeps, obs_stride=w.obs_stride,
                   prec=w.prec if prec is None else prec, dt=w.dt,
                   ess_threshold=w.ess_threshold if thr is None else thr,
                   flow_peak=w.flow_peak, flow_period=w.flow_period)


@pytest.mark.parametrize("substeps", [1, 3])
def test_windkessel_noiseless_fixed_start_equals_kalman(substeps):
    # q = 0 and s0 = 0: every particle follows the same deterministic path, the
    # filter is exact and must reproduce the Kalman likelihood at any P.
    th = (1.0, 1.5, 0.03, 0.0, 4.0, 90.0, 0.0)
    w = W.windkessel(P=64, T=100, substeps=substeps, theta=W.WK_THETA)
    m = _om(w)
    kf = O.kalman_windkessel(m, th, w.y)
    for P in (1, 64, 1000):
        r = O.pf_run(m, th, w.y, 5, P, w.T)
        assert r["status"] == O.OK
        assert r["loglik"] == pytest.approx(kf, rel=1e-12)


def test_windkessel_converges_to_kalman():
    w = W.windkessel(P=1024, T=100)
    m = _om(w)
    kf = O.kalman_windkessel(m, w.theta, w.y)
    stats = {}
    for P in (256, 4096):
        lls = np.array([O.pf_run(m, w.theta, w.y, s, P, w.T, want_x=False, want_anc=False,
                                 want_diag=False)["loglik"] for s in range(1, 33)])
        stats[P] = (lls.mean(), lls.var(ddof=1))
    mean, var = stats[4096]
    se = math.sqrt(var / 32)
    # E[log lhat] = log l - Var/2 to leading order (Jensen), lhat unbiased
    assert abs(mean - (kf - var / 2)) < 4 * se + 0.02
    # Var(log lhat) ~ c / P
    ratio = stats[256][1] / stats[4096][1]
    assert 4.0 < ratio < 64.0


def test_windkessel_adaptive_ess_branch():
    w = W.windkessel(P=2048, T=100, ess_threshold=0.5)
    m = _om(w)
    kf = O.kalman_windkessel(m, w.theta, w.y)
    r = O.pf_run(m, w.theta, w.y, 3, w.P, w.T)
    res = r["diag"][:, 4]
    assert 0 < res[:-1].sum() < w.T - 1
    for i in range(1, w.T):
        if res[i - 1] == 0:
            assert np.array_equal(r["anc"][i], np.arange(w.P))
    lls = [O.pf_run(m, w.theta, w.y, s, w.P, w.T, want_x=False, want_anc=False)["loglik"]
           for s in range(1, 17)]
    assert abs(np.mean(lls) - kf) < 1.0


def test_lorenz96_deterministic_closed_form():
    # q = 0, s0 = 0: deterministic trajectory from x0 = m0, every particle alike.
    F, r = 8.0, 0.25
    th = (F, 0.0, r, 1.3, 0.0)
    w = W.lorenz96_8(P=16, T=30)
    m = _om(w)
    x = np.full(8, 1.3)
    ll = 0.0
    for i in range(w.T):
        x = O.l96_rk4(x, F, w.dt, w.substeps)
        d = w.y[i] - x
        ll += -0.5 * 8 * math.log(2 * math.pi * r) - 0.5 * float(np.sum(d * d)) / r
    res = O.pf_run(m, th, w.y, 9, 16, w.T)
    assert res["loglik"] == pytest.approx(ll, rel=1e-12)
    assert np.allclose(res["x"], x[:, None], rtol=0, atol=0)


def test_degenerate_inputs():
    w = W.windkessel(P=64, T=10)
    m = _om(w)
    th = list(w.theta)
    th[4] = 0.0  # zero observation variance: every weight is zero
    r = O.pf_run(m, th, w.y, 1, 64, w.T)
    assert r["status"] == O.EDEGENERATE and r["loglik"] == -math.inf
    th = list(w.theta)
    th[0] = float("nan")
    r = O.pf_run(m, th, w.y, 1, 64, w.T)
    assert r["status"] == O.EDEGENERATE and r["loglik"] == -math.inf


def test_invalid_arguments():
    w = W.windkessel(P=64, T=10)
    m = _om(w)
    assert O.pf_run(m, w.theta, w.y, 1, 0, w.T)["status"] == O.EINVAL
    m2 = O.model(O.LORENZ96, N=3, substeps=1)
    assert O.pf_run(m2, W.L96_THETA_8, np.zeros((10, 3)), 1, 8, 10)["status"] == O.EINVAL


@pytest.mark.parametrize("prec", [O.FP64, O.MIXED])
def test_thread_count_invariance_and_ancestor_validity(prec):
    w = W.lorenz96_8(P=512, T=20, prec=prec)
    m = _om(w)
    a = O.pf_run(m, w.theta, w.y, 4, w.P, w.T, nthreads=1)
    b = O.pf_run(m, w.theta, w.y, 4, w.P, w.T, nthreads=3)
    assert a["loglik"] == b["loglik"]
    assert np.array_equal(a["x"], b["x"]) and np.array_equal(a["anc"], b["anc"])
    assert np.array_equal(a["anc"][0], np.arange(w.P))
    assert np.all(np.diff(a["anc"], axis=1) >= 0)
    assert a["anc"].min() >= 0 and a["anc"].max() < w.P
    assert np.all(a["diag"][:-1, 4] == 1) and a["diag"][-1, 4] == 0
    assert np.isfinite(a["loglik"])


def test_mixed_close_to_fp64_windkessel():
    w = W.windkessel(P=2048, T=100)
    m64, m32 = _om(w, prec=O.FP64), _om(w, prec=O.MIXED)
    kf = O.kalman_windkessel(m64, w.theta, w.y)
    d = [O.pf_run(m32, w.theta, w.y, s, w.P, w.T, want_x=False, want_anc=False)["loglik"] - kf
         for s in range(1, 9)]
    assert abs(np.mean(d)) < 1.0


def test_seed_changes_result():
    w = W.lorenz96_8(P=256, T=10)
    m = _om(w)
    a = O.pf_run(m, w.theta, w.y, 1, w.P, w.T)["loglik"]
    b = O.pf_run(m, w.theta, w.y, 2, w.P, w.T)["loglik"]
    assert a != b


def test_seed_schedule_constant_is_plain_run_and_still_converges():
    w = W.windkessel(P=1024, T=100)
    m = _om(w)
    a = O.pf_run(m, w.theta, w.y, 7, w.P, w.T)
    b = O.pf_run_sched(m, w.theta, w.y, [7] * (w.T + 1), w.P, w.T)
    assert a["loglik"] == b["loglik"] and np.array_equal(a["anc"], b["anc"])
    # a new key at every step is still a particle filter: unbiased for the
    # Kalman likelihood with the same Jensen offset as the plain runs
    kf = O.kalman_windkessel(m, w.theta, w.y)
    rng = np.random.default_rng(12)
    lls = np.array([O.pf_run_sched(m, w.theta, w.y, rng.integers(1, 2 ** 63, w.T + 1,
                                                                 dtype=np.uint64),
                                   w.P, w.T)["loglik"] for _ in range(32)])
    se = math.sqrt(lls.var(ddof=1) / 32)
    assert abs(lls.mean() - (kf - lls.var(ddof=1) / 2)) < 4 * se + 0.02


# ---- sparse observations (Sec. 5: the first four components every other step) ----
def _brute_force_sparse(theta, y, s, dt, every, flow_fn):
    """log N(y_obs; mu, Sigma) of the Euler windkessel at the observed steps only."""
    from scipy import stats
    R, C, Z, q, r, m0, s0 = theta
    a = 1.0 - dt / (R * C)
    obs = [i for i in range(1, len(y) + 1) if i % every == 0]
    K = [i * s for i in obs]
    flow = flow_fn(max(K) + 1)
    mu = np.array([a ** k * m0 + sum(a ** (k - 1 - m) * dt * flow[m] / C for m in range(k))
                   + Z * flow[k] for k in K])
    Sig = np.array([[a ** (ki + kj) * s0 ** 2 +
                     q * sum(a ** (ki - 1 - m) * a ** (kj - 1 - m) for m in range(min(ki, kj)))
                     + (r if ii == jj else 0.0) for jj, kj in enumerate(K)]
                    for ii, ki in enumerate(K)])
    return stats.multivariate_normal(mean=mu, cov=Sig).logpdf(np.array([y[i - 1] for i in obs]))


@pytest.mark.parametrize("every", [2, 3])
def test_sparse_kalman_against_joint_gaussian(every):
    theta = (1.1, 1.4, 0.04, 0.3, 3.0, 85.0, 10.0)
    m = O.model(O.WINDKESSEL, substeps=2, dt=0.01, obs_every=every)
    y = np.array([92.0, 97.0, 101.5, 99.0, 95.5, 94.0, 96.5])
    ref = _brute_force_sparse(theta, y, 2, 0.01, every,
                              lambda n: O.flow_table(400.0, 1.0, 0.01, n))
    assert O.kalman_windkessel(m, theta, y) == pytest.approx(ref, rel=1e-12, abs=1e-10)


def test_sparse_windkessel_filter_exact_and_convergent():
    w = W.windkessel(P=1024, T=100).with_(obs_every=3)
    m = _om(w)
    m.obs_every = 3
    th0 = (1.0, 1.5, 0.03, 0.0, 4.0, 90.0, 0.0)
    kf0 = O.kalman_windkessel(m, th0, w.y)
    assert O.pf_run(m, th0, w.y, 5, 64, w.T)["loglik"] == pytest.approx(kf0, rel=1e-12)
    kf = O.kalman_windkessel(m, w.theta, w.y)
    lls = np.array([O.pf_run(m, w.theta, w.y, s, w.P, w.T, want_x=False, want_anc=False)["loglik"]
                    for s in range(1, 25)])
    se = math.sqrt(lls.var(ddof=1) / len(lls))
    assert abs(lls.mean() - (kf - lls.var(ddof=1) / 2)) < 4 * se + 0.02
    r = O.pf_run(m, w.theta, w.y, 1, 256, 30)
    for i in range(1, 31):
        if i % 3:
            assert r["diag"][i - 1, 6] == 0.0 and r["diag"][i - 1, 4] == 0.0
            if i < 30:
                assert np.array_equal(r["anc"][i], np.arange(256))  # no resampling after it


def test_sparse_lorenz96_deterministic_closed_form():
    F, r = 8.0, 0.25
    th = (F, 0.0, r, 1.3, 0.0)
    w = W.lorenz96_sparse(P=16, T=20)
    m = O.model(O.LORENZ96, N=8, substeps=w.substeps, dt=w.dt, obs_every=2, obs_count=4)
    x = np.full(8, 1.3)
    ll = 0.0
    for i in range(1, w.T + 1):
        x = O.l96_rk4(x, F, w.dt, w.substeps)
        if i % 2 == 0:
            d = w.y[i - 1] - x[:4]
            ll += -0.5 * 4 * math.log(2 * math.pi * r) - 0.5 * float(np.sum(d * d)) / r
    res = O.pf_run(m, th, w.y, 9, 16, w.T)
    assert res["loglik"] == pytest.approx(ll, rel=1e-12)


# ---- the mixed-precision Lorenz '96 branch (FP32 state, RK4 and noise; FP64
# ---- residuals and weights): Sec. 2.1.2's model and observation, Algorithm 2's
# ---- propagate and weight lines, pinned without the oracle's own integrator
def _rk4_l96(x, F, dt, n):
    """Classic RK4 of dx_n/dt = (x_{n+1} - x_{n-2}) x_{n-1} - x_n + F, numpy,
    in the dtype of x (float64, or float32 with every operation rounded)."""
    t = x.dtype.type
    F, dt = t(F), t(dt)

    def f(v):
        return (np.roll(v, -1) - np.roll(v, 2)) * np.roll(v, 1) - v + F

    for _ in range(n):
        k1 = f(x)
        k2 = f(x + t(0.5) * dt * k1)
        k3 = f(x + t(0.5) * dt * k2)
        k4 = f(x + dt * k3)
        x = x + dt / t(6) * (k1 + t(2) * k2 + t(2) * k3 + k4)
    return x


def _normal32_math(seed, j, i, n, purpose=O.PURPOSE_PROP):
    """Normal number n of stream (j, i, purpose) in the FP32 layout (two
    Box-Muller pairs per Philox block from 24-bit uniforms), evaluated with
    math.log / math.cos / math.sin in double precision from the raw words."""
    w = O.philox4x32_10([j, i, (purpose << 16) | (n // 4), 0],
                        [seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF])
    pair = (n // 2) % 2
    wa, wb = int(w[2 * pair]), int(w[2 * pair + 1])
    u1 = ((wa >> 8) + 1) * 2.0 ** -24
    u2 = (wb >> 8) * 2.0 ** -24
    rho = math.sqrt(-2.0 * math.log(u1))
    return rho * (math.sin(2 * math.pi * u2) if n % 2 else math.cos(2 * math.pi * u2))


L96_MIXED_SHAPES = [
    # name, workload, observed components
    ("N=8, all components", lambda **kw: W.lorenz96_8(prec=W.MIXED, **kw), slice(0, 8)),
    ("N=40, every 2nd component", lambda **kw: W.lorenz96_large(prec=W.MIXED, **kw),
     slice(0, 40, 2)),
]


@pytest.mark.parametrize("name,factory,obs", L96_MIXED_SHAPES, ids=[s[0] for s in L96_MIXED_SHAPES])
def test_mixed_lorenz96_deterministic_closed_form(name, factory, obs):
    """q = 0, one particle: x(t_0) = m0 + s0 z (z_n the normal number n of stream
    (0, 0, INIT), recomputed from the raw Philox words; a random start, since
    a uniform one stays uniform under Lorenz '96 and would hide a misplaced
    component), then the deterministic FP32 RK4 trajectory, so the mixed
    filter's log-likelihood is the closed form sum_i sum_{n observed}
    log N(y_in; x_n(t_i), r).  The FP32 trajectory differs from the FP64 one
    by rounding only; its distance delta_i at each t_i is measured here on an
    independent float32 integration (unfused numpy), and the likelihood
    tolerance is the first-order bound sum_i sum_n (|y_in - x_n| + delta)
    delta / r with a tenfold margin on delta."""
    w = factory(P=1, T=12)
    F, r, m0, s0 = w.theta[0], w.theta[2], 1.25, 1.0
    th = (F, 0.0, r, m0, s0)
    seed = 0x5EED0
    z0 = np.array([_normal32_math(seed, 0, 0, n, O.PURPOSE_INIT) for n in range(w.N)])
    x64 = m0 + s0 * z0
    x32 = x64.astype(np.float32)
    ll, tol = 0.0, 0.0
    ny = len(range(w.N)[obs])
    for i in range(w.T):
        x64 = _rk4_l96(x64, F, w.dt, w.substeps)
        x32 = _rk4_l96(x32, F, w.dt, w.substeps)
        delta = 10.0 * float(np.max(np.abs(x32.astype(np.float64) - x64))) + 1e-5
        d = w.y[i] - x64[obs]
        ll += -0.5 * ny * math.log(2 * math.pi * r) - 0.5 * float(np.sum(d * d)) / r
        tol += float(np.sum((np.abs(d) + delta) * delta)) / r
    assert tol < 0.05  # the bound is informative: far below the effect of any slip
    res = O.pf_run(_om(w), th, w.y, seed, 1, w.T)
    assert res["status"] == O.OK
    assert abs(res["loglik"] - ll) <= tol, (res["loglik"], ll, tol)
    assert np.allclose(res["x"][:, 0], x64, rtol=0, atol=1e-3)


@pytest.mark.parametrize("name,factory,obs", L96_MIXED_SHAPES, ids=[s[0] for s in L96_MIXED_SHAPES])
def test_mixed_lorenz96_noise_placement_closed_form(name, factory, obs):
    """One particle, s0 = 0, q > 0: x(t_i) = RK4(x(t_{i-1})) + sqrt(q) z with z_n
    the normal number n of stream (j = 0, i, PROP), recomputed here from the
    raw Philox words with math.log / math.cos / math.sin (FP32 block layout);
    the filter's log-likelihood is then the closed form of Sec. 2.1.2's
    observation density at those states (one particle: weight = density).
    Tolerance: the FP32 normals agree with the double-precision ones to 2e-6
    and the FP32 RK4 with the FP64 one to the measured delta (as above), so
    the states agree to delta + 2e-6 sqrt(q); a wrong normal index, a wrong
    noise scale or a wrong observed component moves the states by about
    sqrt(q) = 0.1 per component and the likelihood by far more than the bound."""
    w = factory(P=1, T=4)
    F, q, r, m0 = w.theta[0], 0.01, w.theta[2], -0.75
    th = (F, q, r, m0, 0.0)
    seed = 0x5EED1
    x = np.full(w.N, m0)
    x32 = np.full(w.N, m0, dtype=np.float32)
    ll, tol = 0.0, 0.0
    ny = len(range(w.N)[obs])
    for i in range(1, w.T + 1):
        z = np.array([_normal32_math(seed, 0, i, n) for n in range(w.N)])
        x64_next = _rk4_l96(x, F, w.dt, w.substeps)
        x32 = _rk4_l96(x32, F, w.dt, w.substeps)
        delta = 10.0 * float(np.max(np.abs(x32.astype(np.float64) - x64_next))) + 1e-5
        x = x64_next + math.sqrt(q) * z
        x32 = (x32 + np.float32(math.sqrt(q)) * z.astype(np.float32)).astype(np.float32)
        d = w.y[i - 1] - x[obs]
        ll += -0.5 * ny * math.log(2 * math.pi * r) - 0.5 * float(np.sum(d * d)) / r
        tol += float(np.sum((np.abs(d) + delta) * delta)) / r
    assert tol < 0.05
    res = O.pf_run(_om(w), th, w.y, seed, 1, w.T)
    assert res["status"] == O.OK
    assert abs(res["loglik"] - ll) <= tol, (res["loglik"], ll, tol)
    assert np.allclose(res["x"][:, 0], x, rtol=0, atol=1e-3)


def test_mixed_lorenz96_unbiased_against_fp64():
    """Over 64 seeds, the mixed filter's log-likelihood minus the FP64
    filter's on the same seeds has mean zero within four standard errors
    (FP32 propagation changes the estimator by rounding, not systematically)."""
    w = W.lorenz96_8(P=512, T=40)
    m64, m32 = _om(w, prec=O.FP64), _om(w, prec=O.MIXED)
    d = np.array([O.pf_run(m32, w.theta, w.y, s, w.P, w.T, want_x=False, want_anc=False,
                           want_diag=False)["loglik"] -
                  O.pf_run(m64, w.theta, w.y, s, w.P, w.T, want_x=False, want_anc=False,
                           want_diag=False)["loglik"] for s in range(1, 65)])
    se = d.std(ddof=1) / math.sqrt(len(d))
    assert abs(d.mean()) < 4 * se + 1e-9, (d.mean(), se)
    assert np.all(np.isfinite(d))


@pytest.mark.parametrize("prec", [O.FP64, O.MIXED])
@pytest.mark.parametrize("thr", [1.0, 0.5])
def test_teacher_forced_step_chain_is_the_run(prec, thr):
    """The oracle's one-step entry (the reference of the teacher-forced GPU
    checks) chained on its own outputs reproduces the whole run: the same
    states, ancestors and, summed, the same log-likelihood.  With adaptive
    resampling the chain is only followed while every step resamples (a
    step's carried weights are not part of the one-step state)."""
    w = W.lorenz96_8(P=300, T=12, prec=prec, ess_threshold=thr)
    m = _om(w)
    full = O.pf_run_ex(m, w.theta, w.y, 5, w.P, w.T)
    run = O.pf_run(m, w.theta, w.y, 5, w.P, w.T)
    x, anc, ll = full["xhist"][0], None, 0.0
    for i in range(1, w.T + 1):
        r = O.pf_step(m, w.theta, w.y, 5, w.P, w.T, i, x, anc)
        assert r["status"] == O.OK
        assert np.array_equal(r["x"], full["xhist"][i])
        ll += r["incr"]
        assert r["incr"] == run["diag"][i - 1, 6]
        if i < w.T:
            assert np.array_equal(r["anc_next"], full["anc"][i])
        x, anc = r["x"], r["anc_next"]
        if run["diag"][i - 1, 4] == 0:
            break  # carried weights: the chain stops here
    else:
        assert ll == pytest.approx(run["loglik"], rel=1e-13)
