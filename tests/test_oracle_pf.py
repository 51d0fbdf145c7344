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
