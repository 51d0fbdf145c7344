"""Pins of the oracle's paper-exact model variants: its own exponential
against libm; the exact windkessel (exponential decay, noise on the flow)
against a brute-force joint Gaussian and its Kalman likelihood; Lorenz '96
with the Wiener increment inside RK4 against the deterministic RK4 (zero
noise) and the energy balance of the Ito equation (F = 0)."""
import math

import numpy as np
import pytest
from scipy import stats

import oracle as O
import workloads as W


def _ulp(a, ref):
    return abs(a - ref) / np.spacing(abs(ref)) if ref != 0 else abs(a)


def test_exp_against_libm_and_special_values():
    assert O.exp(0.0) == 1.0
    assert O.exp(1000.0) == math.inf and O.exp(-1000.0) == 0.0 and math.isnan(O.exp(math.nan))
    rng = np.random.default_rng(21)
    xs = np.concatenate([rng.uniform(-700, 700, 20000), rng.uniform(-1, 1, 20000),
                         rng.uniform(-1e-6, 1e-6, 2000), [-0.5 * math.log(2), 0.5 * math.log(2)]])
    worst = max(_ulp(O.exp(float(x)), math.exp(x)) for x in xs)
    assert worst <= 2.0, worst
    for k in range(-60, 60, 7):  # near the reduction's breakpoints k ln2
        x = k * math.log(2.0)
        for t in (x, np.nextafter(x, -np.inf), np.nextafter(x, np.inf)):
            assert _ulp(O.exp(float(t)), math.exp(t)) <= 2.0


def _brute_force_exact(theta, y, s, dt, flow):
    """log N(y; mu, Sigma) of the exact windkessel written out as one joint Gaussian."""
    R, C, Z, sig2, r, m0, s0 = theta
    a = math.exp(-dt / (R * C))
    b = R * (1.0 - a)
    qv = b * b * dt * dt * sig2
    T = len(y)
    K = [i * s for i in range(1, T + 1)]
    mu = np.array([a ** k * m0 + sum(a ** (k - 1 - m) * b * flow[m] for m in range(k)) + Z * flow[k]
                   for k in K])
    Sig = np.array([[a ** (ki + kj) * s0 ** 2 +
                     qv * sum(a ** (ki - 1 - m) * a ** (kj - 1 - m) for m in range(min(ki, kj)))
                     + (r if ii == jj else 0.0) for jj, kj in enumerate(K)]
                    for ii, ki in enumerate(K)])
    return stats.multivariate_normal(mean=mu, cov=Sig).logpdf(y)


@pytest.mark.parametrize("T,s", [(1, 1), (3, 1), (3, 4)])
def test_exact_windkessel_kalman_against_joint_gaussian(T, s):
    theta = (1.1, 1.4, 0.04, 9.0e4, 3.0, 85.0, 10.0)
    m = O.model(O.WINDKESSEL_EXP, substeps=s, dt=0.01)
    y = np.array([92.0, 97.0, 101.5][:T])
    flow = O.flow_table(400.0, 1.0, 0.01, T * s + 1)
    ref = _brute_force_exact(theta, y, s, 0.01, flow)
    assert O.kalman_windkessel(m, theta, y) == pytest.approx(ref, rel=1e-12, abs=1e-10)


def test_exact_windkessel_filter_noiseless_and_convergent():
    w = W.windkessel_exact(P=1024, T=100, theta=(1.0, 1.5, 0.03, 4.0e4, 4.0, 90.0, 15.0))
    m = O.model(w.kind, dt=w.dt)
    th0 = (1.0, 1.5, 0.03, 0.0, 4.0, 90.0, 0.0)
    kf0 = O.kalman_windkessel(m, th0, w.y)
    for P in (1, 64):
        assert O.pf_run(m, th0, w.y, 3, P, w.T)["loglik"] == pytest.approx(kf0, rel=1e-12)
    kf = O.kalman_windkessel(m, w.theta, w.y)
    lls = np.array([O.pf_run(m, w.theta, w.y, s, w.P, w.T, want_x=False, want_anc=False)["loglik"]
                    for s in range(1, 25)])
    se = math.sqrt(lls.var(ddof=1) / len(lls))
    assert abs(lls.mean() - (kf - lls.var(ddof=1) / 2)) < 4 * se + 0.02
    # FP32 state: close to the FP64 filter on the same seeds
    m32 = O.model(w.kind, dt=w.dt, prec=O.MIXED)
    d = [O.pf_run(m32, w.theta, w.y, s, w.P, w.T, want_x=False, want_anc=False)["loglik"] - kf
         for s in range(1, 9)]
    assert abs(np.mean(d)) < 1.0


def test_sde_lorenz96_zero_noise_is_deterministic_rk4():
    F, r = 8.0, 0.25
    w = W.lorenz96_sde(P=8, T=20)
    m = O.model(w.kind, N=8, substeps=w.substeps, dt=w.dt)
    th = (F, 0.0, r, 1.3, 0.0)
    res = O.pf_run(m, th, w.y, 9, 8, w.T)
    x = np.full(8, 1.3)
    ll = 0.0
    for i in range(w.T):
        x = O.l96_rk4(x, F, w.dt, w.substeps)
        d = w.y[i] - x
        ll += -0.5 * 8 * math.log(2 * math.pi * r) - 0.5 * float(np.sum(d * d)) / r
    assert np.array_equal(res["x"], np.repeat(x[:, None], 8, axis=1))
    assert res["loglik"] == pytest.approx(ll, rel=1e-12)


@pytest.mark.parametrize("prec", [O.FP64, O.MIXED])
def test_sde_lorenz96_energy_balance(prec):
    """F = 0: the advection conserves sum x^2, so E[sum x^2] obeys
    d/dt E = -2 E + N sigma2 (Ito); from x = 0 it is N sigma2 (1 - e^{-2t}) / 2."""
    N, sig2, dt, s, T = 8, 1.0, 0.01, 10, 10  # t = 1
    m = O.model(O.LORENZ96_SDE, N=N, substeps=s, dt=dt, prec=prec, ess_threshold=0.0)
    th = (0.0, sig2, 1e12, 0.0, 0.0)  # uninformative observations, never resample
    P = 8192
    x = O.pf_run(m, th, np.zeros((T, N)), 4, P, T, want_anc=False, want_diag=False)["x"]
    e = (x ** 2).sum(axis=0)
    ref = N * sig2 * (1 - math.exp(-2.0)) / 2
    se = e.std(ddof=1) / math.sqrt(P)
    assert abs(e.mean() - ref) < 4 * se + 0.02 * ref, (e.mean(), ref, se)
