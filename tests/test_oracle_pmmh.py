"""Pins of the oracle's marginal Metropolis-Hastings (Algorithm 3, Eq. mh):
prior densities and proposal draws against scipy's distributions, the
Hastings correction against scipy's log densities, prior-only chains that
must sample the prior (a dropped correction term moves them off it), and
chains with the exact Kalman likelihood that must reproduce the posterior
computed on a grid."""
import math

import numpy as np
import pytest
from scipy import stats

import oracle as O
import workloads as W

INF = float("inf")
F_UNIFORM = (O.PRIOR_UNIFORM, O.PROPOSE_TRUNC_GAUSSIAN, 8.0, 12.0, 0.5, 8.0, 12.0)
Q_INVGAMMA = (O.PRIOR_INV_GAMMA, O.PROPOSE_INV_GAMMA, 2.0, 0.25, 2.0, 3.0)
FIXED = (O.PRIOR_FIXED, O.PROPOSE_FIXED)


def test_log_prior_against_scipy():
    spec = [(O.PRIOR_GAMMA, 0, 2.0, 0.9), (O.PRIOR_GAMMA, 0, 2.0, 1.5),
            (O.PRIOR_UNIFORM, 0, 8.0, 12.0), (O.PRIOR_INV_GAMMA, 0, 2.0, 25.0),
            (O.PRIOR_GAUSSIAN, 0, 90.0, 15.0), FIXED]
    rng = np.random.default_rng(3)
    for _ in range(50):
        th = [rng.gamma(2, 0.9), rng.gamma(2, 1.5), rng.uniform(8, 12),
              stats.invgamma(2, scale=25).rvs(random_state=rng), rng.normal(90, 15), 7.0]
        ref = (stats.gamma(2, scale=0.9).logpdf(th[0]) + stats.gamma(2, scale=1.5).logpdf(th[1])
               + stats.uniform(8, 4).logpdf(th[2]) + stats.invgamma(2, scale=25).logpdf(th[3])
               + stats.norm(90, 15).logpdf(th[4]))
        assert O.log_prior(spec, th) == pytest.approx(ref, rel=1e-12, abs=1e-12)
    assert O.log_prior(spec, [-1.0, 1, 9, 1, 0, 0]) == -INF
    assert O.log_prior(spec, [1.0, 1, 12.5, 1, 0, 0]) == -INF


def _draws(spec, theta, n, d):
    out, lqr = [], []
    for i in range(n):
        t, l = O.propose(spec, theta, 77, i % 13, i)
        out.append(t[d])
        lqr.append(l)
    return np.array(out), np.array(lqr)


@pytest.mark.parametrize("x", [8.05, 10.0, 11.9])
def test_truncated_gaussian_proposal_distribution_and_correction(x):
    spec = [F_UNIFORM, FIXED]
    xs, lqr = _draws(spec, [x, 0.1], 4000, 0)
    dist = stats.truncnorm((8.0 - x) / 0.5, (12.0 - x) / 0.5, loc=x, scale=0.5)
    assert np.all((xs >= 8.0) & (xs <= 12.0))
    assert stats.kstest(xs, dist.cdf).pvalue > 1e-3
    for xn, l in zip(xs[:200], lqr[:200]):
        back = stats.truncnorm((8.0 - xn) / 0.5, (12.0 - xn) / 0.5, loc=xn, scale=0.5)
        ref = back.logpdf(x) - dist.logpdf(xn)
        assert l == pytest.approx(ref, abs=1e-10)


def test_inverse_gamma_proposal_distribution_and_correction():
    spec = [FIXED, Q_INVGAMMA]
    x = 0.1
    xs, lqr = _draws(spec, [9.0, x], 4000, 1)
    dist = stats.invgamma(2.0, scale=3.0 * x)
    assert stats.kstest(xs, dist.cdf).pvalue > 1e-3
    for xn, l in zip(xs[:200], lqr[:200]):
        ref = stats.invgamma(2.0, scale=3.0 * xn).logpdf(x) - dist.logpdf(xn)
        assert l == pytest.approx(ref, rel=1e-11, abs=1e-11)


def _ecdf_check(chains, cdf_points, cdf_values, nbatch=40):
    """Empirical CDF of the pooled chains against exact values; the error bar
    comes from batch means of each chain."""
    nc, n = chains.shape
    b = n // nbatch
    for x, p in zip(cdf_points, cdf_values):
        ind = (chains[:, :b * nbatch] <= x).astype(float)
        bm = ind.reshape(nc, nbatch, b).mean(axis=2).ravel()
        se = bm.std(ddof=1) / math.sqrt(len(bm))
        assert abs(bm.mean() - p) < 5 * se + 0.005, (x, bm.mean(), p, se)


def test_prior_only_chains_sample_the_prior_lorenz96():
    w = W.lorenz96_8(P=16, T=5)
    m = O.model(w.kind, N=w.N, substeps=w.substeps, dt=w.dt)
    spec = [F_UNIFORM, Q_INVGAMMA, FIXED, FIXED, FIXED]
    th0 = np.tile(np.array(w.theta, dtype=float), (8, 1))
    r = O.pmmh(m, w.y, 16, w.T, O.LIK_NONE, spec, th0, 6000, 5)
    assert r["status"] == O.OK
    F = r["samples"][1000:, :, 0].T
    q = r["samples"][1000:, :, 1].T
    pts = [8.1, 8.25, 9.0, 10.0, 11.0, 11.75, 11.9]
    _ecdf_check(F, pts, [(p - 8.0) / 4.0 for p in pts])
    ig = stats.invgamma(2.0, scale=0.25)
    qs = [0.05, 0.25, 0.5, 0.75, 0.95]
    _ecdf_check(q, ig.ppf(qs), qs)
    assert np.all(r["samples"][:, :, 2:] == th0[None, :, 2:])


def test_prior_only_chains_sample_the_prior_windkessel():
    w = W.windkessel(P=16, T=5)
    m = O.model(w.kind, dt=w.dt)
    spec = [(O.PRIOR_GAMMA, O.PROPOSE_TRUNC_GAUSSIAN, 2.0, 0.9, 0.5, 0.0, INF),
            (O.PRIOR_GAUSSIAN, O.PROPOSE_TRUNC_GAUSSIAN, 1.5, 0.3, 0.25, -INF, INF),
            FIXED, FIXED, FIXED, FIXED, FIXED]
    th0 = np.tile(np.array(w.theta, dtype=float), (8, 1))
    r = O.pmmh(m, w.y, 16, w.T, O.LIK_NONE, spec, th0, 6000, 6)
    R = r["samples"][1000:, :, 0].T
    C = r["samples"][1000:, :, 1].T
    g = stats.gamma(2.0, scale=0.9)
    qs = [0.02, 0.1, 0.25, 0.5, 0.75, 0.95]
    _ecdf_check(R, g.ppf(qs), qs)
    n = stats.norm(1.5, 0.3)
    _ecdf_check(C, n.ppf(qs), qs)


def test_kalman_likelihood_chains_reproduce_the_grid_posterior():
    """Exact likelihood (Algorithm 1): the chain targets p(R, Z | y) exactly;
    compare its marginal means and sds with a 2-D grid of prior x Kalman."""
    w = W.windkessel(P=16, T=60)
    m = O.model(w.kind, dt=w.dt)
    prior_R, prior_Z = stats.gamma(2.0, scale=0.9), stats.gamma(2.0, scale=0.03)
    spec = [(O.PRIOR_GAMMA, O.PROPOSE_TRUNC_GAUSSIAN, 2.0, 0.9, 0.03, 0.0, INF), FIXED,
            (O.PRIOR_GAMMA, O.PROPOSE_TRUNC_GAUSSIAN, 2.0, 0.03, 0.002, 0.0, INF),
            FIXED, FIXED, FIXED, FIXED]
    th0 = np.tile(np.array(w.theta, dtype=float), (6, 1))
    r = O.pmmh(m, w.y, 16, w.T, O.LIK_KALMAN, spec, th0, 5000, 8)
    assert r["status"] == O.OK
    # grid posterior
    Rg = np.linspace(0.80, 1.25, 121)
    Zg = np.linspace(0.0, 0.08, 121)[1:]
    lp = np.zeros((len(Rg), len(Zg)))
    for a, R in enumerate(Rg):
        for b, Z in enumerate(Zg):
            th = list(w.theta)
            th[0], th[2] = R, Z
            lp[a, b] = O.kalman_windkessel(m, th, w.y) + prior_R.logpdf(R) + prior_Z.logpdf(Z)
    p = np.exp(lp - lp.max())
    p /= p.sum()
    assert p[0, :].sum() + p[-1, :].sum() + p[:, -1].sum() < 1e-6  # grid covers the mass
    mR, mZ = (p.sum(1) * Rg).sum(), (p.sum(0) * Zg).sum()
    sR = math.sqrt((p.sum(1) * (Rg - mR) ** 2).sum())
    sZ = math.sqrt((p.sum(0) * (Zg - mZ) ** 2).sum())
    s = r["samples"][1000:]
    for d, mu, sd in ((0, mR, sR), (2, mZ, sZ)):
        x = s[:, :, d].T  # chains x iterations
        bm = x[:, :4000].reshape(x.shape[0], 40, 100).mean(axis=2).ravel()
        se = bm.std(ddof=1) / math.sqrt(len(bm))
        assert abs(x.mean() - mu) < 5 * se + 1e-3 * sd, (d, x.mean(), mu, se)
        assert 0.8 < x.std() / sd < 1.25
    assert np.all(r["accepted"] > 500)


def test_pmmh_with_particle_filter_runs_and_is_reproducible():
    w = W.windkessel(P=128, T=30)
    m = O.model(w.kind, dt=w.dt)
    spec = [(O.PRIOR_GAMMA, O.PROPOSE_TRUNC_GAUSSIAN, 2.0, 0.9, 0.03, 0.0, INF), FIXED,
            (O.PRIOR_GAMMA, O.PROPOSE_TRUNC_GAUSSIAN, 2.0, 0.03, 0.002, 0.0, INF),
            FIXED, FIXED, FIXED, FIXED]
    th0 = np.tile(np.array(w.theta, dtype=float), (3, 1))
    a = O.pmmh(m, w.y, 128, w.T, O.LIK_PF, spec, th0, 20, 9)
    b = O.pmmh(m, w.y, 128, w.T, O.LIK_PF, spec, th0, 20, 9, nthreads=1)
    assert np.array_equal(a["samples"], b["samples"]) and np.array_equal(a["logliks"], b["logliks"])
    # each recorded log-likelihood is the filter's at the recorded parameters:
    # iteration 0 runs theta0 with the key of block (chain, 0, purpose 5, 1)
    for c in range(3):
        wds = O.philox4x32_10([c, 0, O.PURPOSE_PMMH << 16 | 1, 0], [9, 0])
        key = (int(wds[1]) << 32) | int(wds[0])
        ll = O.pf_run(m, th0[c], w.y, key, 128, w.T, want_x=False, want_anc=False)["loglik"]
        assert a["logliks"][0, c] == ll
    assert np.all(np.isfinite(a["logliks"]))
