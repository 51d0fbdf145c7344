"""Pins of the oracle's SMC^2 (Algorithm 4).  With the exact Kalman
likelihood increments of the linear-Gaussian windkessel the sampler is an
exact-likelihood SMC over the parameters, so its evidence and posterior must
match quadrature of prior x Kalman likelihood; with particle filters the
evidence estimate must stay unbiased around the same value."""
import math

import numpy as np
import pytest
from scipy import stats

import oracle as O
import workloads as W

INF = math.inf
FIXED = (O.PRIOR_FIXED, O.PROPOSE_FIXED)


def _quadrature(m, w, T, d, grid, prior, f=lambda v: v):
    lp = []
    for v in grid:
        th = list(w.theta)
        th[d] = v
        lp.append(O.kalman_windkessel(m, th, w.y[:T]))
    lp = np.array(lp) + prior.logpdf(grid)
    M = lp.max()
    p = np.exp(lp - M)
    log_ev = M + math.log(np.trapezoid(p, grid))
    p = p * np.gradient(grid)  # quadrature weights of a possibly non-uniform grid
    p /= p.sum()
    g = f(grid)  # moments of f(theta_d) (log for a heavy-tailed variance)
    mean = (p * g).sum()
    sd = math.sqrt((p * (g - mean) ** 2).sum())
    return log_ev, mean, sd


CASES = [
    # component, prior / proposal, quadrature grid, prior distribution, compared moment
    ("Z", 2, (O.PRIOR_GAMMA, O.PROPOSE_TRUNC_GAUSSIAN, 2.0, 0.03, 0.005, 0.0, INF),
     np.linspace(1e-5, 0.4, 8001), stats.gamma(2.0, scale=0.03), lambda v: v),
    ("q", 3, (O.PRIOR_INV_GAMMA, O.PROPOSE_INV_GAMMA, 2.0, 0.01, 2.0, 3.0),
     np.geomspace(1e-6, 50.0, 20001), stats.invgamma(2.0, scale=0.01), np.log),
]


@pytest.mark.parametrize("name,d,param,grid,prior,f", CASES, ids=[c[0] for c in CASES])
def test_exact_likelihood_smc2_matches_quadrature(name, d, param, grid, prior, f):
    w = W.windkessel(P=16, T=30)
    m = O.model(w.kind, dt=w.dt)
    spec = [FIXED] * 7
    spec[d] = param
    log_ev, mean, sd = _quadrature(m, w, 30, d, grid, prior, f)
    evs, means, sds = [], [], []
    for seed in range(1, 5):
        r = O.smc2(m, w.y, 16, 30, O.LIK_KALMAN, 256, spec, w.theta, seed)
        assert r["status"] == O.OK and r["near"].sum() == 0
        wt = np.exp(r["logv"] - r["logv"].max())
        x = f(r["theta"][:, d])
        mu = np.average(x, weights=wt)
        evs.append(r["log_evidence"])
        means.append(mu)
        sds.append(math.sqrt(np.average((x - mu) ** 2, weights=wt)))
        assert np.all(r["accepted"] > 0)
    se = np.std(evs, ddof=1) / 2.0
    assert abs(np.mean(evs) - log_ev) < 4 * se + 0.05, (np.mean(evs), log_ev, se)
    assert abs(np.mean(means) - mean) < 0.25 * sd, (np.mean(means), mean, sd)
    assert 0.7 < np.mean(sds) / sd < 1.4


def test_particle_filter_smc2_evidence_near_exact():
    w = W.windkessel(P=256, T=20)
    m = O.model(w.kind, dt=w.dt)
    spec = [FIXED] * 7
    spec[2] = CASES[0][2]
    log_ev, _, _ = _quadrature(m, w, 20, 2, CASES[0][3], CASES[0][4])
    evs = [O.smc2(m, w.y, 256, 20, O.LIK_PF, 32, spec, w.theta, s)["log_evidence"]
           for s in (1, 2)]
    assert abs(np.mean(evs) - log_ev) < 1.5, (evs, log_ev)


def test_smc2_reproducible_and_thread_invariant():
    w = W.lorenz96_8(P=64, T=8)
    m = O.model(w.kind, N=8, substeps=w.substeps, dt=w.dt)
    spec = [(O.PRIOR_UNIFORM, O.PROPOSE_TRUNC_GAUSSIAN, 8.0, 12.0, 0.1, 8.0, 12.0),
            (O.PRIOR_INV_GAMMA, O.PROPOSE_INV_GAMMA, 2.0, 0.25, 2.0, 3.0), FIXED, FIXED, FIXED]
    a = O.smc2(m, w.y, 64, 8, O.LIK_PF, 12, spec, w.theta, 3, nthreads=1)
    b = O.smc2(m, w.y, 64, 8, O.LIK_PF, 12, spec, w.theta, 3, nthreads=4)
    assert a["status"] == O.OK
    assert np.array_equal(a["theta"], b["theta"]) and a["log_evidence"] == b["log_evidence"]
    assert np.all((a["theta"][:, 0] >= 8.0) & (a["theta"][:, 0] <= 12.0))
    assert np.all(a["theta"][:, 1] > 0.0)
    assert np.isfinite(a["log_evidence"])


def test_smc2_rejects_non_integer_prior_shape():
    w = W.windkessel(P=16, T=4)
    m = O.model(w.kind, dt=w.dt)
    spec = [FIXED] * 7
    spec[0] = (O.PRIOR_GAMMA, O.PROPOSE_TRUNC_GAUSSIAN, 2.5, 0.9, 0.03, 0.0, INF)
    assert O.smc2(m, w.y, 16, 4, O.LIK_KALMAN, 8, spec, w.theta, 1)["status"] == O.EINVAL
