"""Pins of the oracle's log-sum-exp and systematic resampling: closed-form
weight patterns, math.fsum, exact rational arithmetic and brute-force
enumeration of the offspring counts over the uniform u on tiny P."""
from fractions import Fraction
import math

import numpy as np
import pytest

import oracle as O


def test_lse_equal_weights():
    for P in (1, 7, 1024):
        M, S, Q = O.lse(np.full(P, -3.25))
        assert M == -3.25 and S == P and Q == P
        assert S * S / Q == P  # ESS = P


def test_lse_one_hot():
    ell = np.full(100, -np.inf)
    ell[37] = -5.0
    M, S, Q = O.lse(ell)
    assert (M, S, Q) == (-5.0, 1.0, 1.0)  # ESS = 1


def test_lse_all_minus_inf():
    M, S, Q = O.lse(np.full(10, -np.inf))
    assert M == -np.inf and S == 0.0 and Q == 0.0


def test_lse_shift_invariance_and_fsum():
    rng = np.random.default_rng(4)
    ell = rng.normal(-20, 5, 5000)
    M, S, Q = O.lse(ell)
    w = [math.exp(e - M) for e in ell]
    assert S == pytest.approx(math.fsum(w), rel=2 ** -52)
    assert Q == pytest.approx(math.fsum(v * v for v in w), rel=2 ** -52)
    M2, S2, Q2 = O.lse(ell + 1024.0)  # adds exactly for these magnitudes
    assert M2 == M + 1024.0 and S2 == pytest.approx(S, rel=1e-15)


def _exact_ancestors(w_exact, u):
    P = len(w_exact)
    C = np.cumsum([Fraction(x) for x in w_exact]).tolist()
    S = C[-1]
    out = []
    for j in range(P):
        tau = (j + Fraction(u)) * S / P
        k = next((k for k in range(P) if C[k] > tau), P - 1)
        out.append(k)
    return out


def test_systematic_zero_one_weights_exact():
    rng = np.random.default_rng(5)
    for trial in range(200):
        P = int(rng.integers(1, 40))
        mask = rng.random(P) < 0.4
        if not mask.any():
            mask[rng.integers(0, P)] = True
        ell = np.where(mask, 0.0, -np.inf)
        u = float(rng.random())
        anc, near = O.systematic(ell, u)
        if near == 0:
            assert anc.tolist() == _exact_ancestors(mask.astype(float), u)
        assert np.all(mask[anc])  # zero-weight particles are never chosen
        assert np.all(np.diff(anc) >= 0)


def test_systematic_matches_exact_rational_on_random_weights():
    rng = np.random.default_rng(6)
    for trial in range(200):
        P = int(rng.integers(2, 64))
        ell = rng.normal(0, 2, P)
        u = float(rng.random())
        anc, near = O.systematic(ell, u)
        M = ell.max()
        w = [math.exp(e - M) for e in ell]
        if near == 0:
            assert anc.tolist() == _exact_ancestors(w, u)


@pytest.mark.parametrize("P", [1, 2, 3, 5, 8])
def test_systematic_offspring_brute_force(P):
    """Enumerate every interval of u between breakpoints frac(P C_k / S):
    offspring o_k is constant there, must lie in {floor(P wbar), ceil(P wbar)},
    sums to P, and integrates over u to exactly P wbar_k (unbiasedness)."""
    rng = np.random.default_rng(100 + P)
    for trial in range(30):
        ell = rng.normal(0, 1.5, P)
        M = ell.max()
        w = [Fraction(math.exp(e - M)) for e in ell]
        S = sum(w)
        C = np.cumsum(w).tolist()
        brk = sorted({0.0, 1.0} | {float((P * c / S) % 1) for c in C})
        integral = [Fraction(0)] * P
        for a, b in zip(brk[:-1], brk[1:]):
            if b - a < 1e-9:
                continue
            mid = 0.5 * (a + b)
            anc, near = O.systematic(ell, mid)
            assert near == 0
            o = np.bincount(anc, minlength=P)
            assert o.sum() == P
            for k in range(P):
                pw = P * w[k] / S
                assert math.floor(pw) <= o[k] <= math.ceil(pw)
                integral[k] += Fraction(b - a) * int(o[k])
        for k in range(P):
            assert float(integral[k]) == pytest.approx(float(P * w[k] / S), abs=1e-8)


# ---- stratified and multinomial resampling --------------------------------
def _uniform(seed, j, i, blk, open_zero=False):
    w = O.philox4x32_10([j, i, (O.PURPOSE_RESAMPLE << 16) | blk, 0],
                        [seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF])
    v = ((int(w[1]) << 32) | int(w[0])) >> 11
    return Fraction(v + (1 if open_zero else 0), 1 << 53)




def test_stratified_matches_exact_rational():
    rng = np.random.default_rng(7)
    for trial in range(150):
        P = int(rng.integers(1, 48))
        ell = rng.normal(0, 2, P)
        seed, i = int(rng.integers(1, 2 ** 40)), int(rng.integers(1, 50))
        anc, near = O.resample(ell, O.RESAMPLE_STRATIFIED, seed, i)
        M = ell.max()
        w = [Fraction(math.exp(e - M)) for e in ell]
        C = np.cumsum(w).tolist()
        S = C[-1]
        if near:
            continue
        ref = []
        for j in range(P):
            tau = (j + _uniform(seed, j, i, 1)) * S / P
            ref.append(next((k for k in range(P) if C[k] > tau), P - 1))
        assert anc.tolist() == ref


def test_multinomial_matches_order_statistics_of_exponential_spacings():
    rng = np.random.default_rng(8)
    for trial in range(100):
        P = int(rng.integers(1, 40))
        ell = rng.normal(0, 2, P)
        seed, i = int(rng.integers(1, 2 ** 40)), int(rng.integers(1, 50))
        anc, near = O.resample(ell, O.RESAMPLE_MULTINOMIAL, seed, i)
        e = [-math.log(float(_uniform(seed, l, i, 2, open_zero=True))) for l in range(P + 1)]
        G = [math.fsum(e[:j + 1]) for j in range(P + 1)]
        M = ell.max()
        w = [math.exp(x - M) for x in ell]
        C = [math.fsum(w[:k + 1]) for k in range(P)]
        targets = [G[j] / G[P] * C[-1] for j in range(P)]
        gap = min(abs(t - c) for t in targets for c in C) / C[-1]
        if near or gap < 1e-12:  # the oracle's own log is within 2 ulp of math.log
            continue
        ref = [next((k for k in range(P) if C[k] > t), P - 1) for t in targets]
        assert anc.tolist() == ref
        assert np.all(np.diff(anc) >= 0)


@pytest.mark.parametrize("kind", [O.RESAMPLE_STRATIFIED, O.RESAMPLE_MULTINOMIAL])
def test_offspring_distribution(kind):
    """Unbiased offspring counts for both; multinomial variance P w (1 - w);
    stratified counts within one of P w and never more variable."""
    P = 6
    ell = np.log(np.array([0.02, 0.3, 0.05, 0.33, 0.1, 0.2]))
    wbar = np.exp(ell) / np.exp(ell).sum()
    n = 4000
    counts = np.zeros((n, P))
    for s in range(n):
        anc, _ = O.resample(ell, kind, 1000 + s, 3)
        counts[s] = np.bincount(anc, minlength=P)
    assert np.all(counts.sum(axis=1) == P)
    mean, var = counts.mean(axis=0), counts.var(axis=0)
    se = np.sqrt(P * wbar * (1 - wbar) / n)
    assert np.all(np.abs(mean - P * wbar) < 5 * se)
    if kind == O.RESAMPLE_MULTINOMIAL:
        assert np.all(np.abs(var / (P * wbar * (1 - wbar)) - 1) < 0.15)
        # the smallest weight still draws: P(o >= 1) = 1 - (1 - w)^P
        p1 = 1 - (1 - wbar[0]) ** P
        assert abs(np.mean(counts[:, 0] >= 1) - p1) < 5 * math.sqrt(p1 * (1 - p1) / n)
    else:
        assert np.all(counts >= np.floor(P * wbar) - 1) and np.all(counts <= np.ceil(P * wbar) + 1)
        assert np.all(var <= P * wbar * (1 - wbar) + 0.02)


@pytest.mark.parametrize("kind", [O.RESAMPLE_STRATIFIED, O.RESAMPLE_MULTINOMIAL])
def test_filter_with_other_resamplers_converges_to_kalman(kind):
    import workloads as W
    w = W.windkessel(P=1024, T=100)
    m = O.model(w.kind, dt=w.dt, resampler=kind)
    kf = O.kalman_windkessel(m, w.theta, w.y)
    lls = np.array([O.pf_run(m, w.theta, w.y, s, w.P, w.T, want_x=False, want_anc=False,
                             want_diag=False)["loglik"] for s in range(1, 25)])
    se = math.sqrt(lls.var(ddof=1) / len(lls))
    assert abs(lls.mean() - (kf - lls.var(ddof=1) / 2)) < 4 * se + 0.02


def _chi2_pvalue(obs, expected):
    from scipy import stats
    obs, expected = np.asarray(obs, float), np.asarray(expected, float)
    chi2 = float(np.sum((obs - expected) ** 2 / expected))
    return stats.chi2.sf(chi2, len(obs) - 1)


@pytest.mark.parametrize("seed", [11, 12, 13])
def test_multinomial_offspring_chi2_at_large_P(seed):
    """P = 2^16 (Algorithm 2's multinomial ancestor draw): one draw's offspring
    counts o_k against Multinomial(P, wbar).  Consecutive particles are pooled
    into bins of expected count >= 64 and Pearson's chi^2 (df = bins - 1) must
    not reject at 1e-6; with equal weights the histogram of o_k over 0..4 and
    >= 5 must match Binomial(P, 1/P) the same way (the deterministic schemes
    would give every particle exactly one offspring)."""
    from scipy import stats
    P = 1 << 16
    rng = np.random.default_rng(seed)
    ell = rng.normal(0, 1.5, P)
    anc, _ = O.resample(ell, O.RESAMPLE_MULTINOMIAL, 0xC0FFEE + seed, 7)
    o = np.bincount(anc, minlength=P)
    assert o.sum() == P and np.all(np.diff(anc) >= 0)
    wbar = np.exp(ell - ell.max())
    wbar /= wbar.sum()
    obs, exp_, acc_o, acc_e = [], [], 0, 0.0
    for k in range(P):
        acc_o += int(o[k])
        acc_e += P * wbar[k]
        if acc_e >= 64:
            obs.append(acc_o)
            exp_.append(acc_e)
            acc_o, acc_e = 0, 0.0
    obs[-1] += acc_o
    exp_[-1] += acc_e
    assert len(obs) > 500
    assert _chi2_pvalue(obs, exp_) > 1e-6
    # equal weights: counts ~ Binomial(P, 1/P)
    anc, _ = O.resample(np.zeros(P), O.RESAMPLE_MULTINOMIAL, 0xBEEF + seed, 3)
    o = np.bincount(anc, minlength=P)
    hist = [int(np.sum(o == c)) for c in range(5)] + [int(np.sum(o >= 5))]
    pmf = [stats.binom.pmf(c, P, 1.0 / P) for c in range(5)]
    pmf.append(1.0 - sum(pmf))
    assert _chi2_pvalue(hist, [P * p for p in pmf]) > 1e-6
    assert abs(hist[0] / P - math.exp(-1)) < 0.01
