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
