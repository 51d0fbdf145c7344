"""Pins of the oracle's model pieces: the windkessel input table (closed form),
Lorenz '96 RK4 (invariants, convergence order, scipy's integrator) and the
scalar Kalman filter (brute-force joint Gaussian)."""
import math

import numpy as np
import pytest
from scipy import integrate, stats

import oracle as O
import workloads as W


def test_flow_table_closed_form():
    dt, n = 0.01, 350
    got = O.flow_table(400.0, 1.0, dt, n)
    t = np.arange(n) * dt
    fr = t - np.floor(t)
    ref = np.where(fr < 0.5, 400.0 * np.sin(2 * np.pi * fr), 0.0)
    assert np.max(np.abs(got - ref)) < 1e-11
    assert np.all(got[(fr >= 0.5)] == 0.0) and np.all(got >= 0.0)
    assert got[25] == 400.0  # t = 0.25: the peak, sin(pi/2) exactly


def test_l96_fixed_point_exact():
    for F in (8.0, 3.5):
        x = np.full(8, F)
        assert np.array_equal(O.l96_rk4(x, F, 0.01, 50), x)
        xf = np.full(40, np.float32(F))
        assert np.array_equal(O.l96_rk4f(xf, F, 0.005, 50), xf)


def test_l96_cyclic_shift_equivariance_bitexact():
    rng = np.random.default_rng(0)
    x = rng.standard_normal(40) + 8
    a = O.l96_rk4(x, 8.0, 0.005, 37)
    for sh in (1, 3, 17):
        b = O.l96_rk4(np.roll(x, sh), 8.0, 0.005, 37)
        assert np.array_equal(np.roll(a, sh), b)


def test_l96_energy_decay_at_zero_forcing():
    # With F = 0 the advection term conserves sum x^2, so d/dt sum x^2 = -2 sum x^2.
    rng = np.random.default_rng(1)
    x0 = rng.standard_normal(8)
    e0 = np.sum(x0 ** 2)
    errs = []
    for dt in (0.02, 0.01):
        nsteps = int(round(0.5 / dt))
        x = O.l96_rk4(x0, 0.0, dt, nsteps)
        errs.append(abs(np.sum(x ** 2) / e0 - math.exp(-1.0)))
    assert errs[1] < 1e-8
    assert errs[0] / errs[1] > 10.0


def _fine(x0, F, T):
    sol = integrate.solve_ivp(lambda t, x: (np.roll(x, -1) - np.roll(x, 2)) * np.roll(x, 1) - x + F,
                              (0.0, T), x0, method="DOP853", rtol=1e-13, atol=1e-13)
    return sol.y[:, -1]


def test_l96_rk4_fourth_order_against_scipy():
    rng = np.random.default_rng(2)
    x0 = 8.0 + rng.standard_normal(8)
    ref = _fine(x0, 8.0, 0.5)
    errs = []
    for dt in (0.02, 0.01, 0.005):
        x = O.l96_rk4(x0, 8.0, dt, int(round(0.5 / dt)))
        errs.append(np.max(np.abs(x - ref)))
    assert errs[2] < 2e-5
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 12.0 < r1 < 20.0 and 12.0 < r2 < 20.0


def test_l96_rk4_fp32_tracks_fp64_short_time():
    rng = np.random.default_rng(3)
    x0 = (8.0 + rng.standard_normal(40)).astype(np.float32)
    a = O.l96_rk4(x0.astype(np.float64), 8.0, 0.005, 10)
    b = O.l96_rk4f(x0, 8.0, 0.005, 10)
    assert np.max(np.abs(a - b)) < 1e-4


def _brute_force_loglik(theta, y, s, dt, flow):
    """log N(y; mu, Sigma) of the Euler windkessel written as one joint Gaussian."""
    R, C, Z, q, r, m0, s0 = theta
    a = 1.0 - dt / (R * C)
    T = len(y)
    K = [i * s for i in range(1, T + 1)]
    mu = np.zeros(T)
    Sig = np.zeros((T, T))
    for ii, Ki in enumerate(K):
        mu[ii] = a ** Ki * m0 + sum(a ** (Ki - 1 - m) * dt * flow[m] / C for m in range(Ki)) \
            + Z * flow[Ki]
        for jj, Kj in enumerate(K):
            c = a ** (Ki + Kj) * s0 ** 2
            c += q * sum(a ** (Ki - 1 - m) * a ** (Kj - 1 - m) for m in range(min(Ki, Kj)))
            Sig[ii, jj] = c + (r if ii == jj else 0.0)
    return stats.multivariate_normal(mean=mu, cov=Sig).logpdf(y)


@pytest.mark.parametrize("T,s", [(1, 1), (2, 1), (3, 1), (3, 4)])
def test_kalman_against_joint_gaussian(T, s):
    theta = (1.1, 1.4, 0.04, 0.3, 3.0, 85.0, 10.0)
    m = O.model(O.WINDKESSEL, substeps=s, dt=0.01)
    y = np.array([92.0, 97.0, 101.5][:T])
    flow = O.flow_table(400.0, 1.0, 0.01, T * s + 1)
    ref = _brute_force_loglik(theta, y, s, 0.01, flow)
    assert O.kalman_windkessel(m, theta, y) == pytest.approx(ref, rel=1e-12, abs=1e-10)
