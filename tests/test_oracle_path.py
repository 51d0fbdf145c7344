"""Pins of the oracle's single-path sample (the ancestry trace at the end of
Algorithm 2): the draw of the final particle against exact rational
arithmetic on the published Philox stream, the trace against the ancestor
history, a noiseless model against its closed-form trajectory, and the
sampled paths of the linear-Gaussian windkessel against the smoothing
distribution of the joint Gaussian (brute force, no Kalman code)."""
from fractions import Fraction
import math

import numpy as np
import pytest

import oracle as O
import workloads as W


def _om(w):
    return O.model(w.kind, N=w.N, substeps=w.substeps, obs_stride=w.obs_stride, prec=w.prec,
                   dt=w.dt, ess_threshold=w.ess_threshold, flow_peak=w.flow_peak,
                   flow_period=w.flow_period)


def _path_uniform(seed, T):
    """53-bit uniform of Philox block (0, T+1, purpose 4 << 16, 0), key = seed halves."""
    w = O.philox4x32_10([0, T + 1, O.PURPOSE_PATH << 16, 0],
                        [seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF])
    v = ((int(w[1]) << 32) | int(w[0])) >> 11
    return Fraction(v, 1 << 53)


@pytest.mark.parametrize("w", [W.windkessel(P=7, T=4), W.lorenz96_8(P=13, T=3),
                               W.lorenz96_8(P=9, T=5, prec=W.MIXED),
                               W.windkessel(P=11, T=6, ess_threshold=0.5)],
                         ids=["wk", "l96", "l96_mixed", "wk_adaptive"])
def test_path_pick_and_trace_exact(w):
    m = _om(w)
    for seed in range(1, 40):
        st, ll, path, idx = O.sample_path(m, w.theta, w.y, seed, w.P, w.T)
        r = O.pf_run_ex(m, w.theta, w.y, seed, w.P, w.T)
        assert st == O.OK and r["status"] == O.OK and ll == r["loglik"]
        # final pick: the first k whose weight prefix exceeds v times the total
        ell = r["ellT"]
        M = ell.max()
        wk = [Fraction(math.exp(e - M)) for e in ell]
        C = np.cumsum(wk).tolist()
        vs = _path_uniform(seed, w.T) * C[-1]
        if min(abs(float(c - vs)) for c in C) > 1e-9 * float(C[-1]):
            assert idx[w.T] == next(k for k in range(w.P) if C[k] > vs)
        # trace: ancestors of the picked particle, states of the traced particles
        for i in range(w.T, 0, -1):
            assert idx[i - 1] == r["anc"][i - 1][idx[i]]
        for i in range(w.T + 1):
            assert np.array_equal(path[i], r["xhist"][i][:, idx[i]])


def test_path_noiseless_windkessel_closed_form():
    th = (1.0, 1.5, 0.03, 0.0, 4.0, 90.0, 0.0)
    w = W.windkessel(P=32, T=40, substeps=2)
    m = _om(w)
    st, _, path, idx = O.sample_path(m, th, w.y, 3, 32, w.T)
    assert st == O.OK and np.all((idx >= 0) & (idx < 32))
    R, C = th[0], th[1]
    a = 1.0 - w.dt / (R * C)
    x, k = 90.0, 0
    ref = [x]
    for i in range(w.T):
        for _ in range(w.substeps):
            t = k * w.dt
            fr = t - math.floor(t)
            flow = 400.0 * math.sin(2 * math.pi * fr) if fr < 0.5 else 0.0
            x = a * x + w.dt * flow / C
            k += 1
        ref.append(x)
    assert np.allclose(path[:, 0], ref, rtol=1e-12, atol=1e-9)


def _smoothing_moments(theta, y, s, dt):
    """Mean and variance of x(t_i), i = 0..T, given y_1..y_T, for the Euler
    windkessel written out as one joint Gaussian over states and observations."""
    R, C, Z, q, r, m0, s0 = theta
    a = 1.0 - dt / (R * C)
    T = len(y)
    K = [i * s for i in range(T + 1)]
    n = K[-1] + 1
    t = np.arange(n) * dt
    fr = t - np.floor(t)
    flow = np.where(fr < 0.5, 400.0 * np.sin(2 * np.pi * fr), 0.0)
    mx = np.array([a ** Ki * m0 + sum(a ** (Ki - 1 - mm) * dt * flow[mm] / C for mm in range(Ki))
                   for Ki in K])
    Cxx = np.zeros((T + 1, T + 1))
    for ii, Ki in enumerate(K):
        for jj, Kj in enumerate(K):
            c = a ** (Ki + Kj) * s0 ** 2
            c += q * sum(a ** (Ki - 1 - mm) * a ** (Kj - 1 - mm) for mm in range(min(Ki, Kj)))
            Cxx[ii, jj] = c
    my = mx[1:] + Z * flow[np.array(K[1:])]
    Cxy = Cxx[:, 1:]
    Cyy = Cxx[1:, 1:] + r * np.eye(T)
    gain = np.linalg.solve(Cyy, Cxy.T).T
    mean = mx + gain @ (np.asarray(y) - my)
    var = np.diag(Cxx - gain @ Cxy.T)
    return mean, var


def test_path_samples_follow_smoothing_distribution():
    T, P, nseed = 20, 1024, 48
    w = W.windkessel(P=P, T=T)
    m = _om(w)
    y = w.y[:T, 0]
    mean, var = _smoothing_moments(w.theta, y, w.substeps, w.dt)
    paths = np.array([O.sample_path(m, w.theta, w.y[:T], s, P, T)[2][:, 0]
                      for s in range(1, nseed + 1)])
    z = (paths.mean(axis=0) - mean) / np.sqrt(var / nseed)
    assert np.max(np.abs(z)) < 4.5
    assert np.mean(z * z) < 3.0
    ratio = paths.var(axis=0, ddof=1) / var
    assert 0.4 < np.mean(ratio) < 2.5
