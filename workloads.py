"""Seeded synthetic workloads shaped like the paper's two examples.

The paper's own input and observation files are not available, and its
experiments run on simulated data too, so every observation series here is
simulated from the state-space model itself with numpy's generator
(``numpy.random.default_rng``), in float64, at the workload's parameters.
This module is data synthesis only: it shares no code with ``oracle/`` or
with the CUDA path, holds none of the filter's arithmetic (no weighting,
likelihood or resampling), and no test compares a filter result against it.

Parameter vectors (the initial-state mean and standard deviation ride along
so that special cases such as a fixed initial state can be expressed):

* windkessel ``theta = (R, C, Z, q, r, m0, s0)``: Euler step
  ``x + dt (F/C - x/(R C)) + N(0, q)``, observation ``N(x + Z F(t), r)``,
  ``x0 ~ N(m0, s0^2)``;
* Lorenz '96 ``theta = (F, q, r, m0, s0)``: RK4 substeps, additive ``N(0, q)``
  once per observation interval, observation ``N(x_n, r)`` on every
  ``obs_stride``-th component, ``x0 ~ N(m0, s0^2)``.
"""
from dataclasses import dataclass, field, replace
import math

import numpy as np

DATA_SEED = 0x13063277

WINDKESSEL = 0
LORENZ96 = 1
WINDKESSEL_EXP = 2  # the paper's exact windkessel transition
LORENZ96_SDE = 3    # the paper's Lorenz '96 with the Wiener increment inside RK4
FP64 = 0
MIXED = 1

WK_THETA = (1.0, 1.5, 0.03, 0.01, 4.0, 90.0, 15.0)
L96_THETA_8 = (8.0, 0.01, 0.25, 0.0, 1.0)
L96_THETA_40 = (8.0, 0.01, 1.0, 0.0, 1.0)


@dataclass
class Workload:
    name: str
    kind: int
    N: int
    substeps: int
    obs_stride: int
    dt: float
    P: int
    T: int
    prec: int
    ess_threshold: float
    theta: tuple
    flow_peak: float = 400.0
    flow_period: float = 1.0
    seed: int = 1
    resampler: int = 0  # 0 systematic, 1 stratified, 2 multinomial
    obs_every: int = 0  # 0/1: every step observed; k: steps i with i % k == 0 only
    obs_count: int = 0  # Lorenz '96: observe only the first obs_count strided components
    y: np.ndarray = field(default=None, repr=False)

    @property
    def Ny(self):
        if self.kind in (WINDKESSEL, WINDKESSEL_EXP):
            return 1
        ny = (self.N + self.obs_stride - 1) // self.obs_stride
        return min(ny, self.obs_count) if self.obs_count > 0 else ny

    def with_(self, **kw):
        return replace(self, **kw)


def windkessel(P=1024, T=100, prec=FP64, ess_threshold=1.0, substeps=1, theta=WK_THETA, seed=1):
    """Plain bootstrap PF on the three-element windkessel (Sec. 2.1.1)."""
    w = Workload("windkessel_P%d_T%d" % (P, T), WINDKESSEL, 1, substeps, 1, 0.01, P, T, prec,
                 ess_threshold, tuple(theta), seed=seed)
    w.y = simulate(w)
    return w


def lorenz96_8(P=1 << 14, T=200, prec=FP64, ess_threshold=1.0, theta=L96_THETA_8, seed=1):
    """Lorenz '96, N=8, F=8, RK4 dt=0.01 x 5 substeps, all components observed."""
    w = Workload("lorenz96_N8_P%d_T%d" % (P, T), LORENZ96, 8, 5, 1, 0.01, P, T, prec,
                 ess_threshold, tuple(theta), seed=seed)
    w.y = simulate(w)
    return w


def lorenz96_large(P=1 << 20, T=500, prec=MIXED, ess_threshold=1.0, theta=L96_THETA_40, seed=1):
    """Lorenz '96, N=40, RK4 dt=0.005 x 10 substeps, every 2nd component observed."""
    w = Workload("lorenz96_N40_P%d_T%d" % (P, T), LORENZ96, 40, 10, 2, 0.005, P, T, prec,
                 ess_threshold, tuple(theta), seed=seed)
    w.y = simulate(w)
    return w


def lorenz96_sparse(P=1 << 14, T=60, prec=FP64, ess_threshold=1.0, theta=L96_THETA_8, seed=1):
    """Lorenz '96, N=8 (step 0.05 = RK4 0.01 x 5) with sparse observations as in
    the paper's Lorenz '96 example (Sec. 5): the first four components at every
    other step.  Rows of y at unobserved steps are simulated but not used."""
    w = Workload("lorenz96_sparse_P%d_T%d" % (P, T), LORENZ96, 8, 5, 1, 0.01, P, T, prec,
                 ess_threshold, tuple(theta), seed=seed, obs_every=2, obs_count=4)
    w.y = simulate(w)
    return w


WKX_THETA = (1.0, 1.5, 0.03, 25.0, 4.0, 90.0, 15.0)  # sigma2 = 25: the prior mean
L96W_THETA_8 = (8.0, 0.25, 0.25, 0.0, 1.0)           # sigma2 = 0.25: the prior mean


def windkessel_exact(P=1024, T=100, prec=FP64, ess_threshold=1.0, substeps=1, theta=WKX_THETA,
                     seed=1):
    """The paper's windkessel transition (Sec. 2.1.1, model listing): exponential
    decay over each step h = dt with noise on the flow,
    x <- exp(-h/(RC)) x + R (1 - exp(-h/(RC))) (F + xi), xi ~ N(0, (h sqrt(sigma2))^2)."""
    w = Workload("windkessel_exact_P%d_T%d" % (P, T), WINDKESSEL_EXP, 1, substeps, 1, 0.01, P, T,
                 prec, ess_threshold, tuple(theta), seed=seed)
    w.y = simulate(w)
    return w


def lorenz96_sde(P=1 << 14, T=200, N=8, prec=FP64, ess_threshold=1.0, theta=L96W_THETA_8,
                 substeps=1, dt=0.05, obs_stride=1, seed=1):
    """The paper's Lorenz '96 transition (Sec. 2.1.2, model listing): one RK4 step
    of h = 0.05 per observation whose right-hand side carries the Wiener increment
    sqrt(sigma2) dW_n / h, dW_n ~ N(0, h), held over the step."""
    w = Workload("lorenz96_sde_N%d_P%d_T%d" % (N, P, T), LORENZ96_SDE, N, substeps, obs_stride,
                 dt, P, T, prec, ess_threshold, tuple(theta), seed=seed)
    w.y = simulate(w)
    return w


def _flow(t, peak, period):
    ph = t / period
    fr = ph - np.floor(ph)
    return np.where(fr < 0.5, peak * np.sin(2.0 * np.pi * fr), 0.0)


def _l96_rhs(x, F):
    return (np.roll(x, -1) - np.roll(x, 2)) * np.roll(x, 1) - x + F


def simulate(w, data_seed=DATA_SEED, T=None):
    """Simulate an observation series y[T][Ny] from the model at w.theta."""
    T = w.T if T is None else T
    rng = np.random.default_rng([data_seed, w.kind, w.N, w.substeps, w.obs_stride])
    th = w.theta
    if w.kind in (WINDKESSEL, WINDKESSEL_EXP):
        R, C, Z, q, r, m0, s0 = th
        a = math.exp(-w.dt / (R * C))
        x = m0 + s0 * rng.standard_normal()
        y = np.zeros((T, 1))
        for i in range(1, T + 1):
            for m in range(w.substeps):
                k = (i - 1) * w.substeps + m
                F = _flow(k * w.dt, w.flow_peak, w.flow_period)
                if w.kind == WINDKESSEL:
                    x = x + w.dt * (F / C - x / (R * C)) + math.sqrt(q) * rng.standard_normal()
                else:
                    xi = w.dt * math.sqrt(q) * rng.standard_normal()
                    x = a * x + R * (1.0 - a) * (F + xi)
            Fo = _flow(i * w.substeps * w.dt, w.flow_peak, w.flow_period)
            y[i - 1, 0] = x + Z * Fo + math.sqrt(r) * rng.standard_normal()
        return y
    F, q, r, m0, s0 = th
    x = m0 + s0 * rng.standard_normal(w.N)
    h = w.dt
    y = np.zeros((T, w.Ny))
    for i in range(T):
        for _ in range(w.substeps):
            Fs = F
            if w.kind == LORENZ96_SDE:  # Wiener increment held over the substep
                Fs = F + math.sqrt(q / h) * rng.standard_normal(w.N)
            k1 = _l96_rhs(x, Fs)
            k2 = _l96_rhs(x + 0.5 * h * k1, Fs)
            k3 = _l96_rhs(x + 0.5 * h * k2, Fs)
            k4 = _l96_rhs(x + h * k3, Fs)
            x = x + h / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
        if w.kind == LORENZ96:
            x = x + math.sqrt(q) * rng.standard_normal(w.N)
        y[i] = x[::w.obs_stride][:w.Ny] + math.sqrt(r) * rng.standard_normal(w.Ny)
    return y


def perturb_theta(theta, kind, rng):
    """Log-uniform +-50% around the given parameters (model parameters only,
    not the initial-state mean and spread)."""
    th = list(theta)
    npar = 5 if kind == WINDKESSEL else 3
    for c in range(npar):
        th[c] = th[c] * math.exp(rng.uniform(math.log(0.5), math.log(1.5)))
    return tuple(th)


def batched(n_wk=128, n_l96=128, seed=0x5EED, prec=MIXED, pmin=8, pmax=14, tmin=50, tmax=500):
    """Many uneven independent filters (PMCMC proposals against one data set
    per model): theta log-uniform +-50%, P = 2^U{pmin..pmax}, T ~ U{tmin..tmax}."""
    rng = np.random.default_rng(seed)
    base_wk = windkessel(P=1 << pmin, T=tmax, prec=prec)
    base_l96 = lorenz96_8(P=1 << pmin, T=tmax, prec=prec)
    out = []
    kinds = [WINDKESSEL] * n_wk + [LORENZ96] * n_l96
    for f, kind in enumerate(kinds):
        base = base_wk if kind == WINDKESSEL else base_l96
        P = 1 << int(rng.integers(pmin, pmax + 1))
        T = int(rng.integers(tmin, tmax + 1))
        th = perturb_theta(base.theta, kind, rng)
        w = base.with_(name="%s_f%d" % ("wk" if kind == WINDKESSEL else "l96", f), P=P, T=T,
                       theta=th, seed=f + 1, y=base.y[:T].copy())
        out.append(w)
    return out


def serving_requests(n, rate, seed=0x5E7E, prec=MIXED, pmin=10, pmax=16, tmin=50, tmax=1000):
    """Poisson stream of likelihood requests: (arrival time, workload).
    Model uniform over {windkessel, Lorenz '96 N=8, Lorenz '96 N=40}."""
    rng = np.random.default_rng(seed)
    bases = [windkessel(P=1 << pmin, T=tmax, prec=prec),
             lorenz96_8(P=1 << pmin, T=tmax, prec=prec),
             lorenz96_large(P=1 << pmin, T=tmax, prec=prec)]
    t = 0.0
    out = []
    for r in range(n):
        t += rng.exponential(1.0 / rate)
        b = bases[int(rng.integers(0, 3))]
        P = 1 << int(rng.integers(pmin, pmax + 1))
        T = int(rng.integers(tmin, tmax + 1))
        w = b.with_(name="req%d" % r, P=P, T=T, seed=r + 1, y=b.y[:T].copy())
        out.append((t, w))
    return out
