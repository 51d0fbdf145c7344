"""Pins of the oracle's random-number pieces against things other than itself:
published Philox known answers, libm / mpmath, and the normal distribution."""
import math
import os

import mpmath as mp
import numpy as np
import pytest
from scipy import stats

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat_rows():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        v = [int(t, 16) for t in line.split()]
        rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,expect", _kat_rows())
def test_philox_known_answers(ctr, key, expect):
    out = O.philox4x32_10(ctr, key)
    assert [int(x) for x in out] == expect


def test_philox_counter_sensitivity():
    base = O.philox4x32_10([1, 2, 3, 4], [5, 6])
    for w in range(4):
        c = [1, 2, 3, 4]
        c[w] ^= 1
        assert not np.array_equal(O.philox4x32_10(c, [5, 6]), base)


def _ulp_err(a, ref):
    return abs(a - ref) / np.spacing(abs(ref)) if ref != 0 else abs(a)


def test_log_special_values():
    assert O.log(1.0) == 0.0
    for k in range(-60, 60, 7):
        assert _ulp_err(O.log(2.0 ** k), k * math.log(2.0)) <= 1.0
    assert O.log(0.0) == -math.inf


def test_log_against_libm():
    rng = np.random.default_rng(11)
    xs = np.exp(rng.uniform(math.log(2.0 ** -53), 0.0, 20000))
    xs = np.concatenate([xs, rng.uniform(0.5, 2.0, 5000), 1.0 + rng.uniform(-1e-6, 1e-6, 500)])
    worst = max(_ulp_err(O.log(x), math.log(x)) for x in xs)
    assert worst <= 2.0


def test_logf_against_libm():
    rng = np.random.default_rng(12)
    us = ((rng.integers(0, 1 << 24, 20000) + 1) * 2.0 ** -24).astype(np.float32)
    worst = 0.0
    for u in us:
        ref = math.log(float(u))
        got = float(O.logf(u))
        worst = max(worst, abs(got - ref) / float(np.spacing(np.float32(abs(ref)) if ref else 1)))
    assert worst <= 2.0


def test_sincos2pi_exact_quadrant_points():
    assert O.sincos2pi(0.0) == (0.0, 1.0)
    assert O.sincos2pi(0.25) == (1.0, 0.0)
    assert O.sincos2pi(0.5) == (0.0, -1.0)
    assert O.sincos2pi(0.75) == (-1.0, 0.0)


def test_sincos2pi_against_mpmath():
    mp.mp.prec = 120
    rng = np.random.default_rng(13)
    us = rng.uniform(0.0, 1.0, 1500)
    worst = 0.0
    for u in us:
        s, c = O.sincos2pi(u)
        rs = float(mp.sin(2 * mp.pi * mp.mpf(u)))
        rc = float(mp.cos(2 * mp.pi * mp.mpf(u)))
        # error in units of 2^-53 (absolute, the functions are bounded by 1)
        worst = max(worst, abs(s - rs) * 2.0 ** 53, abs(c - rc) * 2.0 ** 53)
    assert worst <= 2.0


def test_sincos2pif_against_mpmath():
    rng = np.random.default_rng(14)
    us = (rng.integers(0, 1 << 24, 3000) * 2.0 ** -24).astype(np.float32)
    worst = 0.0
    for u in us:
        s, c = O.sincos2pif(u)
        rs = math.sin(2 * math.pi * float(u))
        rc = math.cos(2 * math.pi * float(u))
        worst = max(worst, abs(float(s) - rs) * 2.0 ** 24, abs(float(c) - rc) * 2.0 ** 24)
    assert worst <= 2.0


@pytest.mark.parametrize("prec", [O.FP64, O.MIXED])
def test_normals_distribution(prec):
    z = O.fill_normals(12345, prec, 3, O.PURPOSE_PROP, 1 << 18, 4).ravel()
    n = z.size
    assert abs(z.mean()) < 5 / math.sqrt(n)
    assert abs(z.var() - 1.0) < 5 * math.sqrt(2.0 / n)
    assert abs(stats.skew(z)) < 5 * math.sqrt(6.0 / n)
    assert abs(stats.kurtosis(z)) < 5 * math.sqrt(24.0 / n)
    assert stats.kstest(z, "norm").pvalue > 1e-4


def test_normals_pairs_uncorrelated_and_streams_distinct():
    z = O.fill_normals(7, O.FP64, 1, O.PURPOSE_PROP, 1 << 16, 2)
    assert abs(np.corrcoef(z[:, 0], z[:, 1])[0, 1]) < 5 / math.sqrt(1 << 16)
    a = O.fill_normals(7, O.FP64, 1, O.PURPOSE_PROP, 64, 2)
    b = O.fill_normals(7, O.FP64, 2, O.PURPOSE_PROP, 64, 2)
    c = O.fill_normals(8, O.FP64, 1, O.PURPOSE_PROP, 64, 2)
    d = O.fill_normals(7, O.FP64, 1, O.PURPOSE_INIT, 64, 2)
    for other in (b, c, d):
        assert not np.any(a == other)


def test_normal_block_layout():
    # FP64: one Philox block per pair; FP32: one block per two pairs.
    seed, j, i = 99, 5, 6
    w = O.philox4x32_10([j, i, (O.PURPOSE_PROP << 16) | 0, 0], [seed & 0xffffffff, seed >> 32])
    u1 = (((int(w[1]) << 32 | int(w[0])) >> 11) + 1) * 2.0 ** -53
    u2 = ((int(w[3]) << 32 | int(w[2])) >> 11) * 2.0 ** -53
    r = math.sqrt(-2.0 * math.log(u1))
    assert O.normal64(seed, j, i, O.PURPOSE_PROP, 0) == pytest.approx(r * math.cos(2 * math.pi * u2),
                                                                      abs=1e-14)
    assert O.normal64(seed, j, i, O.PURPOSE_PROP, 1) == pytest.approx(r * math.sin(2 * math.pi * u2),
                                                                      abs=1e-14)
    for pair in range(2):
        wa, wb = int(w[2 * pair]), int(w[2 * pair + 1])
        u1 = ((wa >> 8) + 1) * 2.0 ** -24
        u2 = (wb >> 8) * 2.0 ** -24
        r = math.sqrt(-2.0 * math.log(u1))
        assert O.normal32(seed, j, i, O.PURPOSE_PROP, 2 * pair) == pytest.approx(
            r * math.cos(2 * math.pi * u2), abs=2e-6)
        assert O.normal32(seed, j, i, O.PURPOSE_PROP, 2 * pair + 1) == pytest.approx(
            r * math.sin(2 * math.pi * u2), abs=2e-6)


def test_resample_uniform_range_and_distribution():
    us = np.array([O.resample_uniform(3, i) for i in range(20000)])
    assert us.min() >= 0.0 and us.max() < 1.0
    assert stats.kstest(us, "uniform").pvalue > 1e-4
