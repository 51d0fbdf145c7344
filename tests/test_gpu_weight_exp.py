"""The propagate kernels' weight exponential (Algorithm 2, weight line:
w = exp(ell - M) with ell - M <= 0) and the step combine's weight-sum
logarithm (likelihood line: log S), evaluated on the GPU through the C ABI and
compared with correctly rounded values: the exponential within 2.5 units of
2^-53 relative on -700 < d <= 0, exact at the special points, the library
exponential below; the logarithm within 4 units of 2^-53 times max(1, log S)
on 1 <= S <= 2^120, the library logarithm outside.  The tile's cumulative
weights (the prefix sums Sec. 3.3's resampling searches) are the exact
rational sums of the weights rounded to multiples of 2^-55, each sum rounded
once to the nearest double."""
import math
from fractions import Fraction

import mpmath
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

mpmath.mp.dps = 40
LN2_256 = math.log(2) / 256


def _exact(d):
    return float(mpmath.exp(mpmath.mpf(d)))


def _rel_units(w, d):
    e = mpmath.exp(mpmath.mpf(d))
    return float(abs(mpmath.mpf(w) - e) / e) / 2.0 ** -53


def test_weight_exp_accuracy():
    import paper_1306_3277_b300 as pf
    rng = np.random.default_rng(7)
    d = np.concatenate([
        -rng.exponential(3.0, 4000),                      # typical log-weight gaps
        -rng.uniform(0.0, 700.0, 3000),
        -10.0 ** rng.uniform(-20.0, math.log10(699.9), 3000),
        -(np.arange(0, 4000, 3) + 0.5) * LN2_256,          # range-reduction ties
        -np.arange(1, 4000, 7) * LN2_256,                  # table points (r = 0)
        np.nextafter(-(np.arange(1, 500) * LN2_256), 0.0),
    ])
    d = d[d > -700.0]
    w = pf.pf_weight_exp(d)
    worst = max(_rel_units(wi, di) for wi, di in zip(w, d))
    assert worst <= 2.5, worst
    # the cheap check on the whole range: within 4 units of the C library
    ref = np.exp(d)
    assert np.all(np.abs(w - ref) <= 4 * 2.0 ** -53 * ref)


def test_weight_exp_special_points():
    import paper_1306_3277_b300 as pf
    d = np.array([0.0, -0.0, -1e-300, -2.0 ** -61, -2.0 ** -60, -1e-17, -699.9999999,
                  -700.0, -720.5, -745.1, -745.2, -746.0, -1e300, -np.inf, 0.5, 3.0])
    w = pf.pf_weight_exp(d)
    assert w[0] == 1.0 and w[1] == 1.0 and w[2] == 1.0 and w[3] == 1.0
    for k in range(4, 7):  # the table-driven path
        assert _rel_units(w[k], d[k]) <= 2.5, (d[k], w[k])
    # (-745.2, -700] and d > 0 take the library exponential (subnormal results
    # near the bottom: compare with an absolute floor of two subnormal units)
    for k in (7, 8, 9, 14, 15):
        e = _exact(d[k])
        assert abs(w[k] - e) <= max(2.5 * 2.0 ** -53 * e, 2 * 2.0 ** -1074), (d[k], w[k], e)
    assert np.all(w[10:14] == 0.0)  # d <= -745.2 and -inf
    assert np.isnan(pf.pf_weight_exp(np.array([np.nan]))[0])


def test_weight_exp_monotone_near_table_points():
    import paper_1306_3277_b300 as pf
    base = -np.arange(1, 300) * LN2_256
    d = np.sort(np.concatenate([base, np.nextafter(base, 0.0), np.nextafter(base, -1.0)]))
    w = pf.pf_weight_exp(d)
    assert np.all(np.diff(w) >= 0.0)


def test_weight_exp_rejects_bad_arguments():
    import paper_1306_3277_b300 as pf
    assert pf.pf_weight_exp(np.zeros(0)).size == 0
    assert pf.lib().pf_weight_exp(None, None, -1) == pf.PF_EINVAL
    assert pf.lib().pf_weight_exp(None, None, 4) == pf.PF_EINVAL


# ---------------------------------------------------------------------------
# The step combine's weight-sum logarithm (Algorithm 2, likelihood line:
# log Z_i = M + log S - log P, S >= 1): an FP32 logarithm refined by one
# Newton step with the weight exponential.  Absolute error within 4 units of
# 2^-53 times max(1, log S) against correctly rounded values.
# ---------------------------------------------------------------------------
def _log_err_units(y, s):
    e = mpmath.log(mpmath.mpf(s))
    return float(abs(mpmath.mpf(y) - e)) / (2.0 ** -53 * max(1.0, float(abs(e))))


def test_weight_sum_log_accuracy():
    import paper_1306_3277_b300 as pf
    rng = np.random.default_rng(11)
    s = np.concatenate([
        2.0 ** rng.uniform(0.0, 31.0, 6000),               # weight sums of up to 2^31 particles
        1.0 + rng.uniform(0.0, 1e-3, 1000),                 # one dominant particle
        1.0 + np.arange(1, 400) * 2.0 ** -52,               # next to 1
        2.0 ** np.arange(0, 121),                           # powers of two
        np.nextafter(2.0 ** np.arange(1, 60), 0.0),
        rng.uniform(1.0, 2.0 ** 120, 500),
    ])
    y = pf.pf_weight_sum_log(s)
    worst = max(_log_err_units(yi, si) for yi, si in zip(y, s))
    assert worst <= 4.0, worst
    assert pf.pf_weight_sum_log(np.array([1.0]))[0] == 0.0  # one particle carries all the weight


def test_weight_sum_log_outside_the_fast_range():
    import paper_1306_3277_b300 as pf
    s = np.array([0.5, 1e-300, 2.0 ** 121, 1e300, 0.0, np.inf, np.nan, -1.0])
    y = pf.pf_weight_sum_log(s)
    for k in range(4):  # the library logarithm
        assert _log_err_units(y[k], s[k]) <= 2.0, (s[k], y[k])
    assert y[4] == -np.inf and y[5] == np.inf and np.isnan(y[6]) and np.isnan(y[7])
    assert pf.pf_weight_sum_log(np.zeros(0)).size == 0
    assert pf.lib().pf_weight_sum_log(None, None, -1) == pf.PF_EINVAL
    assert pf.lib().pf_weight_sum_log(None, None, 4) == pf.PF_EINVAL


def _exact_prefix(w):
    """Per tile of 256: each weight rounded to the nearest multiple of 2^-55
    (ties to even: Python's round of a Fraction), exact running sums, each
    rounded to the nearest double (float of a Fraction)."""
    pre, tot = [], []
    for t0 in range(0, len(w), 256):
        acc = Fraction(0)
        for v in w[t0:t0 + 256]:
            acc += Fraction(round(Fraction(float(v)) * 2 ** 55), 2 ** 55)
            pre.append(float(acc))
        tot.append(float(acc))
    return np.array(pre), np.array(tot)


def test_tile_prefix_is_the_rounded_exact_sum():
    import paper_1306_3277_b300 as pf
    rng = np.random.default_rng(11)
    ulp55 = 2.0 ** -55
    w = np.concatenate([
        rng.uniform(0.0, 1.0, 1024),
        np.exp(-rng.exponential(5.0, 1024)),               # weights of a spread tile
        10.0 ** rng.uniform(-320.0, 0.0, 1024),            # down to subnormal weights
        (rng.integers(0, 2 ** 20, 768) + 0.5) * ulp55,     # ties of the 2^-55 rounding
        (rng.integers(0, 2 ** 20, 256) + 0.5) * ulp55 * 2 ** 30,
        np.zeros(100), np.ones(300),                       # exact 0 and 1
        np.full(256, 1.0), np.full(256, ulp55 / 2),        # a full tile of ones; half ulps
        np.full(77, 5e-324),                               # the smallest subnormal
        rng.uniform(0.0, 1.0, 333),                        # ragged last tile
    ])
    prefix, totals = pf.pf_weight_prefix(w)
    ep, et = _exact_prefix(w)
    assert np.array_equal(prefix, ep)
    assert np.array_equal(totals, et)
    # the tile's last prefix is its total, and prefixes never decrease in a tile
    for t in range(len(totals)):
        seg = prefix[256 * t:256 * (t + 1)]
        assert seg[-1] == totals[t]
        assert np.all(np.diff(seg) >= 0.0)


def test_tile_prefix_rejects_weights_outside_unit_interval():
    import paper_1306_3277_b300 as pf
    for bad in ([0.5, 1.0000000000000002], [-1e-300], [np.nan], [np.inf]):
        with pytest.raises(pf.PFError):
            pf.pf_weight_prefix(np.array(bad))
    p, t = pf.pf_weight_prefix(np.zeros(0))
    assert p.size == 0 and t.size == 0
    p, t = pf.pf_weight_prefix(np.array([-0.0, 0.25, -0.0]))  # -0 counts as 0
    assert list(p) == [0.0, 0.25, 0.25] and list(t) == [0.25]
