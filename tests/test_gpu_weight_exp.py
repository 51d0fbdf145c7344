"""The propagate kernels' weight exponential (Algorithm 2, weight line:
w = exp(ell - M) with ell - M <= 0), evaluated on the GPU through the C ABI and
compared with correctly rounded values: within 2.5 units of 2^-53 relative on
-700 < d <= 0, exact at the special points, the library exponential below."""
import math

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
