"""The checked build (PF_CHECKED=1, loaded with PF_B300_CHECKED=1): the kernels
count violations of the path's invariants on the device -- ancestors outside
[0, P), non-finite propagated states, non-monotone in-tile cumulative weights,
invalid offspring ranges -- instead of trusting them. On the parity shapes
(tiled and cluster paths, every resampler, adaptive resampling, FP64 and
mixed) the counts must be zero and the results the plain build's bits; a NaN
parameter must show up as non-finite states."""
import json
import os
import subprocess
import sys

import pytest

import workloads as W

pytestmark = pytest.mark.gpu

ROOT = os.path.join(os.path.dirname(__file__), "..")


def _cases():
    return [W.windkessel(P=777, T=30, seed=2),
            W.windkessel(P=(1 << 16) + 5, T=8, prec=W.MIXED, seed=3),
            W.lorenz96_8(P=1000, T=20, prec=W.MIXED, ess_threshold=0.5, seed=4),
            W.lorenz96_large(P=300, T=5, seed=5),
            W.lorenz96_8(P=700, T=15, prec=W.MIXED, seed=6).with_(resampler=1),
            W.lorenz96_8(P=600, T=10, seed=7).with_(resampler=2),
            W.lorenz96_sde(P=256, T=6, prec=W.MIXED, seed=8),
            W.windkessel_exact(P=512, T=12, seed=9)]


_CHILD = r"""
import json, math, sys
sys.path.insert(0, sys.argv[1]); sys.path.insert(0, sys.argv[1] + "/tests")
import paper_1306_3277_b300 as pf
from test_gpu_checked import _cases
out = {"single": [], "cluster": []}
ws = _cases()
fs = [pf.pf_create(pf.model_from_workload(w), w.P, w.T, w.dt) for w in ws]
for w, f in zip(ws, fs):
    st, ll = f.run(w.theta, w.y, w.seed)[:2]
    out["single"].append([int(st), ll])
pf.pf_batch_configure(fs, 2048)  # small filters on one thread-block cluster each
lls, sts = pf.pf_batch_run(fs, [w.theta for w in ws], [w.y for w in ws], [w.seed for w in ws])
out["cluster"] = [[int(s), l] for s, l in zip(sts, lls)]
out["checked"], out["clean"] = pf.pf_debug_check_counts()
th = list(ws[2].theta)
th[0] = float("nan")  # Lorenz '96 forcing
st, ll = fs[2].run(th, ws[2].y, 1)[:2]
out["nan_status"] = int(st)
out["nan_counts"] = pf.pf_debug_check_counts()[1]
for f in fs:
    f.destroy()
print(json.dumps(out))
"""


def test_checked_build_counts_nothing_and_changes_nothing():
    import paper_1306_3277_b300 as pf
    ref = []
    for w in _cases():
        f = pf.pf_create(pf.model_from_workload(w), w.P, w.T, w.dt)
        st, ll = f.run(w.theta, w.y, w.seed)[:2]
        f.destroy()
        ref.append([int(st), ll])
    env = dict(os.environ, PF_B300_CHECKED="1")
    r = subprocess.run([sys.executable, "-c", _CHILD, os.path.abspath(ROOT)], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["checked"] is True
    assert out["clean"] == {"ancestor_out_of_range": 0, "state_not_finite": 0,
                            "prefix_not_monotone": 0, "offspring_range_invalid": 0}
    assert out["single"] == ref and out["cluster"] == ref
    assert out["nan_status"] == pf.PF_EDEGENERATE
    assert out["nan_counts"]["state_not_finite"] > 0
    assert out["nan_counts"]["ancestor_out_of_range"] == 0


def test_plain_build_reports_unchecked():
    import paper_1306_3277_b300 as pf
    if os.environ.get("PF_B300_CHECKED") == "1":
        pytest.skip("running the checked build")
    checked, counts = pf.pf_debug_check_counts()
    assert checked is False and set(counts.values()) == {0}
