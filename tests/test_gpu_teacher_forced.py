"""Teacher-forced GPU parity (Algorithm 2 one step at a time, through the C
ABI's pf_debug_step): every step of the CUDA path starts from the oracle's
own state x(t_{i-1}) and ancestors a(t_i), so every step is compared in full,
also after a free-running pair of runs would have parted at a near-boundary
target.  Per step: the propagated particles bit-exact, the likelihood
increment within 1e-9 relative, and the ancestors of the next step (as the
resample kernel writes them) equal to the oracle's except at most at the
targets the oracle counts as near a cumulative-weight boundary (1e-12 S),
each of those at most one particle off."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from pf_parity import oracle_model

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1306_3277_b300 as pf
    pf.lib()


def _teacher_forced(w, seed, steps=None):
    import paper_1306_3277_b300 as pf
    m = oracle_model(w)
    f = pf.pf_create(pf.model_from_workload(w), w.P, w.T, w.dt)
    T = w.T if steps is None else steps
    # x(t_0): the oracle's initial draw (the initial-draw kernel is checked by
    # the free-running parity tests)
    x0 = O.pf_run_ex(m, w.theta, w.y[:1], seed, w.P, 1)["xhist"][0]
    x, anc = x0, None
    compared = near_total = mismatch_total = 0
    try:
        for i in range(1, T + 1):
            r = O.pf_step(m, w.theta, w.y, seed, w.P, w.T, i, x, anc)
            st, inc, xg, ag = f.debug_step(w.theta, w.y, seed, i, x.astype(f.state_dtype), anc)
            assert st == pf.PF_OK and r["status"] == O.OK
            assert np.array_equal(xg, r["x"].astype(f.state_dtype)), (
                "step %d: particles differ (max |d| %g)" % (
                    i, np.max(np.abs(xg.astype(np.float64) - r["x"]))))
            assert abs(inc - r["incr"]) <= 1e-9 * abs(r["incr"]), (i, inc, r["incr"])
            if i < w.T:
                oa = r["anc_next"]
                assert ag.min() >= 0 and ag.max() < w.P
                assert np.all(np.diff(ag) >= 0)
                d = np.nonzero(ag != oa)[0]
                near = int(r["diag"][7])
                assert len(d) <= near, "step %d: %d ancestors differ, %d near targets" % (
                    i, len(d), near)
                assert np.all(np.abs(ag[d].astype(np.int64) - oa[d]) <= 1)
                near_total += near
                mismatch_total += len(d)
                anc = oa
            x = r["x"]
            compared += 1
    finally:
        f.destroy()
    return compared, near_total, mismatch_total


CASES = [
    ("lorenz96 N=40 P=2^20 T=6 mixed (Large shape)", lambda: W.lorenz96_large(T=6), 11),
    ("lorenz96 N=8 P=2^14 T=200 FP64", lambda: W.lorenz96_8(), 3),
    ("lorenz96 N=8 P=2^14 T=200 mixed", lambda: W.lorenz96_8(prec=W.MIXED), 4),
    ("windkessel P=1024 T=100 FP64", lambda: W.windkessel(), 5),
    ("windkessel P=2^16+5 T=20 FP64 stratified",
     lambda: W.windkessel(P=(1 << 16) + 5, T=20).with_(resampler=O.RESAMPLE_STRATIFIED), 6),
    ("windkessel P=2^16+5 T=20 mixed multinomial",
     lambda: W.windkessel(P=(1 << 16) + 5, T=20, prec=W.MIXED).with_(
         resampler=O.RESAMPLE_MULTINOMIAL), 7),
]


@pytest.mark.parametrize("name,factory,seed", CASES, ids=[c[0] for c in CASES])
def test_teacher_forced_every_step(name, factory, seed):
    w = factory()
    compared, near, mismatches = _teacher_forced(w, seed)
    assert compared == w.T
    assert mismatches <= near


def test_teacher_forced_step_then_continuation():
    """A state loaded by the teacher-forced step is a resident state: the
    filter continues from it with pf_run_range, and the continuation equals
    the oracle's run from the same state."""
    import paper_1306_3277_b300 as pf
    w = W.lorenz96_8(P=4096, T=20, prec=W.MIXED)
    m = oracle_model(w)
    seed = 21
    ex = O.pf_run_ex(m, w.theta, w.y, seed, w.P, w.T)
    full = O.pf_run(m, w.theta, w.y, seed, w.P, w.T)
    if np.any(full["diag"][:, 7] > 0):
        pytest.skip("near-boundary target in this run")
    f = pf.pf_create(pf.model_from_workload(w), w.P, w.T, w.dt)
    try:
        i = 8
        st, inc, xg, ag = f.debug_step(w.theta, w.y, seed, i, ex["xhist"][i - 1].astype(np.float32),
                                       full["anc"][i - 1])
        assert st == pf.PF_OK and inc == pytest.approx(full["diag"][i - 1, 6], rel=1e-9)
        st, ll, x = f.run_range(None, w.y[i:], seed, i, w.T, want_particles=True)
        assert st == pf.PF_OK
        assert np.array_equal(x, full["x"].astype(np.float32))
        assert ll == pytest.approx(full["diag"][i - 1:, 6].sum(), rel=1e-9)
    finally:
        f.destroy()
