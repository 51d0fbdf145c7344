"""Shared helpers of the parity tests: run one workload through the CUDA path
(C ABI) and through the oracle on the same seeded inputs and compare."""
import numpy as np

import oracle as O


def oracle_model(w):
    return O.model(w.kind, N=w.N, substeps=w.substeps, obs_stride=w.obs_stride, prec=w.prec,
                   dt=w.dt, ess_threshold=w.ess_threshold, flow_peak=w.flow_peak,
                   flow_period=w.flow_period, resampler=w.resampler, obs_every=w.obs_every,
                   obs_count=w.obs_count)


def run_oracle(w, seed, theta=None, nthreads=0):
    th = w.theta if theta is None else theta
    return O.pf_run(oracle_model(w), th, w.y, seed, w.P, w.T, nthreads=nthreads)


def run_gpu(w, seed, theta=None, particles=True, ancestors=True):
    import paper_1306_3277_b300 as pf
    m = pf.model_from_workload(w)
    f = pf.pf_create(m, w.P, w.T, w.dt)
    try:
        th = w.theta if theta is None else theta
        st, ll, x, anc = f.run(th, w.y, seed, want_particles=particles, want_ancestors=ancestors)
    finally:
        f.destroy()
    return dict(status=st, loglik=ll, x=x, anc=anc)


def compare(w, g, o, ll_rtol=1e-9):
    """Compare a GPU run with the oracle's.  Ancestors and particles must be
    bit-exact up to the first step at which the oracle saw a systematic target
    within 1e-12 (relative) of a cumulative-weight boundary; after such a step
    the two paths may legitimately take different ancestors.  Returns the
    number of compared steps and the first near-boundary step (or None)."""
    assert g["status"] == o["status"], (g["status"], o["status"])
    near = np.nonzero(o["diag"][:, 7] > 0)[0]
    first_near = int(near[0]) + 1 if len(near) else None  # 1-based step
    ok_rows = w.T if first_near is None else first_near  # rows 0..first_near-1 match
    if g["anc"] is not None:
        ga, oa = g["anc"], o["anc"]
        assert np.array_equal(ga[:ok_rows], oa[:ok_rows]), _first_diff(ga, oa)
        assert ga.min() >= 0 and ga.max() < w.P
        assert np.all(np.diff(ga, axis=1) >= 0)
    if first_near is None:
        if g["x"] is not None:
            ox = o["x"].astype(g["x"].dtype)
            assert np.array_equal(g["x"], ox), "final particles differ: max |d| %g" % np.max(
                np.abs(g["x"].astype(np.float64) - o["x"]))
        assert abs(g["loglik"] - o["loglik"]) <= ll_rtol * abs(o["loglik"]), (g["loglik"],
                                                                                o["loglik"])
    return ok_rows, first_near


def _first_diff(a, b):
    d = np.argwhere(a != b)
    if len(d) == 0:
        return "equal"
    i, j = d[0]
    return "first ancestor difference at step row %d particle %d: gpu %d oracle %d" % (
        i, j, a[i, j], b[i, j])
