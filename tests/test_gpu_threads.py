"""GPU tests of the boundary's threading contract: each host thread drives
its own filters (pf_create, pf_run, pf_batch_run, pf_destroy), and those
threads run at the same time (ctypes releases the interpreter lock during a
call).  Plans are captured with thread-local stream capture, so a capture in
one thread and an allocation in another do not interfere, and every result
must be the bits the same call gives when the threads run one after
another."""
import threading

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1306_3277_b300 as pf
    pf.lib()


def _workloads():
    return [W.windkessel(P=1024, T=40),
            W.windkessel(P=5000, T=30, prec=W.MIXED),
            W.lorenz96_8(P=3000, T=25),
            W.lorenz96_8(P=2049, T=30, prec=W.MIXED, ess_threshold=0.5),
            W.lorenz96_sparse(P=1500, T=20),
            W.windkessel(P=700, T=50, seed=3).with_(resampler=2)]


def _job(w, seeds):
    """Create a filter, run it once per seed (log-likelihood and final
    particles), run it in a batch of two with a second filter of its own,
    destroy both: everything a thread does with its own filters."""
    import paper_1306_3277_b300 as pf
    f = pf.pf_create(pf.model_from_workload(w), w.P, w.T, w.dt)
    g = pf.pf_create(pf.model_from_workload(w), w.P, w.T, w.dt)
    try:
        out = []
        for s in seeds:
            st, ll, x, _ = f.run(w.theta, w.y, s, want_particles=True)
            out.append((int(st), ll, x.tobytes()))
        lls, sts = pf.pf_batch_run([f, g], [w.theta, w.theta], [w.y, w.y],
                                   [seeds[0], seeds[-1]])
        out.append(tuple(int(v) for v in sts) + tuple(float(v) for v in lls))
        return out
    finally:
        f.destroy()
        g.destroy()


def test_threads_each_with_their_own_filters_match_sequential_runs():
    ws = _workloads()
    seeds = [[11 + 7 * k, 12 + 7 * k, 13 + 7 * k] for k in range(len(ws))]
    ref = [_job(w, s) for w, s in zip(ws, seeds)]
    got = [None] * len(ws)
    errors = []

    def work(k):
        try:
            for _ in range(2):  # every thread repeats its job while the others run
                got[k] = _job(ws[k], seeds[k])
        except Exception as e:  # reported below, in the test's own thread
            errors.append((k, repr(e)))

    threads = [threading.Thread(target=work, args=(k,)) for k in range(len(ws))]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=600)
    assert not any(t.is_alive() for t in threads), "a thread did not finish"
    assert not errors, errors
    for k, (a, b) in enumerate(zip(ref, got)):
        assert a == b, "workload %d: results differ from the sequential run" % k
        assert all(r[0] == 0 for r in a[:-1])


def test_last_error_is_per_thread():
    """pf_last_error is thread-local: a failing call in one thread leaves the
    message another thread reads unchanged."""
    import paper_1306_3277_b300 as pf
    msgs = {}

    def bad():
        with pytest.raises(pf.PFError):
            pf.pf_create(pf.model_from_workload(W.windkessel()), 0, 10, 0.01)
        msgs["bad"] = pf.pf_last_error()

    def good():
        w = W.windkessel(P=256, T=5)
        f = pf.pf_create(pf.model_from_workload(w), w.P, w.T, w.dt)
        f.run(w.theta, w.y, 1)
        f.destroy()
        msgs["good"] = pf.pf_last_error()

    t1 = threading.Thread(target=bad)
    t1.start()
    t1.join()
    t2 = threading.Thread(target=good)
    t2.start()
    t2.join()
    assert msgs["bad"]
    assert msgs["good"] == ""
