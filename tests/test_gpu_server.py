"""GPU tests of the continuous-batching server: every request's result is
bit-identical to pf_run of the same request, alone or in a mix that is
admitted piecewise by memory budget and slots."""
import time

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _mix(n, seed):
    rng = np.random.default_rng(seed)
    bases = [W.windkessel(P=256, T=300), W.lorenz96_8(P=256, T=300, prec=W.MIXED),
             W.lorenz96_large(P=256, T=300), W.lorenz96_8(P=256, T=300, prec=W.FP64,
                                                          ess_threshold=0.5)]
    out = []
    for r in range(n):
        b = bases[int(rng.integers(0, len(bases)))]
        P = int(2 ** rng.integers(6, 13)) + int(rng.integers(0, 3))
        T = int(rng.integers(5, 300))
        out.append(b.with_(name="r%d" % r, P=P, T=T, seed=r + 11, y=b.y[:T].copy()))
    return out


def _serve(pf, ws, budget, slots, stagger=0.0, branches=None, regroup_to=None):
    srv = pf.pf_server_create(budget, slots, branches=branches)
    tickets = []
    for n, w in enumerate(ws):
        tickets.append(srv.submit(pf.model_from_workload(w), w.P, w.T, w.dt, w.theta, w.y, w.seed))
        if stagger:
            time.sleep(stagger)
        if regroup_to is not None and n == len(ws) // 2:
            srv.configure(regroup_to)  # while filters run
    res = {}
    deadline = time.time() + 120
    while len(res) < len(tickets) and time.time() < deadline:
        for t in tickets:
            if t not in res:
                r = srv.poll(t)
                if r is not None:
                    res[t] = r
        time.sleep(0.001)
    stats = srv.stats()
    srv.destroy()
    assert len(res) == len(tickets), "server did not finish"
    return [res[t] for t in tickets], stats


def test_server_results_equal_pf_run():
    import paper_1306_3277_b300 as pf
    ws = _mix(24, 1)
    ref = []
    for w in ws:
        f = pf.pf_create(pf.model_from_workload(w), w.P, w.T, w.dt)
        st, ll, _, _ = f.run(w.theta, w.y, w.seed)
        f.destroy()
        ref.append((st, ll))
    # generous budget, staggered arrivals: requests join while others run
    got, stats = _serve(pf, ws, 8 << 30, 16, stagger=0.002)
    for (st, ll), (gst, gll, lat) in zip(ref, got):
        assert gst == st and gll == ll and lat > 0
    assert stats["completed"] == len(ws)
    # tight budget: a few requests at a time, admitted as memory frees up
    budget = max(pf.pf_device_bytes(pf.model_from_workload(w), w.P, w.T) for w in ws) * 3
    got2, stats2 = _serve(pf, ws, budget, 4)
    for (st, ll), (gst, gll, _) in zip(ref, got2):
        assert gst == st and gll == ll
    assert stats2["iterations"] >= max(w.T for w in ws)


def test_server_alone_equals_in_mix():
    import paper_1306_3277_b300 as pf
    ws = _mix(10, 2)
    alone = [_serve(pf, [w], 1 << 30, 4)[0][0] for w in ws[:3]]
    mixed, _ = _serve(pf, ws, 8 << 30, 32)
    for a, m in zip(alone, mixed[:3]):
        assert a[0] == m[0] and a[1] == m[1]


@pytest.mark.parametrize("branches,regroup_to", [(2, None), (3, None), (8, None), (4, 1),
                                                 (1, 5)])
def test_server_branches_equal_pf_run(branches, regroup_to):
    """Filters dealt into concurrent launch groups (and regrouped while they
    run) give pf_run's results bit for bit."""
    import paper_1306_3277_b300 as pf
    ws = _mix(20, 5)
    ref = []
    for w in ws:
        f = pf.pf_create(pf.model_from_workload(w), w.P, w.T, w.dt)
        st, ll, _, _ = f.run(w.theta, w.y, w.seed)
        f.destroy()
        ref.append((st, ll))
    got, stats = _serve(pf, ws, 8 << 30, 12, stagger=0.002, branches=branches,
                        regroup_to=regroup_to)
    for (st, ll), (gst, gll, _) in zip(ref, got):
        assert gst == st and gll == ll
    assert stats["completed"] == len(ws)


def test_server_configure_rejects_bad_branch_counts():
    import paper_1306_3277_b300 as pf
    srv = pf.pf_server_create(1 << 30, 2)
    try:
        for b in (0, -1, 9):
            with pytest.raises(pf.PFError) as e:
                srv.configure(b)
            assert e.value.status == pf.PF_EINVAL
        srv.configure(8)
    finally:
        srv.destroy()


def test_server_rejects_oversized_and_bad_requests():
    import paper_1306_3277_b300 as pf
    srv = pf.pf_server_create(1 << 20, 2)
    w = W.lorenz96_large(P=1 << 16, T=10)
    with pytest.raises(pf.PFError) as e:
        srv.submit(pf.model_from_workload(w), w.P, w.T, w.dt, w.theta, w.y, 1)
    assert e.value.status == pf.PF_ENOMEM
    with pytest.raises(pf.PFError) as e:
        srv.submit(pf.model(pf.PF_LORENZ96, N=7), 10, 10, 0.01, w.theta, w.y, 1)
    assert e.value.status == pf.PF_EINVAL
    with pytest.raises(pf.PFError):
        srv.poll(12345)
    srv.destroy()


def test_server_ticket_is_collected_once():
    import paper_1306_3277_b300 as pf
    w = W.windkessel(P=256, T=20)
    srv = pf.pf_server_create(1 << 30, 2)
    try:
        t = srv.submit(pf.model_from_workload(w), w.P, w.T, w.dt, w.theta, w.y, 3)
        deadline = time.time() + 60
        r = None
        while r is None and time.time() < deadline:
            r = srv.poll(t)  # None (PF_EBUSY) while queued or running
            time.sleep(0.001)
        assert r is not None and r[0] == pf.PF_OK
        with pytest.raises(pf.PFError) as e:
            srv.poll(t)
        assert e.value.status == pf.PF_EINVAL
    finally:
        srv.destroy()
