"""Failure handling, with the failure made on the host (no GPU fault): a device
allocation of a filter or of a served request is made to fail through
pf_debug_fail_allocation. pf_create must return PF_ENOMEM at every one of its
allocations without leaking the others, a served request must finish with
PF_ENOMEM while the server goes on, and filters created afterwards give the
same bits as before.  A server whose scheduler sees a CUDA error (reported by
pf_debug_fail_server_wait in place of the real wait's result) must end every
running and queued request with PF_ECUDA, refuse new ones and still shut
down."""
import time

import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_create_fails_cleanly_at_each_allocation():
    import torch
    import paper_1306_3277_b300 as pf
    # adaptive resampling: the carried log-weight buffers are allocated too
    w = W.lorenz96_8(P=4096, T=20, prec=W.MIXED, ess_threshold=0.5)
    m = pf.model_from_workload(w)
    f = pf.pf_create(m, w.P, w.T, w.dt)
    st_ref, ll_ref = f.run(w.theta, w.y, 3)[:2]
    f.destroy()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    failed = 0
    try:
        for k in range(1, 16):
            pf.pf_debug_fail_allocation(k)
            try:
                f = pf.pf_create(m, w.P, w.T, w.dt)
            except pf.PFError as e:
                assert e.status == pf.PF_ENOMEM, e
                failed += 1
                continue
            pf.pf_debug_fail_allocation(0)  # k is past the filter's allocations
            st, ll = f.run(w.theta, w.y, 3)[:2]
            f.destroy()
            assert (st, ll) == (st_ref, ll_ref)
    finally:
        pf.pf_debug_fail_allocation(0)
    assert failed == 9  # x[0], x[1], ctil, ell, lam, anc, tile and group partials, control
    torch.cuda.synchronize()
    assert abs(torch.cuda.mem_get_info()[0] - free0) < (64 << 20)


def _wait(srv, ticket, limit=60.0):
    import paper_1306_3277_b300 as pf
    deadline = time.time() + limit
    while time.time() < deadline:
        try:
            r = srv.poll(ticket)
        except pf.PFError as e:
            return e.status, None
        if r is not None:
            return r[0], r[1]
        time.sleep(0.001)
    raise AssertionError("server did not finish the request")


def test_served_request_fails_cleanly_and_the_server_goes_on():
    import paper_1306_3277_b300 as pf
    w = W.windkessel(P=1024, T=50, prec=W.MIXED)
    m = pf.model_from_workload(w)
    f = pf.pf_create(m, w.P, w.T, w.dt)
    ref = f.run(w.theta, w.y, 5)[:2]
    f.destroy()
    srv = pf.pf_server_create(1 << 30, 4)
    try:
        pf.pf_debug_fail_allocation(1)  # the first allocation of the next admitted request
        bad = srv.submit(m, w.P, w.T, w.dt, w.theta, w.y, 5)
        assert _wait(srv, bad)[0] == pf.PF_ENOMEM
        pf.pf_debug_fail_allocation(0)
        good = srv.submit(m, w.P, w.T, w.dt, w.theta, w.y, 5)
        assert _wait(srv, good) == ref
        assert srv.stats()["running"] == 0
    finally:
        pf.pf_debug_fail_allocation(0)
        srv.destroy()


def test_fault_injection_rejects_negative_k():
    import paper_1306_3277_b300 as pf
    with pytest.raises(pf.PFError) as e:
        pf.pf_debug_fail_allocation(-1)
    assert e.value.status == pf.PF_EINVAL


def test_server_ends_its_requests_after_a_cuda_error():
    import paper_1306_3277_b300 as pf
    w = W.windkessel(P=512, T=400, prec=W.MIXED)
    m = pf.model_from_workload(w)
    srv = pf.pf_server_create(1 << 30, 2)
    try:
        pf.pf_debug_fail_server_wait(1)  # the scheduler's first wait for an iteration
        tickets = [srv.submit(m, w.P, w.T, w.dt, w.theta, w.y, k) for k in range(3)]
        # two requests run (two slots), the third waits in the queue: all three end
        assert [_wait(srv, t)[0] for t in tickets] == [pf.PF_ECUDA] * 3
        with pytest.raises(pf.PFError) as e:
            srv.submit(m, w.P, w.T, w.dt, w.theta, w.y, 9)
        assert e.value.status == pf.PF_ECUDA
        st = srv.stats()
        assert st["running"] == 0 and st["queued"] == 0 and st["completed"] == 3
    finally:
        pf.pf_debug_fail_server_wait(0)
        srv.destroy()
    # the GPU was never at fault: a new server serves the same request exactly
    f = pf.pf_create(m, w.P, w.T, w.dt)
    ref = f.run(w.theta, w.y, 5)[:2]
    f.destroy()
    srv = pf.pf_server_create(1 << 30, 2)
    try:
        assert _wait(srv, srv.submit(m, w.P, w.T, w.dt, w.theta, w.y, 5)) == ref
    finally:
        srv.destroy()
    with pytest.raises(pf.PFError) as e:
        pf.pf_debug_fail_server_wait(-1)
    assert e.value.status == pf.PF_EINVAL
