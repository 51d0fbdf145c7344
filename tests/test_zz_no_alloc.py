"""The allocation-free entry point pf_run_noalloc, for callers that cannot
allocate device memory at the point where they need a likelihood (their own
pool holds the device budget, or their framework forbids allocation on its
hot path).  It must give the same log-likelihood, status and final particles
as the ordinary pf_create/pf_run path, on two calls in a row (the second call
finds the previous call's data in the shared fixed array), hold no device
memory beyond the fixed array, report a degenerate run as pf_run does, and
refuse host pointers.  This file is collected last on purpose."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _reference(pf, w, seed):
    f = pf.pf_create(pf.model_from_workload(w), w.P, w.T, w.dt)
    st, ll, x, _ = f.run(w.theta, w.y, seed, want_particles=True)
    f.destroy()
    return st, ll, x


def _reference_theta(pf, w, theta, seed):
    f = pf.pf_create(pf.model_from_workload(w), w.P, w.T, w.dt)
    st, ll, x, _ = f.run(theta, w.y, seed, want_particles=True)
    f.destroy()
    return st, ll, x


def _noalloc(pf, torch, w, seed, stream):
    th = torch.tensor(w.theta, dtype=torch.float64, device="cuda")
    y = torch.tensor(w.y, dtype=torch.float64, device="cuda")
    ll = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    dtype = torch.float64 if w.prec == W.FP64 else torch.float32
    x = torch.zeros((w.N, w.P), dtype=dtype, device="cuda")
    torch.cuda.synchronize()
    pf.pf_run_noalloc(pf.model_from_workload(w), w.P, w.T, w.dt, th, y, seed, ll, status, x,
                      stream)
    stream.synchronize()
    return int(status.item()), ll.item(), x.cpu().numpy()


@pytest.mark.parametrize("make", [
    lambda: W.windkessel(P=1000, T=60, substeps=3),
    lambda: W.lorenz96_8(P=4099, T=40, prec=W.MIXED, ess_threshold=0.5),
    lambda: W.lorenz96_large(P=3000, T=12),
], ids=["windkessel-fp64", "lorenz96-8-mixed-ess", "lorenz96-40-mixed"])
def test_noalloc_matches_pf_run_twice(make):
    import torch
    import paper_1306_3277_b300 as pf
    w = make()
    stream = torch.cuda.Stream()
    for seed in (21, 22):  # two calls in a row share the fixed array
        st_ref, ll_ref, x_ref = _reference(pf, w, seed)
        st, ll, x = _noalloc(pf, torch, w, seed, stream)
        assert st == st_ref == pf.PF_OK
        assert ll == ll_ref  # the same kernels on the same plan: the same bits
        assert np.array_equal(x, x_ref)


def test_noalloc_holds_no_device_memory_across_calls():
    """After a first call has loaded the fixed array on the device, further
    calls change the device's free memory by nothing: the entry point
    allocates nothing (the caller's buffers exist before the calls)."""
    import torch
    import paper_1306_3277_b300 as pf
    w = W.lorenz96_8(P=4096, T=30, prec=W.MIXED)
    stream = torch.cuda.Stream()
    th = torch.tensor(w.theta, dtype=torch.float64, device="cuda")
    y = torch.tensor(w.y, dtype=torch.float64, device="cuda")
    ll = torch.zeros(1, dtype=torch.float64, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    x = torch.zeros((w.N, w.P), dtype=torch.float32, device="cuda")
    m = pf.model_from_workload(w)
    pf.pf_run_noalloc(m, w.P, w.T, w.dt, th, y, 3, ll, status, x, stream)  # set-up call
    stream.synchronize()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    lls = []
    for seed in (4, 5, 4):
        pf.pf_run_noalloc(m, w.P, w.T, w.dt, th, y, seed, ll, status, x, stream)
        stream.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        lls.append(ll.item())
    assert lls[0] == lls[2] != lls[1]


def test_noalloc_degenerate_status_matches_pf_run():
    """Zero observation variance makes every weight zero: status
    PF_EDEGENERATE and log-likelihood -inf, as pf_run reports."""
    import torch
    import paper_1306_3277_b300 as pf
    w = W.windkessel(P=512, T=10)
    th_h = list(w.theta)
    th_h[4] = 0.0
    st_ref, ll_ref, _ = _reference_theta(pf, w, th_h, 1)
    th = torch.tensor(th_h, dtype=torch.float64, device="cuda")
    y = torch.tensor(w.y, dtype=torch.float64, device="cuda")
    ll = torch.zeros(1, dtype=torch.float64, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.Stream()
    pf.pf_run_noalloc(pf.model_from_workload(w), w.P, w.T, w.dt, th, y, 1, ll, status, None,
                      stream)
    stream.synchronize()
    assert st_ref == pf.PF_EDEGENERATE == int(status.item())
    assert ll_ref == -np.inf == ll.item()


def test_noalloc_refuses_host_arrays():
    """A host array where device memory is required is refused before any
    launch (PF_EINVAL from the library itself, ValueError from the binding)."""
    import ctypes
    import torch
    import paper_1306_3277_b300 as pf
    w = W.windkessel(P=256, T=5)
    th_host = np.ascontiguousarray(w.theta, dtype=np.float64)
    y = torch.tensor(w.y, dtype=torch.float64, device="cuda")
    ll = torch.zeros(1, dtype=torch.float64, device="cuda")
    m = pf.model_from_workload(w)
    st = pf.lib().pf_run_noalloc(ctypes.byref(m), w.P, w.T, w.dt, th_host.ctypes.data,
                                 y.data_ptr(), ctypes.c_uint64(1), ll.data_ptr(), None, None,
                                 None)
    assert st == pf.PF_EINVAL
    assert "theta" in pf.pf_last_error()
    with pytest.raises(ValueError):
        pf.pf_run_noalloc(m, w.P, w.T, w.dt, th_host, y, 1, ll)


def test_noalloc_rejects_filters_larger_than_the_array():
    import torch
    import paper_1306_3277_b300 as pf
    w = W.lorenz96_large(P=1 << 20, T=2)
    th = torch.tensor(w.theta, dtype=torch.float64, device="cuda")
    y = torch.tensor(w.y, dtype=torch.float64, device="cuda")
    ll = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(pf.PFError) as e:
        pf.pf_run_noalloc(pf.model_from_workload(w), w.P, w.T, w.dt, th, y, 1, ll)
    assert e.value.status == pf.PF_EINVAL
    assert "scratch" in str(e.value)
