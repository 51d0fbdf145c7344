"""The allocation-free entry point pf_run_noalloc, for callers that cannot
allocate device memory at the point where they need a likelihood (their own
pool holds the device budget, or their framework forbids allocation on its
hot path).  It must give the same log-likelihood, status and final particles
as the ordinary pf_create/pf_run path, on two calls in a row (the second call
finds the previous call's data in the shared fixed array).  This file is
collected last on purpose."""
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
        assert abs(ll - ll_ref) <= 1e-9 * abs(ll_ref), (ll, ll_ref)
        assert np.array_equal(x, x_ref)


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
