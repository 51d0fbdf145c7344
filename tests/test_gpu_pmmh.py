"""GPU parity of the marginal Metropolis-Hastings chains (Algorithm 3): the
chains run on the GPU (proposals, batched filters, acceptance) follow the
oracle's chains sample for sample -- parameters bit-exact, log-likelihoods
within 1e-9 relative -- up to the first iteration the oracle flags as near
(a filter with a near-boundary resampling target, or an acceptance test
within 1e-9 of its threshold)."""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W
from pf_parity import oracle_model

pytestmark = pytest.mark.gpu
INF = math.inf


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


WK_SPEC = [(3, 1, 2.0, 0.9, 0.03, 0.0, INF), (0, 0), (3, 1, 2.0, 0.03, 0.002, 0.0, INF),
           (4, 2, 2.0, 0.01, 2.0, 3.0), (0, 0), (0, 0), (0, 0)]
L96_SPEC = [(1, 1, 8.0, 12.0, 0.1, 8.0, 12.0), (4, 2, 2.0, 0.25, 2.0, 3.0), (0, 0), (0, 0), (0, 0)]

CASES = [
    ("windkessel P=256 T=50 FP64", lambda: W.windkessel(P=256, T=50), WK_SPEC, 4, 40),
    ("windkessel P=300 T=40 ESS 0.5 mixed", lambda: W.windkessel(P=300, T=40, ess_threshold=0.5,
                                                                 prec=W.MIXED), WK_SPEC, 3, 30),
    ("lorenz96 N=8 P=1024 T=40 mixed", lambda: W.lorenz96_8(P=1024, T=40, prec=W.MIXED),
     L96_SPEC, 4, 30),
    ("lorenz96 N=8 P=700 T=30 FP64", lambda: W.lorenz96_8(P=700, T=30), L96_SPEC, 2, 25),
]


@pytest.mark.parametrize("name,factory,spec,nc,niter", CASES, ids=[c[0] for c in CASES])
def test_pmmh_chains_match_oracle(name, factory, spec, nc, niter):
    import paper_1306_3277_b300 as pf
    w = factory()
    th0 = np.tile(np.array(w.theta, dtype=float), (nc, 1))
    th0[:, 0] *= 1.0 + 0.01 * np.arange(nc)  # chains start apart
    fs = [pf.pf_create(pf.model_from_workload(w), w.P, w.T, w.dt) for _ in range(nc)]
    try:
        samples, lls, acc = pf.pf_pmmh_run(fs, w.y, spec, th0, niter, 31)
        # the same chains again: the library is deterministic
        s2, l2, a2 = pf.pf_pmmh_run(fs, w.y, spec, th0, niter, 31)
        assert np.array_equal(samples, s2) and np.array_equal(lls, l2)
    finally:
        for f in fs:
            f.destroy()
    o = O.pmmh(oracle_model(w), w.y, w.P, w.T, O.LIK_PF, spec, th0, niter, 31)
    compared = 0
    for c in range(nc):
        flagged = np.nonzero(o["near"][:, c])[0]
        upto = int(flagged[0]) if len(flagged) else niter + 1
        assert np.array_equal(samples[:upto, c], o["samples"][:upto, c]), c
        ref = o["logliks"][:upto, c]
        assert np.all(np.abs(lls[:upto, c] - ref) <= 1e-9 * np.abs(ref)), c
        if upto == niter + 1:
            assert acc[c] == o["accepted"][c]
        compared += upto
    assert compared >= nc * niter // 2
    assert acc.sum() > 0  # the chains move


def test_pmmh_rejects_bad_spec_and_mixed_kinds():
    import paper_1306_3277_b300 as pf
    w = W.windkessel(P=64, T=10)
    v = W.lorenz96_8(P=64, T=10)
    f1 = pf.pf_create(pf.model_from_workload(w), 64, 10, w.dt)
    f2 = pf.pf_create(pf.model_from_workload(v), 64, 10, v.dt)
    try:
        bad = list(WK_SPEC)
        bad[3] = (4, 2, 2.0, 0.01, 2.5, 3.0)  # non-integer inverse-gamma shape
        with pytest.raises(pf.PFError) as e:
            pf.pf_pmmh_run([f1], w.y, bad, [w.theta], 2, 1)
        assert e.value.status == pf.PF_EINVAL
        with pytest.raises(pf.PFError) as e:
            pf.pf_pmmh_run([f1, f2], w.y, WK_SPEC, [w.theta, w.theta], 2, 1)
        assert e.value.status == pf.PF_EINVAL
        with pytest.raises(pf.PFError):
            pf.pf_pmmh_run([f1, f1], w.y, WK_SPEC, [w.theta, w.theta], 2, 1)
    finally:
        f1.destroy()
        f2.destroy()
