"""GPU parity of the Lorenz '96 state sizes the C ABI accepts beyond those
the other tests run (N = 16, 20, 24, 32; Sec. 2.1.2 with N a free
parameter): each propagate kernel instantiation against the oracle, in FP64
and in mixed precision (the packed FP32 pairs of the RK4 need N/2 pairs with
their cyclic wrap), with every, every 2nd and every 3rd component observed
(Ny = ceil(N / stride)), the additive and the stochastic transitions; then
the same filters in one batch give the bits of their single runs.
Particles and ancestors bit-exact away from the oracle's near-boundary
window, log-likelihood within 1e-9."""
import pytest

import workloads as W
from pf_parity import compare, run_gpu, run_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _l96(N, stride, prec, P, T, seed=1):
    w = W.lorenz96_8(P=P, T=T, prec=prec, seed=seed).with_(N=N, obs_stride=stride)
    w.y = W.simulate(w)
    return w


def _l96_sde(N, stride, prec, P, T):
    w = W.lorenz96_sde(P=P, T=T, N=N, prec=prec, obs_stride=stride)
    w.y = W.simulate(w)
    return w


CASES = [
    ("N16 stride1 fp64", lambda: _l96(16, 1, W.FP64, 2500, 10)),
    ("N16 stride2 mixed", lambda: _l96(16, 2, W.MIXED, 3001, 12)),
    ("N20 stride3 fp64", lambda: _l96(20, 3, W.FP64, 1800, 8)),
    ("N20 stride1 mixed", lambda: _l96(20, 1, W.MIXED, 2600, 10)),
    ("N24 stride2 fp64", lambda: _l96(24, 2, W.FP64, 2100, 8)),
    ("N24 stride3 mixed", lambda: _l96(24, 3, W.MIXED, 2305, 10)),
    ("N32 stride2 fp64", lambda: _l96(32, 2, W.FP64, 1500, 8)),
    ("N32 stride1 mixed", lambda: _l96(32, 1, W.MIXED, 2049, 10)),
    ("N32 stride3 mixed adaptive", lambda: _l96(32, 3, W.MIXED, 1700, 12).with_(
        ess_threshold=0.5)),
    ("sde N16 stride2 mixed", lambda: _l96_sde(16, 2, W.MIXED, 2000, 8)),
    ("sde N24 stride1 fp64", lambda: _l96_sde(24, 1, W.FP64, 1300, 6)),
    ("sde N32 stride2 mixed", lambda: _l96_sde(32, 2, W.MIXED, 1600, 8)),
]


@pytest.mark.parametrize("name,factory", CASES, ids=[c[0] for c in CASES])
def test_dimension_parity(name, factory):
    w = factory()
    for seed in (3, 4):
        compare(w, run_gpu(w, seed), run_oracle(w, seed))


def test_dimensions_in_one_batch_equal_single_runs():
    import paper_1306_3277_b300 as pf
    ws = [f() for _, f in CASES]
    fs = [pf.pf_create(pf.model_from_workload(w), w.P, w.T, w.dt) for w in ws]
    try:
        ref = [f.run(w.theta, w.y, 7 + k)[:2] for k, (w, f) in enumerate(zip(ws, fs))]
        for shape in ((0, 1, 8, 0, 1), (0, 3, 4, 0, 1), (4096, 2, 8, 0, 1)):
            pf.pf_batch_set_shape(fs, *shape)
            lls, sts = pf.pf_batch_run(fs, [w.theta for w in ws], [w.y for w in ws],
                                       [7 + k for k in range(len(ws))])
            assert [(int(a), b) for a, b in zip(sts, lls)] == [(int(a), b) for a, b in ref], shape
    finally:
        for f in fs:
            f.destroy()
