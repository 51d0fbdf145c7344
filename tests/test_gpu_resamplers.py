"""GPU parity of the stratified and multinomial resamplers (Sec. 3.3;
Algorithm 2's multinomial draw): ancestors and final particles bit-exact and
log-likelihood within 1e-9 relative against the oracle, outside near-boundary
targets; batched runs that mix the three schemes equal their single runs;
the server takes stratified requests and refuses multinomial ones."""
import numpy as np
import pytest

import workloads as W
from pf_parity import compare, run_gpu, run_oracle

pytestmark = pytest.mark.gpu
STRAT, MULTI = 1, 2


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


CASES = [
    ("windkessel P=1000 T=60 stratified", lambda: W.windkessel(P=1000, T=60).with_(resampler=STRAT),
     (1, 2)),
    ("windkessel P=1000 T=60 multinomial", lambda: W.windkessel(P=1000, T=60).with_(resampler=MULTI),
     (1, 2)),
    ("windkessel P=777 T=80 ESS 0.5 multinomial",
     lambda: W.windkessel(P=777, T=80, ess_threshold=0.5).with_(resampler=MULTI), (3,)),
    ("lorenz96 N=8 P=5000 T=40 mixed stratified",
     lambda: W.lorenz96_8(P=5000, T=40, prec=W.MIXED).with_(resampler=STRAT), (4,)),
    ("lorenz96 N=8 P=5000 T=40 mixed multinomial",
     lambda: W.lorenz96_8(P=5000, T=40, prec=W.MIXED).with_(resampler=MULTI), (5,)),
    ("lorenz96 N=40 P=2^16+5 T=6 FP64 multinomial",
     lambda: W.lorenz96_large(P=(1 << 16) + 5, T=6, prec=W.FP64).with_(resampler=MULTI), (6,)),
    ("lorenz96 N=40 P=2^16+5 T=6 FP64 stratified",
     lambda: W.lorenz96_large(P=(1 << 16) + 5, T=6, prec=W.FP64).with_(resampler=STRAT), (7,)),
    ("windkessel P=256 T=20 multinomial", lambda: W.windkessel(P=256, T=20).with_(resampler=MULTI),
     (8,)),
    ("windkessel P=1 T=5 stratified", lambda: W.windkessel(P=1, T=5).with_(resampler=STRAT), (9,)),
    ("windkessel P=257 T=20 multinomial", lambda: W.windkessel(P=257, T=20).with_(resampler=MULTI),
     (10,)),
]


@pytest.mark.parametrize("name,factory,seeds", CASES, ids=[c[0] for c in CASES])
def test_parity(name, factory, seeds):
    w = factory()
    for seed in seeds:
        o = run_oracle(w, seed)
        g = run_gpu(w, seed)
        rows, _ = compare(w, g, o)
        assert rows >= 1


def test_large_shape_full_particle_count_multinomial():
    w = W.lorenz96_large(T=3).with_(resampler=MULTI)
    o = run_oracle(w, 12)
    g = run_gpu(w, 12)
    compare(w, g, o)


def test_batch_mixing_schemes_equals_single_runs():
    import paper_1306_3277_b300 as pf
    ws = []
    for k, base in enumerate([W.windkessel(P=300, T=25), W.lorenz96_8(P=700, T=12, prec=W.MIXED),
                              W.windkessel(P=513, T=30, ess_threshold=0.5)]):
        for rs in (0, STRAT, MULTI):
            ws.append(base.with_(resampler=rs, seed=10 * k + rs + 1))
    fs = [pf.pf_create(pf.model_from_workload(w), w.P, w.T, w.dt) for w in ws]
    try:
        ref = [f.run(w.theta, w.y, w.seed)[:2] for w, f in zip(ws, fs)]
        # the default shape, one launch chain, the cluster path for the small
        # filters (multinomial ones stay tiled), the persistent launch
        for shape in (None, (0, 1, 8, 0, 1), (4096, 2, 4, 0, 1), (0, 1, 8, 4, 2)):
            if shape is not None:
                pf.pf_batch_set_shape(fs, *shape)
            lls, sts = pf.pf_batch_run(fs, [w.theta for w in ws], [w.y for w in ws],
                                       [w.seed for w in ws])
            for k, (st, ll) in enumerate(ref):
                assert sts[k] == st and lls[k] == ll, (k, ws[k].resampler, shape)
    finally:
        for f in fs:
            f.destroy()


def test_server_takes_stratified_and_refuses_multinomial():
    import time
    import paper_1306_3277_b300 as pf
    w = W.lorenz96_8(P=1000, T=20, prec=W.MIXED).with_(resampler=STRAT)
    f = pf.pf_create(pf.model_from_workload(w), w.P, w.T, w.dt)
    _, ll_ref, _, _ = f.run(w.theta, w.y, 3)
    f.destroy()
    srv = pf.pf_server_create(1 << 30, 4)
    try:
        t = srv.submit(pf.model_from_workload(w), w.P, w.T, w.dt, w.theta, w.y, 3)
        res, deadline = None, time.time() + 60
        while res is None and time.time() < deadline:
            res = srv.poll(t)
            time.sleep(0.001)
        assert res is not None and res[0] == pf.PF_OK and res[1] == ll_ref
        m = w.with_(resampler=MULTI)
        with pytest.raises(pf.PFError) as e:
            srv.submit(pf.model_from_workload(m), m.P, m.T, m.dt, m.theta, m.y, 3)
        assert e.value.status == pf.PF_EINVAL
    finally:
        srv.destroy()


def test_unknown_resampler_rejected():
    import paper_1306_3277_b300 as pf
    with pytest.raises(pf.PFError) as e:
        pf.pf_create(pf.model(pf.PF_WINDKESSEL, resampler=3), 10, 10, 0.01)
    assert e.value.status == pf.PF_EINVAL
