"""GPU parity of the paper-exact model variants: sparse observations (steps
without an observation, the first components only, as in the paper's
Lorenz '96 example), the exact windkessel transition (exponential decay,
noise on the flow) and Lorenz '96 with the Wiener increment inside RK4.
Ancestors and final particles bit-exact and log-likelihood within 1e-9
relative against the oracle, outside near-boundary targets; batched,
sampled-path and server runs agree too."""
import numpy as np
import pytest

import workloads as W
from pf_parity import compare, run_gpu, run_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _resim(w):
    w.y = W.simulate(w)
    return w


SPARSE = [
    ("lorenz96 sparse N=8 P=2^14 T=60 FP64", lambda: W.lorenz96_sparse(), (1, 2)),
    ("lorenz96 sparse N=8 P=2^14 T=60 mixed", lambda: W.lorenz96_sparse(prec=W.MIXED), (3,)),
    ("lorenz96 sparse P=3000 T=40 ESS 0.5", lambda: W.lorenz96_sparse(P=3000, T=40,
                                                                      ess_threshold=0.5), (4,)),
    ("windkessel every 3rd step P=1000 T=60",
     lambda: W.windkessel(P=1000, T=60).with_(obs_every=3), (5,)),
    ("windkessel every 2nd step, never resample",
     lambda: W.windkessel(P=300, T=30, ess_threshold=0.0).with_(obs_every=2), (6,)),
    ("windkessel every 4th step multinomial",
     lambda: W.windkessel(P=500, T=40).with_(obs_every=4, resampler=2), (7,)),
    ("lorenz96 N=40 first 10 of the even components every 3rd step",
     lambda: _resim(W.lorenz96_large(P=3000, T=21).with_(obs_count=10, obs_every=3)), (8,)),
]


@pytest.mark.parametrize("name,factory,seeds", SPARSE, ids=[c[0] for c in SPARSE])
def test_sparse_parity(name, factory, seeds):
    w = factory()
    for seed in seeds:
        o = run_oracle(w, seed)
        g = run_gpu(w, seed)
        rows, _ = compare(w, g, o)
        assert rows >= 1
        steps = np.arange(1, w.T + 1)
        unobserved = steps % max(w.obs_every, 1) != 0
        assert np.all(o["diag"][unobserved, 6] == 0.0)


def test_sparse_batch_and_path():
    import oracle as O
    import paper_1306_3277_b300 as pf
    from pf_parity import oracle_model
    ws = [W.lorenz96_sparse(P=1000, T=30, seed=3), W.windkessel(P=700, T=33).with_(obs_every=3),
          W.lorenz96_8(P=900, T=20)]
    fs = [pf.pf_create(pf.model_from_workload(w), w.P, w.T, w.dt) for w in ws]
    try:
        lls, sts = pf.pf_batch_run(fs, [w.theta for w in ws], [w.y for w in ws],
                                   [w.seed for w in ws])
        for k, (w, f) in enumerate(zip(ws, fs)):
            st, ll, _, _ = f.run(w.theta, w.y, w.seed)
            assert sts[k] == st and lls[k] == ll
        w, f = ws[0], fs[0]
        st, ll, path, idx = f.sample_path(w.theta, w.y, 5)
        ost, oll, opath, oidx = O.sample_path(oracle_model(w), w.theta, w.y, 5, w.P, w.T)
        assert st == ost == pf.PF_OK and abs(ll - oll) <= 1e-9 * abs(oll)
        assert np.array_equal(idx, oidx) and np.array_equal(path, opath)
    finally:
        for f in fs:
            f.destroy()


BIG = (1.0, 1.5, 0.03, 4.0e4, 4.0, 90.0, 15.0)  # flow noise large enough to matter
L96W_40 = (8.0, 0.25, 1.0, 0.0, 1.0)

EXACT = [
    ("exact windkessel P=1024 T=100 FP64", lambda: W.windkessel_exact(), (1, 2)),
    ("exact windkessel sigma2=4e4 P=1000 T=60 s=3 FP64",
     lambda: W.windkessel_exact(P=1000, T=60, substeps=3, theta=BIG), (3,)),
    ("exact windkessel sigma2=4e4 P=1000 T=60 s=3 mixed",
     lambda: W.windkessel_exact(P=1000, T=60, substeps=3, theta=BIG, prec=W.MIXED), (4,)),
    ("exact windkessel ESS 0.5 P=777 T=80",
     lambda: W.windkessel_exact(P=777, T=80, ess_threshold=0.5, theta=BIG), (5,)),
    ("sde lorenz96 N=8 P=2^14 T=100 FP64", lambda: W.lorenz96_sde(T=100), (6,)),
    ("sde lorenz96 N=8 P=2^14 T=100 mixed", lambda: W.lorenz96_sde(T=100, prec=W.MIXED), (7,)),
    ("sde lorenz96 N=8 s=5 dt=0.01 P=5000 T=40 mixed",
     lambda: W.lorenz96_sde(P=5000, T=40, substeps=5, dt=0.01, prec=W.MIXED), (8,)),
    ("sde lorenz96 N=40 s=10 dt=0.005 P=3000 T=10 mixed",
     lambda: W.lorenz96_sde(P=3000, T=10, N=40, substeps=10, dt=0.005, obs_stride=2,
                            prec=W.MIXED, theta=L96W_40), (9,)),
    ("sde lorenz96 N=40 FP64 P=2^12+5 T=6",
     lambda: W.lorenz96_sde(P=4101, T=6, N=40, substeps=10, dt=0.005, obs_stride=2,
                            theta=L96W_40), (10,)),
]


@pytest.mark.parametrize("name,factory,seeds", EXACT, ids=[c[0] for c in EXACT])
def test_exact_variant_parity(name, factory, seeds):
    w = factory()
    for seed in seeds:
        o = run_oracle(w, seed)
        g = run_gpu(w, seed)
        rows, _ = compare(w, g, o)
        assert rows >= 1


def test_exact_variants_in_batch_and_server():
    import time
    import paper_1306_3277_b300 as pf
    ws = [W.windkessel_exact(P=600, T=25, theta=BIG, seed=2),
          W.lorenz96_sde(P=800, T=20, prec=W.MIXED, seed=3), W.windkessel(P=300, T=20),
          W.lorenz96_8(P=500, T=15, prec=W.MIXED)]
    fs = [pf.pf_create(pf.model_from_workload(w), w.P, w.T, w.dt) for w in ws]
    try:
        ref, singles = [], []
        for w, f in zip(ws, fs):
            st, ll, _, _ = f.run(w.theta, w.y, w.seed)
            singles.append((st, ll))
            ref.append(ll)
        # the default shape, one launch chain, the cluster path, the persistent
        # launch (whose classes these variants are not: they take launch chains)
        for shape in (None, (0, 1, 8, 0, 1), (4096, 2, 4, 0, 1), (0, 1, 8, 4, 2)):
            if shape is not None:
                pf.pf_batch_set_shape(fs, *shape)
            lls, sts = pf.pf_batch_run(fs, [w.theta for w in ws], [w.y for w in ws],
                                       [w.seed for w in ws])
            for k, (st, ll) in enumerate(singles):
                assert sts[k] == st and lls[k] == ll, (k, shape)
    finally:
        for f in fs:
            f.destroy()
    srv = pf.pf_server_create(1 << 30, 8)
    try:
        ts = [srv.submit(pf.model_from_workload(w), w.P, w.T, w.dt, w.theta, w.y, w.seed)
              for w in ws]
        got, deadline = {}, time.time() + 60
        while len(got) < len(ts) and time.time() < deadline:
            for t in ts:
                if t not in got:
                    r = srv.poll(t)
                    if r is not None:
                        got[t] = r
            time.sleep(0.001)
        assert [got[t][1] for t in ts] == ref
    finally:
        srv.destroy()
