"""GPU tests of Algorithm 2 over intervals t_{r:s} and of the single-path
sample: consecutive intervals give the bits of one whole run, every interval
end matches the oracle's state history and running likelihood, and the path
drawn on the GPU is the oracle's path (indices exact, states bit-exact)
outside near-boundary draws."""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W
from pf_parity import oracle_model

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


RANGE_CASES = [
    ("windkessel P=1000 T=60 ESS 0.5 FP64", lambda: W.windkessel(P=1000, T=60, ess_threshold=0.5),
     (0, 1, 17, 18, 45, 60)),
    ("windkessel P=300 T=30 never resample", lambda: W.windkessel(P=300, T=30, ess_threshold=0.0),
     (0, 10, 30)),
    ("lorenz96 N=8 P=5000 T=40 mixed", lambda: W.lorenz96_8(P=5000, T=40, prec=W.MIXED),
     (0, 7, 8, 39, 40)),
    ("lorenz96 N=40 P=3000 T=20 mixed", lambda: W.lorenz96_large(P=3000, T=20), (0, 5, 20)),
    ("lorenz96 N=8 P=2^12+3 T=25 FP64", lambda: W.lorenz96_8(P=4099, T=25), (0, 12, 25)),
]


def _near_step(o):
    near = np.nonzero(o["diag"][:, 7] > 0)[0]
    return int(near[0]) + 1 if len(near) else None


@pytest.mark.parametrize("name,factory,cuts", RANGE_CASES, ids=[c[0] for c in RANGE_CASES])
def test_range_pieces_equal_whole_run_and_oracle(name, factory, cuts):
    import paper_1306_3277_b300 as pf
    w = factory()
    seed = 21
    m = pf.model_from_workload(w)
    f = pf.pf_create(m, w.P, w.T, w.dt)
    try:
        st_full, ll_full, x_full, _ = f.run(w.theta, w.y, seed, want_particles=True)
        o = O.pf_run(oracle_model(w), w.theta, w.y, seed, w.P, w.T)
        ox = O.pf_run_ex(oracle_model(w), w.theta, w.y, seed, w.P, w.T)
        running = np.cumsum(o["diag"][:, 6])
        first_near = _near_step(o)
        for _ in range(2):  # a second pass over the same filter starts again at r = 0
            for r, s in zip(cuts[:-1], cuts[1:]):
                st, ll, x = f.run_range(w.theta if r == 0 else None, w.y[r:s], seed, r, s,
                                        want_particles=True)
                assert st == pf.PF_OK
                if first_near is None or s < first_near:
                    assert np.array_equal(x, ox["xhist"][s].astype(x.dtype))
                    assert abs(ll - running[s - 1]) <= 1e-9 * abs(running[s - 1])
            assert ll == ll_full and np.array_equal(x, x_full)
        assert st_full == pf.PF_OK
    finally:
        f.destroy()


@pytest.mark.parametrize("name,factory,cuts", RANGE_CASES[:4], ids=[c[0] for c in RANGE_CASES[:4]])
def test_range_fresh_key_per_interval_matches_oracle_schedule(name, factory, cuts):
    import paper_1306_3277_b300 as pf
    w = factory()
    keys = [1000003 * (k + 1) + 17 for k in range(len(cuts) - 1)]
    sched = np.zeros(w.T + 1, dtype=np.uint64)
    sched[0] = keys[0]
    for k, (r, s) in enumerate(zip(cuts[:-1], cuts[1:])):
        sched[r + 1:s + 1] = keys[k]
    o = O.pf_run_sched(oracle_model(w), w.theta, w.y, sched, w.P, w.T, want_xhist=True)
    running = np.cumsum(o["diag"][:, 6])
    first_near = _near_step(o)
    f = pf.pf_create(pf.model_from_workload(w), w.P, w.T, w.dt)
    try:
        for k, (r, s) in enumerate(zip(cuts[:-1], cuts[1:])):
            st, ll, x = f.run_range(w.theta if r == 0 else None, w.y[r:s], keys[k], r, s,
                                    want_particles=True)
            assert st == pf.PF_OK
            if first_near is None or s < first_near:
                assert np.array_equal(x, o["xhist"][s].astype(x.dtype))
                assert abs(ll - running[s - 1]) <= 1e-9 * abs(running[s - 1])
    finally:
        f.destroy()


def test_range_observations_from_device_memory():
    import torch
    import paper_1306_3277_b300 as pf
    w = W.lorenz96_8(P=2048, T=30, prec=W.MIXED)
    m = pf.model_from_workload(w)
    f = pf.pf_create(m, w.P, w.T, w.dt)
    try:
        _, ll_full, x_full, _ = f.run(w.theta, w.y, 5, want_particles=True)
        th = torch.tensor(w.theta, dtype=torch.float64, device="cuda")
        y = torch.tensor(w.y, dtype=torch.float64, device="cuda")
        ll = torch.zeros(1, dtype=torch.float64, device="cuda")
        x = torch.zeros((w.N, w.P), dtype=torch.float32, device="cuda")
        for r, s in ((0, 11), (11, 30)):
            pf.pf_run_range(f, th if r == 0 else None, y[r:s].contiguous(), 5, r, s, ll,
                            x if s == 30 else None)
        assert float(ll.item()) == ll_full
        assert np.array_equal(x.cpu().numpy(), x_full)
    finally:
        f.destroy()


def test_range_argument_errors():
    import paper_1306_3277_b300 as pf
    w = W.windkessel(P=256, T=20)
    f = pf.pf_create(pf.model_from_workload(w), w.P, w.T, w.dt)
    try:
        with pytest.raises(pf.PFError) as e:  # nothing to continue
            f.run_range(None, w.y[5:10], 1, 5, 10)
        assert e.value.status == pf.PF_EINVAL
        f.run_range(w.theta, w.y[:5], 1, 0, 5)
        for r, s in ((4, 10), (6, 10), (5, 5), (5, 21)):
            with pytest.raises(pf.PFError) as e:
                f.run_range(None, w.y[r:max(s, r + 1)], 1, r, s)
            assert e.value.status == pf.PF_EINVAL
        with pytest.raises(pf.PFError):  # r = 0 needs theta
            f.run_range(None, w.y[:5], 1, 0, 5)
        f.run_range(w.theta, w.y[:5], 1, 0, 5)
        f.run(w.theta, w.y, 1)  # a whole run ends the interval sequence
        with pytest.raises(pf.PFError) as e:
            f.run_range(None, w.y[5:10], 1, 5, 10)
        assert e.value.status == pf.PF_EINVAL
    finally:
        f.destroy()


def _pick_is_near(ellT, seed, T, P):
    w = O.philox4x32_10([0, T + 1, O.PURPOSE_PATH << 16, 0],
                        [seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF])
    v = (((int(w[1]) << 32) | int(w[0])) >> 11) / float(1 << 53)
    e = np.exp(ellT - ellT.max())
    C = np.cumsum(e)
    E = C * (P / C[-1])
    return np.min(np.abs(E - v * P)) <= 1e-9 * P


PATH_CASES = [
    ("windkessel P=1024 T=100 FP64", lambda: W.windkessel(), (1, 2)),
    ("windkessel P=777 T=80 ESS 0.5 FP64", lambda: W.windkessel(P=777, T=80, ess_threshold=0.5),
     (3,)),
    ("windkessel P=300 T=30 never resample", lambda: W.windkessel(P=300, T=30, ess_threshold=0.0),
     (4,)),
    ("lorenz96 N=8 P=2^14 T=60 mixed", lambda: W.lorenz96_8(T=60, prec=W.MIXED), (5,)),
    ("lorenz96 N=8 P=5000 T=40 ESS 0.5 FP64", lambda: W.lorenz96_8(P=5000, T=40,
                                                                   ess_threshold=0.5), (6,)),
    ("lorenz96 N=40 P=2^16+5 T=6 FP64", lambda: W.lorenz96_large(P=(1 << 16) + 5, T=6,
                                                                 prec=W.FP64), (7, 8)),
    ("lorenz96 N=40 P=3000 T=20 mixed", lambda: W.lorenz96_large(P=3000, T=20), (8,)),
]


@pytest.mark.parametrize("name,factory,seeds", PATH_CASES, ids=[c[0] for c in PATH_CASES])
def test_sample_path_matches_oracle(name, factory, seeds):
    import paper_1306_3277_b300 as pf
    w = factory()
    m = pf.model_from_workload(w)
    f = pf.pf_create(m, w.P, w.T, w.dt)
    compared = 0
    try:
        for seed in seeds:
            st, ll, path, idx = f.sample_path(w.theta, w.y, seed)
            ost, oll, opath, oidx = O.sample_path(oracle_model(w), w.theta, w.y, seed, w.P, w.T)
            assert st == ost == pf.PF_OK
            assert abs(ll - oll) <= 1e-9 * abs(oll)
            # the trace is a valid ancestry on the GPU's own history
            _, _, _, anc = f.run(w.theta, w.y, seed, want_ancestors=True)
            assert 0 <= idx.min() and idx.max() < w.P
            for i in range(w.T, 0, -1):
                assert idx[i - 1] == anc[i - 1][idx[i]]
            o = O.pf_run(oracle_model(w), w.theta, w.y, seed, w.P, w.T)
            ex = O.pf_run_ex(oracle_model(w), w.theta, w.y, seed, w.P, w.T)
            if _near_step(o) is None and not _pick_is_near(ex["ellT"], seed, w.T, w.P):
                assert np.array_equal(idx, oidx)
                assert np.array_equal(path, opath)
                compared += 1
    finally:
        f.destroy()
    assert compared >= 1


def test_sample_path_is_deterministic_and_leaves_runs_alone():
    import paper_1306_3277_b300 as pf
    w = W.lorenz96_8(P=4096, T=30, prec=W.MIXED)
    f = pf.pf_create(pf.model_from_workload(w), w.P, w.T, w.dt)
    try:
        _, ll0, x0, _ = f.run(w.theta, w.y, 9, want_particles=True)
        a = f.sample_path(w.theta, w.y, 9)
        b = f.sample_path(w.theta, w.y, 9)
        assert a[1] == b[1] == ll0
        assert np.array_equal(a[2], b[2]) and np.array_equal(a[3], b[3])
        _, ll1, x1, _ = f.run(w.theta, w.y, 9, want_particles=True)
        assert ll1 == ll0 and np.array_equal(x1, x0)
    finally:
        f.destroy()


def test_sample_path_degenerate_filter():
    import paper_1306_3277_b300 as pf
    w = W.windkessel(P=256, T=10)
    th = list(w.theta)
    th[4] = 0.0  # zero observation variance: every weight is zero
    f = pf.pf_create(pf.model_from_workload(w), w.P, w.T, w.dt)
    try:
        st, ll, path, idx = f.sample_path(th, w.y, 1)
        assert st == pf.PF_EDEGENERATE and ll == -math.inf
        assert np.all(np.isnan(path)) and np.all(idx == -1)
    finally:
        f.destroy()
