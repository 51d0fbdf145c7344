"""GPU tests of the batched form's persistent launch: the tiled filters of a
batch run in one grid of resident CTAs that take (filter, phase, tiles) work
items from a device queue, the CTA finishing a phase queueing the filter's
next one.  Every filter must give the bits of its own single run, whatever
the CTAs per SM and the tiles per item, on the first run (plan and graph
built) and on a replay; filters that stop early (a degenerate step) must not
hold up the others; shapes outside the kernel's classes fall back to the
per-step chains with the same bits; a wait that runs out (a slot nothing
fills, planted on the host) ends the launch with PF_ETIMEOUT and leaves the
device usable."""
import math
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


def _mix(prec):
    """Windkessel and Lorenz '96 N = 8 filters of one precision: uneven P
    (one tile to more than one group of 256 tiles, ragged last tiles) and T,
    every resampling mode the queue distinguishes (every step, adaptive,
    never), stratified resampling and sparse observations."""
    ws = W.batched(n_wk=5, n_l96=5, pmin=6, pmax=13, tmin=1, tmax=70, prec=prec)
    ws += [W.windkessel(P=300, T=40, ess_threshold=0.5, seed=3, prec=prec),
           W.windkessel(P=500, T=30, ess_threshold=0.0, seed=4, prec=prec),
           W.lorenz96_8(P=700, T=25, prec=prec, seed=5).with_(resampler=1),
           W.lorenz96_sparse(P=1500, T=30, seed=7, prec=prec),
           W.windkessel(P=256, T=1, seed=8, prec=prec),
           W.windkessel(P=70000, T=6, seed=9, prec=prec),  # 274 tiles: two groups
           W.lorenz96_8(P=3000, T=9, prec=prec, ess_threshold=0.5, seed=10)]
    return ws


def _run_batch(pf, fs, ws, thetas=None):
    return pf.pf_batch_run(fs, thetas or [w.theta for w in ws], [w.y for w in ws],
                           [w.seed for w in ws])


@pytest.mark.parametrize("prec", [W.MIXED, W.FP64], ids=["mixed", "fp64"])
@pytest.mark.parametrize("bps,kt", [(1, 1), (3, 1), (2, 2), (4, 8), (3, 4)])
def test_persistent_launch_is_bit_identical(prec, bps, kt):
    import paper_1306_3277_b300 as pf
    ws = _mix(prec)
    fs = [pf.pf_create(pf.model_from_workload(w), w.P, w.T, w.dt) for w in ws]
    try:
        ref = [f.run(w.theta, w.y, w.seed)[:2] for w, f in zip(ws, fs)]
        pf.pf_batch_set_shape(fs, 0, 1, 8, bps, kt)
        assert pf.pf_batch_get_shape(fs)["persistent_blocks_per_sm"] == bps
        for _ in range(2):  # the second run replays the cached graph
            lls, sts = _run_batch(pf, fs, ws)
            for k, (st, ll) in enumerate(ref):
                assert sts[k] == st and lls[k] == ll, (k, ws[k].name, lls[k], ll)
    finally:
        for f in fs:
            f.destroy()


@pytest.mark.parametrize("kt", [1, 2])
def test_persistent_edge_sizes(kt):
    """One-particle filters, exact and ragged tiles, one- to three-step runs,
    in both model classes and the queue's two forms (whole run on one CTA,
    queued items): every filter gives its single run's bits."""
    import paper_1306_3277_b300 as pf
    ws = []
    for k, (P, T) in enumerate([(1, 1), (1, 3), (2, 2), (255, 1), (256, 2), (257, 3), (513, 2),
                                (769, 3), (1, 2), (300, 1)]):
        if k % 2:
            ws.append(W.lorenz96_8(P=P, T=T, prec=W.MIXED, seed=k + 1))
        else:
            ws.append(W.windkessel(P=P, T=T, prec=W.MIXED, seed=k + 1))
    fs = [pf.pf_create(pf.model_from_workload(w), w.P, w.T, w.dt) for w in ws]
    try:
        ref = [f.run(w.theta, w.y, w.seed)[:2] for w, f in zip(ws, fs)]
        pf.pf_batch_set_shape(fs, 0, 1, 8, 3, kt)
        for _ in range(2):
            lls, sts = _run_batch(pf, fs, ws)
            assert [(int(a), b) for a, b in zip(sts, lls)] == [(int(a), b) for a, b in ref]
    finally:
        for f in fs:
            f.destroy()


@pytest.mark.parametrize("kt", [1, 4])
def test_persistent_degenerate_filters_end_early(kt):
    """Zero observation variance makes every weight zero at the first step: the
    filter reports PF_EDEGENERATE with log-likelihood -inf, and its remaining
    work items are struck from the queue's total (a 12-tile filter in queued
    items, a 1-tile filter on its own CTA), so the others finish unchanged."""
    import paper_1306_3277_b300 as pf
    ws = [W.windkessel(P=3000, T=20, seed=1, prec=W.MIXED),
          W.windkessel(P=256, T=15, seed=2, prec=W.MIXED),
          W.windkessel(P=2000, T=12, seed=3, prec=W.MIXED),
          W.lorenz96_8(P=1000, T=10, seed=4, prec=W.MIXED)]
    thetas = [list(w.theta) for w in ws]
    thetas[0][4] = 0.0
    thetas[1][4] = 0.0
    fs = [pf.pf_create(pf.model_from_workload(w), w.P, w.T, w.dt) for w in ws]
    try:
        ref = [f.run(th, w.y, w.seed)[:2] for th, w, f in zip(thetas, ws, fs)]
        assert ref[0][0] == ref[1][0] == pf.PF_EDEGENERATE
        pf.pf_batch_set_shape(fs, 0, 1, 8, 2, kt)
        for _ in range(2):
            lls, sts = _run_batch(pf, fs, ws, thetas)
            assert sts[0] == sts[1] == pf.PF_EDEGENERATE
            assert lls[0] == lls[1] == -math.inf
            for k in (2, 3):
                assert sts[k] == ref[k][0] and lls[k] == ref[k][1]
    finally:
        for f in fs:
            f.destroy()


def test_classes_outside_the_kernel_fall_back_to_the_chains():
    """A Lorenz '96 N = 40 filter, an exact windkessel, a multinomial filter or
    mixed precisions keep the batch on the per-step chains: same bits."""
    import paper_1306_3277_b300 as pf
    cases = [
        [W.windkessel(P=600, T=10, seed=1, prec=W.MIXED), W.lorenz96_large(P=700, T=4, seed=2)],
        [W.windkessel(P=600, T=10, seed=1), W.windkessel_exact(P=256, T=12, seed=3)],
        [W.windkessel(P=600, T=10, seed=1), W.lorenz96_8(P=600, T=8, seed=4).with_(resampler=2)],
        [W.windkessel(P=600, T=10, seed=1), W.windkessel(P=900, T=7, seed=5, prec=W.MIXED)],
    ]
    for ws in cases:
        fs = [pf.pf_create(pf.model_from_workload(w), w.P, w.T, w.dt) for w in ws]
        try:
            ref = [f.run(w.theta, w.y, w.seed)[:2] for w, f in zip(ws, fs)]
            pf.pf_batch_set_shape(fs, 0, 2, 8, 2, 1)
            lls, sts = _run_batch(pf, fs, ws)
            assert [(int(a), b) for a, b in zip(sts, lls)] == [(int(a), b) for a, b in ref]
        finally:
            for f in fs:
                f.destroy()


def test_persistent_with_cluster_filters_and_invalid_shapes():
    """Cluster-path filters beside the persistent launch (a side branch of the
    same graph) keep their bits; out-of-range persistent fields are refused."""
    import paper_1306_3277_b300 as pf
    ws = _mix(W.MIXED)
    fs = [pf.pf_create(pf.model_from_workload(w), w.P, w.T, w.dt) for w in ws]
    try:
        ref = [f.run(w.theta, w.y, w.seed)[:2] for w, f in zip(ws, fs)]
        pf.pf_batch_set_shape(fs, 1024, 1, 8, 2, 2)
        lls, sts = _run_batch(pf, fs, ws)
        assert [(int(a), b) for a, b in zip(sts, lls)] == [(int(a), b) for a, b in ref]
        for bad in ((0, 1, 8, -1, 1), (0, 1, 8, 9, 1), (0, 1, 8, 2, 3), (0, 1, 8, 2, 16),
                    (0, 1, 8, 2, 0)):
            with pytest.raises(pf.PFError) as e:
                pf.pf_batch_set_shape(fs, *bad)
            assert e.value.status == pf.PF_EINVAL
    finally:
        for f in fs:
            f.destroy()


def test_autotuner_searches_the_persistent_fields():
    import paper_1306_3277_b300 as pf
    ws = W.batched(n_wk=8, n_l96=8, pmin=8, pmax=12, tmin=20, tmax=60)
    fs = [pf.pf_create(pf.model_from_workload(w), w.P, w.T, w.dt) for w in ws]
    try:
        ref = [f.run(w.theta, w.y, w.seed)[:2] for w, f in zip(ws, fs)]
        pf.pf_batch_autotune(fs, [w.theta for w in ws], [w.y for w in ws], [w.seed for w in ws])
        shape = pf.pf_batch_get_shape(fs)
        assert shape["persistent_blocks_per_sm"] in (0, 2, 3, 4)
        assert shape["tiles_per_item"] in (1, 2, 4)
        lls, sts = _run_batch(pf, fs, ws)
        assert [(int(a), b) for a, b in zip(sts, lls)] == [(int(a), b) for a, b in ref]
    finally:
        for f in fs:
            f.destroy()


def test_pmmh_chains_on_the_persistent_launch():
    """PMMH runs its chains' filters through the batch plan's graph: on the
    persistent launch every sample is the one the per-step chains give."""
    import paper_1306_3277_b300 as pf
    w = W.windkessel(P=512, T=30)
    spec = [(3, 1, 2.0, 0.9, 0.03, 0.0, math.inf), (0, 0), (3, 1, 2.0, 0.03, 0.002, 0.0, math.inf),
            (4, 2, 2.0, 0.01, 2.0, 3.0), (0, 0), (0, 0), (0, 0)]
    th0 = np.tile(np.array(w.theta), (8, 1))
    out = []
    for shape in ((0, 1, 8, 0, 1), (0, 1, 8, 2, 1), (0, 1, 8, 3, 2)):
        fs = [pf.pf_create(pf.model_from_workload(w), w.P, w.T, w.dt) for _ in range(8)]
        try:
            pf.pf_batch_set_shape(fs, *shape)
            out.append(pf.pf_pmmh_run(fs, w.y, spec, th0, 10, 5))
        finally:
            for f in fs:
                f.destroy()
    for o in out[1:]:
        assert np.array_equal(out[0][0], o[0]) and np.array_equal(out[0][1], o[1])


def test_persistent_wait_runs_out_and_the_device_stays_usable():
    """A slot that nothing fills (one slot more than the filters fill, counted
    by the host) makes a CTA's bounded wait run out: the launch ends with
    PF_ETIMEOUT, every kernel having returned, and the next batch on the same
    device gives the bits of the single runs."""
    import paper_1306_3277_b300 as pf
    def make():
        ws = [W.windkessel(P=2000, T=12, seed=1, prec=W.MIXED),
              W.lorenz96_8(P=1500, T=10, seed=2, prec=W.MIXED),
              W.windkessel(P=256, T=9, seed=3, prec=W.MIXED)]
        return ws, [pf.pf_create(pf.model_from_workload(w), w.P, w.T, w.dt) for w in ws]
    pf.pf_debug_persist_wait_limit(0.25)
    try:
        ws, fs = make()
        try:
            pf.pf_debug_persist_unfilled_slot(True)
            pf.pf_batch_set_shape(fs, 0, 1, 8, 2, 1)
            t0 = time.perf_counter()
            with pytest.raises(pf.PFError) as e:
                _run_batch(pf, fs, ws)
            assert e.value.status == pf.PF_ETIMEOUT
            assert time.perf_counter() - t0 < 10.0
        finally:
            pf.pf_debug_persist_unfilled_slot(False)
            for f in fs:
                f.destroy()
        ws, fs = make()
        try:
            ref = [f.run(w.theta, w.y, w.seed)[:2] for w, f in zip(ws, fs)]
            pf.pf_batch_set_shape(fs, 0, 1, 8, 2, 1)
            lls, sts = _run_batch(pf, fs, ws)
            assert [(int(a), b) for a, b in zip(sts, lls)] == [(int(a), b) for a, b in ref]
        finally:
            for f in fs:
                f.destroy()
        for bad in (0.0, -1.0, 61.0):
            with pytest.raises(pf.PFError) as e:
                pf.pf_debug_persist_wait_limit(bad)
            assert e.value.status == pf.PF_EINVAL
    finally:
        pf.pf_debug_persist_wait_limit(4.0)
