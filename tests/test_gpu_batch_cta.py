"""GPU tests of the batched form's launch shapes: filters sent to the cluster
path (one thread-block cluster runs a whole filter, one CTA per tile, on a
side branch of the plan's graph) or dealt into several independent branches of
per-step launches give the bits of their single runs, whatever the shape and
whatever the autotuner chooses; PMMH chains over such batches are unchanged
too."""
import math

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _mix():
    ws = W.batched(n_wk=6, n_l96=6, pmin=6, pmax=13, tmin=5, tmax=80)
    ws += [W.windkessel(P=300, T=40, ess_threshold=0.5, seed=3),
           W.windkessel(P=500, T=30, ess_threshold=0.0, seed=4),
           W.lorenz96_8(P=700, T=25, prec=W.MIXED, seed=5).with_(resampler=1),
           W.lorenz96_8(P=600, T=20, seed=6).with_(resampler=2),  # multinomial: tiled path
           W.lorenz96_sparse(P=512, T=30, seed=7),
           W.windkessel_exact(P=256, T=25, seed=8),
           W.lorenz96_sde(P=256, T=15, prec=W.MIXED, seed=9),
           W.lorenz96_large(P=1000, T=6, seed=10),
           W.lorenz96_8(P=1 << 15, T=10, prec=W.MIXED, seed=11)]  # more than one group
    return ws


def _single(pf, ws, fs):
    return [f.run(w.theta, w.y, w.seed)[:2] for w, f in zip(ws, fs)]


@pytest.mark.parametrize("cta_max", [2048, 1024, 300])
def test_cluster_path_is_bit_identical(cta_max):
    import paper_1306_3277_b300 as pf
    ws = _mix()
    fs = [pf.pf_create(pf.model_from_workload(w), w.P, w.T, w.dt) for w in ws]
    try:
        ref = _single(pf, ws, fs)
        pf.pf_batch_configure(fs, cta_max)
        for _ in range(2):  # the second run replays the cached graph
            lls, sts = pf.pf_batch_run(fs, [w.theta for w in ws], [w.y for w in ws],
                                       [w.seed for w in ws])
            for k, (st, ll) in enumerate(ref):
                assert sts[k] == st and lls[k] == ll, (k, ws[k].name, lls[k], ll)
    finally:
        for f in fs:
            f.destroy()


def test_degenerate_filter_on_the_cluster_path():
    import paper_1306_3277_b300 as pf
    ws = [W.windkessel(P=256, T=10, seed=1), W.windkessel(P=512, T=12, seed=2)]
    th_bad = list(ws[0].theta)
    th_bad[4] = 0.0  # zero observation variance
    fs = [pf.pf_create(pf.model_from_workload(w), w.P, w.T, w.dt) for w in ws]
    try:
        ref = [fs[0].run(th_bad, ws[0].y, 1)[:2], fs[1].run(ws[1].theta, ws[1].y, 2)[:2]]
        pf.pf_batch_configure(fs, 1024)
        lls, sts = pf.pf_batch_run(fs, [th_bad, ws[1].theta], [w.y for w in ws], [1, 2])
        assert sts[0] == pf.PF_EDEGENERATE and lls[0] == -math.inf
        assert sts[1] == ref[1][0] and lls[1] == ref[1][1]
    finally:
        for f in fs:
            f.destroy()


def test_autotuner_choice_keeps_results_and_pmmh():
    import paper_1306_3277_b300 as pf
    ws = W.batched(n_wk=8, n_l96=8, pmin=8, pmax=12, tmin=20, tmax=60)
    fs = [pf.pf_create(pf.model_from_workload(w), w.P, w.T, w.dt) for w in ws]
    try:
        ref = _single(pf, ws, fs)
        chosen = pf.pf_batch_autotune(fs, [w.theta for w in ws], [w.y for w in ws],
                                      [w.seed for w in ws])
        assert chosen in (0, 256, 512, 1024, 2048)
        shape = pf.pf_batch_get_shape(fs)
        assert shape["cta_max_particles"] == chosen
        assert shape["branches"] in (1, 2, 4, 8, 16)
        assert shape["resample_blocks_per_sm"] in (2, 4, 8)
        lls, sts = pf.pf_batch_run(fs, [w.theta for w in ws], [w.y for w in ws],
                                   [w.seed for w in ws])
        assert [(int(a), b) for a, b in zip(sts, lls)] == [(int(a), b) for a, b in ref]
    finally:
        for f in fs:
            f.destroy()
    # PMMH chains over one windkessel shape: tiled and cluster splits agree
    w = W.windkessel(P=512, T=40)
    spec = [(3, 1, 2.0, 0.9, 0.03, 0.0, math.inf), (0, 0), (3, 1, 2.0, 0.03, 0.002, 0.0, math.inf),
            (4, 2, 2.0, 0.01, 2.0, 3.0), (0, 0), (0, 0), (0, 0)]
    th0 = np.tile(np.array(w.theta), (6, 1))
    out = []
    for cta in (0, 1024):
        fs = [pf.pf_create(pf.model_from_workload(w), w.P, w.T, w.dt) for _ in range(6)]
        try:
            pf.pf_batch_configure(fs, cta)
            out.append(pf.pf_pmmh_run(fs, w.y, spec, th0, 15, 3))
        finally:
            for f in fs:
                f.destroy()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


@pytest.mark.parametrize("branches,cta,rs", [(2, 0, 8), (3, 0, 4), (8, 1024, 2), (64, 0, 1)])
def test_branches_are_bit_identical(branches, cta, rs):
    """The tiled filters dealt into independent launch chains (parallel branches
    of the captured graph) give the bits of their single runs; the first run
    builds and captures the plan, the second replays it."""
    import paper_1306_3277_b300 as pf
    ws = [w for w in _mix() if w.resampler != 2]
    fs = [pf.pf_create(pf.model_from_workload(w), w.P, w.T, w.dt) for w in ws]
    try:
        ref = _single(pf, ws, fs)
        pf.pf_batch_set_shape(fs, cta, branches, rs)
        assert pf.pf_batch_get_shape(fs) == {"cta_max_particles": cta, "branches": branches,
                                             "resample_blocks_per_sm": rs,
                                             "persistent_blocks_per_sm": 0,
                                             "tiles_per_item": 1}
        for _ in range(2):
            lls, sts = pf.pf_batch_run(fs, [w.theta for w in ws], [w.y for w in ws],
                                       [w.seed for w in ws])
            for k, (st, ll) in enumerate(ref):
                assert sts[k] == st and lls[k] == ll, (k, ws[k].name, lls[k], ll)
    finally:
        for f in fs:
            f.destroy()


def test_branches_with_a_multinomial_filter_and_invalid_shapes():
    """A multinomial filter keeps the plan on one chain (same bits); shapes out
    of range are refused."""
    import paper_1306_3277_b300 as pf
    ws = _mix()
    fs = [pf.pf_create(pf.model_from_workload(w), w.P, w.T, w.dt) for w in ws]
    try:
        ref = _single(pf, ws, fs)
        pf.pf_batch_set_shape(fs, 0, 4, 8)
        lls, sts = pf.pf_batch_run(fs, [w.theta for w in ws], [w.y for w in ws],
                                   [w.seed for w in ws])
        assert [(int(a), b) for a, b in zip(sts, lls)] == [(int(a), b) for a, b in ref]
        for bad in ((-1, 1, 8), (0, 0, 8), (0, 1, 0), (0, 1, 9)):
            with pytest.raises(pf.PFError) as e:
                pf.pf_batch_set_shape(fs, *bad)
            assert e.value.status == pf.PF_EINVAL
    finally:
        for f in fs:
            f.destroy()


def test_samplers_unchanged_by_branches():
    """PMMH chains run their filters through a batch plan: dealing the chains
    into branches changes none of their samples."""
    import paper_1306_3277_b300 as pf
    w = W.windkessel(P=512, T=30)
    spec = [(3, 1, 2.0, 0.9, 0.03, 0.0, math.inf), (0, 0), (3, 1, 2.0, 0.03, 0.002, 0.0, math.inf),
            (4, 2, 2.0, 0.01, 2.0, 3.0), (0, 0), (0, 0), (0, 0)]
    th0 = np.tile(np.array(w.theta), (8, 1))
    out = []
    for branches in (1, 4):
        fs = [pf.pf_create(pf.model_from_workload(w), w.P, w.T, w.dt) for _ in range(8)]
        try:
            pf.pf_batch_set_shape(fs, 0, branches, 8)
            out.append(pf.pf_pmmh_run(fs, w.y, spec, th0, 10, 5))
        finally:
            for f in fs:
                f.destroy()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
