"""GPU tests of the sub-tile propagate launch.  FP64 filters whose plan's tiles
would leave most SMs idle (a filter running alone, a small batch) propagate
each 256-particle tile with 2 or 4 blocks; the last block of the tile gathers
the tile's log-weights and runs its reductions in the canonical order.
Results must be the bits of the same filter inside a batch whose tiles fill
the GPU (one block per tile),
on both sides of the 4 / 2 / 1 block-per-tile thresholds, with ragged last
tiles, for every model class that has the kernel, and the oracle's (ancestors
and particles bit-exact away from the near-boundary window, log-likelihood
within 1e-9)."""
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


# tile counts 12 and 20 (4 blocks per tile), 77 and 130 (2 blocks per tile for
# the two-blocks-per-SM FP64 Lorenz '96 kernels), 330 (one)
CASES = [
    ("l96_8_P3000", lambda: W.lorenz96_8(P=3000, T=12)),
    ("l96_8_P19700", lambda: W.lorenz96_8(P=19700, T=8)),
    ("l96_8_P33280_ess", lambda: W.lorenz96_8(P=33280, T=8, ess_threshold=0.5)),
    ("l96_8_P84480", lambda: W.lorenz96_8(P=84480, T=4)),
    ("l96_4_P5000", lambda: W.lorenz96_8(P=5000, T=10).with_(N=4, obs_stride=1)),
    ("l96_12_P9000", lambda: W.lorenz96_8(P=9000, T=6).with_(N=12, obs_stride=2)),
    ("l96_sparse_P4000", lambda: W.lorenz96_sparse(P=4000, T=12)),
    ("l96_sde_P3000", lambda: W.lorenz96_sde(P=3000, T=10)),
    ("l96_8_P2305_one_in_last", lambda: W.lorenz96_8(P=2305, T=6)),  # empty sub-blocks
    ("l96_8_P2433", lambda: W.lorenz96_8(P=2433, T=5)),  # 129 particles in the last tile
    ("wk_P5000_unsplit", lambda: W.windkessel(P=5000, T=30)),  # no sub-tile kernel
]


def _prepare(w):
    """y simulated for the workload's own shape (a with_() change of N or
    observed components needs its own observations)."""
    w.y = W.simulate(w)
    return w


@pytest.mark.parametrize("name,factory", CASES, ids=[c[0] for c in CASES])
def test_subtile_equals_batch_and_oracle(name, factory):
    import paper_1306_3277_b300 as pf
    w = _prepare(factory())
    seed = 5
    g = run_gpu(w, seed)  # alone: the sub-tile launch where it applies
    o = run_oracle(w, seed)
    compare(w, g, o)
    # the same filter in a batch whose tiles fill the GPU keeps one block per tile
    other = W.windkessel(P=1 << 18, T=3, seed=2, prec=W.MIXED)
    fs = [pf.pf_create(pf.model_from_workload(x), x.P, x.T, x.dt) for x in (w, other)]
    try:
        lls, sts = pf.pf_batch_run(fs, [w.theta, other.theta], [w.y, other.y], [seed, 2])
        assert int(sts[0]) == g["status"] and lls[0] == g["loglik"], (lls[0], g["loglik"])
    finally:
        for f in fs:
            f.destroy()


def test_small_fp64_batch_on_subtiles_equals_single_runs():
    """A batch of few FP64 Lorenz '96 filters takes the sub-tile launch too
    (beside windkessel filters, which keep one block per tile): every filter
    gives the bits of its single run."""
    import paper_1306_3277_b300 as pf
    ws = [W.lorenz96_8(P=1024, T=9, seed=50 + k) for k in range(6)]
    ws += [W.lorenz96_sde(P=512, T=7, seed=60 + k) for k in range(4)]
    ws += [W.windkessel(P=256, T=12, seed=k + 1) for k in range(10)]
    fs = [pf.pf_create(pf.model_from_workload(w), w.P, w.T, w.dt) for w in ws]
    try:
        ref = [f.run(w.theta, w.y, w.seed)[:2] for w, f in zip(ws, fs)]
        for branches in (1, 3):
            pf.pf_batch_set_shape(fs, 0, branches, 8)
            lls, sts = pf.pf_batch_run(fs, [w.theta for w in ws], [w.y for w in ws],
                                       [w.seed for w in ws])
            assert [(int(a), b) for a, b in zip(sts, lls)] == [(int(a), b) for a, b in ref]
    finally:
        for f in fs:
            f.destroy()


def test_subtile_step_entries_share_the_plan():
    """pf_run_range over two intervals and a teacher-forced step run the
    single-filter plan (with the sub-tile launch): the intervals give pf_run's
    log-likelihood and particles."""
    import paper_1306_3277_b300 as pf
    w = W.lorenz96_8(P=6000, T=10)
    f = pf.pf_create(pf.model_from_workload(w), w.P, w.T, w.dt)
    try:
        st, ll, x, _ = f.run(w.theta, w.y, 9, want_particles=True)
        st1, ll1, _ = f.run_range(w.theta, w.y[0:4], 9, 0, 4)
        st2, ll2, x2 = f.run_range(None, w.y[4:], 9, 4, w.T, want_particles=True)
        assert st == st1 == st2 == pf.PF_OK
        assert ll2 == ll
        assert np.array_equal(x2, x)
    finally:
        f.destroy()
