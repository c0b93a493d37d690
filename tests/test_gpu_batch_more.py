"""GPU parity of the batched counts (Sect. 4.2 task queue) with weights and on
non-periodic catalogues: each row of one launch over several catalogues must
equal the oracle's count of that catalogue (counts bit-exact, weighted sums
within 1e-10 relative per bin), with and without CUDA-graph replay, for the
grid batch and the k-d tree batch.
"""

import numpy as np
import pytest

import oracle
import synth

P = pytest.importorskip("paper_2301_12557_gb300")
torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

WREL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P.build()
    oracle.build()
    torch.cuda.init()
    yield


def _check(got, want, gw=None, ww=None, what=""):
    if not np.array_equal(got, want):
        bad = np.nonzero(got != want)[0]
        raise AssertionError(f"{what}: {bad.size} bins differ, first {bad[:8].tolist()}: "
                             f"gpu {got[bad[:8]].tolist()} oracle {want[bad[:8]].tolist()}")
    if ww is not None:
        zero = ww == 0
        assert np.all(gw[zero] == 0), what
        rel = np.abs(gw[~zero] - ww[~zero]) / np.abs(ww[~zero])
        assert rel.size == 0 or rel.max() <= WREL, f"{what}: weighted rel err {rel.max():.3e}"


@pytest.mark.parametrize("wdtype", [np.float32, np.float64])
def test_grid_batch_weighted(wdtype):
    L = 300.0
    mocks = synth.batch_mocks(5, 800, 4000, 3.0, 8.0, L, 991)
    ws = [synth.lognormal_weights(m.shape[0], 0.3, 992 + k, wdtype) for k, m in enumerate(mocks)]
    ea = np.linspace(0.0, 40.0, 21)
    mu = np.linspace(0.0, 1.0, 11)
    bins = P.Bins("smu", "z", ea, mu)
    box = P.make_box(L, True)
    opts = P.make_opts("f32", 20.0)
    grids = [P.pc_build_grid(m, w, box=box, r_max=bins.r_max, opts=opts)
             for m, w in zip(mocks, ws)]
    try:
        for use_graph in (0, 1):
            opts.use_graph = use_graph
            c, wc, _ = P.pc_count_batch(grids, bins, opts, weighted=True)
            c = c.reshape(len(mocks), -1)
            wc = wc.reshape(len(mocks), -1)
            for k, (m, w) in enumerate(zip(mocks, ws)):
                want, wantw = oracle.count(m, w1=w.astype(np.float64), box=L, periodic=True,
                                           mode="smu", edges_a=ea, edges_b=mu, method="grid")
                _check(c[k], want, wc[k], wantw, f"mock {k} graph {use_graph}")
    finally:
        for g in grids:
            g.free()


def test_batch_of_survey_shells_midpoint():
    """Four survey-shell catalogues (different sizes, FKP weights) counted in
    (sigma, pi) along the midpoint line of sight in one launch: the grid
    batch on common bounds and one cell side, and the tree batch."""
    cats = [synth.survey_shell(n, True, 1001 + k) for k, n in enumerate([3000, 500, 2000, 1])]
    ws = [synth.fkp_weights(c, 3000) for c in cats]
    ea = np.linspace(0.0, 30.0, 11)
    eb = np.linspace(0.0, 30.0, 7)
    bins = P.Bins("sigpi", "mid", ea, eb)
    lo = np.min([c.min(0) for c in cats], axis=0) - 1.0
    hi = np.max([c.max(0) for c in cats], axis=0) + 1.0
    want = [oracle.count(c, w1=w, periodic=False, mode="sigpi", los="mid", edges_a=ea,
                         edges_b=eb, method="grid") for c, w in zip(cats, ws)]
    assert want[0][0].sum() > 0
    box = P.make_box(None, False, lo, hi)
    opts = P.make_opts("f32", 40.0)
    grids = [P.pc_build_grid(c, w, box=box, r_max=bins.r_max, opts=opts)
             for c, w in zip(cats, ws)]
    try:
        for use_graph in (0, 1):
            opts.use_graph = use_graph
            c, wc, st = P.pc_count_batch(grids, bins, opts, weighted=True)
            assert st.prec == P.PC_PREC_F32_RESCUE
            c = c.reshape(len(cats), -1)
            wc = wc.reshape(len(cats), -1)
            for k in range(len(cats)):
                _check(c[k], want[k][0], wc[k], want[k][1], f"grid shell {k} graph {use_graph}")
    finally:
        for g in grids:
            g.free()
    tb = P.make_box(None, False)
    trees = [P.pc_build_tree(c, w, box=tb) for c, w in zip(cats, ws)]
    try:
        c, wc, _ = P.pc_count_tree_batch(trees, bins, P.make_opts("f32", 0.0, 2), weighted=True)
        c = c.reshape(len(cats), -1)
        wc = wc.reshape(len(cats), -1)
        for k in range(len(cats)):
            _check(c[k], want[k][0], wc[k], want[k][1], f"tree shell {k}")
    finally:
        for t in trees:
            t.free()
