"""Whole histograms of full-size catalogues against stored oracle results.

tests/golden/fullsize/<target>.json hold the oracle's counts of every pair of
a whole catalogue (cell-list driver, binary64 definition), written by
tests/golden/make_fullsize.py, which calls only the oracle.  Each test here
regenerates the catalogue from its seed, checks that its bytes hash to the
stored value (so the GPU counts the very catalogue the oracle counted),
counts it through the C ABI in the launch configuration the benchmark times
(the options the autotuner picks on the same catalogue), and compares every
bin: counts bit-exact, weighted sums within 1e-10 relative (exact where the
oracle's sum is zero).  Sect. 5 of the paper reports identical results
between its two codes; this is that check for the GPU path against the
definition, at full size.

The 256-mock batch is checked against its stored mocks in
test_zy_full_size.py, which generates the whole batch once.
"""

import hashlib
import json
import os

import numpy as np
import pytest

from synth import catalogs as C
from synth import workloads as W

P = pytest.importorskip("paper_2301_12557_gb300")
torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "fullsize")
WREL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P.build()
    yield


def load_golden(target):
    with open(os.path.join(GOLDEN, target + ".json")) as f:
        rec = json.load(f)
    c = np.asarray(rec["counts"], dtype=np.int64)
    wc = np.asarray(rec["wcounts"], dtype=np.float64) if rec["wcounts"] is not None else None
    return rec, c, wc


def check_catalogue(rec, x, wt=None):
    h = hashlib.sha256(np.ascontiguousarray(x, dtype=np.float64).tobytes())
    if wt is not None:
        h.update(np.ascontiguousarray(wt).tobytes())
    assert x.shape[0] == rec["n"], f"{rec['target']}: size {x.shape[0]} != {rec['n']}"
    assert h.hexdigest() == rec["catalogue_sha256"], (
        f"{rec['target']}: the regenerated catalogue differs from the one the stored "
        "histogram was computed on (regenerate it with tests/golden/make_fullsize.py)")


def check_hist(got, want, gw=None, ww=None, what=""):
    bad = np.nonzero(got != want)[0]
    assert bad.size == 0, (f"{what}: counts differ in {bad.size} bins, first "
                           f"{bad[:5].tolist()}: {got[bad[:5]].tolist()} vs {want[bad[:5]].tolist()}")
    if ww is not None:
        zero = ww == 0
        assert np.all(gw[zero] == 0), what
        rel = np.abs(gw[~zero] - ww[~zero]) / np.abs(ww[~zero])
        assert rel.size == 0 or rel.max() <= WREL, f"{what}: weighted rel err {rel.max():.3e}"


def count_grid(x, wt, box, bins, opts):
    g = P.pc_build_grid(x, wt, box=box, r_max=bins.r_max, opts=opts)
    try:
        c, wc, st = P.pc_count_auto(g, bins, opts, weighted=wt is not None)
    finally:
        g.free()
    return c, wc, st


def count_tree(x, wt, box, bins):
    opts, cap, _ = P.pc_tune_tree(x, wt, box=box, bins=bins)
    t = P.pc_build_tree(x, wt, box=box, list_cap=cap)
    try:
        c, wc, st = P.pc_count_tree(t, None, bins, opts, weighted=wt is not None)
    finally:
        t.free()
    return c, wc, st


@pytest.mark.parametrize("name", ["uniform_periodic_n20k_s40", "ns_periodic_n2m_smu40x100"])
def test_periodic_cube_whole_histogram(name):
    """Configs 1 and 2 whole: the tuned FP32 + rescue grid path, the k-d tree
    path and the plain FP64 path all equal the oracle bin for bin."""
    rec, want, _ = load_golden(name)
    w = W.WORKLOADS[name]
    D = W.make_inputs(w)["D"]
    check_catalogue(rec, D)
    xd = torch.from_numpy(D).cuda()
    bins = P.Bins(w.mode, w.los, w.edges_a, w.edges_b)
    box = P.make_box(w.L, True)
    opts, _ = P.pc_tune(xd, box=box, bins=bins)
    got, _, st = count_grid(xd, None, box, bins, opts)
    check_hist(got, want, what=f"{name}: grid, tuned (cell {opts.cell_size:.3g}, ipt {opts.ipt})")
    assert st.prec == P.PC_PREC_F32_RESCUE and st.rescued > 0
    got, _, _ = count_tree(xd, None, box, bins)
    check_hist(got, want, what=f"{name}: k-d tree, tuned")
    o64 = P.make_opts("f64", P.pc_suggest_cell_size(D.shape[0], w.L ** 3, bins.r_max), 1)
    got, _, st = count_grid(xd, None, box, bins, o64)
    check_hist(got, want, what=f"{name}: plain FP64")
    assert st.prec == P.PC_PREC_F64


def test_survey_shell_dd_whole_histogram():
    """The survey shell's weighted DD (FKP weights, (sigma, pi) 40 x 40 along
    the midpoint line of sight) whole: grid and tree paths, tuned."""
    name = "survey_shell_d1m_r20m_sigpi40x40_DD"
    rec, want, wwant = load_golden(name)
    w = W.WORKLOADS["survey_shell_d1m_r20m_sigpi40x40"]
    nd = w.extra["n_data"]
    D = C.survey_shell(nd, True, w.seed)
    wD = C.fkp_weights(D, nd)
    check_catalogue(rec, D, wD)
    xd, wd = torch.from_numpy(D).cuda(), torch.from_numpy(wD).cuda()
    bins = P.Bins("sigpi", "mid", w.edges_a, w.edges_b)
    box = P.make_box(None, False, D.min(0), D.max(0))
    opts, _ = P.pc_tune(xd, wd, box=box, bins=bins)
    got, gw, st = count_grid(xd, wd, box, bins, opts)
    assert st.prec == P.PC_PREC_F32_RESCUE
    check_hist(got, want, gw, wwant, what=f"{name}: grid, tuned (cell {opts.cell_size:.3g})")
    got, gw, _ = count_tree(xd, wd, box, bins)
    check_hist(got, want, gw, wwant, what=f"{name}: k-d tree, tuned")
