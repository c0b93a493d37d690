"""Full-size parity for the weighted cube, the batched mocks and the survey
shell, in the launch configuration the benchmark times (the options pc_tune
picks on the same catalogue).  The oracle checks sampled outputs it can
compute: every pair of a random sample of i-points with the whole catalogue
(the cross form of the same pair set), bit-exact counts and weighted sums
within 1e-10; the batch is also tied to single counts of every mock.

The 256-mock batch is also compared whole, row by row, with the oracle's
histograms of four of its mocks stored in tests/golden/fullsize/ (smallest,
largest, two of median size), for the grid batch and the tree batch.

(Collected after the main parity file: these cases take tens of seconds.)
"""

import glob
import hashlib
import json
import os

import numpy as np
import pytest

import oracle
from synth import workloads as W

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
    yield


def _check(got, want, gw=None, ww=None, what=""):
    assert np.array_equal(got, want), f"{what}: counts differ in {np.count_nonzero(got != want)} bins"
    if ww is not None:
        zero = ww == 0
        assert np.all(gw[zero] == 0), what
        rel = np.abs(gw[~zero] - ww[~zero]) / np.abs(ww[~zero])
        assert rel.size == 0 or rel.max() <= WREL, f"{what}: weighted rel err {rel.max():.3e}"


def _opts_kw(opts):
    return dict(cell_size=opts.cell_size, ipt=opts.ipt, priv=opts.priv)


def test_weighted_cube_100m_sampled():
    w = W.WORKLOADS["mixed_periodic_n100m_s40_w"]
    inp = W.make_inputs(w)
    D, wD = inp["D"], inp["wD"]
    xd, wd = torch.from_numpy(D).cuda(), torch.from_numpy(wD).cuda()
    bins = P.Bins("s", "z", w.edges_a)
    opts, _ = P.pc_tune(xd, wd, box=P.make_box(w.L, True), bins=bins)
    idx = np.random.default_rng(11).choice(D.shape[0], 300, replace=False)
    S, wS = np.ascontiguousarray(D[idx]), np.ascontiguousarray(wD[idx])
    kw = dict(box=w.L, periodic=True, edges_a=w.edges_a)
    g, gw, st = P.count(S, xd, w1=wS, w2=wd, return_stats=True, **kw, **_opts_kw(opts))
    o, ow = oracle.count(S, D, w1=wS, w2=wD, method="grid", **kw)
    assert st.wsum in (1, 2, 3)
    _check(g, o, gw, ow, "weighted cube, sampled cross")


def _mock_goldens():
    """{mock index: (stored record, counts)} of the stored whole-mock histograms."""
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "fullsize")
    out = {}
    for path in sorted(glob.glob(os.path.join(here, "mocks256_ns_smu40x100_mock*.json"))):
        rec = json.load(open(path))
        k = int(rec["target"].rsplit("mock", 1)[1])
        out[k] = (rec, np.asarray(rec["counts"], dtype=np.int64))
    return out


def test_batched_mocks_256_vs_single_counts_and_sampled_oracle():
    w = W.WORKLOADS["mocks256_ns_smu40x100"]
    mocks = W.make_inputs(w)["mocks"]
    goldens = _mock_goldens()
    assert len(goldens) == 4
    for k, (rec, _) in goldens.items():
        h = hashlib.sha256(np.ascontiguousarray(mocks[k]).tobytes()).hexdigest()
        assert h == rec["catalogue_sha256"], f"mock {k} differs from the stored one"
    X = [torch.from_numpy(x).cuda() for x in mocks]
    bins = P.Bins("smu", "z", w.edges_a, w.edges_b)
    box = P.make_box(w.L, True)
    med = sorted(range(len(X)), key=lambda k: X[k].shape[0])[len(X) // 2]
    opts, _ = P.pc_tune(X[med], box=box, bins=bins)
    opts.use_graph = 1
    gs = [P.pc_build_grid(x, box=box, r_max=bins.r_max, opts=opts) for x in X]
    try:
        batch, _, _ = P.pc_count_batch(gs, bins, opts)
        batch = batch.reshape(len(X), -1)
        for k, g in enumerate(gs):
            single, _, _ = P.pc_count_auto(g, bins, opts)
            assert np.array_equal(batch[k], single), f"mock {k}"
        for k, (_, want) in goldens.items():
            _check(batch[k], want, what=f"mock {k}: grid batch row vs whole oracle histogram")
    finally:
        for g in gs:
            g.free()
    # the tree batch (every tree built in one level loop, one persistent
    # launch over every tree's lists), tuned on the median mock as the
    # benchmark does
    topts, cap, _ = P.pc_tune_tree(X[med], box=box, bins=bins)
    ts = P.pc_build_tree_batch(X, box=box, list_cap=cap)
    try:
        tb, _, _ = P.pc_count_tree_batch(ts, bins, topts)
        tb = tb.reshape(len(X), -1)
        assert np.array_equal(tb, batch), "tree batch differs from the grid batch"
        for k, (_, want) in goldens.items():
            _check(tb[k], want, what=f"mock {k}: tree batch row vs whole oracle histogram")
    finally:
        for t in ts:
            t.free()
    kw = dict(box=w.L, periodic=True, mode="smu", edges_a=w.edges_a, edges_b=w.edges_b)
    for k in (0, len(X) - 1):
        D = mocks[k]
        idx = np.random.default_rng(12 + k).choice(D.shape[0], 400, replace=False)
        S = np.ascontiguousarray(D[idx])
        g, _ = P.count(S, X[k], **kw, **_opts_kw(opts))
        o, _ = oracle.count(S, D, method="grid", **kw)
        _check(g, o, what=f"mock {k}, sampled cross")


def test_survey_shell_sampled_dr():
    w = W.WORKLOADS["survey_shell_d1m_r20m_sigpi40x40"]
    inp = W.make_inputs(w)
    D, R, wD, wR = inp["D"], inp["R"], inp["wD"], inp["wR"]
    xr, wr = torch.from_numpy(R).cuda(), torch.from_numpy(wR).cuda()
    bins = P.Bins("sigpi", "mid", w.edges_a, w.edges_b)
    lo = np.minimum(D.min(0), R.min(0))
    hi = np.maximum(D.max(0), R.max(0))
    opts, _ = P.pc_tune(xr, wr, box=P.make_box(None, False, lo, hi), bins=bins)
    idx = np.random.default_rng(13).choice(D.shape[0], 300, replace=False)
    S, wS = np.ascontiguousarray(D[idx]), np.ascontiguousarray(wD[idx])
    kw = dict(periodic=False, mode="sigpi", los="mid", edges_a=w.edges_a, edges_b=w.edges_b)
    g, gw, st = P.count(S, xr, w1=wS, w2=wr, return_stats=True, **kw, **_opts_kw(opts))
    o, ow = oracle.count(S, R, w1=wS, w2=wR, method="grid", **kw)
    assert st.prec == P.PC_PREC_F32_RESCUE
    _check(g, o, gw, ow, "survey shell, sampled DR")
