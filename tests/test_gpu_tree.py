"""GPU parity of the k-d tree path (Alg. 1 build, Alg. 3 traversal).

The GPU tree is compared node by node with the oracle's tree (the same
median splits along the same axes give the same point sets, hence the same
minimum bounding boxes), and the counts of the tree path are compared with
the oracle's counts: integer counts bit-identical, weighted sums within 1e-10
relative per bin.
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


def _both(x1, x2=None, w1=None, w2=None, n_leaf=32, list_cap=0, ipt=2, **kw):
    got = P.count_tree(x1, x2, w1=w1, w2=w2, n_leaf=n_leaf, list_cap=list_cap, ipt=ipt, **kw)
    want = oracle.count(x1, x2, w1=w1, w2=w2, method="grid", **kw)
    return got, want


# --------------------------------------------------------------------------
# tree structure against the oracle's tree
# --------------------------------------------------------------------------

def _compare_trees(x, gpu, ref):
    assert gpu["depth"] == ref["depth"]
    cg, cr = gpu["count"], ref["count"]
    assert np.array_equal(cg, cr)
    assert np.array_equal(gpu["start"][cr >= 0], ref["start"][cr >= 0])
    n = x.shape[0]
    assert sorted(gpu["ord"].tolist()) == list(range(n))
    # compare each node's point set, descending only below nodes whose split
    # axis is not a near-tie of two variances (either axis is then correct)
    todo = [0]
    checked = 0
    while todo:
        h = todo.pop()
        c = int(cr[h])
        s = int(ref["start"][h])
        a = set(gpu["ord"][s:s + c].tolist())
        b = set(ref["ord"][s:s + c].tolist())
        assert a == b, f"slot {h}: point sets differ"
        np.testing.assert_array_equal(gpu["box"][h], ref["box"][h])
        checked += 1
        if ref["axis"][h] < 0:
            assert gpu["axis"][h] == -1
            continue
        v = np.sort(x[ref["ord"][s:s + c]].var(axis=0))
        if v[2] - v[1] <= 1e-9 * v[2]:
            continue
        assert gpu["axis"][h] == ref["axis"][h], f"slot {h}"
        todo += [2 * h + 1, 2 * h + 2]
    return checked


@pytest.mark.parametrize("n,n_leaf,periodic", [(1, 8, False), (100, 8, False), (257, 32, True),
                                              (5000, 8, False), (20001, 32, True),
                                              (4096, 1, False), (30000, 128, False)])
def test_tree_structure_matches_oracle(n, n_leaf, periodic):
    L = 200.0
    x = synth.neyman_scott(n, max(1, n // 20), 20.0, 3.0, L, 700 + n) if n > 50 else \
        synth.uniform_box(n, L, 700 + n)
    x[:, 2] *= 0.7
    if not periodic:
        x = x + np.array([1000.0, -300.0, 50.0])
    b = P.make_box(L, True) if periodic else P.make_box(None, False)
    t = P.pc_build_tree(x, box=b, n_leaf=n_leaf)
    try:
        g = P.pc_tree_export(t)
    finally:
        t.free()
    ref = oracle.kdtree(x, n_leaf=n_leaf, box=L, periodic=periodic)
    xc = x - L * np.floor(x / L) if periodic else x
    checked = _compare_trees(xc, g, ref)
    assert checked >= min(n, 3) if n > n_leaf else checked == 1
    # the automatic list level: nodes of 129..2048 points (or the root)
    ll = g["list_level"]
    assert 0 <= ll <= g["depth"]
    largest = int(np.ceil(n / 2 ** ll))
    assert largest <= 2048 or ll == 0
    assert largest > 128 or ll == 0


# --------------------------------------------------------------------------
# counts
# --------------------------------------------------------------------------

MODES = [("s", "z", None), ("smu", "z", np.linspace(0.0, 1.0, 11)),
         ("sigpi", "z", np.linspace(0.0, 25.0, 11))]


@pytest.mark.parametrize("mode,los,eb", MODES)
@pytest.mark.parametrize("periodic", [True, False])
def test_tree_auto_and_cross_clustered(mode, los, eb, periodic):
    L = 200.0
    x = synth.neyman_scott(20000, 1000, 20.0, 2.0, L, 711)
    y = synth.uniform_box(12000, L, 712)
    ea = np.linspace(0.0, 25.0, 26)
    kw = dict(box=L, periodic=periodic, mode=mode, los=los, edges_a=ea, edges_b=eb)
    (g, _), (w, _) = _both(x, **kw)
    _check(g, w, what=f"tree auto {mode} periodic={periodic}")
    (g, _), (w, _) = _both(x, y, **kw)
    _check(g, w, what=f"tree cross {mode} periodic={periodic}")


@pytest.mark.parametrize("mode,eb", [("smu", np.linspace(0, 1, 6)), ("sigpi", np.linspace(0, 40, 9))])
def test_tree_survey_midpoint_weighted(mode, eb):
    d = synth.survey_shell(4000, True, 721)
    r = synth.survey_shell(9000, False, 722)
    wd = synth.fkp_weights(d, 4000)
    wr = synth.fkp_weights(r, 4000)
    ea = np.linspace(0.0, 40.0, 9)
    kw = dict(periodic=False, mode=mode, los="mid", edges_a=ea, edges_b=eb)
    (g, gw), (w, ww) = _both(d, w1=wd, **kw)
    _check(g, w, gw, ww, f"tree DD {mode}")
    (g, gw), (w, ww) = _both(d, r, w1=wd, w2=wr, **kw)
    _check(g, w, gw, ww, f"tree DR {mode}")


def test_tree_weighted_binary32_weights_integer_products():
    """binary32 weights: the integer weight products (wsum 2) on the tree path."""
    L = 150.0
    x = synth.neyman_scott(15000, 800, 18.0, 2.0, L, 731)
    w = synth.lognormal_weights(x.shape[0], 0.3, 732, np.float32)
    ea = np.linspace(0.0, 20.0, 21)
    kw = dict(box=L, periodic=True, mode="s", edges_a=ea)
    g, gw, st = P.count_tree(x, w1=w, return_stats=True, **kw)
    o, ow = oracle.count(x, w1=w.astype(np.float64), method="grid", **kw)
    _check(g, o, gw, ow, "tree wint")
    assert st.wsum == 2


def test_tree_near_edges_and_lattice_ties():
    L = 400.0
    ea = np.linspace(0.0, 50.0, 26)
    offs = [0.0, 2.0 ** -52, -2.0 ** -52, 1e-9, -1e-9, 1e-7, -1e-7, 2e-6, -2e-6, 1e-5, -1e-5]
    x = synth.catalogs.near_edge_pairs(ea, L, 6000, offs, 741)
    mu = np.linspace(0.0, 1.0, 41)
    for mode, eb in (("s", None), ("smu", mu), ("sigpi", np.linspace(0.0, 50.0, 26))):
        (g, _), (w, _) = _both(x, box=L, periodic=True, mode=mode, edges_a=ea, edges_b=eb)
        _check(g, w, what=f"tree near-edge {mode}")
    ea5 = np.linspace(5.0, 50.0, 19)
    x5 = synth.catalogs.near_edge_pairs(ea5[:3], L, 3000, offs, 742)
    (g, _), (w, _) = _both(x5, box=L, periodic=True, mode="s", edges_a=ea5)
    _check(g, w, what="tree near-edge e0 > 0")
    z = synth.lattice_points(3000, 24, 743)
    (g, _), (w, _) = _both(z, box=24.0, periodic=True, mode="smu", edges_a=np.arange(0, 11.0),
                           edges_b=[0, 0.25, 0.5, 0.75, 1.0])
    _check(g, w, what="tree lattice")


def test_tree_log_and_table_bins():
    L = 300.0
    x = synth.neyman_scott(25000, 1200, 20.0, 1.0, L, 751)
    ea = np.geomspace(0.1, 30.0, 25)
    (g, _), (w, _) = _both(x, box=L, periodic=True, mode="s", edges_a=ea)
    _check(g, w, what="tree log bins")
    eap = ea.copy()
    eap[1:-1] *= 1.0 + 1e-5 * np.cos(np.arange(1, ea.size - 1))
    (g, _), (w, _) = _both(x, box=L, periodic=True, mode="smu", edges_a=eap,
                           edges_b=np.linspace(0, 1, 11))
    _check(g, w, what="tree table bins")


def test_tree_large_histogram():
    L = 400.0
    x = synth.neyman_scott(30000, 3000, 10.0, 2.0, L, 761)
    ea = np.linspace(0.0, 40.0, 201)
    eb = np.linspace(0.0, 1.0, 121)
    (g, _), (w, _) = _both(x, box=L, periodic=True, mode="smu", edges_a=ea, edges_b=eb)
    _check(g, w, what="tree 200 x 120")


@pytest.mark.parametrize("n", [1, 2, 3, 255, 256, 257, 513, 1000])
@pytest.mark.parametrize("n_leaf", [1, 32, 128])
def test_tree_small_and_ragged_sizes(n, n_leaf):
    L = 50.0
    x = synth.uniform_box(n, L, 770 + n)
    ea = np.linspace(0.0, 20.0, 11)
    for periodic in (True, False):
        (g, _), (w, _) = _both(x, box=L, periodic=periodic, mode="smu", edges_a=ea,
                               edges_b=np.linspace(0, 1, 5), n_leaf=n_leaf)
        _check(g, w, what=f"tree n={n} leaf={n_leaf} periodic={periodic}")
    y = synth.uniform_box(max(n // 2, 1), L, 780 + n)
    (g, _), (w, _) = _both(x, y, box=L, periodic=True, mode="s", edges_a=ea, n_leaf=n_leaf)
    _check(g, w, what=f"tree cross n={n}")


def test_tree_matches_grid_and_sampled_oracle_at_size():
    """2e5 clustered points: tree and grid counts identical (both exact), and
    the tree path's cross counts of 600 sampled points against all points
    equal the oracle's brute-force counts."""
    L = 500.0
    x = synth.neyman_scott(200000, 10000, 20.0, 2.0, L, 791)
    ea = np.linspace(0.0, 50.0, 26)
    mu = np.linspace(0.0, 1.0, 21)
    kw = dict(box=L, periodic=True, mode="smu", edges_a=ea, edges_b=mu)
    gt, _, st = P.count_tree(x, return_stats=True, **kw)
    gg, _ = P.count(x, **kw)
    assert np.array_equal(gt, gg)
    assert st.tree_pairs > 0 and st.blocks >= 200000 / 256
    rng = np.random.default_rng(792)
    s = x[rng.choice(x.shape[0], 600, replace=False)]
    g, _ = P.count_tree(s, x, **kw)
    w, _ = oracle.count(s, x, **kw)
    _check(g, w, what="tree sampled cross")


@pytest.mark.parametrize("list_cap,ipt", [(0, 2), (256, 2), (512, 4), (1024, 2), (1024, 4),
                                          (4096, 4), (0, 4)])
def test_tree_list_levels_keep_counts(list_cap, ipt):
    """List nodes of any size (several balanced blocks each, the own-node
    rest of an auto count as a segment) give the same counts."""
    L = 300.0
    x = synth.neyman_scott(60000, 3000, 20.0, 2.0, L, 801)
    y = synth.uniform_box(7000, L, 802)
    ea = np.linspace(0.0, 30.0, 16)
    mu = np.linspace(0.0, 1.0, 11)
    kw = dict(box=L, periodic=True, mode="smu", edges_a=ea, edges_b=mu)
    (g, _), (w, _) = _both(x, list_cap=list_cap, ipt=ipt, **kw)
    _check(g, w, what=f"tree auto list_cap={list_cap} ipt={ipt}")
    (g, _), (w, _) = _both(x, y, list_cap=list_cap, ipt=ipt, **kw)
    _check(g, w, what=f"tree cross list_cap={list_cap} ipt={ipt}")
    b = P.make_box(L, True)
    t = P.pc_build_tree(x, box=b, list_cap=list_cap)
    try:
        n, depth, ll, slots = t.info()
    finally:
        t.free()
    if list_cap:
        assert int(np.ceil(n / 2 ** ll)) <= list_cap < int(np.ceil(n / 2 ** (ll - 1)))


def test_tree_errors():
    x = synth.uniform_box(100, 10.0, 799)
    with pytest.raises(P.PairCountError):
        P.pc_build_tree(x, box=P.make_box(10.0, True), n_leaf=0)
    with pytest.raises(P.PairCountError):
        P.pc_build_tree(x, box=P.make_box(10.0, True), n_leaf=129)
    with pytest.raises(P.PairCountError):
        P.pc_build_tree(x[:0], box=P.make_box(10.0, True))
    with pytest.raises(P.PairCountError):
        P.pc_build_tree(x, box=P.make_box(10.0, True), list_cap=300)
    with pytest.raises(P.PairCountError):   # separation of L/2 or more in a periodic box
        P.count_tree(x, box=10.0, periodic=True, mode="s", edges_a=[0.0, 6.0])
    t = P.pc_build_tree(x, box=P.make_box(10.0, True))
    try:
        with pytest.raises(P.PairCountError):   # plain FP64 is a grid-path option
            P.pc_count_tree(t, None, P.Bins("s", "z", [0.0, 1.0]), P.make_opts("f64"))
    finally:
        t.free()


def test_tree_tuner_and_shards():
    """pc_tune_tree's options keep the counts, and block shards of a tree count
    sum to the full count."""
    L = 300.0
    x = synth.neyman_scott(80000, 4000, 20.0, 2.0, L, 811)
    ea = np.linspace(0.0, 30.0, 16)
    mu = np.linspace(0.0, 1.0, 11)
    bins = P.Bins("smu", "z", ea, mu)
    b = P.make_box(L, True)
    o, cap, trials = P.pc_tune_tree(x, box=b, bins=bins)
    assert o.ipt in (2, 4) and cap in (0, 512, 1024, 2048, 4096) and len(trials) >= 2
    want, _ = oracle.count(x, box=L, periodic=True, mode="smu", edges_a=ea, edges_b=mu,
                           method="grid")
    t = P.pc_build_tree(x, box=b, list_cap=cap)
    try:
        got, _, _ = P.pc_count_tree(t, None, bins, o)
        _check(got, want, what="tuned tree")
        tot = np.zeros_like(want)
        for k in range(3):
            os_ = P.make_opts("f32", 0.0, o.ipt, shard_index=k, shard_count=3)
            part, _, _ = P.pc_count_tree(t, None, bins, os_)
            tot += part
        _check(tot, want, what="tree shards")
    finally:
        t.free()


def test_tree_batch_matches_single_counts_and_oracle():
    """A batch of trees of very different sizes (1 point to 40k) in one launch
    equals each tree's own count; two of them against the oracle."""
    L = 200.0
    cats = [synth.neyman_scott(n, max(1, n // 20), 20.0, 2.0, L, 820 + i)
            if n > 50 else synth.uniform_box(n, L, 820 + i)
            for i, n in enumerate([40000, 1, 3000, 257, 25000, 90, 12000])]
    ws = [synth.lognormal_weights(c.shape[0], 0.3, 840 + i, np.float32) for i, c in enumerate(cats)]
    ea = np.linspace(0.0, 25.0, 26)
    mu = np.linspace(0.0, 1.0, 11)
    bins = P.Bins("smu", "z", ea, mu)
    b = P.make_box(L, True)
    for ipt in (2, 4):
        trees = [P.pc_build_tree(c, w, box=b) for c, w in zip(cats, ws)]
        try:
            o = P.make_opts("f32", 0.0, ipt)
            cb, wb, st = P.pc_count_tree_batch(trees, bins, o, weighted=True)
            cb = cb.reshape(len(cats), -1)
            wb = wb.reshape(len(cats), -1)
            for k, t in enumerate(trees):
                c1, w1, _ = P.pc_count_tree(t, None, bins, o, weighted=True)
                assert np.array_equal(cb[k], c1), (ipt, k)
                np.testing.assert_allclose(wb[k], w1, rtol=1e-12, atol=0)
            assert st.tree_pairs > 0
        finally:
            for t in trees:
                t.free()
    for k in (0, 2):
        want, wwant = oracle.count(cats[k], w1=ws[k].astype(np.float64), box=L, periodic=True,
                                   mode="smu", edges_a=ea, edges_b=mu, method="grid")
        _check(cb[k], want, wb[k], wwant, f"tree batch mock {k}")


def _same_tree(a, b, what):
    """Two builds of one catalogue: the same heap slots, node ranges and point
    order; boxes and split axes equal except below a node whose variance sums
    (rounded in another order) broke an exact tie the other way."""
    ea, eb = P.pc_tree_export(a), P.pc_tree_export(b)
    assert ea["depth"] == eb["depth"] and ea["list_level"] == eb["list_level"], what
    assert np.array_equal(ea["count"], eb["count"]), what
    assert np.array_equal(ea["start"], eb["start"]), what
    same_axis = ea["axis"] == eb["axis"]
    if same_axis.all():
        assert np.array_equal(ea["box"], eb["box"]), what
        assert np.array_equal(ea["ord"], eb["ord"]), what
    return bool(same_axis.all())


def test_batched_tree_build_equals_single_builds():
    """pc_build_tree_batch (one level loop over all catalogues, the deepest
    first) gives each catalogue the tree pc_build_tree gives it, and a tree
    batch over those trees the same counts and weighted sums as the single
    builds and the oracle: very different sizes (1 to 40,000 points) and
    depths, binary32 weights, periodic; and a non-periodic batch with
    binary64 weights along the midpoint line of sight."""
    L = 200.0
    cats = [synth.neyman_scott(n, max(1, n // 20), 20.0, 2.0, L, 860 + i)
            if n > 50 else synth.uniform_box(n, L, 860 + i)
            for i, n in enumerate([40000, 1, 3000, 257, 25000, 90, 12000])]
    ws = [synth.lognormal_weights(c.shape[0], 0.3, 880 + i, np.float32) for i, c in enumerate(cats)]
    ea = np.linspace(0.0, 25.0, 26)
    mu = np.linspace(0.0, 1.0, 11)
    bins = P.Bins("smu", "z", ea, mu)
    b = P.make_box(L, True)
    dev = [torch.from_numpy(c).cuda() for c in cats]      # device and host inputs mixed
    inputs = [dev[k] if k % 2 else cats[k] for k in range(len(cats))]
    tb = P.pc_build_tree_batch(inputs, ws, box=b)
    ts = [P.pc_build_tree(c, w, box=b) for c, w in zip(cats, ws)]
    try:
        for k in range(len(cats)):
            _same_tree(tb[k], ts[k], f"catalogue {k}")
        o = P.make_opts("f32", 0.0, 2)
        cb, wb, _ = P.pc_count_tree_batch(tb, bins, o, weighted=True)
        cs, ws_, _ = P.pc_count_tree_batch(ts, bins, o, weighted=True)
        assert np.array_equal(cb, cs)
        np.testing.assert_allclose(wb, ws_, rtol=1e-12, atol=0)
        cb = cb.reshape(len(cats), -1)
        wb = wb.reshape(len(cats), -1)
        for k in (0, 2, 4):
            want, wwant = oracle.count(cats[k], w1=ws[k].astype(np.float64), box=L, periodic=True,
                                       mode="smu", edges_a=ea, edges_b=mu, method="grid")
            _check(cb[k], want, wb[k], wwant, f"batch-built tree {k}")
    finally:
        for t in tb + ts:
            t.free()
    # non-periodic shells, binary64 weights, midpoint line of sight
    shells = [synth.survey_shell(n, k % 2 == 0, 890 + k) for k, n in enumerate([3000, 500, 2000])]
    sw = [synth.fkp_weights(s, s.shape[0]) for s in shells]
    sp = np.linspace(0.0, 40.0, 9)
    bins = P.Bins("sigpi", "mid", sp, sp)
    b = P.make_box(None, False)
    tb = P.pc_build_tree_batch(shells, sw, box=b)
    try:
        for k, (s, w) in enumerate(zip(shells, sw)):
            got, gw, _ = P.pc_count_tree(tb[k], None, bins, weighted=True)
            want, wwant = oracle.count(s, w1=w, periodic=False, mode="sigpi", los="mid",
                                       edges_a=sp, edges_b=sp, method="grid")
            _check(got, want, gw, wwant, f"batch-built shell {k}")
    finally:
        for t in tb:
            t.free()
