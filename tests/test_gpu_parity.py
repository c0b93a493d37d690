"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Integer counts must be bit-identical.  Weighted sums must agree within 1e-10
relative per bin (exactly where the oracle's bin is zero): the oracle sums
binary64 products with Neumaier compensation, the GPU sums the same binary64
products in a different order, so only summation rounding separates them.
"""

import numpy as np
import pytest

import oracle
import synth
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


def _both(x1, x2=None, w1=None, w2=None, prec="f32", **kw):
    got = P.count(x1, x2, w1=w1, w2=w2, prec=prec, **kw)
    kw2 = {k: v for k, v in kw.items() if k not in ("cell_size", "ipt", "priv",
                                                      "rescue_capacity")}
    want = oracle.count(x1, x2, w1=w1, w2=w2, method="grid", **kw2)
    return got, want


MODES = [
    ("s", "z", None),
    ("smu", "z", np.linspace(0.0, 1.0, 11)),
    ("sigpi", "z", np.linspace(0.0, 30.0, 16)),
]


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("mode,los,eb", MODES)
def test_periodic_auto_clustered(mode, los, eb, prec):
    L = 150.0
    x = synth.neyman_scott(6000, 600, 10.0, 2.0, L, 101)
    ea = np.linspace(0.0, 30.0, 16)
    (g, _), (w, _) = _both(x, box=L, periodic=True, mode=mode, los=los, edges_a=ea,
                           edges_b=eb, prec=prec)
    _check(g, w, what=f"{mode}/{prec}")


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("mode,los,eb", MODES)
def test_periodic_cross(mode, los, eb, prec):
    L = 120.0
    d = synth.neyman_scott(3000, 300, 10.0, 3.0, L, 111)
    r = synth.uniform_box(4000, L, 112)
    ea = np.linspace(0.0, 25.0, 11)
    (g, _), (w, _) = _both(d, r, box=L, periodic=True, mode=mode, los=los, edges_a=ea,
                           edges_b=eb, prec=prec)
    _check(g, w, what=f"cross {mode}/{prec}")


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("mode,eb", [("smu", np.linspace(0, 1, 6)),
                                     ("sigpi", np.linspace(0, 40, 9))])
def test_survey_midpoint_weighted(mode, eb, prec):
    d = synth.survey_shell(3000, True, 121)
    r = synth.survey_shell(6000, False, 122)
    wd = synth.fkp_weights(d, 3000)
    wr = synth.fkp_weights(r, 3000)
    ea = np.linspace(0.0, 40.0, 9)
    kw = dict(periodic=False, mode=mode, los="mid", edges_a=ea, edges_b=eb)
    (g, gw), (w, ww) = _both(d, w1=wd, prec=prec, **kw)
    _check(g, w, gw, ww, f"DD {mode}/{prec}")
    (g, gw), (w, ww) = _both(d, r, w1=wd, w2=wr, prec=prec, **kw)
    _check(g, w, gw, ww, f"DR {mode}/{prec}")


def test_cross_self_identity_and_symmetry():
    L = 100.0
    x = synth.neyman_scott(5000, 500, 10.0, 2.0, L, 131)
    y = synth.uniform_box(3000, L, 132)
    ea = np.linspace(0.0, 20.0, 21)
    mu = np.linspace(0.0, 1.0, 21)
    kw = dict(box=L, periodic=True, mode="smu", edges_a=ea, edges_b=mu)
    a, _ = P.count(x, **kw)
    c, _ = P.count(x, x, **kw)
    want = 2 * a
    want[0] += x.shape[0]
    assert np.array_equal(c, want)
    dr, _ = P.count(x, y, **kw)
    rd, _ = P.count(y, x, **kw)
    assert np.array_equal(dr, rd)


def test_near_edge_adversarial():
    """Pairs placed at bin edges * (1 + tiny): the FP32 decision is within
    rounding of the edge, so these exercise the binary64 rescue."""
    L = 400.0
    ea = np.linspace(0.0, 50.0, 26)
    offs = [0.0, 2.0 ** -52, -2.0 ** -52, 4 * 2.0 ** -52, -8 * 2.0 ** -52, 1e-9, -1e-9,
            3e-8, -3e-8, 1e-7, -1e-7, 5e-7, -5e-7, 2e-6, -2e-6, 1e-5, -1e-5]
    x = synth.catalogs.near_edge_pairs(ea, L, 6000, offs, 141)
    mu = np.linspace(0.0, 1.0, 41)
    for mode, eb in (("s", None), ("smu", mu), ("sigpi", np.linspace(0.0, 50.0, 26))):
        (g, _), (w, _) = _both(x, box=L, periodic=True, mode=mode, edges_a=ea, edges_b=eb)
        _check(g, w, what=f"near-edge {mode}")
    # evenly spaced edges starting above zero: pairs just below the first edge
    # fall below the histogram, pairs just above it into bin 0
    ea5 = np.linspace(5.0, 50.0, 19)
    x5 = synth.catalogs.near_edge_pairs(ea5[:3], L, 3000, offs, 142)
    for mode, eb in (("s", None), ("smu", mu)):
        (g, _), (w, _) = _both(x5, box=L, periodic=True, mode=mode, edges_a=ea5, edges_b=eb)
        _check(g, w, what=f"near-edge {mode}, e0 > 0")


@pytest.mark.parametrize("mode", ["s", "smu"])
def test_log_bins_clustered_and_near_edges(mode):
    """Logarithmic s bins in [0.1, R) (the other binning scheme of the paper,
    Sect. 3.2: monotone non-uniform edges through the table path), on a
    clustered catalogue and on pairs planted at the log edges * (1 + tiny)."""
    L = 300.0
    ea = np.geomspace(0.1, 30.0, 25)
    eb = np.linspace(0.0, 1.0, 11) if mode == "smu" else None
    x = synth.neyman_scott(30000, 1500, 20.0, 1.0, L, 601)
    (g, _), (w, _) = _both(x, box=L, periodic=True, mode=mode, edges_a=ea, edges_b=eb)
    _check(g, w, what=f"log bins {mode}")
    offs = [0.0, 2.0 ** -52, -2.0 ** -52, 1e-9, -1e-9, 1e-7, -1e-7, 2e-6, -2e-6]
    y = synth.catalogs.near_edge_pairs(ea, L, 6000, offs, 602)
    (g, _), (w, _) = _both(y, box=L, periodic=True, mode=mode, edges_a=ea, edges_b=eb)
    _check(g, w, what=f"log bins near edges {mode}")
    # edges a little off a geometric sequence: the table path instead
    eap = ea.copy()
    eap[1:-1] *= 1.0 + 1e-5 * np.cos(np.arange(1, ea.size - 1))
    (g, _), (w, _) = _both(x, box=L, periodic=True, mode=mode, edges_a=eap, edges_b=eb)
    _check(g, w, what=f"near-log bins {mode}")
    y = synth.catalogs.near_edge_pairs(eap, L, 6000, offs, 604)
    (g, _), (w, _) = _both(y, box=L, periodic=True, mode=mode, edges_a=eap, edges_b=eb)
    _check(g, w, what=f"near-log bins near edges {mode}")


def test_headline_binning_200x120_scaled():
    """The paper's headline binning, 200 s bins x 120 mu bins (24,000 bins,
    a histogram larger than the 16 KB shared budget), on a scaled clustered
    periodic catalogue with the separation range scaled to fit the box."""
    L = 400.0
    x = synth.neyman_scott(40000, 4000, 10.0, 2.0, L, 603)
    ea = np.linspace(0.0, 40.0, 201)
    eb = np.linspace(0.0, 1.0, 121)
    (g, _), (w, _) = _both(x, box=L, periodic=True, mode="smu", edges_a=ea, edges_b=eb)
    _check(g, w, what="200 x 120 bins")


def test_large_weighted_histogram_grouped_ctas():
    """6,000 (s, mu) bins with binary64 weighted sums: counts plus sums fill
    72 KB of shared memory, so the kernel runs CTAs of four thread groups
    sharing one histogram; counts and sums match the oracle."""
    L = 400.0
    x = synth.neyman_scott(30000, 3000, 10.0, 2.0, L, 605)
    w = synth.lognormal_weights(x.shape[0], 0.3, 606)
    ea = np.linspace(0.0, 40.0, 61)
    eb = np.linspace(0.0, 1.0, 101)
    (g, gw), (o, ow) = _both(x, w1=w, box=L, periodic=True, mode="smu", edges_a=ea, edges_b=eb)
    _check(g, o, gw, ow, "6000 bins weighted")


def test_lattice_ties_exact():
    """Integer lattice with integer edges: many exact ties on bin edges."""
    x = synth.lattice_points(3000, 24, 151)
    ea = np.arange(0, 11, dtype=np.float64)
    for mode, eb in (("s", None), ("smu", [0, 0.25, 0.5, 0.75, 1.0]), ("sigpi", np.arange(0, 6.0))):
        for prec in ("f32", "f64"):
            (g, _), (w, _) = _both(x, box=24.0, periodic=True, mode=mode, edges_a=ea,
                                   edges_b=eb, prec=prec)
            _check(g, w, what=f"lattice {mode}/{prec}")


@pytest.mark.parametrize("n", [0, 1, 2, 3, 255, 256, 257, 1000])
def test_small_and_ragged_sizes(n):
    L = 50.0
    x = synth.uniform_box(n, L, 161 + n) if n else np.zeros((0, 3))
    ea = np.linspace(0.0, 10.0, 11)
    (g, _), (w, _) = _both(x, box=L, periodic=True, mode="smu", edges_a=ea,
                           edges_b=np.linspace(0, 1, 5))
    _check(g, w, what=f"n={n}")


@pytest.mark.parametrize("n1,n2", [(0, 500), (500, 0), (1, 500), (500, 1), (1, 1)])
def test_cross_with_empty_and_single_catalogues(n1, n2):
    L = 60.0
    x1 = synth.uniform_box(n1, L, 171) if n1 else np.zeros((0, 3))
    x2 = synth.uniform_box(n2, L, 172) if n2 else np.zeros((0, 3))
    ea = np.linspace(0.0, 20.0, 11)
    (g, _), (w, _) = _both(x1, x2, box=L, periodic=True, mode="smu", edges_a=ea,
                           edges_b=np.linspace(0, 1, 5))
    _check(g, w, what=f"cross {n1} x {n2}")


def test_batch_with_empty_and_single_mocks():
    L = 100.0
    ea = np.linspace(0.0, 20.0, 11)
    eb = np.linspace(0.0, 1.0, 6)
    bins = P.Bins("smu", "z", ea, eb)
    box = P.make_box(L, True)
    cats = [np.zeros((0, 3)), synth.uniform_box(1, L, 181), synth.uniform_box(3000, L, 182),
            np.zeros((0, 3)), synth.neyman_scott(2000, 200, 10.0, 2.0, L, 183)]
    opts = P.make_opts("f32", 25.0)
    gs = [P.pc_build_grid(c, box=box, r_max=bins.r_max, opts=opts) for c in cats]
    try:
        for use_graph in (0, 1):
            opts.use_graph = use_graph
            got, _, _ = P.pc_count_batch(gs, bins, opts)
            got = got.reshape(len(cats), -1)
            for k, c in enumerate(cats):
                want, _ = oracle.count(c, box=L, periodic=True, mode="smu", edges_a=ea,
                                       edges_b=eb, method="grid")
                _check(got[k], want, what=f"batch mock {k} (graph {use_graph})")
    finally:
        for g in gs:
            g.free()


def test_periodic_coordinates_on_and_outside_the_box():
    """Coordinates at 0, at L, just inside and outside [0, L) and several box
    lengths away are folded into the box (canonical form) on both sides."""
    L = 80.0
    rng = np.random.default_rng(191)
    base = synth.uniform_box(3000, L, 192)
    special = np.array([[0.0, 0.0, 0.0], [L, L, L], [L - 1e-12, 0.5, 79.9], [-1e-12, 40.0, 40.0],
                        [-L, 2 * L, 3 * L + 1.0], [1.0, -0.5, L + 0.5], [0.0, 0.0, 1e-9]])
    shifted = base + L * rng.integers(-3, 4, size=base.shape)
    x = np.vstack([base[:1500], shifted[1500:], special])
    ea = np.linspace(0.0, 30.0, 16)
    for mode, eb in (("s", None), ("smu", np.linspace(0, 1, 9)), ("sigpi", np.linspace(0, 20, 5))):
        (g, _), (w, _) = _both(x, box=L, periodic=True, mode=mode, edges_a=ea, edges_b=eb)
        _check(g, w, what=f"folded coordinates {mode}")


def test_catalogue_far_from_the_origin():
    """A non-periodic catalogue offset by 1e5 Mpc/h: the FP32 path works on
    cell-relative offsets, and its band carries the coordinate magnitude."""
    x = synth.neyman_scott(6000, 600, 10.0, 2.0, 200.0, 193) + np.array([1.0e5, -2.5e5, 7.0e4])
    ea = np.linspace(0.0, 25.0, 26)
    for mode, los, eb in (("s", "z", None), ("smu", "z", np.linspace(0, 1, 11)),
                          ("sigpi", "mid", np.linspace(0, 20, 11))):
        (g, _), (w, _) = _both(x, periodic=False, mode=mode, los=los, edges_a=ea, edges_b=eb)
        _check(g, w, what=f"far catalogue {mode}/{los}")


def test_dense_cell_and_duplicates():
    """One dense clump (thousands of points in one cell) plus exact duplicates
    (s = 0 pairs go to bin 0 / mu bin 0)."""
    L = 100.0
    rng = np.random.default_rng(171)
    clump = 50.0 + rng.normal(0, 0.3, size=(3000, 3))
    dup = np.repeat(rng.random((50, 3)) * L, 3, axis=0)
    x = np.concatenate([clump, dup, synth.uniform_box(2000, L, 172)])
    ea = np.linspace(0.0, 12.0, 25)
    for mode, eb in (("s", None), ("smu", np.linspace(0, 1, 8))):
        for prec in ("f32", "f64"):
            (g, _), (w, _) = _both(x, box=L, periodic=True, mode=mode, edges_a=ea, edges_b=eb,
                                   prec=prec)
            _check(g, w, what=f"clump {mode}/{prec}")


def test_rescue_queue_overflow_goes_inline():
    L = 80.0
    x = synth.catalogs.near_edge_pairs(np.linspace(0, 20, 11), L, 3000, [0.0, 1e-7, -1e-7],
                                       181)
    ea = np.linspace(0.0, 20.0, 11)
    for cap in (1, -1):
        g, _, st = P.count(x, box=L, periodic=True, edges_a=ea, rescue_capacity=cap,
                           return_stats=True)
        w, _ = oracle.count(x, box=L, periodic=True, edges_a=ea)
        _check(g, w, what=f"capacity {cap}")
        assert st.rescue_inline > 0


@pytest.mark.parametrize("cell", [6.0, 9.5, 17.0, 30.0])
def test_cell_size_does_not_change_counts(cell):
    L = 200.0
    x = synth.neyman_scott(8000, 800, 10.0, 3.0, L, 191)
    ea = np.linspace(0.0, 30.0, 31)
    mu = np.linspace(0.0, 1.0, 21)
    want, _ = oracle.count(x, box=L, periodic=True, mode="smu", edges_a=ea, edges_b=mu,
                           method="grid")
    for ipt in (2, 4):
        g, _ = P.count(x, box=L, periodic=True, mode="smu", edges_a=ea, edges_b=mu,
                       cell_size=cell, ipt=ipt)
        _check(g, want, what=f"cell {cell} ipt {ipt}")


@pytest.mark.parametrize("nb", [8, 40, 400])
def test_histogram_replication_modes(nb):
    """Automatic lane copies (up to 32), one count copy per warp and one shared
    copy all give the oracle's counts and weighted sums; few bins stress the
    collisions that the lane copies remove."""
    L = 300.0
    x = synth.neyman_scott(20000, 2000, 10.0, 3.0, L, 211)
    w = synth.lognormal_weights(x.shape[0], 0.3, 212)
    ea = np.linspace(0.0, 30.0, nb + 1)
    want, wantw = oracle.count(x, w1=w, box=L, periodic=True, edges_a=ea, method="grid")
    for priv in (0, 1, 2):
        got, gotw = P.count(x, w1=w, box=L, periodic=True, edges_a=ea, priv=priv)
        _check(got, want, gotw, wantw, f"{nb} bins, priv {priv}")
        got64, gotw64 = P.count(x, w1=w, box=L, periodic=True, edges_a=ea, priv=priv, prec="f64")
        _check(got64, want, gotw64, wantw, f"{nb} bins, priv {priv}, f64")


def test_integer_weight_products_match_binary64():
    """binary32 weights on floor-based bins with few bins run the integer
    product path (stats.wsum == 2) and stay within 1e-10 of the binary64
    oracle; zero weights, a cross count of grids with different exponent
    ranges and the exponent-span limit are covered."""
    L = 300.0
    rng = np.random.default_rng(515)
    x = synth.neyman_scott(20000, 2000, 10.0, 3.0, L, 516)
    y = synth.neyman_scott(15000, 1500, 10.0, 3.0, L, 517)
    ea = np.linspace(0.0, 30.0, 31)
    kw = dict(box=L, periodic=True, edges_a=ea)
    # lognormal weights with some exact zeros
    wx = synth.lognormal_weights(x.shape[0], 0.3, 518)
    wx[rng.choice(x.shape[0], 500, replace=False)] = 0.0
    g, gw, st = P.count(x, w1=wx, return_stats=True, **kw)
    o, ow = oracle.count(x, w1=wx, method="grid", **kw)
    assert st.wsum == 2
    _check(g, o, gw, ow, "integer weights, auto")
    # cross count: the two grids' weights sit in different binades
    wy = (2.0 + 2.0 * rng.random(y.shape[0])).astype(np.float32)
    g, gw, st = P.count(x, y, w1=wx, w2=wy, return_stats=True, **kw)
    o, ow = oracle.count(x, y, w1=wx, w2=wy, method="grid", **kw)
    assert st.wsum == 2
    _check(g, o, gw, ow, "integer weights, cross")
    # exponent spans 6 + 6: at the limit, still integer
    w6 = np.exp2(rng.uniform(-3.0, 3.0, x.shape[0])).astype(np.float32)
    g, gw, st = P.count(x, w1=w6, return_stats=True, **kw)
    o, ow = oracle.count(x, w1=w6, method="grid", **kw)
    assert st.wsum == 2
    _check(g, o, gw, ow, "integer weights, span 12")
    # spans 12 + 12: beyond the limit, binary64 products
    w12 = np.exp2(rng.uniform(-6.0, 6.0, x.shape[0])).astype(np.float32)
    g, gw, st = P.count(x, w1=w12, return_stats=True, **kw)
    o, ow = oracle.count(x, w1=w12, method="grid", **kw)
    assert st.wsum == 1
    _check(g, o, gw, ow, "wide weights, binary64")
    # binary64 weights that are not binary32 values: integer products of
    # their binary32 roundings plus the remainders' terms
    w64 = rng.uniform(0.5, 1.5, x.shape[0])
    g, gw, st = P.count(x, w1=w64, return_stats=True, **kw)
    o, ow = oracle.count(x, w1=w64, method="grid", **kw)
    assert st.wsum == 3
    _check(g, o, gw, ow, "binary64 weights")


def test_integer_weight_products_with_binary64_remainders():
    """Binary64 weights (wsum 3): each weight's binary32 rounding goes
    through the integer products and its remainder through the binary32
    correction term, rounded to the accumulators' unit; within 1e-10 of the
    binary64 oracle for an auto count at the span limit (6 + 6 binades, the
    products' smallest at 2^34 units), a cross count of binary64 against
    binary32 weights (one side without remainders) and of two binary64
    catalogues in different binades, (s, mu) and (sigma, pi) bins along the
    midpoint line of sight (FKP-like weights of a non-periodic shell), the
    k-d tree path, and weights so small that their remainders would
    underflow binary32, which take the binary64 products."""
    L = 300.0
    rng = np.random.default_rng(531)
    x = synth.neyman_scott(20000, 2000, 10.0, 3.0, L, 532)
    y = synth.neyman_scott(15000, 1500, 10.0, 3.0, L, 533)
    ea = np.linspace(0.0, 30.0, 31)
    kw = dict(box=L, periodic=True, edges_a=ea)
    w6 = np.exp2(rng.uniform(-3.0, 3.0, x.shape[0]))           # binary64, 6 binades
    w6[:5] = 2.0 ** -3 * (1.0 + 2.0 ** -40)                   # the smallest, with remainders
    g, gw, st = P.count(x, w1=w6, return_stats=True, **kw)
    o, ow = oracle.count(x, w1=w6, method="grid", **kw)
    assert st.wsum == 3
    _check(g, o, gw, ow, "binary64 weights, span 6 + 6")
    wy32 = synth.lognormal_weights(y.shape[0], 0.3, 534)      # binary32: no remainders
    g, gw, st = P.count(x, y, w1=w6, w2=wy32, return_stats=True, **kw)
    o, ow = oracle.count(x, y, w1=w6, w2=wy32, method="grid", **kw)
    assert st.wsum == 3
    _check(g, o, gw, ow, "binary64 x binary32 weights")
    wy64 = 3.0 + 5.0 * rng.random(y.shape[0])
    g, gw, st = P.count(x, y, w1=w6, w2=wy64, return_stats=True, **kw)
    o, ow = oracle.count(x, y, w1=w6, w2=wy64, method="grid", **kw)
    assert st.wsum == 3
    _check(g, o, gw, ow, "two binary64 catalogues")
    mu = np.linspace(0.0, 1.0, 11)
    kws = dict(box=L, periodic=True, mode="smu", edges_a=np.linspace(0.0, 25.0, 26), edges_b=mu)
    g, gw, st = P.count(x, w1=w6, return_stats=True, **kws)
    o, ow = oracle.count(x, w1=w6, method="grid", **kws)
    assert st.wsum == 3
    _check(g, o, gw, ow, "binary64 weights, (s, mu)")
    shell = synth.survey_shell(30000, True, 535)
    fkp = synth.fkp_weights(shell, shell.shape[0])
    sp = np.linspace(0.0, 40.0, 9)
    kwp = dict(periodic=False, mode="sigpi", los="mid", edges_a=sp, edges_b=sp)
    g, gw, st = P.count(shell, w1=fkp, return_stats=True, **kwp)
    o, ow = oracle.count(shell, w1=fkp, method="grid", **kwp)
    assert st.wsum == 3
    _check(g, o, gw, ow, "FKP weights, (sigma, pi), midpoint")
    t = P.pc_build_tree(x, w6, box=P.make_box(L, True))
    try:
        g, gw, st = P.pc_count_tree(t, None, P.Bins("s", "z", ea), weighted=True)
    finally:
        t.free()
    o, ow = oracle.count(x, w1=w6, method="grid", **kw)
    assert st.wsum == 3
    _check(g, o, gw, ow, "binary64 weights, k-d tree")
    tiny = w6 * 2.0 ** -80                                    # his below 2^-78
    g, gw, st = P.count(x, w1=tiny, return_stats=True, **kw)
    o, ow = oracle.count(x, w1=tiny, method="grid", **kw)
    assert st.wsum == 1
    _check(g, o, gw, ow, "tiny binary64 weights: binary64 products")



def test_integer_weights_on_large_histograms_fold_into_exact_sums():
    """Histograms of thousands of bins leave fewer than 16 lane copies, so the
    integer weight records are folded into each CTA's exact 128-bit sums at
    every product limit instead of being flushed (fold mode).  Within 1e-10
    of the oracle: (s, mu) 40 x 100 with binary32 weights (wsum 2) on a dense
    clustered catalogue (many folds per CTA), a cross count with binary64
    weights (wsum 3), (sigma, pi) 40 x 40 along the midpoint line of sight
    with FKP weights on a shell, the k-d tree path, and a batch of catalogues
    (one histogram row each, so the folded sums change rows between tasks),
    launched directly and replayed as a CUDA graph."""
    L = 200.0
    x = synth.neyman_scott(40000, 4000, 10.0, 3.0, L, 541)
    y = synth.neyman_scott(20000, 2000, 10.0, 3.0, L, 542)
    ea = np.linspace(0.0, 40.0, 41)
    mu = np.linspace(0.0, 1.0, 101)
    kw = dict(box=L, periodic=True, mode="smu", edges_a=ea, edges_b=mu)
    wx = synth.lognormal_weights(x.shape[0], 0.3, 543)
    g, gw, st = P.count(x, w1=wx, return_stats=True, **kw)
    o, ow = oracle.count(x, w1=wx, method="grid", **kw)
    assert st.wsum == 2
    _check(g, o, gw, ow, "4000 bins, binary32 weights")
    wx64 = synth.lognormal_weights(x.shape[0], 0.3, 544, np.float64)
    wy64 = 1.0 + np.random.default_rng(545).random(y.shape[0])
    g, gw, st = P.count(x, y, w1=wx64, w2=wy64, return_stats=True, **kw)
    o, ow = oracle.count(x, y, w1=wx64, w2=wy64, method="grid", **kw)
    assert st.wsum == 3
    _check(g, o, gw, ow, "4000 bins, binary64 weights, cross")
    shell = synth.survey_shell(40000, True, 546)
    fkp = synth.fkp_weights(shell, shell.shape[0])
    sp = np.linspace(0.0, 40.0, 41)
    kwp = dict(periodic=False, mode="sigpi", los="mid", edges_a=sp, edges_b=sp)
    g, gw, st = P.count(shell, w1=fkp, return_stats=True, **kwp)
    o, ow = oracle.count(shell, w1=fkp, method="grid", **kwp)
    assert st.wsum == 3
    _check(g, o, gw, ow, "1600 (sigma, pi) bins, FKP weights, midpoint")
    bins = P.Bins("smu", "z", ea, mu)
    t = P.pc_build_tree(x, wx, box=P.make_box(L, True))
    try:
        g, gw, st = P.pc_count_tree(t, None, bins, weighted=True)
    finally:
        t.free()
    o, ow = oracle.count(x, w1=wx, method="grid", **kw)
    assert st.wsum == 2
    _check(g, o, gw, ow, "4000 bins, k-d tree")
    mocks = synth.batch_mocks(4, 3000, 8000, 3.0, 8.0, L, 547)
    mws = [synth.lognormal_weights(m.shape[0], 0.3, 548 + k) for k, m in enumerate(mocks)]
    box = P.make_box(L, True)
    want = [oracle.count(m, w1=w, method="grid", **kw) for m, w in zip(mocks, mws)]
    for use_graph in (0, 1):
        opts = P.make_opts("f32", 20.0)
        opts.use_graph = use_graph
        grids = [P.pc_build_grid(m, w, box=box, r_max=bins.r_max, opts=opts) for m, w in zip(mocks, mws)]
        try:
            for _ in range(2):
                c, cw, st = P.pc_count_batch(grids, bins, opts, weighted=True)
                assert st.wsum == 2
                c = c.reshape(len(mocks), -1)
                cw = cw.reshape(len(mocks), -1)
                for k in range(len(mocks)):
                    _check(c[k], want[k][0], cw[k], want[k][1], f"batch mock {k}, graph {use_graph}")
        finally:
            for gg in grids:
                gg.free()


def test_integer_weight_packing_limits_and_sixteen_copies():
    """The packed significand M << (8 - k) at both ends of an 8-binade
    catalogue (k = 0 and k = 8) in a cross count with a 4-binade catalogue
    (spans 8 + 4 = 12: integer products); a 9-binade catalogue takes the
    binary64 products even beside a one-binade one; and a 250-bin (s, mu)
    histogram, whose counts and weight records get 16 lane copies instead of
    32, still runs the integer path.  All within 1e-10 of the oracle."""
    L = 300.0
    rng = np.random.default_rng(521)
    x = synth.neyman_scott(20000, 2000, 10.0, 3.0, L, 522)
    y = synth.neyman_scott(15000, 1500, 10.0, 3.0, L, 523)
    ea = np.linspace(0.0, 30.0, 31)
    kw = dict(box=L, periodic=True, edges_a=ea)
    w8 = np.exp2(rng.uniform(-4.0, 4.0, x.shape[0])).astype(np.float32)
    w8[:5] = np.float32(2.0 ** -4)                           # the smallest binade (k = 8)
    w8[5:10] = np.float32(16.0)                               # the largest (k = 0)
    w4 = np.exp2(rng.uniform(0.0, 4.0, y.shape[0])).astype(np.float32)
    w4[:5] = np.float32(1.0)
    w4[5:10] = np.float32(16.0)
    g, gw, st = P.count(x, y, w1=w8, w2=w4, return_stats=True, **kw)
    o, ow = oracle.count(x, y, w1=w8, w2=w4, method="grid", **kw)
    assert st.wsum == 2
    _check(g, o, gw, ow, "integer weights, spans 8 + 4")
    w9 = np.exp2(rng.uniform(-4.5, 4.5, x.shape[0])).astype(np.float32)
    w9[:5] = np.float32(2.0 ** -5)
    w9[5:10] = np.float32(16.0)
    w1 = np.full(y.shape[0], 1.5, dtype=np.float32)
    g, gw, st = P.count(x, y, w1=w9, w2=w1, return_stats=True, **kw)
    o, ow = oracle.count(x, y, w1=w9, w2=w1, method="grid", **kw)
    assert st.wsum == 1
    _check(g, o, gw, ow, "9 binades: binary64 products")
    wx = synth.lognormal_weights(x.shape[0], 0.3, 524)
    mu = np.linspace(0.0, 1.0, 11)
    kws = dict(box=L, periodic=True, mode="smu", edges_a=np.linspace(0.0, 25.0, 26), edges_b=mu)
    g, gw, st = P.count(x, w1=wx, return_stats=True, **kws)
    o, ow = oracle.count(x, w1=wx, method="grid", **kws)
    assert st.wsum == 2
    _check(g, o, gw, ow, "integer weights, 250 bins (16 lane copies)")


def test_shards_are_the_same_pairs_in_both_precisions():
    """A shard is a set of cells: the FP32 + rescue path (256-point blocks)
    and the plain FP64 path (128-point blocks) count identical pairs shard by
    shard at the same cell side, auto and cross, weighted."""
    L = 150.0
    x = synth.neyman_scott(9000, 900, 10.0, 3.0, L, 251)
    y = synth.uniform_box(6000, L, 252)
    wx = synth.lognormal_weights(x.shape[0], 0.3, 253)
    wy = synth.lognormal_weights(y.shape[0], 0.3, 254)
    bins = P.Bins("s", "z", np.linspace(0.0, 30.0, 16))
    box = P.make_box(L, True)
    o = P.make_opts("f32", 10.0)
    gx = P.pc_build_grid(x, wx, box=box, r_max=bins.r_max, opts=o)
    gy = P.pc_build_grid(y, wy, box=box, r_max=bins.r_max, opts=o)
    try:
        for r in range(3):
            o32 = P.make_opts("f32", 10.0, 2, shard_index=r, shard_count=3)
            o64 = P.make_opts("f64", 10.0, 1, shard_index=r, shard_count=3)
            a32, aw32, _ = P.pc_count_auto(gx, bins, o32, weighted=True)
            a64, aw64, _ = P.pc_count_auto(gx, bins, o64, weighted=True)
            assert a32.sum() > 0 and np.array_equal(a32, a64), r
            np.testing.assert_allclose(aw32, aw64, rtol=1e-10, atol=0)
            c32, cw32, _ = P.pc_count_cross(gx, gy, bins, o32, weighted=True)
            c64, cw64, _ = P.pc_count_cross(gx, gy, bins, o64, weighted=True)
            assert np.array_equal(c32, c64), r
            np.testing.assert_allclose(cw32, cw64, rtol=1e-10, atol=0)
    finally:
        gx.free()
        gy.free()


def test_device_tensors_and_device_outputs():
    L = 100.0
    x = synth.neyman_scott(4000, 400, 10.0, 2.0, L, 201)
    ea = np.linspace(0.0, 20.0, 11)
    xd = torch.from_numpy(x).cuda()
    bins = P.Bins("s", "z", ea)
    g = P.pc_build_grid(xd, box=P.make_box(L, True), r_max=bins.r_max)
    out = torch.zeros(bins.nbins, dtype=torch.int64, device="cuda")
    P.pc_count_auto(g, bins, counts=out)
    g.free()
    want, _ = oracle.count(x, box=L, periodic=True, edges_a=ea)
    _check(out.cpu().numpy(), want, what="device io")


def test_weighted_f32_weights_periodic():
    L = 150.0
    x = synth.mixed_box(8000, L, 0.5, 10.0, 3.0, 211)
    w = synth.lognormal_weights(x.shape[0], 0.3, 212)   # float32
    ea = np.linspace(0.0, 30.0, 7)
    for prec in ("f32", "f64"):
        (g, gw), (o, ow) = _both(x, w1=w, box=L, periodic=True, edges_a=ea, prec=prec)
        _check(g, o, gw, ow, f"lognormal weights {prec}")


def test_batch_matches_per_mock_oracle():
    mocks = synth.batch_mocks(6, 1500, 4000, 3.0, 8.0, 300.0, 221)
    ea = np.linspace(0.0, 40.0, 21)
    mu = np.linspace(0.0, 1.0, 11)
    bins = P.Bins("smu", "z", ea, mu)
    box = P.make_box(300.0, True)
    opts = P.make_opts("f32", 20.0)
    grids = [P.pc_build_grid(m, box=box, r_max=bins.r_max, opts=opts) for m in mocks]
    c, _, st = P.pc_count_batch(grids, bins, opts)
    for g in grids:
        g.free()
    c = c.reshape(len(mocks), -1)
    for k, m in enumerate(mocks):
        w, _ = oracle.count(m, box=300.0, periodic=True, mode="smu", edges_a=ea, edges_b=mu,
                            method="grid")
        _check(c[k], w, what=f"mock {k}")


def test_batch_graph_replay_matches_and_survives_free():
    mocks = synth.batch_mocks(5, 1200, 3000, 3.0, 8.0, 300.0, 225)
    ea = np.linspace(0.0, 40.0, 21)
    mu = np.linspace(0.0, 1.0, 11)
    bins = P.Bins("smu", "z", ea, mu)
    box = P.make_box(300.0, True)
    opts = P.make_opts("f32", 20.0)
    opts.use_graph = 1
    grids = [P.pc_build_grid(m, box=box, r_max=bins.r_max, opts=opts) for m in mocks]
    want = np.concatenate([oracle.count(m, box=300.0, periodic=True, mode="smu", edges_a=ea,
                                        edges_b=mu, method="grid")[0] for m in mocks])
    for _ in range(3):   # capture once, then replay
        c, _, st = P.pc_count_batch(grids, bins, opts)
        _check(c, want, what="graph batch")
        assert st.launches >= 3
    dev = torch.zeros(bins.nbins * len(mocks), dtype=torch.int64, device="cuda")
    P.pc_count_batch(grids, bins, opts, counts=dev)
    _check(dev.cpu().numpy(), want, what="graph batch, device output")
    grids[2].free()          # drops the cached graph that uses it
    rest = [g for k, g in enumerate(grids) if k != 2]
    c, _, _ = P.pc_count_batch(rest, bins, opts)
    want_rest = np.concatenate([want.reshape(len(mocks), -1)[k] for k in range(len(mocks)) if k != 2])
    _check(c, want_rest, what="graph batch after free")
    for g in rest:
        g.free()


@pytest.mark.parametrize("nshard", [2, 3])
def test_block_shards_sum_to_the_full_count(nshard):
    """Multi-GPU shards (pc_opts.shard_index/count) run one after the other on
    one GPU; their int64 histograms must sum to the unsharded count."""
    L = 150.0
    x = synth.neyman_scott(9000, 900, 10.0, 3.0, L, 241)
    y = synth.uniform_box(5000, L, 242)
    bins = P.Bins("smu", "z", np.linspace(0.0, 30.0, 16), np.linspace(0.0, 1.0, 11))
    box = P.make_box(L, True)
    o = P.make_opts("f32", 10.0)
    gx = P.pc_build_grid(x, box=box, r_max=bins.r_max, opts=o)
    gy = P.pc_build_grid(y, box=box, r_max=bins.r_max, opts=o)
    full_a, _, _ = P.pc_count_auto(gx, bins, o)
    full_c, _, _ = P.pc_count_cross(gx, gy, bins, o)
    part_a = np.zeros_like(full_a)
    part_c = np.zeros_like(full_c)
    for r in range(nshard):
        so = P.make_opts("f32", 10.0, shard_index=r, shard_count=nshard)
        part_a += P.pc_count_auto(gx, bins, so)[0]
        part_c += P.pc_count_cross(gx, gy, bins, so)[0]
    gx.free()
    gy.free()
    assert np.array_equal(part_a, full_a)
    assert np.array_equal(part_c, full_c)
    w, _ = oracle.count(x, box=L, periodic=True, mode="smu", edges_a=bins.ea, edges_b=bins.eb,
                        method="grid")
    _check(full_a, w, what="unsharded")


def test_errors_are_reported():
    L = 100.0
    x = synth.uniform_box(100, L, 231)
    with pytest.raises(P.PairCountError):
        P.count(x, box=L, periodic=True, edges_a=[0.0, 60.0])   # R >= L/2
    with pytest.raises(P.PairCountError):
        P.count(x, box=L, periodic=True, edges_a=[0.0, 5.0, 3.0])
    with pytest.raises(P.PairCountError):
        P.count(x, box=L, periodic=True, mode="smu", los="mid", edges_a=[0, 5.0],
                edges_b=[0, 1.0])


# --------------------------------------------------------------------------
# the five workloads
# --------------------------------------------------------------------------

def test_workload_uniform_n20k_full():
    w = W.WORKLOADS["uniform_periodic_n20k_s40"]
    inp = W.make_inputs(w)
    for prec in ("f32", "f64"):
        g, _ = P.count(inp["D"], box=w.L, periodic=True, edges_a=w.edges_a, prec=prec)
        o, _ = oracle.count(inp["D"], box=w.L, periodic=True, edges_a=w.edges_a)
        _check(g, o, what=f"uniform n20k {prec}")


def test_workload_ns_smu_scaled():
    w = W.WORKLOADS["ns_periodic_n2m_smu40x100"]
    inp = W.make_inputs(w, scale=0.02)     # 40,000 points, same cluster shape
    kw = dict(box=w.L, periodic=True, mode="smu", edges_a=w.edges_a, edges_b=w.edges_b)
    g, _ = P.count(inp["D"], **kw)
    o, _ = oracle.count(inp["D"], method="grid", **kw)
    _check(g, o, what="ns smu scaled")


def test_workload_survey_scaled_weighted():
    """The survey shell: its bounding box comes within ~430 Mpc/h of the
    observer, but every point lies at r >= 1000, so the FP32 midpoint bound
    holds and the FP32 path must run (stats.prec == 0)."""
    w = W.WORKLOADS["survey_shell_d1m_r20m_sigpi40x40"]
    inp = W.make_inputs(w, scale=0.004)    # D 4,000, R 80,000
    kw = dict(periodic=False, mode="sigpi", los="mid", edges_a=w.edges_a, edges_b=w.edges_b)
    g, gw, st = P.count(inp["D"], w1=inp["wD"], return_stats=True, **kw)
    o, ow = oracle.count(inp["D"], w1=inp["wD"], method="grid", **kw)
    assert st.prec == P.PC_PREC_F32_RESCUE
    _check(g, o, gw, ow, "survey DD")
    g, gw, st = P.count(inp["D"], inp["R"], w1=inp["wD"], w2=inp["wR"], return_stats=True, **kw)
    o, ow = oracle.count(inp["D"], inp["R"], w1=inp["wD"], w2=inp["wR"], method="grid", **kw)
    assert st.prec == P.PC_PREC_F32_RESCUE
    _check(g, o, gw, ow, "survey DR")


def test_midpoint_near_observer_runs_fp64():
    """Points around the observer: |x_i + x_j| has no useful lower bound, the
    FP32 error band does not hold, and the library runs the FP64 path."""
    rng = np.random.default_rng(404)
    x = rng.uniform(-60.0, 60.0, size=(3000, 3))
    kw = dict(periodic=False, mode="sigpi", los="mid", edges_a=np.linspace(0, 20, 5),
              edges_b=np.linspace(0, 20, 5))
    g, _, st = P.count(x, return_stats=True, **kw)
    o, _ = oracle.count(x, method="grid", **kw)
    assert st.prec == P.PC_PREC_F64
    _check(g, o, what="midpoint near the observer")


def test_workload_mixed_weighted_scaled():
    w = W.WORKLOADS["mixed_periodic_n100m_s40_w"]
    inp = W.make_inputs(w, scale=0.0015)   # 150,000 points in L = 3000
    (g, gw), (o, ow) = _both(inp["D"], w1=inp["wD"], box=w.L, periodic=True,
                             edges_a=w.edges_a)
    _check(g, o, gw, ow, "mixed weighted")


def test_tuned_options_keep_counts_and_pruning_is_sound():
    """pc_tune's choice counts exactly like the oracle, and every pair the
    group bounds pruned is out of range: in-range pairs <= candidates - pruned."""
    L = 400.0
    x = synth.neyman_scott(60000, 6000, 10.0, 4.0, L, 311)
    ea = np.linspace(0.0, 40.0, 41)
    mu = np.linspace(0.0, 1.0, 51)
    box = P.make_box(L, True)
    bins = P.Bins("smu", "z", ea, mu)
    opts, trials = P.pc_tune(x, box=box, bins=bins)
    assert len(trials) >= 3
    assert opts.ipt in (2, 4) and opts.priv in (0, 1)
    assert any(t[0] == opts.cell_size and t[1] == opts.ipt for t in trials)
    assert all(np.isfinite(t[3]) and t[3] > 0 for t in trials)
    want, _ = oracle.count(x, box=L, periodic=True, mode="smu", edges_a=ea, edges_b=mu,
                           method="grid")
    g = P.pc_build_grid(x, box=box, r_max=bins.r_max, opts=opts)
    got, _, st = P.pc_count_auto(g, bins, opts)
    g.free()
    _check(got, want, what=f"tuned {opts.cell_size} ipt {opts.ipt} priv {opts.priv}")
    assert st.pruned > 0
    assert int(want.sum()) <= st.candidates - st.pruned


def _bench_opts(D, w, bins):
    """The options the benchmark times: pc_tune on the same catalogue."""
    opts, _ = P.pc_tune(D, box=P.make_box(w.L, True), bins=bins)
    return dict(cell_size=opts.cell_size, ipt=opts.ipt, priv=opts.priv)


def test_full_size_ns_smu_auto_vs_cross_and_sampled_oracle():
    """N = 2,000,000 clustered points, (s, mu) 40 x 100, in the launch
    configuration the benchmark times (the tuned options).  Auto counts are
    tied to the cross path (cross(D, D) = 2 auto(D) + N self-pairs in bin 0),
    and the cross path is checked against the oracle on a sampled subset of
    i-points."""
    w = W.WORKLOADS["ns_periodic_n2m_smu40x100"]
    D = W.make_inputs(w)["D"]
    kw = dict(box=w.L, periodic=True, mode="smu", edges_a=w.edges_a, edges_b=w.edges_b)
    xd = torch.from_numpy(D).cuda()
    tuned = _bench_opts(xd, w, P.Bins("smu", "z", w.edges_a, w.edges_b))
    a, _ = P.count(xd, **kw, **tuned)
    a0, _ = P.count(xd, **kw)
    assert np.array_equal(a, a0)
    c, _ = P.count(xd, xd, **kw)
    want = 2 * a
    want[0] += D.shape[0]
    assert np.array_equal(c, want)
    idx = np.random.default_rng(7).choice(D.shape[0], 1500, replace=False)
    S = np.ascontiguousarray(D[idx])
    g, _ = P.count(S, xd, **kw)
    o, _ = oracle.count(S, D, method="grid", **kw)
    _check(g, o, what="sampled cross at full size")


def test_estimators_on_gpu_counts_of_uniform_randoms():
    """End to end: GPU pair counts of uniform periodic randoms give a
    Peebles-Hauser xi (with the analytic RR) and a Landy-Szalay xi (with a
    second random catalogue) that vanish within Poisson noise."""
    from paper_2301_12557_gb300 import estimators as E
    L, n = 500.0, 60000
    d = synth.uniform_box(n, L, 801)
    r = synth.uniform_box(2 * n, L, 802)
    ea = np.linspace(0.0, 50.0, 11)
    kw = dict(box=L, periodic=True, edges_a=ea)
    dd, _ = P.count(d, **kw)
    dr, _ = P.count(d, r, **kw)
    rr, _ = P.count(r, **kw)
    ndd, ndr, nrr = (E.normalise(dd, E.pair_norm(n)), E.normalise(dr, E.pair_norm(n, 2 * n, auto=False)),
                     E.normalise(rr, E.pair_norm(2 * n)))
    rr_a = E.analytic_rr(ea, box=L)
    sig = 1.0 / np.sqrt(rr_a * E.pair_norm(n))          # relative Poisson noise of DD
    assert np.all(np.abs(E.peebles_hauser(ndd, rr_a)) <= 5 * sig)
    assert np.all(np.abs(E.landy_szalay(ndd, ndr, nrr)) <= 5 * sig)
