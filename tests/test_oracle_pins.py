"""Pins for the CPU oracle: it is checked against things other than itself.

* hand-derived golden fixtures (tests/golden/*.json, each with its citation);
* exact rational arithmetic (fractions.Fraction) on integer lattices, where
  every tie between a separation and a bin edge is exercised;
* a library special case (scipy cKDTree neighbour counts, a single s range);
* closed forms for uniform periodic randoms (Eq. npair_valid generalised to
  shells; uniform mu; cylinder volumes for (sigma, pi));
* exact rational weighted sums with dyadic weights on the same lattices, and
  weighted sums within one ulp of the exactly rounded sum (math.fsum);
* invariants: cross(D, D) vs auto(D), DR = RD, permutations, scaling by a
  power of two (Sect. 3.2.4), unit weights, brute force vs cell list, the mu
  marginal of H(s, mu) equal to H(s).
"""

import itertools
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# golden fixtures
# --------------------------------------------------------------------------

def test_cube_corner_golden():
    g = json.load(open(os.path.join(GOLD, "cube_corners.json")))
    pts = np.array(g["points"], dtype=np.float64)
    for case in g["cases"]:
        for method in ("brute", "grid"):
            c, _ = oracle.count(pts, mode=case["mode"], los=case["los"],
                                edges_a=case["edges_a"], edges_b=case["edges_b"],
                                method=method)
            assert c.tolist() == case["counts"], (case, method)


def test_midpoint_golden():
    g = json.load(open(os.path.join(GOLD, "midpoint_pairs.json")))
    for case in g["cases"]:
        b = oracle.pair_bin(case["a"], case["b"], mode=case["mode"], los="mid",
                            edges_a=case["edges_a"], edges_b=case["edges_b"])
        assert b == case["bin"], case


# --------------------------------------------------------------------------
# exact rational recomputation on lattices
# --------------------------------------------------------------------------

def _exact_bin(a, b, L, periodic, mode, los, ea, eb):
    """Exact-arithmetic bin of a pair (Fractions; no floating point)."""
    d = []
    for q in range(3):
        v = Fraction(b[q]) - Fraction(a[q])
        if periodic:
            h = Fraction(L) / 2
            if v > h:
                v -= Fraction(L)
            elif v < -h:
                v += Fraction(L)
        d.append(v)
    s2 = d[0] ** 2 + d[1] ** 2 + d[2] ** 2
    Ea = [Fraction(e) ** 2 for e in ea]

    def loc(v, E):
        if not (E[0] <= v < E[-1]):
            return None
        k = 0
        while k + 1 < len(E) - 1 and v >= E[k + 1]:
            k += 1
        return k

    if mode == "s":
        k = loc(s2, Ea)
        return -1 if k is None else k
    if los == "z":
        p2 = d[2] ** 2
    else:
        lv = [Fraction(a[q]) + Fraction(b[q]) for q in range(3)]
        sl = d[0] * lv[0] + d[1] * lv[1] + d[2] * lv[2]
        ll = lv[0] ** 2 + lv[1] ** 2 + lv[2] ** 2
        p2 = sl * sl / ll if ll > 0 else Fraction(0)
    Eb = [Fraction(e) ** 2 for e in eb]
    if mode == "smu":
        k = loc(s2, Ea)
        if k is None:
            return -1
        j = 0
        if s2 > 0:
            while j + 1 < len(Eb) - 1 and p2 >= Eb[j + 1] * s2:
                j += 1
        return k * (len(eb) - 1) + j
    q2 = max(s2 - p2, Fraction(0))
    k = loc(q2, Ea)
    j = loc(p2, Eb)
    if k is None or j is None:
        return -1
    return k * (len(eb) - 1) + j


def _exact_counts(x, L, periodic, mode, los, ea, eb):
    nb = (len(ea) - 1) * (1 if mode == "s" else len(eb) - 1)
    h = np.zeros(nb, dtype=np.int64)
    pts = [tuple(int(v) for v in p) for p in x]
    for i, j in itertools.combinations(range(len(pts)), 2):
        b = _exact_bin(pts[i], pts[j], L, periodic, mode, los, ea, eb)
        if b >= 0:
            h[b] += 1
    return h


def _exact_wsums(x, w, y, wy, L, periodic, mode, los, ea, eb):
    """Exact per-bin sums of w_i w_j over the pairs of x (auto, i < j) or
    x x y (cross), in rational arithmetic."""
    nb = (len(ea) - 1) * (1 if mode == "s" else len(eb) - 1)
    h = [Fraction(0)] * nb
    px = [tuple(int(v) for v in p) for p in x]
    if y is None:
        pairs = ((i, j, px[i], px[j], w[i], w[j])
                 for i, j in itertools.combinations(range(len(px)), 2))
    else:
        py = [tuple(int(v) for v in p) for p in y]
        pairs = ((i, j, px[i], py[j], w[i], wy[j])
                 for i in range(len(px)) for j in range(len(py)))
    for _, _, a, b, wa, wb in pairs:
        k = _exact_bin(a, b, L, periodic, mode, los, ea, eb)
        if k >= 0:
            h[k] += Fraction(wa) * Fraction(wb)
    return h


LATTICE_CASES = [
    # (mode, los, periodic, edges_a, edges_b)
    ("s", "z", True, [0, 1, 2, 3, 4, 5], None),
    ("s", "z", False, [1, 1.5, 2, 3, 4.5, 7], None),
    ("smu", "z", True, [0, 1, 2, 3, 4], [0, 0.25, 0.5, 0.75, 1]),
    ("smu", "z", False, [0, 2, 4, 6], [0, 0.5, 0.625, 1]),
    ("sigpi", "z", True, [0, 1, 2, 3], [0, 1, 2, 3, 4]),
    ("sigpi", "z", False, [0, 0.5, 1, 2.5, 4], [0, 2, 4]),
    ("smu", "mid", False, [0, 1, 2, 3, 5], [0, 0.25, 0.5, 0.75, 1]),
    ("sigpi", "mid", False, [0, 1, 2, 3, 4], [0, 1, 2, 3]),
]


@pytest.mark.parametrize("mode,los,periodic,ea,eb", LATTICE_CASES)
def test_lattice_exact(mode, los, periodic, ea, eb):
    side = 9
    for seed in range(3):
        x = synth.lattice_points(60, side, 11 + seed, unique=(seed != 2))
        if los == "mid":
            x = x + np.array([20.0, -3.0, 5.0])  # keep the observer outside
        got, _ = oracle.count(x, box=float(side), periodic=periodic, mode=mode, los=los,
                              edges_a=ea, edges_b=eb)
        want = _exact_counts(x, side, periodic, mode, los, ea, eb)
        assert got.tolist() == want.tolist(), (mode, los, periodic, seed)
        got_g, _ = oracle.count(x, box=float(side), periodic=periodic, mode=mode, los=los,
                                edges_a=ea, edges_b=eb, method="grid")
        assert got_g.tolist() == want.tolist()


@pytest.mark.parametrize("mode,los,periodic,ea,eb", LATTICE_CASES[::2] + [LATTICE_CASES[-1]])
def test_lattice_weighted_exact(mode, los, periodic, ea, eb):
    """Weighted sums (Sect. 2.5: each pair adds w_i w_j) with dyadic weights
    k/8: every product and partial sum is exact in binary64, so the sums must
    equal the rational ones bit for bit, for auto and cross counts and for
    every method."""
    side = 9
    rng = np.random.default_rng(5)
    x = synth.lattice_points(50, side, 31, unique=False)
    y = synth.lattice_points(40, side, 32, unique=False)
    if los == "mid":
        x, y = x + np.array([20.0, -3.0, 5.0]), y + np.array([20.0, -3.0, 5.0])
    w = rng.integers(1, 8, x.shape[0]) / 8.0
    wy = rng.integers(1, 8, y.shape[0]) / 8.0
    kw = dict(box=float(side), periodic=periodic, mode=mode, los=los, edges_a=ea, edges_b=eb)
    want_a = [float(v) for v in _exact_wsums(x, w, None, None, side, periodic, mode, los, ea, eb)]
    want_x = [float(v) for v in _exact_wsums(x, w, y, wy, side, periodic, mode, los, ea, eb)]
    for method in ("brute", "grid", "kdtree"):
        _, got = oracle.count(x, w1=w, method=method, n_leaf=3, **kw)
        assert got.tolist() == want_a, (method, "auto")
        _, got = oracle.count(x, y, w1=w, w2=wy, method=method, n_leaf=3, **kw)
        assert got.tolist() == want_x, (method, "cross")


# --------------------------------------------------------------------------
# library special case: cKDTree neighbour counts
# --------------------------------------------------------------------------

@pytest.mark.parametrize("periodic", [True, False])
def test_ckdtree_single_range_and_shells(periodic):
    spatial = pytest.importorskip("scipy.spatial")
    L = 100.0
    x = synth.neyman_scott(3000, 300, 10.0, 2.0, L, 5)
    y = synth.uniform_box(2000, L, 6)
    edges = np.array([0.0, 2.0, 5.0, 9.5, 14.0, 20.0])
    kw = {"boxsize": L} if periodic else {}
    tx = spatial.cKDTree(x, **kw)
    ty = spatial.cKDTree(y, **kw)
    # auto: ordered pairs with d <= r including self-pairs
    cum = tx.count_neighbors(tx, edges)
    auto_cum = (cum - x.shape[0]) // 2
    want = np.diff(auto_cum)
    got, _ = oracle.count(x, box=L, periodic=periodic, edges_a=edges)
    assert got.tolist() == want.tolist()
    # single range [0, R): the paper's grid benchmark quantity (Sect. 2.1)
    got1, _ = oracle.count(x, box=L, periodic=periodic, edges_a=[0.0, 20.0])
    assert int(got1[0]) == int(auto_cum[-1])
    # cross
    cumx = tx.count_neighbors(ty, edges)
    gotx, _ = oracle.count(x, y, box=L, periodic=periodic, edges_a=edges)
    assert gotx.tolist() == np.diff(cumx).tolist()


# --------------------------------------------------------------------------
# closed forms for uniform randoms in a periodic box
# --------------------------------------------------------------------------

def _check_expectation(got, exp, N, vol_frac):
    # pair-count variance for uniform randoms: Poisson term inflated by the
    # shared-point (triplet) term ~ 2 N V_bin / V
    sig = np.sqrt(exp * (1.0 + 2.0 * N * vol_frac))
    z = (got - exp) / np.maximum(sig, 1.0)
    assert np.all(np.abs(z) < 5.0), z
    assert abs(got.sum() - exp.sum()) < 5.0 * np.sqrt(exp.sum() * (1 + 2 * N * vol_frac.sum()))


def test_closed_form_uniform_s_smu_sigpi():
    L, N = 100.0, 4000
    x = synth.uniform_box(N, L, 21)
    npairs = N * (N - 1) / 2
    e = np.linspace(0.0, 20.0, 11)
    vf = 4.0 / 3.0 * np.pi * (e[1:] ** 3 - e[:-1] ** 3) / L ** 3
    got, _ = oracle.count(x, box=L, periodic=True, edges_a=e, method="grid")
    _check_expectation(got.astype(float), npairs * vf, N, vf)
    # Eq. npair_valid total: N^2 (4 pi / 3) (R / L)^3, for unordered pairs / 2
    assert abs(got.sum() - npairs * 4 / 3 * np.pi * (20 / L) ** 3) < 5 * np.sqrt(
        npairs * vf.sum() * (1 + 2 * N * vf.sum()))
    # (s, mu): mu uniform on [0, 1] for isotropic randoms
    m = np.linspace(0.0, 1.0, 6)
    g2, _ = oracle.count(x, box=L, periodic=True, mode="smu", edges_a=e, edges_b=m,
                         method="grid")
    exp2 = (npairs * vf)[:, None] * np.diff(m)[None, :]
    _check_expectation(g2.astype(float), exp2.ravel(), N, (vf[:, None] * np.diff(m)).ravel())
    # (sigma, pi) along z: cylinder shells, pi counted on |dz|
    sg = np.linspace(0.0, 15.0, 6)
    pi = np.linspace(0.0, 12.0, 5)
    g3, _ = oracle.count(x, box=L, periodic=True, mode="sigpi", edges_a=sg, edges_b=pi,
                         method="grid")
    vf3 = (np.pi * np.diff(sg ** 2))[:, None] * (2 * np.diff(pi))[None, :] / L ** 3
    _check_expectation(g3.astype(float), (npairs * vf3).ravel(), N, vf3.ravel())


# --------------------------------------------------------------------------
# invariants
# --------------------------------------------------------------------------

MODES = [("s", "z", None), ("smu", "z", np.linspace(0, 1, 11)), ("sigpi", "z", np.linspace(0, 12, 7))]


@pytest.mark.parametrize("mode,los,eb", MODES)
def test_cross_self_equals_twice_auto_plus_self_pairs(mode, los, eb):
    L = 60.0
    x = synth.neyman_scott(1500, 150, 10.0, 1.5, L, 31)
    ea = np.linspace(0.0, 12.0, 9)
    a, _ = oracle.count(x, box=L, periodic=True, mode=mode, los=los, edges_a=ea, edges_b=eb)
    c, _ = oracle.count(x, x, box=L, periodic=True, mode=mode, los=los, edges_a=ea, edges_b=eb)
    want = 2 * a
    want[0] += x.shape[0]  # self-pairs: s = 0 (mu bin 0; sigma = pi = 0)
    assert c.tolist() == want.tolist()


@pytest.mark.parametrize("mode,los,eb", MODES + [("smu", "mid", np.linspace(0, 1, 5)),
                                                 ("sigpi", "mid", np.linspace(0, 30, 6))])
def test_dr_equals_rd_and_permutation(mode, los, eb):
    periodic = los == "z"
    L = 80.0
    d = synth.neyman_scott(900, 90, 10.0, 2.0, L, 41)
    r = synth.uniform_box(1100, L, 42)
    if not periodic:
        d = d + 500.0
        r = r + 500.0
    ea = np.linspace(0.0, 20.0, 6)
    wd = synth.lognormal_weights(d.shape[0], 0.3, 1, np.float64)
    wr = synth.lognormal_weights(r.shape[0], 0.3, 2, np.float64)
    kw = dict(box=L, periodic=periodic, mode=mode, los=los, edges_a=ea, edges_b=eb)
    c1, w1 = oracle.count(d, r, w1=wd, w2=wr, **kw)
    c2, w2 = oracle.count(r, d, w1=wr, w2=wd, **kw)
    assert c1.tolist() == c2.tolist()
    np.testing.assert_allclose(w1, w2, rtol=1e-13, atol=0)
    p = np.random.default_rng(0).permutation(d.shape[0])
    c3, w3 = oracle.count(d[p], w1=wd[p], **kw)
    c4, w4 = oracle.count(d, w1=wd, **kw)
    assert c3.tolist() == c4.tolist()
    np.testing.assert_allclose(w3, w4, rtol=1e-13, atol=0)


@pytest.mark.parametrize("k", [-3, 4])
def test_power_of_two_rescaling_is_exact(k):
    """Scaling coordinates, box and edges by 2^k only changes exponents
    (Sect. 3.2.4), so counts are bit-identical."""
    L = 100.0
    x = synth.neyman_scott(2000, 200, 10.0, 2.0, L, 51)
    ea = np.linspace(0.0, 20.0, 41)
    mu = np.linspace(0.0, 1.0, 21)
    f = 2.0 ** k
    for mode, eb in (("s", None), ("smu", mu), ("sigpi", np.linspace(0, 20, 11))):
        a, _ = oracle.count(x, box=L, periodic=True, mode=mode, edges_a=ea, edges_b=eb)
        eb2 = None if eb is None else (eb if mode == "smu" else eb * f)
        b, _ = oracle.count(x * f, box=L * f, periodic=True, mode=mode, edges_a=ea * f,
                            edges_b=eb2)
        assert a.tolist() == b.tolist(), mode


@pytest.mark.parametrize("los,periodic", [("z", True), ("z", False), ("mid", False)])
def test_mu_marginal_equals_s_histogram(los, periodic):
    """mu edges spanning [0, 1] put every in-range pair in exactly one mu bin
    (Sect. 2.5: mu = |pi| / s lies in [0, 1], the top edge closed), so the
    sum over mu of H(s, mu) is H(s), bit for bit, and the weighted sums
    agree to rounding."""
    L = 90.0
    x = synth.neyman_scott(2000, 200, 10.0, 2.0, L, 91)
    x[:5] = x[5]                        # coincident points: s = 0, mu bin 0
    x[7] = x[6] + np.array([0.0, 0.0, 3.0])   # a pair along the z axis: mu = 1
    if not periodic:
        x = x + 400.0
    w = synth.lognormal_weights(x.shape[0], 0.3, 9, np.float64)
    ea = np.linspace(0.0, 18.0, 10)
    mu = np.linspace(0.0, 1.0, 13)
    kw = dict(box=L, periodic=periodic, los=los, edges_a=ea, w1=w)
    for method in ("brute", "grid", "kdtree"):
        hs, ws = oracle.count(x, mode="s", method=method, **kw)
        hm, wm = oracle.count(x, mode="smu", edges_b=mu, method=method, **kw)
        assert hm.reshape(len(ea) - 1, -1).sum(axis=1).tolist() == hs.tolist(), method
        np.testing.assert_allclose(wm.reshape(len(ea) - 1, -1).sum(axis=1), ws, rtol=1e-13)


@pytest.mark.parametrize("method", ["brute", "grid", "kdtree"])
def test_weighted_sums_are_the_exactly_rounded_sums(method):
    """Each bin's weighted sum is the sum of the rounded products
    fl(w_i w_j) over its pairs (Sect. 2.5 pair weight); the compensated sum
    must lie within one ulp of that sum rounded once (math.fsum), where a
    plain running sum drifts by tens of ulps over the thousands of pairs per
    bin.  Bins come from numpy's own evaluation of the definition (generic
    reals, so no pair sits on an edge), checked against the oracle's counts."""
    import math
    L, N = 50.0, 2000
    x = synth.uniform_box(N, L, 77)
    w = synth.lognormal_weights(N, 0.3, 78, np.float64)
    ea = np.linspace(0.0, 10.0, 11)
    i, j = np.triu_indices(N, 1)
    d = x[j] - x[i]
    d = np.where(d > L / 2, d - L, np.where(d < -L / 2, d + L, d))
    s2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
    E = ea * ea
    k = np.searchsorted(E, s2, side="right") - 1
    ok = (k >= 0) & (s2 < E[-1])
    prod = w[i] * w[j]
    exact = np.array([math.fsum(prod[ok & (k == b)]) for b in range(ea.size - 1)])
    cnt = np.array([int((ok & (k == b)).sum()) for b in range(ea.size - 1)])
    c, ws = oracle.count(x, w1=w, box=L, periodic=True, edges_a=ea, method=method)
    assert c.tolist() == cnt.tolist()
    assert np.all(np.abs(ws - exact) <= np.spacing(exact)), (ws - exact) / np.spacing(exact)


def test_unit_weights_reproduce_counts():
    L = 50.0
    x = synth.uniform_box(1200, L, 61)
    ea = np.linspace(0.0, 10.0, 6)
    c, w = oracle.count(x, w1=np.ones(x.shape[0]), box=L, periodic=True, edges_a=ea)
    assert np.array_equal(w, c.astype(np.float64))


@pytest.mark.parametrize("mode,los,eb", MODES + [("sigpi", "mid", np.linspace(0, 25, 6))])
@pytest.mark.parametrize("periodic", [True, False])
def test_brute_equals_grid(mode, los, eb, periodic):
    if los == "mid" and periodic:
        pytest.skip("midpoint LOS is for non-periodic catalogues")
    L = 120.0
    x = synth.neyman_scott(2500, 250, 10.0, 3.0, L, 71)
    y = synth.uniform_box(1500, L, 72)
    if not periodic:
        x, y = x + 300.0, y + 300.0
    ea = np.linspace(0.0, 25.0, 11)
    w = synth.lognormal_weights(x.shape[0], 0.3, 3, np.float64)
    wy = synth.lognormal_weights(y.shape[0], 0.3, 4, np.float64)
    kw = dict(box=L, periodic=periodic, mode=mode, los=los, edges_a=ea, edges_b=eb)
    a, wa = oracle.count(x, w1=w, **kw)
    b, wb = oracle.count(x, w1=w, method="grid", **kw)
    assert a.tolist() == b.tolist()
    np.testing.assert_allclose(wa, wb, rtol=1e-13, atol=0)
    a, _ = oracle.count(x, y, **kw)
    b, _ = oracle.count(x, y, method="grid", **kw)
    assert a.tolist() == b.tolist()


def test_thread_count_does_not_change_counts():
    L = 100.0
    x = synth.neyman_scott(3000, 300, 10.0, 2.0, L, 81)
    ea = np.linspace(0.0, 20.0, 21)
    a, _ = oracle.count(x, box=L, periodic=True, edges_a=ea, threads=1)
    b, _ = oracle.count(x, box=L, periodic=True, edges_a=ea, threads=7)
    assert a.tolist() == b.tolist()


def test_periodic_wrap_and_canonical_form():
    L = 10.0
    ea = [0.0, 0.5, 1.5, 3.0]
    # across the boundary: |dx| = 1 through the wrap
    assert oracle.pair_bin([0.5, 5, 5], [9.5, 5, 5], box=L, periodic=True, edges_a=ea) == 1
    # coordinates outside [0, L) fold back before the separation is taken
    assert oracle.pair_bin([10.5, 5, 5], [-0.5, 5, 5], box=L, periodic=True, edges_a=ea) == 1
    # non-periodic: no wrap, far apart
    assert oracle.pair_bin([0.5, 5, 5], [9.5, 5, 5], edges_a=ea) == -1


def test_mu_closed_top_and_zero_separation():
    mu = [0.0, 0.5, 1.0]
    ea = [0.0, 2.0]
    # mu = 1 exactly (along z) lands in the last mu bin
    assert oracle.pair_bin([0, 0, 0], [0, 0, 1], mode="smu", edges_a=ea, edges_b=mu) == 1
    # mu = 0 in the first
    assert oracle.pair_bin([0, 0, 0], [1, 0, 0], mode="smu", edges_a=ea, edges_b=mu) == 0
    # a tie p2 == M_j * s2 goes to the upper mu bin.  M = 0.5^2 = 0.25 and
    # dz = 1 give p2 = 1; pick dx, dy so that s2 rounds to exactly 4.0.
    dx = 3.0 ** 0.5
    dy = 0.0
    while (dx * dx + dy * dy) + 1.0 != 4.0:
        dy = dy * 2.0 if dy else 2.0 ** -30
    assert oracle.pair_bin([0, 0, 0], [dx, dy, 1.0], mode="smu", edges_a=[0.0, 3.0],
                           edges_b=[0.0, 0.5, 1.0]) == 1
    assert oracle.pair_bin([0, 0, 0], [dx, dy, 1.0 - 2.0 ** -40], mode="smu",
                           edges_a=[0.0, 3.0], edges_b=[0.0, 0.5, 1.0]) == 0
    # coincident points: s = 0 goes to mu bin 0
    assert oracle.pair_bin([1, 1, 1], [1, 1, 1], mode="smu", edges_a=ea, edges_b=mu) == 0


def test_radial_pairs_have_zero_sigma():
    """Pairs on a ray from the observer lie along their own midpoint line of
    sight (Sect. 2.5: l = x_i + x_j parallel to d), so sigma vanishes up to
    the rounding of the coordinates and pi = |d|.  In binary64 pi^2 often
    exceeds s^2 by a rounding error; the definition clamps sigma^2 at 0, and
    every pair must land in the first sigma bin and the pi bin of |d|, as the
    exact rational evaluation of the same coordinates says."""
    rng = np.random.default_rng(5)
    n = 2000
    u = rng.normal(size=(n, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    r1 = rng.uniform(500.0, 1500.0, n)
    dd = rng.uniform(0.5, 19.5, n)
    dd[np.abs(dd - np.round(dd / 5.0) * 5.0) < 1e-6] += 0.1    # keep off the pi edges
    a = u * r1[:, None]
    b = u * (r1 + dd)[:, None]
    ea, eb = [0.0, 1.0, 2.0, 4.0], [0.0, 5.0, 10.0, 20.0]
    for k in range(n):
        got = oracle.pair_bin(a[k], b[k], mode="sigpi", los="mid", edges_a=ea, edges_b=eb)
        ex = _exact_bin(tuple(a[k]), tuple(b[k]), 0, False, "sigpi", "mid", ea, eb)
        assert got == ex, (k, got, ex)
        assert 0 <= got < 3          # sigma bin 0
        if k < 40:                   # the count drivers take the same decision
            for method in ("brute", "grid", "kdtree"):
                c, _ = oracle.count(np.stack([a[k], b[k]]), mode="sigpi", los="mid",
                                    edges_a=ea, edges_b=eb, method=method)
                assert c.sum() == 1 and c[ex] == 1, (k, method)


def test_invalid_arguments_raise():
    x = synth.uniform_box(10, 10.0, 1)
    with pytest.raises(ValueError):
        oracle.count(x, edges_a=[0.0, 2.0, 1.0])
    with pytest.raises(ValueError):
        oracle.count(x, mode="smu", edges_a=[0.0, 1.0], edges_b=[0.0, 0.5])
    with pytest.raises(ValueError):
        oracle.count(x, box=10.0, periodic=True, mode="smu", los="mid", edges_a=[0.0, 1.0],
                     edges_b=[0.0, 1.0])
