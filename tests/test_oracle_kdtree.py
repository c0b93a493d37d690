"""Pins for the oracle's k-d tree (Alg. 1) and dual-tree count (Alg. 3).

The tree is checked against the defining properties of Alg. 1, recomputed
here with numpy on each node's own points: balanced halving (left child
floor(n / 2) points), the split axis of largest coordinate variance, every
left point at or below every right point along that axis, leaves of at most
n_leaf points, and minimum bounding boxes.  The dual-tree count is checked
against the brute-force definition and against exact rational counts on
integer lattices (where many separations equal a bin edge exactly, so a
pruning test without its margin, or a dropped child pair, changes a count).
"""

import numpy as np
import pytest

import oracle
import synth
from test_oracle_pins import _exact_counts


def _check_tree(x, T, n_leaf):
    n = x.shape[0]
    order = T["ord"]
    assert sorted(order.tolist()) == list(range(n))
    start, count, axis, box = T["start"], T["count"], T["axis"], T["box"]
    assert start[0] == 0 and count[0] == n
    nodes = 0
    for h in range(count.size):
        c = int(count[h])
        if c < 0:
            continue
        nodes += 1
        pts = x[order[start[h]:start[h] + c]]
        np.testing.assert_array_equal(box[h, :3], pts.min(axis=0))
        np.testing.assert_array_equal(box[h, 3:], pts.max(axis=0))
        if c <= n_leaf:
            assert axis[h] == -1
            if 2 * h + 1 < count.size:
                assert count[2 * h + 1] == -1 and count[2 * h + 2] == -1
            continue
        a = int(axis[h])
        var = pts.var(axis=0)
        top = np.sort(var)
        if top[2] - top[1] > 1e-9 * top[2]:      # no near-tie between two axes
            assert a == int(np.argmax(var)), (h, var)
        l, r = 2 * h + 1, 2 * h + 2
        assert count[l] == c // 2 and count[r] == c - c // 2
        assert start[l] == start[h] and start[r] == start[h] + c // 2
        left = x[order[start[l]:start[l] + count[l]], a]
        right = x[order[start[r]:start[r] + count[r]], a]
        assert left.max() <= right.min()
    return nodes


@pytest.mark.parametrize("n,n_leaf", [(1, 8), (7, 8), (9, 8), (1000, 1), (3001, 8), (5000, 33)])
def test_kdtree_properties(n, n_leaf):
    x = synth.uniform_box(n, 100.0, 5 + n)
    x[:, 1] *= 0.6                      # distinct variances per axis at the top
    T = oracle.kdtree(x, n_leaf=n_leaf)
    nodes = _check_tree(x, T, n_leaf)
    # a balanced tree with leaves of at most n_leaf points
    assert T["depth"] == int(np.ceil(np.log2(max(n / n_leaf, 1.0)))) or n <= n_leaf
    assert nodes <= 2 * n - 1


def test_kdtree_clustered_and_periodic():
    L = 80.0
    x = synth.neyman_scott(4000, 200, 10.0, 1.0, L, 9)
    x[:7] += L                           # outside the box: folded first
    T = oracle.kdtree(x, n_leaf=8, box=L, periodic=True)
    xc = x - L * np.floor(x / L)
    _check_tree(xc, T, 8)
    assert T["box"][0, :3].min() >= 0.0 and T["box"][0, 3:].max() < L


MODES = [("s", "z", None), ("smu", "z", np.linspace(0, 1, 11)),
         ("sigpi", "z", np.linspace(0, 12, 7)), ("smu", "mid", np.linspace(0, 1, 6)),
         ("sigpi", "mid", np.linspace(0, 12, 5))]


@pytest.mark.parametrize("mode,los,eb", MODES)
@pytest.mark.parametrize("periodic", [True, False])
@pytest.mark.parametrize("n_leaf", [1, 8, 40])
def test_dualtree_equals_brute(mode, los, eb, periodic, n_leaf):
    if los == "mid" and periodic:
        pytest.skip("midpoint LOS is for non-periodic catalogues")
    L = 60.0
    x = synth.neyman_scott(1800, 150, 10.0, 2.0, L, 41)
    y = synth.uniform_box(900, L, 42)
    if not periodic:
        x, y = x + 200.0, y + 200.0
    ea = np.linspace(0.5, 14.0, 9)
    w = synth.lognormal_weights(x.shape[0], 0.3, 3, np.float64)
    wy = synth.lognormal_weights(y.shape[0], 0.3, 4, np.float64)
    kw = dict(box=L, periodic=periodic, mode=mode, los=los, edges_a=ea, edges_b=eb)
    a, wa = oracle.count(x, w1=w, **kw)
    b, wb = oracle.count(x, w1=w, method="kdtree", n_leaf=n_leaf, **kw)
    assert a.tolist() == b.tolist()
    np.testing.assert_allclose(wb, wa, rtol=1e-13, atol=0)
    a, wa = oracle.count(x, y, w1=w, w2=wy, **kw)
    b, wb = oracle.count(x, y, w1=w, w2=wy, method="kdtree", n_leaf=n_leaf, **kw)
    assert a.tolist() == b.tolist()
    np.testing.assert_allclose(wb, wa, rtol=1e-13, atol=0)


@pytest.mark.parametrize("mode,los,periodic,ea,eb", [
    ("s", "z", True, [0, 1, 2, 3, 4], None),
    ("s", "z", False, [1, 1.5, 2, 3, 4.5], None),
    ("smu", "z", True, [0, 1, 2, 3, 4], [0, 0.25, 0.5, 0.75, 1]),
    ("sigpi", "z", False, [0, 0.5, 1, 2.5, 4], [0, 2, 4]),
])
def test_dualtree_lattice_exact(mode, los, periodic, ea, eb):
    side = 9
    for seed in range(2):
        x = synth.lattice_points(60, side, 21 + seed, unique=(seed == 0))
        want = _exact_counts(x, side, periodic, mode, los, ea, eb)
        for n_leaf in (1, 3, 8):
            got, _ = oracle.count(x, box=float(side), periodic=periodic, mode=mode, los=los,
                                  edges_a=ea, edges_b=eb, method="kdtree", n_leaf=n_leaf)
            assert got.tolist() == want.tolist(), (seed, n_leaf)


def test_dualtree_empty_and_single():
    ea = [0.0, 1.0, 2.0]
    one = np.array([[1.0, 2.0, 3.0]])
    c, _ = oracle.count(one, edges_a=ea, method="kdtree")
    assert c.tolist() == [0, 0]
    c, _ = oracle.count(one, one + 0.5, edges_a=ea, method="kdtree")
    assert c.tolist() == [1, 0]
    c, _ = oracle.count(np.zeros((0, 3)), one, edges_a=ea, method="kdtree")
    assert c.tolist() == [0, 0]
