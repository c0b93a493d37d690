"""GPU parity on degenerate non-periodic catalogues: points on a plane, on a
line, and all at one position, so the bounding box has no extent along one,
two or three axes (the grid then has one cell along those axes, the k-d tree
splits along axes of zero variance, and every pair of the single position
has s = 0, mu bin 0 and sigma = pi = 0).  Both lines of sight, grid (FP32 +
rescue and FP64) and tree paths, auto and cross counts; counts bit-exact,
weighted sums within 1e-10 relative per bin.
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


ORIGIN = np.array([1000.5, 1200.25, 1300.125])   # away from the observer at 0


def _shape(kind, n, seed):
    rng = np.random.default_rng(seed)
    x = np.repeat(ORIGIN[None, :], n, axis=0)
    if kind == "plane":
        x[:, :2] += rng.uniform(0.0, 60.0, size=(n, 2))
    elif kind == "line":
        x[:, 0] += rng.uniform(0.0, 60.0, size=n)
    return np.ascontiguousarray(x)


CASES = [("s", "z", None), ("smu", "z", np.linspace(0.0, 1.0, 6)),
         ("smu", "mid", np.linspace(0.0, 1.0, 6)), ("sigpi", "mid", np.linspace(0.0, 20.0, 6))]


@pytest.mark.parametrize("kind", ["plane", "line", "point"])
def test_zero_extent_axes(kind):
    x = _shape(kind, 1500 if kind != "point" else 300, 931)
    y = _shape(kind, 700 if kind != "point" else 200, 932)
    w = synth.lognormal_weights(x.shape[0], 0.3, 933, np.float64)
    for mode, los, eb in CASES:
        kw = dict(periodic=False, mode=mode, los=los, edges_a=np.linspace(0.0, 20.0, 11),
                  edges_b=eb)
        want, wantw = oracle.count(x, w1=w, method="grid", **kw)
        if kind == "point":
            assert want[0] == x.shape[0] * (x.shape[0] - 1) // 2
        for prec in ("f32", "f64"):
            got, gotw = P.count(x, w1=w, prec=prec, **kw)
            _check(got, want, gotw, wantw, f"{kind} grid {mode}/{los} {prec}")
        got, gotw = P.count_tree(x, w1=w, **kw)
        _check(got, want, gotw, wantw, f"{kind} tree {mode}/{los}")
        want, _ = oracle.count(x, y, method="grid", **kw)
        got, _ = P.count(x, y, **kw)
        _check(got, want, what=f"{kind} grid cross {mode}/{los}")
        got, _ = P.count_tree(x, y, **kw)
        _check(got, want, what=f"{kind} tree cross {mode}/{los}")


@pytest.mark.parametrize("n", [1, 2])
def test_one_and_two_points_without_a_box(n):
    x = _shape("point", n, 941)
    if n == 2:
        x[1, 2] += 3.0                       # s = 3 along z (mu = 1 for the z line of sight)
    for mode, los, eb in CASES:
        kw = dict(periodic=False, mode=mode, los=los, edges_a=np.linspace(0.0, 20.0, 11),
                  edges_b=eb)
        want, _ = oracle.count(x, method="grid", **kw)
        assert want.sum() == n - 1
        got, _ = P.count(x, **kw)
        _check(got, want, what=f"grid n={n} {mode}/{los}")
        got, _ = P.count_tree(x, **kw)
        _check(got, want, what=f"tree n={n} {mode}/{los}")
