"""GPU parity at the limits of the periodic definition: the largest
separation close to half the box, and boxes with a different side per axis.

A periodic count takes the minimum image of every pair (Sect. 2.5), which is
unique only for separations below L/2.  Near that bound the grid path needs
enough cells per axis that no two stencil offsets reach the same cell (it
raises the cell count to 2k + 1 for a reach of k cells, and reports
PC_EOVERFLOW once that exceeds 2^26 cells); the k-d tree path pairs nodes
under explicit periodic images and has no such limit.  Counts must equal the
oracle's bit for bit, weighted sums within 1e-10 relative per bin.
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


def _catalogue(L, n, seed):
    """Half clustered, half uniform, in the box [0, L) (L a scalar or 3 sides)."""
    Ls = np.broadcast_to(np.asarray(L, dtype=np.float64), (3,))
    u = synth.uniform_box(n - n // 2, 1.0, seed) * Ls
    c = synth.neyman_scott(n // 2, max(1, n // 20), 10.0, 0.015, 1.0, seed + 1) * Ls
    x = np.ascontiguousarray(np.concatenate([u, c]))
    x[x >= Ls] = 0.0
    return x


def _bins(mode, r):
    if mode == "s":
        return dict(mode="s", edges_a=np.linspace(0.0, r, 10))
    if mode == "smu":
        return dict(mode="smu", edges_a=np.linspace(0.0, r, 10), edges_b=np.linspace(0, 1, 9))
    c = r / np.sqrt(2.0)          # sqrt(sigma_max^2 + pi_max^2) = r
    return dict(mode="sigpi", edges_a=np.linspace(0.0, c, 7), edges_b=np.linspace(0.0, c, 7))


@pytest.mark.parametrize("mode", ["s", "smu", "sigpi"])
def test_largest_separation_at_0p45_of_the_box(mode):
    """r = 0.45 L: the grid needs 21 cells per axis (a reach of 10 cells each
    way without aliasing); grid (FP32 + rescue and FP64) and tree paths."""
    L = 100.0
    x = _catalogue(L, 2500, 901)
    w = synth.lognormal_weights(x.shape[0], 0.3, 902, np.float64)
    kw = dict(box=L, periodic=True, **_bins(mode, 45.0))
    want, wantw = oracle.count(x, w1=w, method="grid", **kw)
    assert want.sum() > 0
    for prec in ("f32", "f64"):
        got, gotw = P.count(x, w1=w, prec=prec, **kw)
        _check(got, want, gotw, wantw, f"grid {mode} {prec}")
    got, gotw = P.count_tree(x, w1=w, **kw)
    _check(got, want, gotw, wantw, f"tree {mode}")
    y = _catalogue(L, 1200, 903)
    want, _ = oracle.count(x, y, method="grid", **kw)
    got, _ = P.count(x, y, **kw)
    _check(got, want, what=f"grid cross {mode}")
    got, _ = P.count_tree(x, y, **kw)
    _check(got, want, what=f"tree cross {mode}")


@pytest.mark.parametrize("mode", ["s", "smu", "sigpi"])
def test_separation_just_below_half_the_box(mode):
    """r = 0.499 L: the tree path counts it exactly; the grid path would need
    more than 2^26 cells and says so (PC_EOVERFLOW) instead of aliasing."""
    L = 100.0
    x = _catalogue(L, 2000, 911)
    kw = dict(box=L, periodic=True, **_bins(mode, 49.9))
    want, _ = oracle.count(x, method="grid", **kw)
    got, _ = P.count_tree(x, **kw)
    _check(got, want, what=f"tree auto {mode}")
    y = _catalogue(L, 700, 912)
    want, _ = oracle.count(x, y, method="grid", **kw)
    got, _ = P.count_tree(x, y, **kw)
    _check(got, want, what=f"tree cross {mode}")
    with pytest.raises(P.PairCountError) as e:
        P.count(x, **kw)
    assert e.value.status == P.PC_EOVERFLOW


@pytest.mark.parametrize("mode", ["s", "smu", "sigpi"])
def test_box_with_a_different_side_per_axis(mode):
    """L = (100, 60, 140): cells, stencil reach and periodic images are per
    axis; the largest separation (25) sits below the smallest half side."""
    L = np.array([100.0, 60.0, 140.0])
    x = _catalogue(L, 4000, 921)
    assert np.all(x < L)
    w = synth.lognormal_weights(x.shape[0], 0.3, 922, np.float64)
    kw = dict(box=L, periodic=True, **_bins(mode, 25.0))
    want, wantw = oracle.count(x, w1=w, method="grid", **kw)
    for prec in ("f32", "f64"):
        got, gotw = P.count(x, w1=w, prec=prec, **kw)
        _check(got, want, gotw, wantw, f"grid {mode} {prec}")
    got, gotw = P.count_tree(x, w1=w, **kw)
    _check(got, want, gotw, wantw, f"tree {mode}")
    y = _catalogue(L, 1500, 923)
    want, _ = oracle.count(x, y, method="grid", **kw)
    got, _ = P.count(x, y, **kw)
    _check(got, want, what=f"grid cross {mode}")
    got, _ = P.count_tree(x, y, **kw)
    _check(got, want, what=f"tree cross {mode}")
