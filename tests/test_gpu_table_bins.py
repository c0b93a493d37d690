"""GPU parity of the lookup-table bins for the second axis: (sigma, pi) with
edges that are neither evenly spaced nor start at zero on either axis, and
(s, mu) with unevenly spaced mu edges (Sect. 3.2.3: any monotone edges go
through the hybrid index table).  Besides clustered catalogues, pairs are
planted with pi, sigma or mu at an edge times (1 + delta) along the z line of
sight, so the binary64 rescue decides them.  Grid (FP32 + rescue, FP64) and
tree paths; counts bit-exact, weighted sums within 1e-10 relative per bin.
"""

import numpy as np
import pytest

import oracle
import synth

P = pytest.importorskip("paper_2301_12557_gb300")
torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

WREL = 1e-10

OFFS = [0.0, 2.0 ** -52, -2.0 ** -52, 1e-9, -1e-9, 1e-7, -1e-7, 2e-6, -2e-6]
SIG_EDGES = np.array([0.5, 1.0, 2.0, 4.0, 8.0, 16.0, 25.0])
PI_EDGES = np.array([1.0, 3.0, 7.0, 12.0, 20.0])
MU_EDGES = np.array([0.0, 0.05, 0.2, 0.21, 0.5, 0.8, 0.95, 1.0])


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


def _planted(L, n_pairs, seed, sep):
    """Point pairs a, b = a + (t cos phi, t sin phi, +-dz), (t, dz) from sep(rng),
    folded into [0, L)."""
    rng = np.random.default_rng(seed)
    t, dz = sep(rng, n_pairs)
    phi = rng.uniform(0.0, 2.0 * np.pi, n_pairs)
    sgn = np.where(rng.random(n_pairs) < 0.5, -1.0, 1.0)
    a = rng.uniform(0.0, L, (n_pairs, 3))
    b = a + np.stack([t * np.cos(phi), t * np.sin(phi), sgn * dz], axis=1)
    x = np.empty((2 * n_pairs, 3))
    x[0::2], x[1::2] = a, b
    x = np.mod(x, L)
    x[x >= L] = 0.0
    return np.ascontiguousarray(x)


def _sigpi_sep(rng, n):
    off = np.asarray(OFFS)
    sg = SIG_EDGES[rng.integers(0, SIG_EDGES.size, n)] * (1 + off[rng.integers(0, off.size, n)])
    pz = PI_EDGES[rng.integers(0, PI_EDGES.size, n)] * (1 + off[rng.integers(0, off.size, n)])
    return sg, pz


def _mu_sep(rng, n):
    off = np.asarray(OFFS)
    s = rng.uniform(2.0, 29.0, n)
    mu = np.minimum(MU_EDGES[rng.integers(0, MU_EDGES.size, n)] *
                    (1 + off[rng.integers(0, off.size, n)]), 1.0)
    return s * np.sqrt(np.maximum(1.0 - mu * mu, 0.0)), s * mu


def _run(x, y, w, what, **kw):
    want, wantw = oracle.count(x, w1=w, method="grid", **kw)
    assert want.sum() > 0
    for prec in ("f32", "f64"):
        got, gotw = P.count(x, w1=w, prec=prec, **kw)
        _check(got, want, gotw, wantw, f"{what} grid {prec}")
    got, gotw = P.count_tree(x, w1=w, **kw)
    _check(got, want, gotw, wantw, f"{what} tree")
    want, _ = oracle.count(x, y, method="grid", **kw)
    got, _ = P.count(x, y, **kw)
    _check(got, want, what=f"{what} grid cross")
    got, _ = P.count_tree(x, y, **kw)
    _check(got, want, what=f"{what} tree cross")


def test_sigpi_table_bins_z():
    L = 150.0
    x = np.vstack([synth.neyman_scott(6000, 600, 10.0, 2.0, L, 951),
                   _planted(L, 3000, 952, _sigpi_sep)])
    y = synth.uniform_box(3000, L, 953)
    w = synth.lognormal_weights(x.shape[0], 0.3, 954, np.float64)
    _run(x, y, w, "sigpi z", box=L, periodic=True, mode="sigpi", los="z",
         edges_a=SIG_EDGES, edges_b=PI_EDGES)


def test_sigpi_table_bins_midpoint():
    x = synth.survey_shell(5000, True, 961)
    y = synth.survey_shell(4000, False, 962)
    w = synth.fkp_weights(x, 5000)
    _run(x, y, w, "sigpi mid", periodic=False, mode="sigpi", los="mid",
         edges_a=SIG_EDGES, edges_b=PI_EDGES)


def test_uneven_mu_edges_z():
    L = 150.0
    x = np.vstack([synth.neyman_scott(6000, 600, 10.0, 2.0, L, 971),
                   _planted(L, 3000, 972, _mu_sep)])
    y = synth.uniform_box(3000, L, 973)
    w = synth.lognormal_weights(x.shape[0], 0.3, 974, np.float64)
    _run(x, y, w, "smu uneven mu z", box=L, periodic=True, mode="smu", los="z",
         edges_a=np.linspace(0.0, 30.0, 16), edges_b=MU_EDGES)


def test_uneven_mu_edges_midpoint():
    x = synth.survey_shell(5000, True, 981)
    y = synth.survey_shell(4000, False, 982)
    w = synth.fkp_weights(x, 5000)
    _run(x, y, w, "smu uneven mu mid", periodic=False, mode="smu", los="mid",
         edges_a=np.linspace(0.0, 30.0, 16), edges_b=MU_EDGES)
