"""The seeded input generators follow their stated recipes (CPU only).

Every parity case and benchmark line draws its catalogues from ``synth``; these
checks tie each generator to the distribution it claims: ranges, exact sizes,
determinism per seed, the Neyman-Scott pair excess from the Gaussian offsets,
the survey shell's geometry and radial selection, FKP normalisation, unit-mean
lognormal weights, and separations of the planted near-edge pairs.
"""

import math

import numpy as np
import pytest

import synth
from synth import catalogs as C
from synth import workloads as W


def test_seeded_and_reproducible():
    for gen in (lambda s: C.uniform_box(500, 10.0, s),
                lambda s: C.neyman_scott(500, 50, 10.0, 1.0, 10.0, s),
                lambda s: C.survey_shell(300, True, s),
                lambda s: C.lognormal_weights(300, 0.3, s)):
        a, b, c = gen(3), gen(3), gen(4)
        assert np.array_equal(a, b)
        assert not np.array_equal(a, c)


def test_uniform_box_moments():
    L, n = 50.0, 200_000
    x = C.uniform_box(n, L, 1)
    assert x.shape == (n, 3) and x.dtype == np.float64 and x.flags.c_contiguous
    assert x.min() >= 0.0 and x.max() < L
    # mean L/2 and variance L^2/12 per axis, within 5 standard errors
    se_mean = L / math.sqrt(12 * n)
    assert np.all(np.abs(x.mean(axis=0) - L / 2) < 5 * se_mean)
    se_var = L * L * math.sqrt(1 / 180 / n) * 2     # var of U^2 terms, generous
    assert np.all(np.abs(x.var(axis=0) - L * L / 12) < 5 * se_var)


def _maxwell_cdf(r, scale):
    """P(|d| < r) for d ~ N(0, scale^2 I_3)."""
    t = r / scale
    return math.erf(t / math.sqrt(2)) - math.sqrt(2 / math.pi) * t * math.exp(-t * t / 2)


def test_neyman_scott_size_range_and_pair_excess():
    spatial = pytest.importorskip("scipy.spatial")
    L, n, lam, sig = 400.0, 40_000, 10.0, 2.0
    x = C.neyman_scott(n, n // 10, lam, sig, L, 7)
    assert x.shape == (n, 3)
    assert x.min() >= 0.0 and x.max() < L
    r = 3 * sig
    t = spatial.cKDTree(x, boxsize=L)
    pairs = (int(t.count_neighbors(t, r)) - n) // 2
    uniform = n * (n - 1) / 2 * 4 / 3 * math.pi * r ** 3 / L ** 3
    # siblings: about n / lam parents with Poisson(lam) children, so
    # (n / lam) lam^2 / 2 sibling pairs, separated by N(0, 2 sig^2 I)
    siblings = n * lam / 2 * _maxwell_cdf(r, sig * math.sqrt(2))
    want = uniform + siblings
    assert abs(pairs - want) < 0.05 * want, (pairs, want)
    assert pairs > 10 * uniform


def test_mixed_box_halves():
    L, n = 300.0, 20_000
    x = C.mixed_box(n, L, 0.5, 10.0, 5.0, 11)
    assert x.shape == (n, 3) and x.min() >= 0.0 and x.max() < L
    assert np.array_equal(x[: n // 2], C.uniform_box(n // 2, L, 11))


def test_survey_shell_geometry_and_selection():
    n = 60_000
    x = C.survey_shell(n, False, 5)
    assert x.shape == (n, 3)
    r = np.sqrt((x * x).sum(axis=1))
    ra = np.arctan2(x[:, 1], x[:, 0])
    dec = np.arcsin(x[:, 2] / r)
    assert r.min() >= C.SURVEY_R_MIN and r.max() < C.SURVEY_R_MAX
    assert ra.min() >= C.SURVEY_RA[0] and ra.max() < C.SURVEY_RA[1]
    assert dec.min() >= C.SURVEY_DEC[0] and dec.max() < C.SURVEY_DEC[1]
    # uniform in volume, thinned by p(r): the radial density is r^2 p(r)
    edges = np.linspace(C.SURVEY_R_MIN, C.SURVEY_R_MAX, 21)
    got, _ = np.histogram(r, edges)
    rr = np.linspace(C.SURVEY_R_MIN, C.SURVEY_R_MAX, 200_001)
    f = rr * rr * C.survey_selection(rr)
    cdf = np.concatenate([[0.0], np.cumsum(0.5 * (f[1:] + f[:-1]) * np.diff(rr))])
    want = np.diff(np.interp(edges, rr, cdf)) / cdf[-1] * n
    assert np.all(np.abs(got - want) < 5 * np.sqrt(want)), (got, want)
    # declination uniform in sin(dec)
    sd = np.sin(dec)
    se = np.linspace(math.sin(C.SURVEY_DEC[0]), math.sin(C.SURVEY_DEC[1]), 11)
    got, _ = np.histogram(sd, se)
    assert np.all(np.abs(got - n / 10) < 5 * math.sqrt(n / 10))
    # clustered data stay inside the same footprint
    d = C.survey_shell(5000, True, 6)
    rd = np.sqrt((d * d).sum(axis=1))
    assert rd.min() >= C.SURVEY_R_MIN and rd.max() < C.SURVEY_R_MAX


def test_fkp_weights_formula_and_normalisation():
    n_data = 1_000_000
    R = C.survey_shell(50_000, False, 8)
    w = C.fkp_weights(R, n_data, P0=1.0e4)
    assert np.all((w > 0) & (w < 1))
    nbar = (1.0 / w - 1.0) / 1.0e4
    r = np.sqrt((R * R).sum(axis=1))
    # nbar is proportional to p(r) ...
    ratio = nbar / C.survey_selection(r)
    assert np.allclose(ratio, ratio[0], rtol=1e-9)
    # ... and integrates to n_data over the footprint
    omega = (C.SURVEY_RA[1] - C.SURVEY_RA[0]) * (math.sin(C.SURVEY_DEC[1]) -
                                                 math.sin(C.SURVEY_DEC[0]))
    rr = np.linspace(C.SURVEY_R_MIN, C.SURVEY_R_MAX, 100_001)
    f = C.survey_selection(rr) * rr * rr
    integral = omega * float(np.sum(0.5 * (f[1:] + f[:-1]) * np.diff(rr)))
    assert abs(ratio[0] * integral - n_data) < 1e-6 * n_data


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_lognormal_weights_unit_mean(dtype):
    n, s = 400_000, 0.3
    w = C.lognormal_weights(n, s, 9, dtype)
    assert w.dtype == dtype and w.shape == (n,) and np.all(w > 0)
    sd = math.sqrt(math.exp(s * s) - 1)          # std of a unit-mean lognormal
    assert abs(float(w.astype(np.float64).mean()) - 1.0) < 5 * sd / math.sqrt(n)
    lg = np.log(w.astype(np.float64))
    assert abs(lg.std() - s) < 0.01
    assert abs(lg.mean() + s * s / 2) < 5 * s / math.sqrt(n)


def test_batch_mocks_ranges_and_independent_seeds():
    mocks = C.batch_mocks(6, 1000, 3000, 3.0, 8.0, 200.0, 123)
    assert len(mocks) == 6
    for k, x in enumerate(mocks):
        assert 1000 <= x.shape[0] <= 3000
        assert x.min() >= 0.0 and x.max() < 200.0
        # mock k regenerates from its own seed alone
        rng = np.random.Generator(np.random.PCG64(123 + 1000 * k))
        n = int(rng.integers(1000, 3001))
        sig = float(3.0 + rng.random() * 5.0)
        assert n == x.shape[0]
        assert np.array_equal(x, C.neyman_scott(n, n // 10, 10.0, sig, 200.0, 123 + 1000 * k + 1))


def test_lattice_points():
    x = C.lattice_points(500, 9, 3, unique=True)
    assert np.array_equal(x, np.round(x)) and x.min() >= 0 and x.max() <= 8
    assert len({tuple(p) for p in x}) == 500
    y = C.lattice_points(2000, 5, 4, unique=False)
    assert np.array_equal(y, np.round(y)) and y.min() >= 0 and y.max() <= 4


def test_near_edge_pairs_sit_at_the_requested_separations():
    L = 1000.0
    edges = W.linear_edges(0.0, 200.0, 40)
    offs = [0.0, 1e-15, -1e-15, 1e-9, -1e-9, 1e-5]
    x = C.near_edge_pairs(edges, L, 5000, offs, 12)
    assert x.shape == (10000, 3) and x.min() >= 0.0 and x.max() < L
    d = x[1::2] - x[0::2]
    d -= L * np.round(d / L)                      # minimum image
    s = np.sqrt((d * d).sum(axis=1))
    pos = edges[edges > 0]
    # each separation is edge * (1 + offset) for some listed edge and offset,
    # up to the rounding of the placement (a few ulps of L)
    cand = pos[:, None] * (1.0 + np.asarray(offs))[None, :]
    err = np.abs(s[:, None, None] - cand[None]).min(axis=(1, 2))
    assert err.max() < 1e-12 * L


def test_linear_edges_and_workloads():
    e = W.linear_edges(0.0, 200.0, 40)
    assert e[0] == 0.0 and e[-1] == 200.0 and np.all(np.diff(e) > 0)
    assert np.allclose(np.diff(e), 5.0, rtol=1e-12)
    for name, w in W.WORKLOADS.items():
        assert w.name == name and w.seed == C.SEED_BASE + w.index
        inp = W.make_inputs(w, 1e-3 if w.index != 5 else 1e-5)
        if w.index == 3:
            assert inp["D"].shape[1] == 3 and inp["R"].shape[0] == int(20_000_000 * 1e-3)
            assert inp["wD"].shape == (inp["D"].shape[0],)
        elif w.index == 4:
            assert len(inp["mocks"]) >= 1
        else:
            assert inp["D"].shape[1] == 3 and inp["D"].max() < w.L
    assert synth.WORKLOADS is W.WORKLOADS
