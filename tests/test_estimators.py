"""Estimators, normalisations, analytic RR, multipoles and w_p (host-side),
pinned to closed forms, library integrals and the oracle's counts."""

import numpy as np
import pytest

import oracle
import synth
from paper_2301_12557_gb300 import estimators as E


def test_pair_norms():
    assert E.pair_norm(10) == 45.0
    assert E.pair_norm(7, 11, auto=False) == 77.0
    w = np.array([0.5, 1.5, 2.0, 3.0])
    brute = sum(w[i] * w[j] for i in range(4) for j in range(i + 1, 4))
    assert E.pair_norm(w1=w) == pytest.approx(brute, rel=1e-15)
    v = np.array([1.0, 2.0])
    assert E.pair_norm(w1=w, w2=v, auto=False) == pytest.approx(w.sum() * 3.0)


def test_analytic_rr_closed_forms():
    L, R = 100.0, 20.0
    ea = np.linspace(0.0, R, 11)
    s = E.analytic_rr(ea, box=L)
    assert s.sum() == pytest.approx(4.0 / 3.0 * np.pi * R ** 3 / L ** 3, rel=1e-14)
    mu = np.linspace(0.0, 1.0, 5)
    smu = E.analytic_rr(ea, mu, box=L, mode="smu").reshape(10, 4)
    assert np.allclose(smu.sum(1), s, rtol=1e-14)
    pe = np.linspace(0.0, 10.0, 6)
    sp = E.analytic_rr(ea, pe, box=L, mode="sigpi")
    assert sp.sum() == pytest.approx(np.pi * R ** 2 * 2 * 10.0 / L ** 3, rel=1e-14)


def test_analytic_rr_matches_uniform_randoms_and_peebles_hauser_is_null():
    """Uniform periodic randoms: the oracle's normalised counts equal the
    volume fractions within 5 sigma, so DD / @@ - 1 is zero within noise."""
    L, n = 200.0, 6000
    x = synth.uniform_box(n, L, 411)
    ea = np.linspace(0.0, 40.0, 9)
    dd, _ = oracle.count(x, box=L, periodic=True, edges_a=ea, method="grid")
    norm = E.pair_norm(n)
    rr = E.analytic_rr(ea, box=L)
    expect = rr * norm
    assert np.all(np.abs(dd - expect) <= 5 * np.sqrt(expect) + 1)
    xi = E.peebles_hauser(E.normalise(dd, norm), rr)
    assert np.all(np.abs(xi) <= 5 / np.sqrt(expect) + 1 / expect)


def test_estimator_formulas():
    assert E.landy_szalay(0.5, 0.2, 0.25) == pytest.approx(1.4)
    assert E.peebles_hauser(0.3, 0.2) == pytest.approx(0.5)
    assert E.szapudi_szalay(0.6, 0.2, 0.3, 0.25) == pytest.approx((0.6 - 0.2 - 0.3 + 0.25) / 0.25)
    same = np.array([0.1, 0.2, 0.4])
    assert np.all(E.landy_szalay(same, same, same) == 0.0)
    assert np.isnan(E.landy_szalay(1.0, 1.0, 0.0))


def test_legendre_bin_integrals_against_quadrature():
    integrate = pytest.importorskip("scipy.integrate")
    from scipy.special import eval_legendre
    mu = np.array([0.0, 0.1, 0.35, 0.7, 1.0])
    for ell in (0, 1, 2, 3, 4, 6):
        got = E.legendre_bin_integrals(mu, ell)
        want = [integrate.quad(lambda t: eval_legendre(ell, t), a, b, epsabs=1e-15)[0]
                for a, b in zip(mu[:-1], mu[1:])]
        assert np.allclose(got, want, rtol=1e-12, atol=1e-15)
    # over [0, 1]: 1 for l = 0, 0 for even l > 0
    full = np.array([0.0, 1.0])
    assert E.legendre_bin_integrals(full, 0)[0] == pytest.approx(1.0)
    for ell in (2, 4, 6):
        assert abs(E.legendre_bin_integrals(full, ell)[0]) < 1e-15


def test_multipoles_and_projected_closed_forms():
    mu = np.linspace(0.0, 1.0, 21)
    c = np.array([0.5, -0.25, 2.0])
    xi = np.repeat(c[:, None], 20, axis=1)          # isotropic: only the monopole
    m = E.multipoles(xi, mu)
    assert np.allclose(m[0], c, rtol=1e-14)
    assert np.allclose(m[1:], 0.0, atol=1e-14)
    # xi(mu) = bin averages of L_2: xi_2 = 5 sum_j (int_j L_2)^2 / dmu_j
    i2 = E.legendre_bin_integrals(mu, 2)
    xi2 = (i2 / np.diff(mu))[None, :]
    m2 = E.multipoles(xi2, mu, ells=(0, 2))
    assert m2[0, 0] == pytest.approx(0.0, abs=1e-14)
    assert m2[1, 0] == pytest.approx(5.0 * np.sum(i2 ** 2 / np.diff(mu)), rel=1e-14)
    assert m2[1, 0] == pytest.approx(1.0, rel=5e-3)   # -> 1 as the bins shrink (O(dmu^2))
    pe = np.linspace(0.0, 40.0, 9)
    wp = E.projected(np.full((3, 8), 0.1), pe)
    assert np.allclose(wp, 2 * 0.1 * 40.0, rtol=1e-14)
