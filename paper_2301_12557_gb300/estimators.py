"""Correlation-function estimators on top of the pair counts (host-side).

The counts from ``pc_count_auto`` / ``pc_count_cross`` are raw: unordered
pairs (auto) or all (i, j) pairs (cross), optionally weighted.  The
estimators of the paper (Sect. 1 and App. D) combine *normalised* counts:

- normalisation: auto counts by the number of distinct pairs,
  N (N - 1) / 2, or ((sum w)^2 - sum w^2) / 2 with weights; cross counts by
  N1 N2, or (sum w1)(sum w2);
- Landy-Szalay:    xi = (DD - 2 DR + RR) / RR
- Peebles-Hauser:  xi = DD / RR - 1, RR analytic for a periodic box ("@@")
- Szapudi-Szalay (cross): xi = (D1D2 - D1R2 - R1D2 + R1R2) / R1R2
- multipoles:      xi_l(s) = (2 l + 1) int_0^1 xi(s, mu) L_l(mu) dmu
- projected:       w_p(sigma) = 2 int_0^pi_max xi(sigma, pi) dpi

With histograms the (s, mu) and (sigma, pi) estimates are constant inside
each bin, so the integrals become exact sums over bins of the bin value
times the integral of L_l (or of 1) over the bin.

These are small host computations over histograms (numpy); the pair counts
themselves come from the GPU library.
"""

from __future__ import annotations

import numpy as np

__all__ = ["pair_norm", "normalise", "analytic_rr", "landy_szalay", "peebles_hauser",
           "szapudi_szalay", "legendre_bin_integrals", "multipoles", "projected"]


def pair_norm(n1=None, n2=None, *, w1=None, w2=None, auto=True) -> float:
    """Number (or weight) of the pairs a count can contain.

    auto: N (N - 1) / 2, or ((sum w)^2 - sum w^2) / 2 with weights;
    cross: N1 N2, or (sum w1)(sum w2).
    """
    if auto:
        if w1 is not None:
            w = np.asarray(w1, dtype=np.float64)
            return float((w.sum() ** 2 - (w * w).sum()) / 2.0)
        n = float(n1)
        return n * (n - 1.0) / 2.0
    if w1 is not None:
        return float(np.asarray(w1, dtype=np.float64).sum() * np.asarray(w2, dtype=np.float64).sum())
    return float(n1) * float(n2)


def normalise(counts, norm: float) -> np.ndarray:
    """Counts divided by their pair normalisation (see ``pair_norm``)."""
    return np.asarray(counts, dtype=np.float64) / float(norm)


def analytic_rr(edges_a, edges_b=None, *, box: float, mode: str = "s") -> np.ndarray:
    """Normalised random-random counts of a periodic box of side ``box``
    (uniform points, separations below box / 2): the fraction of the box
    volume inside each bin.

    s bins: spherical shells 4 pi / 3 (s_{k+1}^3 - s_k^3);
    (s, mu): the shell times the mu width (mu = |cos| is uniform on [0, 1]);
    (sigma, pi): annulus pi (sigma_{k+1}^2 - sigma_k^2) times 2 (pi_{j+1} - pi_j)
    (|pi| counts both signs along the line of sight).
    Layout as the counts: row-major, first axis outermost.
    """
    ea = np.asarray(edges_a, dtype=np.float64)
    V = float(box) ** 3
    if mode == "s":
        return (4.0 * np.pi / 3.0) * np.diff(ea ** 3) / V
    eb = np.asarray(edges_b, dtype=np.float64)
    if mode == "smu":
        shell = (4.0 * np.pi / 3.0) * np.diff(ea ** 3)
        return np.outer(shell, np.diff(eb)).ravel() / V
    if mode == "sigpi":
        ring = np.pi * np.diff(ea ** 2)
        return np.outer(ring, 2.0 * np.diff(eb)).ravel() / V
    raise ValueError(f"unknown mode {mode!r}")


def landy_szalay(dd, dr, rr) -> np.ndarray:
    """(DD - 2 DR + RR) / RR on normalised counts (NaN where RR = 0)."""
    dd, dr, rr = (np.asarray(a, dtype=np.float64) for a in (dd, dr, rr))
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.where(rr != 0, (dd - 2.0 * dr + rr) / rr, np.nan)


def peebles_hauser(dd, rr) -> np.ndarray:
    """DD / RR - 1 on normalised counts (NaN where RR = 0)."""
    dd, rr = np.asarray(dd, dtype=np.float64), np.asarray(rr, dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.where(rr != 0, dd / rr - 1.0, np.nan)


def szapudi_szalay(d1d2, d1r2, r1d2, r1r2) -> np.ndarray:
    """Cross correlation (D1D2 - D1R2 - R1D2 + R1R2) / R1R2 on normalised counts."""
    a, b, c, d = (np.asarray(x, dtype=np.float64) for x in (d1d2, d1r2, r1d2, r1r2))
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.where(d != 0, (a - b - c + d) / d, np.nan)


def _legendre_antiderivative(ell: int, x: np.ndarray) -> np.ndarray:
    """int_0^x L_ell(t) dt, from (2 l + 1) L_l = d/dx (L_{l+1} - L_{l-1})
    for l >= 1; int_0^x L_0 = x."""
    from numpy.polynomial import legendre as Leg
    x = np.asarray(x, dtype=np.float64)
    if ell == 0:
        return x.copy()
    c_up = np.zeros(ell + 2)
    c_up[ell + 1] = 1.0
    c_dn = np.zeros(ell + 2)
    c_dn[ell - 1] = 1.0
    f = (Leg.legval(x, c_up) - Leg.legval(x, c_dn)) / (2 * ell + 1)
    f0 = (Leg.legval(0.0, c_up) - Leg.legval(0.0, c_dn)) / (2 * ell + 1)
    return f - f0


def legendre_bin_integrals(mu_edges, ell: int) -> np.ndarray:
    """int_{mu_j}^{mu_{j+1}} L_ell(mu) dmu for every mu bin."""
    F = _legendre_antiderivative(ell, np.asarray(mu_edges, dtype=np.float64))
    return np.diff(F)


def multipoles(xi_smu, mu_edges, ells=(0, 2, 4)) -> np.ndarray:
    """xi_l(s) = (2 l + 1) sum_j xi(s, mu_j) int_{bin j} L_l(mu) dmu.

    xi_smu: (n_s, n_mu) array (or flat row-major).  Returns (len(ells), n_s).
    """
    mu_edges = np.asarray(mu_edges, dtype=np.float64)
    nmu = mu_edges.size - 1
    xi = np.asarray(xi_smu, dtype=np.float64).reshape(-1, nmu)
    out = np.empty((len(ells), xi.shape[0]))
    for k, ell in enumerate(ells):
        out[k] = (2 * ell + 1) * xi @ legendre_bin_integrals(mu_edges, ell)
    return out


def projected(xi_sigpi, pi_edges) -> np.ndarray:
    """w_p(sigma) = 2 sum_j xi(sigma, pi_j) (pi_{j+1} - pi_j).

    xi_sigpi: (n_sigma, n_pi) array (or flat row-major).
    """
    pi_edges = np.asarray(pi_edges, dtype=np.float64)
    xi = np.asarray(xi_sigpi, dtype=np.float64).reshape(-1, pi_edges.size - 1)
    return 2.0 * xi @ np.diff(pi_edges)
