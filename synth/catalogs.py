"""Seeded catalogue generators (positions and weights only).

Every generator takes an explicit integer seed and uses numpy's PCG64, so the
same call gives the same catalogue on any machine.  Coordinates are float64.
Periodic catalogues lie in [0, L) on every axis.

Shapes follow the workloads the paper benchmarks: uniform periodic randoms
(Sect. 2.1, Fig. 3 and Sect. 5), octant/survey shells (Sect. 2.4, Sect. 5 with
the BOSS DR12 randoms) and clustered mocks.  The paper's survey files are not
available, so ``survey_shell`` stands in for them with the same geometry class
(observer at the origin, a shell in comoving distance inside an angular patch,
a smooth radial selection and FKP-like weights).
"""

from __future__ import annotations

import numpy as np

SEED_BASE = 2301125570


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def _wrap_unit(x: np.ndarray, L: float) -> np.ndarray:
    """Fold generated coordinates into [0, L) (generator-side only)."""
    x = np.mod(x, L)
    x[x >= L] = 0.0
    return x


def uniform_box(n: int, L: float, seed: int) -> np.ndarray:
    """n points uniform in the periodic cube [0, L)^3."""
    x = _rng(seed).random((int(n), 3)) * float(L)
    x[x >= L] = 0.0
    return np.ascontiguousarray(x)


def neyman_scott(n: int, n_parents: int, mean_children: float, sigma: float,
                 L: float, seed: int) -> np.ndarray:
    """Neyman-Scott cluster process in a periodic cube, trimmed to exactly n.

    Parents are uniform in [0, L)^3; each parent gets Poisson(mean_children)
    children displaced by isotropic Gaussian offsets of width sigma; children
    are wrapped into the box.  If the children fall short of n, more parents
    are drawn; the first n children (in generation order) are returned.
    """
    rng = _rng(seed)
    n = int(n)
    chunks = []
    total = 0
    n_par = int(n_parents)
    while total < n:
        parents = rng.random((n_par, 3)) * L
        counts = rng.poisson(mean_children, size=n_par)
        reps = np.repeat(parents, counts, axis=0)
        kids = reps + rng.normal(0.0, sigma, size=reps.shape)
        chunks.append(kids)
        total += kids.shape[0]
        n_par = max(1000, int(1.2 * (n - total) / max(mean_children, 1e-9)) + 1)
    x = np.concatenate(chunks, axis=0)[:n]
    return np.ascontiguousarray(_wrap_unit(x, float(L)))


def mixed_box(n: int, L: float, frac_clustered: float, mean_children: float,
              sigma: float, seed: int) -> np.ndarray:
    """Union of a uniform part and a Neyman-Scott part in one periodic cube."""
    n_cl = int(round(n * frac_clustered))
    n_un = int(n) - n_cl
    a = uniform_box(n_un, L, seed)
    b = neyman_scott(n_cl, max(1, int(n_cl / mean_children)), mean_children,
                     sigma, L, seed + 1)
    return np.ascontiguousarray(np.concatenate([a, b], axis=0))


# --------------------------------------------------------------------------
# Survey-like shell (non-periodic)
# --------------------------------------------------------------------------

SURVEY_R_MIN = 1000.0
SURVEY_R_MAX = 2000.0
SURVEY_RA = (0.0, np.deg2rad(60.0))
SURVEY_DEC = (np.deg2rad(-30.0), np.deg2rad(30.0))


def survey_selection(r: np.ndarray) -> np.ndarray:
    """Smooth radial selection p(r) in (0, 1], peaked at r = 1500 Mpc/h."""
    return np.exp(-((r - 1500.0) / 500.0) ** 2)


def _shell_uniform(rng, m):
    u = rng.random(m)
    r = np.cbrt(SURVEY_R_MIN ** 3 + u * (SURVEY_R_MAX ** 3 - SURVEY_R_MIN ** 3))
    ra = SURVEY_RA[0] + rng.random(m) * (SURVEY_RA[1] - SURVEY_RA[0])
    sd = np.sin(SURVEY_DEC[0]) + rng.random(m) * (np.sin(SURVEY_DEC[1]) - np.sin(SURVEY_DEC[0]))
    dec = np.arcsin(sd)
    return np.stack([r * np.cos(dec) * np.cos(ra), r * np.cos(dec) * np.sin(ra),
                     r * np.sin(dec)], axis=1)


def _in_shell(x):
    r = np.sqrt((x * x).sum(axis=1))
    ra = np.arctan2(x[:, 1], x[:, 0])
    dec = np.arcsin(np.clip(x[:, 2] / np.maximum(r, 1e-300), -1, 1))
    ok = (r >= SURVEY_R_MIN) & (r < SURVEY_R_MAX)
    ok &= (ra >= SURVEY_RA[0]) & (ra < SURVEY_RA[1])
    ok &= (dec >= SURVEY_DEC[0]) & (dec < SURVEY_DEC[1])
    return ok, r


def survey_shell(n: int, clustered: bool, seed: int, sigma: float = 5.0,
                 mean_children: float = 10.0) -> np.ndarray:
    """n points in the shell 1000 <= r < 2000 Mpc/h inside a 60x60 deg patch.

    Points are thinned by ``survey_selection``.  ``clustered`` draws
    Neyman-Scott children around parents spread uniformly in the shell.
    """
    rng = _rng(seed)
    n = int(n)
    out = []
    total = 0
    while total < n:
        need = n - total
        if clustered:
            n_par = max(1000, int(need / (0.5 * mean_children)) + 1)
            parents = _shell_uniform(rng, n_par)
            counts = rng.poisson(mean_children, size=n_par)
            reps = np.repeat(parents, counts, axis=0)
            cand = reps + rng.normal(0.0, sigma, size=reps.shape)
        else:
            cand = _shell_uniform(rng, max(1000, int(need * 2.0) + 1))
        ok, r = _in_shell(cand)
        cand, r = cand[ok], r[ok]
        keep = rng.random(cand.shape[0]) < survey_selection(r)
        cand = cand[keep]
        out.append(cand)
        total += cand.shape[0]
    return np.ascontiguousarray(np.concatenate(out, axis=0)[:n])


def fkp_weights(x: np.ndarray, n_data: int, P0: float = 1.0e4) -> np.ndarray:
    """FKP-like weights w = 1 / (1 + nbar(r) P0), float64.

    nbar(r) = n_data * p(r) / integral(p dV) over the shell and patch, i.e.
    the expected data density with the survey selection p(r).
    """
    rr = np.linspace(SURVEY_R_MIN, SURVEY_R_MAX, 20001)
    omega = (SURVEY_RA[1] - SURVEY_RA[0]) * (np.sin(SURVEY_DEC[1]) - np.sin(SURVEY_DEC[0]))
    f = survey_selection(rr) * rr * rr
    integral = omega * float(np.sum(0.5 * (f[1:] + f[:-1]) * np.diff(rr)))
    r = np.sqrt((x * x).sum(axis=1))
    nbar = n_data * survey_selection(r) / integral
    return np.ascontiguousarray(1.0 / (1.0 + nbar * P0))


def lognormal_weights(n: int, sigma_ln: float, seed: int,
                      dtype=np.float32) -> np.ndarray:
    """Unit-mean lognormal weights exp(sigma g - sigma^2 / 2)."""
    g = _rng(seed).standard_normal(int(n))
    return np.ascontiguousarray(np.exp(sigma_ln * g - 0.5 * sigma_ln ** 2).astype(dtype))


def batch_mocks(m: int, n_min: int, n_max: int, sigma_lo: float, sigma_hi: float,
                L: float, seed: int, mean_children: float = 10.0):
    """m Neyman-Scott mocks with N ~ U[n_min, n_max] and sigma ~ U[lo, hi].

    Mock k is seeded with seed + 1000 * k, so any single mock can be
    regenerated on its own.
    """
    return [batch_mock(k, n_min, n_max, sigma_lo, sigma_hi, L, seed, mean_children)
            for k in range(int(m))]


def batch_mock_size(k: int, n_min: int, n_max: int, seed: int) -> int:
    """Number of points of mock k of ``batch_mocks`` (no positions drawn)."""
    return int(_rng(seed + 1000 * int(k)).integers(n_min, n_max + 1))


def batch_mock(k: int, n_min: int, n_max: int, sigma_lo: float, sigma_hi: float,
               L: float, seed: int, mean_children: float = 10.0) -> np.ndarray:
    """Mock k of ``batch_mocks`` on its own (the same array, from its own seed)."""
    rng = _rng(seed + 1000 * int(k))
    n = int(rng.integers(n_min, n_max + 1))
    sig = float(sigma_lo + rng.random() * (sigma_hi - sigma_lo))
    return neyman_scott(n, max(1, n // int(mean_children)), mean_children,
                        sig, L, seed + 1000 * int(k) + 1)


def lattice_points(n: int, side: int, seed: int, unique: bool = True) -> np.ndarray:
    """n integer-valued points in [0, side)^3 (exact in any float format)."""
    rng = _rng(seed)
    if unique:
        idx = rng.choice(side ** 3, size=int(n), replace=False)
        pts = np.stack([idx % side, (idx // side) % side, idx // (side * side)], axis=1)
    else:
        pts = rng.integers(0, side, size=(int(n), 3))
    return np.ascontiguousarray(pts.astype(np.float64))


def near_edge_pairs(edges_len: np.ndarray, L: float, n_pairs: int, rel_offsets,
                    seed: int, spacing: float | None = None) -> np.ndarray:
    """Point pairs whose separation sits at edge * (1 + offset).

    For each pair an edge value and an offset are drawn from the given lists;
    the two points are placed along a random direction.  Pair anchors are laid
    out on a coarse jittered lattice so different pairs are mostly far apart
    (they are still all counted; only the pair geometry is controlled).
    Returns a (2 * n_pairs, 3) array inside [0, L).
    """
    rng = _rng(seed)
    e = np.asarray(edges_len, dtype=np.float64)
    e = e[e > 0]
    off = np.asarray(rel_offsets, dtype=np.float64)
    k = rng.integers(0, e.size, size=n_pairs)
    o = off[rng.integers(0, off.size, size=n_pairs)]
    d = e[k] * (1.0 + o)
    v = rng.standard_normal((n_pairs, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    a = rng.random((n_pairs, 3)) * L
    b = a + v * d[:, None]
    pts = np.empty((2 * n_pairs, 3))
    pts[0::2] = a
    pts[1::2] = b
    return np.ascontiguousarray(_wrap_unit(pts, float(L)))


def s2_samples(n: int, r_max: float, seed: int) -> np.ndarray:
    """n squared pair separations in [0, r_max^2) with the distribution of
    uniform pairs, s ~ s^2 ds (App. C: s^2 = x^(2/3) r_max^2 for x uniform in
    [0, 1)), rounded to binary32 (the benchmark streams 4-byte samples)."""
    x = _rng(seed).random(int(n))
    s2 = (x ** (2.0 / 3.0)) * (float(r_max) ** 2)
    out = s2.astype(np.float32)
    top = np.float32(float(r_max) ** 2)
    out[out >= top] = np.nextafter(top, np.float32(0))
    return np.ascontiguousarray(out)
