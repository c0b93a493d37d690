"""The five synthetic workloads (catalogue recipe + binning), by name.

Bin layouts follow the paper's binning schemes (Sect. 5): linear s bins on
[0, 200) Mpc/h, linear mu bins on [0, 1], linear sigma/pi bins.  Seeds are
SEED_BASE + workload index (mocks additionally + 1000 * mock index).
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import catalogs as C


def linear_edges(lo: float, hi: float, n: int) -> np.ndarray:
    """n + 1 evenly spaced float64 edges from lo to hi (exact endpoints)."""
    e = lo + (hi - lo) * np.arange(n + 1, dtype=np.float64) / n
    e[0], e[-1] = lo, hi
    return e


@dataclass
class Workload:
    name: str
    index: int
    description: str
    periodic: bool
    L: float                      # periodic box side (0 for survey geometry)
    mode: str                     # "s", "smu", "sigpi"
    los: str                      # "z" or "mid"
    edges_a: np.ndarray           # s or sigma edges
    edges_b: np.ndarray | None    # mu or pi edges
    weighted: bool
    pair_kinds: tuple = ("DD",)
    extra: dict = field(default_factory=dict)

    @property
    def seed(self) -> int:
        return C.SEED_BASE + self.index


S40 = linear_edges(0.0, 200.0, 40)
MU100 = linear_edges(0.0, 1.0, 100)

WORKLOADS = {
    "uniform_periodic_n20k_s40": Workload(
        "uniform_periodic_n20k_s40", 1,
        "periodic cube L=1000, N=20,000 uniform, auto DD, 40 linear s bins on [0,200)",
        True, 1000.0, "s", "z", S40, None, False, ("DD",), {"n": 20_000}),
    "ns_periodic_n2m_smu40x100": Workload(
        "ns_periodic_n2m_smu40x100", 2,
        "periodic cube L=1000, N=2,000,000 Neyman-Scott (200k parents, Poisson(10), sigma=5), "
        "auto DD in (s, mu) 40x100, LOS z",
        True, 1000.0, "smu", "z", S40, MU100, False, ("DD",),
        {"n": 2_000_000, "parents": 200_000, "children": 10.0, "sigma": 5.0}),
    "survey_shell_d1m_r20m_sigpi40x40": Workload(
        "survey_shell_d1m_r20m_sigpi40x40", 3,
        "survey shell 1000-2000 Mpc/h, 60x60 deg, D=1,000,000 clustered, R=20,000,000 uniform, "
        "FKP weights, weighted DD/DR/RR in (sigma, pi) 40x40 on [0,200)^2, midpoint LOS",
        False, 0.0, "sigpi", "mid", S40, S40, True, ("DD", "DR", "RR"),
        {"n_data": 1_000_000, "n_rand": 20_000_000}),
    "mocks256_ns_smu40x100": Workload(
        "mocks256_ns_smu40x100", 4,
        "256 periodic Neyman-Scott mocks L=1000, N~U[200k,800k], sigma~U[3,8], "
        "auto (s, mu) 40x100, LOS z, one batched launch",
        True, 1000.0, "smu", "z", S40, MU100, False, ("DD",),
        {"m": 256, "n_min": 200_000, "n_max": 800_000}),
    "mixed_periodic_n100m_s40_w": Workload(
        "mixed_periodic_n100m_s40_w", 5,
        "periodic cube L=3000, N=100,000,000 (50% uniform, 50% Neyman-Scott sigma=5), "
        "float32 lognormal weights (sigma_ln=0.3), weighted auto in 40 s bins on [0,200)",
        True, 3000.0, "s", "z", S40, None, True, ("DD",), {"n": 100_000_000}),
}


def make_inputs(w: Workload, scale: float = 1.0):
    """Generate the catalogue(s) of a workload, optionally scaled down in N.

    ``scale`` < 1 shrinks every N (and the number of cluster parents in
    proportion) inside the same volume, so the oracle can finish quickly while
    the geometry, cluster shape and binning stay the same.  Returns a dict.
    """
    s = float(scale)
    if w.index == 1:
        n = max(2, int(w.extra["n"] * s))
        L = w.L
        return {"D": C.uniform_box(n, L, w.seed), "L": L}
    if w.index == 2:
        n = max(2, int(w.extra["n"] * s))
        L = w.L
        par = max(1, int(w.extra["parents"] * s))
        return {"D": C.neyman_scott(n, par, w.extra["children"], w.extra["sigma"], L, w.seed),
                "L": L}
    if w.index == 3:
        nd = max(2, int(w.extra["n_data"] * s))
        nr = max(2, int(w.extra["n_rand"] * s))
        D = C.survey_shell(nd, True, w.seed)
        R = C.survey_shell(nr, False, w.seed + 7)
        return {"D": D, "R": R, "wD": C.fkp_weights(D, nd), "wR": C.fkp_weights(R, nd), "L": 0.0}
    if w.index == 4:
        m = max(1, int(w.extra["m"] * min(1.0, s * 64))) if s < 1 else w.extra["m"]
        nmin = max(2, int(w.extra["n_min"] * s))
        nmax = max(nmin, int(w.extra["n_max"] * s))
        L = w.L
        return {"mocks": C.batch_mocks(m, nmin, nmax, 3.0, 8.0, L, w.seed), "L": L}
    if w.index == 5:
        n = max(2, int(w.extra["n"] * s))
        L = w.L
        D = C.mixed_box(n, L, 0.5, 10.0, 5.0, w.seed)
        return {"D": D, "wD": C.lognormal_weights(n, 0.3, w.seed + 3), "L": L}
    raise KeyError(w.name)
