#!/usr/bin/env python
"""Write the full-size expected histograms, with the CPU oracle alone.

Each target regenerates one workload catalogue with ``synth`` (seeded),
records a SHA-256 of its bytes (coordinates, then weights), counts every pair
with the oracle's cell list (``oracle.count(method="grid")``, all host cores)
and writes ``tests/golden/fullsize/<target>.json``: the workload name, seed,
catalogue hash, size, oracle method, thread count and run time, the git
commit of this script, the int64 counts and, for weighted targets, the
binary64 weighted sums.  Nothing here touches the CUDA library.

The targets are the catalogues whose whole histogram the oracle can produce
in minutes on a many-core host: the 20,000-point uniform cube, the 2,000,000-
point clustered cube in (s, mu), the survey shell's weighted DD in
(sigma, pi) along the midpoint line of sight, and four of the 256 mocks (the
smallest, the largest and the two of median size).

Usage:
  python tests/golden/make_fullsize.py [--commit SHA] [--hash-only] [target ...]
``--hash-only`` prints each target's catalogue hash and size and writes
nothing (to check that another machine draws the same catalogues).
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
OUT = os.path.join(HERE, "fullsize")
sys.path.insert(0, ROOT)

from synth import catalogs as C  # noqa: E402
from synth import workloads as W  # noqa: E402


def mock_indices():
    """Mocks of the 256-mock batch: smallest, largest, two of median size."""
    w = W.WORKLOADS["mocks256_ns_smu40x100"]
    sizes = [C.batch_mock_size(k, w.extra["n_min"], w.extra["n_max"], w.seed)
             for k in range(w.extra["m"])]
    order = sorted(range(len(sizes)), key=lambda k: (sizes[k], k))
    m = len(order)
    return {"smallest": order[0], "largest": order[-1],
            "median_lo": order[m // 2 - 1], "median_hi": order[m // 2]}


def targets():
    """name -> (workload, builder returning (x, weights or None))."""
    t = {}
    w1 = W.WORKLOADS["uniform_periodic_n20k_s40"]
    t["uniform_periodic_n20k_s40"] = (w1, lambda: (W.make_inputs(w1)["D"], None))
    w2 = W.WORKLOADS["ns_periodic_n2m_smu40x100"]
    t["ns_periodic_n2m_smu40x100"] = (w2, lambda: (W.make_inputs(w2)["D"], None))
    w3 = W.WORKLOADS["survey_shell_d1m_r20m_sigpi40x40"]

    def shell_dd():
        nd = w3.extra["n_data"]
        D = C.survey_shell(nd, True, w3.seed)
        return D, C.fkp_weights(D, nd)
    t["survey_shell_d1m_r20m_sigpi40x40_DD"] = (w3, shell_dd)
    w4 = W.WORKLOADS["mocks256_ns_smu40x100"]
    for tag, k in mock_indices().items():
        def one(k=k):
            return C.batch_mock(k, w4.extra["n_min"], w4.extra["n_max"], 3.0, 8.0, w4.L,
                                w4.seed), None
        t[f"mocks256_ns_smu40x100_mock{k}"] = (w4, one)
    return t


def catalogue_hash(x, wt) -> str:
    h = hashlib.sha256(np.ascontiguousarray(x, dtype=np.float64).tobytes())
    if wt is not None:
        h.update(np.ascontiguousarray(wt).tobytes())
    return h.hexdigest()


def script_commit(given):
    if given:
        return given
    try:
        sha = subprocess.run(["git", "-C", ROOT, "rev-parse", "HEAD"], capture_output=True,
                             text=True, check=True).stdout.strip()
        dirty = subprocess.run(["git", "-C", ROOT, "status", "--porcelain", "--",
                                os.path.relpath(__file__, ROOT)],
                               capture_output=True, text=True).stdout.strip()
        return sha + ("+modified" if dirty else "")
    except Exception:
        return "unknown"


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("names", nargs="*")
    ap.add_argument("--commit", default=None)
    ap.add_argument("--hash-only", action="store_true")
    ap.add_argument("--out", default=OUT)
    a = ap.parse_args()
    tg = targets()
    names = a.names or list(tg)
    for nm in names:
        if nm not in tg:
            raise SystemExit(f"unknown target {nm}; known: {', '.join(tg)}")
    if not a.hash_only:
        import oracle
        oracle.build()
        os.makedirs(a.out, exist_ok=True)
    commit = script_commit(a.commit)
    for nm in names:
        w, make = tg[nm]
        x, wt = make()
        hsh = catalogue_hash(x, wt)
        if a.hash_only:
            print(json.dumps({"target": nm, "n": int(x.shape[0]), "sha256": hsh}), flush=True)
            continue
        threads = oracle.default_threads()
        t0 = time.perf_counter()
        c, wc = oracle.count(x, w1=wt, box=w.L if w.periodic else None, periodic=w.periodic,
                             mode=w.mode, los=w.los, edges_a=w.edges_a, edges_b=w.edges_b,
                             method="grid", threads=threads)
        dt = time.perf_counter() - t0
        rec = {"target": nm, "workload": w.name, "seed": int(w.seed),
               "n": int(x.shape[0]), "catalogue_sha256": hsh, "weighted": wt is not None,
               "oracle": "oracle.count(method='grid'): cell list, binary64 definition",
               "threads": int(threads), "seconds": round(dt, 1), "script_commit": commit,
               "counts": [int(v) for v in c],
               "wcounts": [float(v) for v in wc] if wc is not None else None}
        path = os.path.join(a.out, nm + ".json")
        with open(path + ".tmp", "w") as f:
            json.dump(rec, f, separators=(",", ":"))
            f.write("\n")
        os.replace(path + ".tmp", path)
        print(f"{nm}: n={x.shape[0]} pairs={int(c.sum())} {dt:.1f} s -> {path}", flush=True)


if __name__ == "__main__":
    main()
