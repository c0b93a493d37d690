"""CPU oracle for exact pair counting -- TEST INFRASTRUCTURE ONLY.

This package is the plain, slow, obviously-correct definition the CUDA path is
checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py`` (its cpu_baseline leg and its ``--impl reference`` arm) may import
it.  The product library never imports, links or calls anything here, and
this package imports nothing from the product.

The arithmetic lives in ``paircount_oracle.c`` (plain C, binary64, compiled
without FMA contraction); this module only compiles it with gcc and marshals
numpy arrays.  Every function cites the paper passage it follows in the C
source header.  Parity pins for it are in ``tests/test_oracle_*.py``.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "paircount_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

MODES = {"s": 0, "smu": 1, "sigpi": 2}
LOS = {"z": 0, "mid": 1}


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-pthread", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _configure(lib):
    """Declare the C signatures on a loaded copy of the oracle library."""
    dp = ctypes.POINTER(ctypes.c_double)
    i64p = ctypes.POINTER(ctypes.c_int64)
    ip = ctypes.POINTER(ctypes.c_int)
    lib.oracle_count.restype = ctypes.c_int
    lib.oracle_count.argtypes = [
        dp, dp, ctypes.c_int64, dp, dp, ctypes.c_int64,
        ctypes.c_int, dp, ctypes.c_int, ctypes.c_int,
        ctypes.c_int, dp, ctypes.c_int, dp,
        ctypes.c_int, ctypes.c_int, i64p, dp]
    lib.oracle_count_kdtree.restype = ctypes.c_int
    lib.oracle_count_kdtree.argtypes = [
        dp, dp, ctypes.c_int64, dp, dp, ctypes.c_int64,
        ctypes.c_int, dp, ctypes.c_int, ctypes.c_int,
        ctypes.c_int, dp, ctypes.c_int, dp,
        ctypes.c_int, i64p, dp]
    lib.oracle_kdtree.restype = ctypes.c_int
    lib.oracle_kdtree.argtypes = [dp, ctypes.c_int64, ctypes.c_int, dp, ctypes.c_int,
                                  ctypes.c_int64, i64p, i64p, ip, dp, i64p]
    lib.oracle_pair_bin.restype = ctypes.c_int
    lib.oracle_pair_bin.argtypes = [dp, dp, ctypes.c_int, dp, ctypes.c_int,
                                    ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, dp]
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _configure(ctypes.CDLL(build()))
    return _lib


def _dptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a, shape=None):
    if a is None:
        return None
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


def default_threads() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def nbins_of(mode: str, edges_a, edges_b) -> int:
    na = len(edges_a) - 1
    return na if mode == "s" else na * (len(edges_b) - 1)


def count(x1, x2=None, *, w1=None, w2=None, box=None, periodic=False,
          mode="s", los="z", edges_a, edges_b=None, method="brute",
          threads=None, weighted=None, n_leaf=8):
    """Exact pair counts of catalogue x1 (auto) or x1 x x2 (cross).

    Returns (counts int64 [nbins], wcounts float64 [nbins] or None).  The bin
    layout is row-major with the s (or sigma) index outermost.
    ``method`` is "brute" (all pairs), "grid" (cell list, same semantics) or
    "kdtree" (k-d tree of Alg. 1 with leaves of at most ``n_leaf`` points and
    the dual-tree traversal of Alg. 3; one thread).
    """
    lib = _load()
    x1 = _f64(x1, (-1, 3))
    x2 = _f64(x2, (-1, 3)) if x2 is not None else None
    if weighted is None:
        weighted = w1 is not None
    if weighted:
        w1 = _f64(w1, (-1,)) if w1 is not None else np.ones(x1.shape[0])
        if x2 is not None:
            w2 = _f64(w2, (-1,)) if w2 is not None else np.ones(x2.shape[0])
    else:
        w1 = w2 = None
    ea = _f64(edges_a, (-1,))
    eb = _f64(edges_b, (-1,)) if edges_b is not None else np.array([0.0, 1.0])
    L = _f64(box if box is not None else [0.0, 0.0, 0.0], (-1,))
    if L.size == 1:
        L = np.repeat(L, 3)
    nb = nbins_of(mode, ea, eb)
    counts = np.zeros(nb, dtype=np.int64)
    wc = np.zeros(nb, dtype=np.float64) if weighted else None
    if method == "kdtree":
        rc = lib.oracle_count_kdtree(
            _dptr(x1), _dptr(w1), x1.shape[0],
            _dptr(x2), _dptr(w2), 0 if x2 is None else x2.shape[0],
            int(bool(periodic)), _dptr(L), MODES[mode], LOS[los],
            ea.size - 1, _dptr(ea), eb.size - 1, _dptr(eb), int(n_leaf),
            counts.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
            _dptr(wc) if wc is not None else None)
        if rc != 0:
            raise ValueError("oracle_count_kdtree rejected its arguments")
        return counts, wc
    rc = lib.oracle_count(
        _dptr(x1), _dptr(w1), x1.shape[0],
        _dptr(x2), _dptr(w2), 0 if x2 is None else x2.shape[0],
        int(bool(periodic)), _dptr(L), MODES[mode], LOS[los],
        ea.size - 1, _dptr(ea), eb.size - 1, _dptr(eb),
        1 if method == "grid" else 0, int(threads or default_threads()),
        counts.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
        _dptr(wc) if wc is not None else None)
    if rc != 0:
        raise ValueError("oracle_count rejected its arguments")
    return counts, wc


def kdtree(x, *, n_leaf=8, box=None, periodic=False) -> dict:
    """The k-d tree of Alg. 1 over x (canonical coordinates when periodic).

    Heap order (children of slot h: 2h + 1, 2h + 2).  Returns a dict with
    ``depth``, ``start``, ``count`` (-1 in empty slots), ``axis`` (-1 for
    leaves and empty slots), ``box`` ([slots, 6]: lo, hi) and ``ord`` (tree
    position -> point index).
    """
    lib = _load()
    x = _f64(x, (-1, 3))
    n = x.shape[0]
    L = _f64(box if box is not None else [0.0, 0.0, 0.0], (-1,))
    if L.size == 1:
        L = np.repeat(L, 3)
    d, m = 0, n
    while m > n_leaf:
        m = (m + 1) // 2
        d += 1
    slots = (2 << d) - 1
    start = np.zeros(slots, dtype=np.int64)
    count = np.zeros(slots, dtype=np.int64)
    axis = np.zeros(slots, dtype=np.int32)
    bx = np.zeros((slots, 6), dtype=np.float64)
    order = np.zeros(n, dtype=np.int64)
    i64 = ctypes.POINTER(ctypes.c_int64)
    rc = lib.oracle_kdtree(_dptr(x), n, int(bool(periodic)), _dptr(L), int(n_leaf), slots,
                           start.ctypes.data_as(i64), count.ctypes.data_as(i64),
                           axis.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dptr(bx),
                           order.ctypes.data_as(i64))
    if rc < 0:
        raise ValueError("oracle_kdtree rejected its arguments")
    return {"depth": rc, "start": start, "count": count, "axis": axis, "box": bx, "ord": order}


def hist_s2(s2, edges) -> np.ndarray:
    """Histogram of squared separations under the pair definition's rule
    (Sect. 3.2): bin k iff E_k <= s2 < E_{k+1} with E_k = e_k^2 in binary64;
    samples outside [E_0, E_n) are not counted.  numpy's searchsorted finds
    the largest k with E_k <= s2."""
    e = np.asarray(edges, dtype=np.float64)
    E = e * e
    v = np.asarray(s2).astype(np.float64)
    keep = (v >= E[0]) & (v < E[-1])
    k = np.searchsorted(E, v[keep], side="right") - 1
    return np.bincount(k, minlength=e.size - 1).astype(np.int64)


def pair_bin(a, b, *, box=None, periodic=False, mode="s", los="z", edges_a,
             edges_b=None) -> int:
    """Bin of a single pair (a, b); -1 when it falls outside all bins."""
    lib = _load()
    a = _f64(a, (3,))
    b = _f64(b, (3,))
    ea = _f64(edges_a, (-1,))
    eb = _f64(edges_b, (-1,)) if edges_b is not None else np.array([0.0, 1.0])
    L = _f64(box if box is not None else [0.0, 0.0, 0.0], (-1,))
    if L.size == 1:
        L = np.repeat(L, 3)
    r = lib.oracle_pair_bin(_dptr(a), _dptr(b), int(bool(periodic)), _dptr(L),
                            MODES[mode], LOS[los], ea.size - 1, _dptr(ea),
                            eb.size - 1, _dptr(eb))
    if r == -2:
        raise ValueError("oracle_pair_bin rejected its arguments")
    return int(r)
