"""Exact grid pair counting on one GB300 -- Python binding of libpaircount.

This module only marshals arguments into the C ABI declared in
``include/paircount.h`` (ctypes); every step of the computation runs in the
CUDA library.  There is no CPU fallback: if ``libpaircount.so`` has not been
built, every call raises.

Functions keep the ABI's names (``pc_build_grid``, ``pc_count_auto``,
``pc_count_cross``, ``pc_count_batch``, ...).  ``count`` is a convenience
wrapper that builds the grid(s), counts and frees them in one call.

Catalogues may be numpy arrays (host memory; the library copies them) or
torch CUDA tensors (device memory; used in place).  Positions are float64
arrays of shape (N, 3); weights are float64 or float32 arrays of shape (N,).
"""

from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_double, c_float, c_int, c_longlong, c_void_p

import numpy as np

from . import _build

PC_OK, PC_EINVAL, PC_ENOMEM, PC_ECUDA, PC_EOVERFLOW, PC_ETIMEOUT, PC_EUNSUPPORTED = (
    0, -1, -2, -3, -4, -5, -6)
PC_BIN_S, PC_BIN_SMU, PC_BIN_SIGPI = 0, 1, 2
PC_LOS_Z, PC_LOS_MIDPOINT = 0, 1
PC_PREC_F32_RESCUE, PC_PREC_F64 = 0, 1
MODES = {"s": PC_BIN_S, "smu": PC_BIN_SMU, "sigpi": PC_BIN_SIGPI}
LOS = {"z": PC_LOS_Z, "mid": PC_LOS_MIDPOINT}
PRECS = {"f32": PC_PREC_F32_RESCUE, "f64": PC_PREC_F64}


class pc_box(ctypes.Structure):
    _fields_ = [("L", c_double * 3), ("periodic", c_int), ("lo", c_double * 3),
                ("hi", c_double * 3)]


class pc_bins(ctypes.Structure):
    _fields_ = [("mode", c_int), ("los", c_int), ("n_a", c_int), ("edges_a", POINTER(c_double)),
                ("n_b", c_int), ("edges_b", POINTER(c_double))]


class pc_opts(ctypes.Structure):
    _fields_ = [("prec", c_int), ("cell_size", c_double), ("ipt", c_int), ("priv", c_int),
                ("rescue_capacity", c_longlong), ("use_graph", c_int),
                ("grid_ctas_per_sm", c_int), ("shard_index", c_int), ("shard_count", c_int)]


class pc_stats(ctypes.Structure):
    _fields_ = [("candidates", c_longlong), ("rescued", c_longlong),
                ("rescue_inline", c_longlong), ("blocks", c_longlong),
                ("cell_size", c_double), ("ms_total", c_float), ("ms_pairs", c_float),
                ("ms_rescue", c_float), ("launches", c_int),
                ("pruned", c_longlong), ("prec", c_int), ("wsum", c_int),
                ("tree_pairs", c_longlong), ("ms_traverse", c_float)]


class pc_tune_trial(ctypes.Structure):
    _fields_ = [("cell_size", c_double), ("ipt", c_int), ("priv", c_int), ("ms", c_float)]


class PairCountError(RuntimeError):
    def __init__(self, status, where, detail):
        super().__init__(f"{where}: {detail or pc_strerror(status)} (status {status})")
        self.status = status


_lib = None

EXPORTS = ["pc_build_grid", "pc_free_grid", "pc_grid_info", "pc_count_auto", "pc_count_cross",
           "pc_count_batch", "pc_aabb", "pc_suggest_cell_size", "pc_strerror", "pc_last_error",
           "pc_version", "pc_launch_count", "pc_count_auto_noalloc", "pc_tune",
           "pc_build_tree", "pc_free_tree", "pc_tree_info", "pc_tree_export", "pc_count_tree",
           "pc_tune_tree", "pc_hist_s2", "pc_count_tree_batch", "pc_stencil", "pc_fp32_bands",
           "pc_fp32_tables", "pc_fp_peak", "pc_alloc_count", "pc_build_tree_batch"]


def library_path() -> str:
    return _build.LIB


def build(force: bool = False) -> str:
    """Compile libpaircount.so with nvcc (sm_103a)."""
    return _build.build(force=force)


def lib():
    """Load libpaircount.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(
            f"libpaircount.so is missing ({path}); build it first "
            "(python -c 'import __graft_entry__ as g; g.build()')")
    L = ctypes.CDLL(path)
    vp = c_void_p
    L.pc_build_grid.restype = c_int
    L.pc_build_grid.argtypes = [vp, vp, c_int, c_longlong, POINTER(pc_box), c_double,
                                POINTER(pc_opts), vp, POINTER(vp)]
    L.pc_free_grid.restype = None
    L.pc_free_grid.argtypes = [vp]
    L.pc_grid_info.restype = c_int
    L.pc_grid_info.argtypes = [vp, POINTER(c_longlong), POINTER(c_double)]
    L.pc_count_auto.restype = c_int
    L.pc_count_auto.argtypes = [vp, POINTER(pc_bins), POINTER(pc_opts), vp, vp, vp,
                                POINTER(pc_stats)]
    L.pc_count_cross.restype = c_int
    L.pc_count_cross.argtypes = [vp, vp, POINTER(pc_bins), POINTER(pc_opts), vp, vp, vp,
                                 POINTER(pc_stats)]
    L.pc_count_batch.restype = c_int
    L.pc_count_batch.argtypes = [POINTER(vp), c_int, POINTER(pc_bins), POINTER(pc_opts), vp,
                                 vp, vp, POINTER(pc_stats)]
    L.pc_aabb.restype = c_int
    L.pc_aabb.argtypes = [vp, c_longlong, vp, POINTER(c_double), POINTER(c_double)]
    L.pc_suggest_cell_size.restype = c_double
    L.pc_suggest_cell_size.argtypes = [c_longlong, c_double, c_double, c_int]
    L.pc_strerror.restype = ctypes.c_char_p
    L.pc_strerror.argtypes = [c_int]
    L.pc_last_error.restype = ctypes.c_char_p
    L.pc_last_error.argtypes = []
    L.pc_version.restype = ctypes.c_char_p
    L.pc_version.argtypes = []
    L.pc_launch_count.restype = c_longlong
    L.pc_launch_count.argtypes = []
    L.pc_alloc_count.restype = c_longlong
    L.pc_alloc_count.argtypes = []
    L.pc_tune.restype = c_int
    L.pc_tune.argtypes = [vp, vp, c_int, c_longlong, POINTER(pc_box), POINTER(pc_bins),
                          POINTER(pc_opts), vp, POINTER(pc_opts), POINTER(pc_tune_trial), c_int,
                          POINTER(c_int)]
    L.pc_count_auto_noalloc.restype = c_int
    L.pc_count_auto_noalloc.argtypes = [vp, POINTER(pc_bins), POINTER(pc_opts), vp, vp, vp]
    L.pc_build_tree.restype = c_int
    L.pc_build_tree.argtypes = [vp, vp, c_int, c_longlong, POINTER(pc_box), c_int, c_int, vp,
                                POINTER(vp)]
    L.pc_build_tree_batch.restype = c_int
    L.pc_build_tree_batch.argtypes = [POINTER(vp), POINTER(vp), c_int, POINTER(c_longlong), c_int,
                                      POINTER(pc_box), c_int, c_int, vp, POINTER(vp)]
    L.pc_free_tree.restype = None
    L.pc_free_tree.argtypes = [vp]
    L.pc_tree_info.restype = c_int
    L.pc_tree_info.argtypes = [vp, POINTER(c_longlong), POINTER(c_int), POINTER(c_int),
                               POINTER(c_longlong)]
    L.pc_tree_export.restype = c_int
    L.pc_tree_export.argtypes = [vp, vp, vp, vp, vp, vp]
    L.pc_tune_tree.restype = c_int
    L.pc_tune_tree.argtypes = [vp, vp, c_int, c_longlong, POINTER(pc_box), POINTER(pc_bins), c_int,
                               POINTER(pc_opts), vp, POINTER(pc_opts), POINTER(c_int),
                               POINTER(pc_tune_trial), c_int, POINTER(c_int)]
    L.pc_fp_peak.restype = c_int
    L.pc_fp_peak.argtypes = [c_int, c_longlong, vp, POINTER(c_double), POINTER(c_float)]
    L.pc_hist_s2.restype = c_int
    L.pc_hist_s2.argtypes = [vp, c_longlong, c_int, POINTER(c_double), c_int, c_int, c_int, vp, vp,
                             POINTER(c_float)]
    L.pc_stencil.restype = c_int
    L.pc_stencil.argtypes = [POINTER(c_double), c_double, c_int, c_int, POINTER(c_int),
                             POINTER(c_int)]
    L.pc_fp32_bands.restype = c_int
    L.pc_fp32_bands.argtypes = [POINTER(pc_bins), POINTER(c_double), POINTER(c_double),
                                POINTER(c_double), POINTER(c_double), c_int, c_double,
                                POINTER(c_double)]
    L.pc_fp32_tables.restype = c_int
    L.pc_fp32_tables.argtypes = [POINTER(pc_bins), POINTER(c_double), POINTER(c_double),
                                 POINTER(c_double), POINTER(c_double), c_int, c_double,
                                 POINTER(c_float), c_int, POINTER(c_int), POINTER(c_double)]
    L.pc_count_tree_batch.restype = c_int
    L.pc_count_tree_batch.argtypes = [POINTER(vp), c_int, POINTER(pc_bins), POINTER(pc_opts), vp,
                                      vp, vp, POINTER(pc_stats)]
    L.pc_count_tree.restype = c_int
    L.pc_count_tree.argtypes = [vp, vp, POINTER(pc_bins), POINTER(pc_opts), vp, vp, vp,
                                POINTER(pc_stats)]
    _lib = L
    return L


def pc_strerror(status: int) -> str:
    return lib().pc_strerror(int(status)).decode()


def pc_last_error() -> str:
    return lib().pc_last_error().decode()


def pc_version() -> str:
    return lib().pc_version().decode()


def pc_alloc_count() -> int:
    """Device (and pinned host) allocations the library has made so far."""
    return int(lib().pc_alloc_count())


def pc_launch_count() -> int:
    """Kernels launched by the library since it was loaded."""
    return int(lib().pc_launch_count())


def _check(status: int, where: str):
    if status != PC_OK:
        raise PairCountError(status, where, pc_last_error())


# --------------------------------------------------------------------------
# marshalling helpers
# --------------------------------------------------------------------------

def _torch():
    try:
        import torch  # noqa: F401
        return torch
    except Exception:  # pragma: no cover
        return None


def _ptr(a, dtype, shape_last=None):
    """(pointer, keepalive, n) for a numpy array or torch tensor."""
    if a is None:
        return None, None, 0
    t = _torch()
    if t is not None and isinstance(a, t.Tensor):
        want = {np.float64: t.float64, np.float32: t.float32, np.int64: t.int64}[dtype]
        if a.dtype != want:
            raise TypeError(f"expected a {want} tensor, got {a.dtype}")
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        if shape_last is not None and (a.dim() != 2 or a.shape[1] != shape_last):
            raise ValueError(f"expected shape (N, {shape_last})")
        return c_void_p(a.data_ptr()), a, a.shape[0] if a.dim() else 0
    arr = np.ascontiguousarray(np.asarray(a, dtype=dtype))
    if shape_last is not None:
        arr = arr.reshape(-1, shape_last)
    return c_void_p(arr.ctypes.data), arr, arr.shape[0]


def _stream_handle(stream):
    if stream is None:
        t = _torch()
        if t is not None and t.cuda.is_available() and t.cuda.is_initialized():
            return c_void_p(t.cuda.current_stream().cuda_stream)
        return c_void_p(0)
    if isinstance(stream, int):
        return c_void_p(stream)
    return c_void_p(stream.cuda_stream)


def make_box(L=None, periodic=False, lo=None, hi=None) -> pc_box:
    b = pc_box()
    if L is not None:
        Ls = np.broadcast_to(np.asarray(L, dtype=np.float64), (3,))
        for a in range(3):
            b.L[a] = float(Ls[a])
    b.periodic = 1 if periodic else 0
    if lo is not None and hi is not None:
        for a in range(3):
            b.lo[a] = float(lo[a])
            b.hi[a] = float(hi[a])
    return b


class Bins:
    """Histogram description (owns its edge arrays)."""

    def __init__(self, mode="s", los="z", edges_a=None, edges_b=None):
        self.mode = mode
        self.los = los
        self.ea = np.ascontiguousarray(np.asarray(edges_a, dtype=np.float64))
        self.eb = (np.ascontiguousarray(np.asarray(edges_b, dtype=np.float64))
                   if edges_b is not None else np.array([0.0, 1.0]))
        self.s = pc_bins()
        self.s.mode = MODES[mode]
        self.s.los = LOS[los]
        self.s.n_a = self.ea.size - 1
        self.s.edges_a = self.ea.ctypes.data_as(POINTER(c_double))
        self.s.n_b = self.eb.size - 1
        self.s.edges_b = self.eb.ctypes.data_as(POINTER(c_double))

    @property
    def nbins(self) -> int:
        return self.s.n_a * (1 if self.mode == "s" else self.s.n_b)

    @property
    def r_max(self) -> float:
        if self.mode == "sigpi":
            return float(np.hypot(self.ea[-1], self.eb[-1]))
        return float(self.ea[-1])


def make_opts(prec="f32", cell_size=0.0, ipt=0, priv=-1, rescue_capacity=0, use_graph=0,
              grid_ctas_per_sm=0, shard_index=0, shard_count=0) -> pc_opts:
    o = pc_opts()
    o.prec = PRECS[prec] if isinstance(prec, str) else int(prec)
    o.cell_size = float(cell_size)
    o.ipt = int(ipt)
    o.priv = int(priv)
    o.rescue_capacity = int(rescue_capacity)
    o.use_graph = int(use_graph)
    o.grid_ctas_per_sm = int(grid_ctas_per_sm)
    o.shard_index = int(shard_index)
    o.shard_count = int(shard_count)
    return o


class Grid:
    """Owner of a pc_grid handle (freed with the object)."""

    def __init__(self, handle, n):
        self.handle = handle
        self.n = n

    @property
    def cell_size(self) -> float:
        n = c_longlong()
        c = c_double()
        _check(lib().pc_grid_info(self.handle, ctypes.byref(n), ctypes.byref(c)), "pc_grid_info")
        return c.value

    def free(self):
        if self.handle:
            lib().pc_free_grid(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


# --------------------------------------------------------------------------
# the ABI, one Python function per entry point
# --------------------------------------------------------------------------

def pc_build_grid(xyz, w=None, *, box: pc_box, r_max: float, opts: pc_opts | None = None,
                  stream=None) -> Grid:
    px, keep_x, n = _ptr(xyz, np.float64, 3)
    w_is_f32 = 0
    pw, keep_w = None, None
    if w is not None:
        t = _torch()
        is32 = (getattr(w, "dtype", None) == np.float32 or
                (t is not None and isinstance(w, t.Tensor) and w.dtype == t.float32))
        w_is_f32 = 1 if is32 else 0
        pw, keep_w, nw = _ptr(w, np.float32 if is32 else np.float64)
        if nw != n:
            raise ValueError("weights and positions differ in length")
    out = c_void_p()
    st = _check(lib().pc_build_grid(px, pw, w_is_f32, n, ctypes.byref(box), float(r_max),
                                    ctypes.byref(opts) if opts is not None else None,
                                    _stream_handle(stream), ctypes.byref(out)), "pc_build_grid")
    del st, keep_x, keep_w
    return Grid(out, n)


def pc_tune(xyz, w=None, *, box: pc_box, bins: Bins, opts: pc_opts | None = None, stream=None,
            max_trials: int = 32):
    """Measured autotuning of cell side, i-points per thread and histogram
    privatisation; returns (tuned pc_opts, list of (cell_size, ipt, priv, ms))."""
    px, keep_x, n = _ptr(xyz, np.float64, 3)
    w_is_f32 = 0
    pw, keep_w = None, None
    if w is not None:
        t = _torch()
        is32 = (getattr(w, "dtype", None) == np.float32 or
                (t is not None and isinstance(w, t.Tensor) and w.dtype == t.float32))
        w_is_f32 = 1 if is32 else 0
        pw, keep_w, nw = _ptr(w, np.float32 if is32 else np.float64)
        if nw != n:
            raise ValueError("weights and positions differ in length")
    out = pc_opts()
    trials = (pc_tune_trial * max_trials)()
    nt = c_int(0)
    _check(lib().pc_tune(px, pw, w_is_f32, n, ctypes.byref(box), ctypes.byref(bins.s),
                         ctypes.byref(opts) if opts is not None else None, _stream_handle(stream),
                         ctypes.byref(out), trials, max_trials, ctypes.byref(nt)), "pc_tune")
    del keep_x, keep_w
    return out, [(t.cell_size, t.ipt, t.priv, t.ms) for t in trials[:nt.value]]


def pc_free_grid(g: Grid):
    g.free()


def pc_grid_info(g: Grid):
    """(number of points, cell side) of a grid."""
    n = c_longlong()
    c = c_double()
    _check(lib().pc_grid_info(g.handle, ctypes.byref(n), ctypes.byref(c)), "pc_grid_info")
    return n.value, c.value


def _outputs(counts, wcounts, rows, nbins, weighted):
    if counts is None:
        counts = np.zeros(rows * nbins, dtype=np.int64)
    if weighted and wcounts is None:
        wcounts = np.zeros(rows * nbins, dtype=np.float64)
    pc_, kc, _ = _ptr(counts, np.int64)
    pw_, kw, _ = _ptr(wcounts, np.float64) if wcounts is not None else (None, None, 0)
    return counts, wcounts, pc_, pw_, (kc, kw)


def pc_count_auto(g: Grid, bins: Bins, opts: pc_opts | None = None, stream=None, counts=None,
                  wcounts=None, weighted=False):
    counts, wcounts, pc_, pw_, keep = _outputs(counts, wcounts, 1, bins.nbins, weighted)
    st = pc_stats()
    _check(lib().pc_count_auto(g.handle, ctypes.byref(bins.s),
                               ctypes.byref(opts) if opts is not None else None,
                               _stream_handle(stream), pc_, pw_, ctypes.byref(st)),
           "pc_count_auto")
    del keep
    return counts, wcounts, st


def pc_count_auto_noalloc(g: Grid, bins: Bins, opts: pc_opts | None = None, stream=None,
                          counts=None, wcounts=None, weighted=False):
    """Auto counts without any device allocation inside the call (all
    temporaries live in a fixed array inside the library).  Pass device
    tensors for counts/wcounts to keep the whole call allocation-free."""
    counts, wcounts, pc_, pw_, keep = _outputs(counts, wcounts, 1, bins.nbins, weighted)
    _check(lib().pc_count_auto_noalloc(g.handle, ctypes.byref(bins.s),
                                       ctypes.byref(opts) if opts is not None else None,
                                       _stream_handle(stream), pc_, pw_),
           "pc_count_auto_noalloc")
    del keep
    return counts, wcounts


def pc_count_cross(g1: Grid, g2: Grid, bins: Bins, opts: pc_opts | None = None, stream=None,
                   counts=None, wcounts=None, weighted=False):
    counts, wcounts, pc_, pw_, keep = _outputs(counts, wcounts, 1, bins.nbins, weighted)
    st = pc_stats()
    _check(lib().pc_count_cross(g1.handle, g2.handle, ctypes.byref(bins.s),
                                ctypes.byref(opts) if opts is not None else None,
                                _stream_handle(stream), pc_, pw_, ctypes.byref(st)),
           "pc_count_cross")
    del keep
    return counts, wcounts, st


def pc_count_batch(grids, bins: Bins, opts: pc_opts | None = None, stream=None, counts=None,
                   wcounts=None, weighted=False):
    m = len(grids)
    counts, wcounts, pc_, pw_, keep = _outputs(counts, wcounts, m, bins.nbins, weighted)
    arr = (c_void_p * m)(*[g.handle for g in grids])
    st = pc_stats()
    _check(lib().pc_count_batch(arr, m, ctypes.byref(bins.s),
                                ctypes.byref(opts) if opts is not None else None,
                                _stream_handle(stream), pc_, pw_, ctypes.byref(st)),
           "pc_count_batch")
    del keep
    return counts, wcounts, st


class Tree:
    """Owner of a pc_tree handle (freed with the object)."""

    def __init__(self, handle, n):
        self.handle = handle
        self.n = n

    def info(self):
        """(points, depth, list level, heap slots)."""
        return pc_tree_info(self)

    def free(self):
        if self.handle:
            lib().pc_free_tree(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def _weights_arg(w, n):
    if w is None:
        return None, None, 0
    t = _torch()
    is32 = (getattr(w, "dtype", None) == np.float32 or
            (t is not None and isinstance(w, t.Tensor) and w.dtype == t.float32))
    pw, keep_w, nw = _ptr(w, np.float32 if is32 else np.float64)
    if nw != n:
        raise ValueError("weights and positions differ in length")
    return pw, keep_w, 1 if is32 else 0


def pc_build_tree(xyz, w=None, *, box: pc_box, n_leaf: int = 32, list_cap: int = 0,
                  stream=None) -> Tree:
    """k-d tree of Alg. 1 built on the GPU (see paircount.h)."""
    px, keep_x, n = _ptr(xyz, np.float64, 3)
    pw, keep_w, w_is_f32 = _weights_arg(w, n)
    out = c_void_p()
    _check(lib().pc_build_tree(px, pw, w_is_f32, n, ctypes.byref(box), int(n_leaf),
                               int(list_cap), _stream_handle(stream), ctypes.byref(out)),
           "pc_build_tree")
    del keep_x, keep_w
    return Tree(out, n)


def pc_build_tree_batch(xyzs, ws=None, *, box: pc_box, n_leaf: int = 32, list_cap: int = 0,
                        stream=None) -> list:
    """The k-d trees of many catalogues built in one level loop (see
    paircount.h); returns one Tree per catalogue, in order."""
    m = len(xyzs)
    if m == 0:
        return []
    px, keep, ns = [], [], []
    for x in xyzs:
        p, k, n = _ptr(x, np.float64, 3)
        px.append(p)
        keep.append(k)
        ns.append(n)
    pw, w_is_f32 = None, 0
    if ws is not None:
        if len(ws) != m:
            raise ValueError("one weight array per catalogue")
        pw = []
        flags = set()
        for w, n in zip(ws, ns):
            p, k, f = _weights_arg(w, n)
            pw.append(p)
            keep.append(k)
            flags.add(f)
        if len(flags) != 1:
            raise ValueError("weights must be all binary32 or all binary64")
        w_is_f32 = flags.pop()
        pw = (c_void_p * m)(*pw)
    out = (c_void_p * m)()
    _check(lib().pc_build_tree_batch((c_void_p * m)(*px), pw, w_is_f32, (c_longlong * m)(*ns), m,
                                     ctypes.byref(box), int(n_leaf), int(list_cap),
                                     _stream_handle(stream), out), "pc_build_tree_batch")
    del keep
    return [Tree(c_void_p(out[k]), ns[k]) for k in range(m)]


def pc_tune_tree(xyz, w=None, *, box: pc_box, bins: Bins, n_leaf: int = 32,
                 opts: pc_opts | None = None, stream=None, max_trials: int = 16):
    """Measured list level and i-points per thread of the tree path; returns
    (pc_opts with ipt, list_cap, list of (list_cap, ipt, ms))."""
    px, keep_x, n = _ptr(xyz, np.float64, 3)
    pw, keep_w, w_is_f32 = _weights_arg(w, n)
    out = pc_opts()
    cap = c_int(0)
    trials = (pc_tune_trial * max_trials)()
    nt = c_int(0)
    _check(lib().pc_tune_tree(px, pw, w_is_f32, n, ctypes.byref(box), ctypes.byref(bins.s),
                              int(n_leaf), ctypes.byref(opts) if opts is not None else None,
                              _stream_handle(stream), ctypes.byref(out), ctypes.byref(cap), trials,
                              max_trials, ctypes.byref(nt)), "pc_tune_tree")
    del keep_x, keep_w
    return out, cap.value, [(int(t.cell_size), t.ipt, t.ms) for t in trials[:nt.value]]


HIST_METHODS = {"bsearch": 0, "reverse": 1, "map_lin": 2, "map_log": 3, "lut": 4}


def pc_hist_s2(s2, edges, method="lut", table_size=0, repeat=1, stream=None, counts=None):
    """Histogram-update micro-benchmark (see paircount.h); returns (counts, ms)."""
    ps, keep, n = _ptr(s2, np.float32)
    e = np.ascontiguousarray(np.asarray(edges, dtype=np.float64))
    nb = e.size - 1
    if counts is None:
        counts = np.zeros(nb, dtype=np.int64)
    pc_, kc, _ = _ptr(counts, np.int64)
    ms = c_float(0.0)
    m = HIST_METHODS[method] if isinstance(method, str) else int(method)
    _check(lib().pc_hist_s2(ps, n, int(repeat), e.ctypes.data_as(POINTER(c_double)), nb, m,
                            int(table_size), _stream_handle(stream), pc_, ctypes.byref(ms)),
           "pc_hist_s2")
    del keep, kc
    return counts, ms.value


PEAK_KINDS = {"ffma": 0, "ffma2": 1, "dfma": 2}


def pc_fp_peak(kind="ffma", iters=0, stream=None):
    """Measured FMA throughput of the current device (see paircount.h).
    Returns (TFLOP/s, ms of the timed launch)."""
    tf = c_double(0.0)
    ms = c_float(0.0)
    k = PEAK_KINDS[kind] if isinstance(kind, str) else int(kind)
    _check(lib().pc_fp_peak(k, int(iters), _stream_handle(stream), ctypes.byref(tf),
                            ctypes.byref(ms)), "pc_fp_peak")
    return tf.value, ms.value


def pc_free_tree(t: Tree):
    t.free()


def pc_tree_info(t: Tree):
    n = c_longlong()
    d = c_int()
    b = c_int()
    s = c_longlong()
    _check(lib().pc_tree_info(t.handle, ctypes.byref(n), ctypes.byref(d), ctypes.byref(b),
                              ctypes.byref(s)), "pc_tree_info")
    return n.value, d.value, b.value, s.value


def pc_tree_export(t: Tree) -> dict:
    """Tree structure in heap order: start, count (-1: empty slot), axis
    (-1: leaf or empty), box [slots, 6] and ord (tree position -> index)."""
    n, depth, blevel, slots = pc_tree_info(t)
    start = np.zeros(slots, dtype=np.int64)
    count = np.zeros(slots, dtype=np.int64)
    axis = np.zeros(slots, dtype=np.int32)
    bx = np.zeros((slots, 6), dtype=np.float64)
    order = np.zeros(n, dtype=np.int64)
    _check(lib().pc_tree_export(t.handle, start.ctypes.data, count.ctypes.data, axis.ctypes.data,
                                bx.ctypes.data, order.ctypes.data), "pc_tree_export")
    return {"depth": depth, "list_level": blevel, "start": start, "count": count,
            "axis": axis, "box": bx, "ord": order}


def pc_count_tree(t1: Tree, t2, bins: Bins, opts: pc_opts | None = None, stream=None,
                  counts=None, wcounts=None, weighted=False):
    """Auto (t2 None) or cross counts through the dual-tree traversal."""
    counts, wcounts, pc_, pw_, keep = _outputs(counts, wcounts, 1, bins.nbins, weighted)
    st = pc_stats()
    _check(lib().pc_count_tree(t1.handle, t2.handle if t2 is not None else None,
                               ctypes.byref(bins.s),
                               ctypes.byref(opts) if opts is not None else None,
                               _stream_handle(stream), pc_, pw_, ctypes.byref(st)),
           "pc_count_tree")
    del keep
    return counts, wcounts, st


def pc_count_tree_batch(trees, bins: Bins, opts: pc_opts | None = None, stream=None,
                        counts=None, wcounts=None, weighted=False):
    """Auto counts of several trees in one pair-kernel launch (row k: tree k)."""
    m = len(trees)
    counts, wcounts, pc_, pw_, keep = _outputs(counts, wcounts, m, bins.nbins, weighted)
    arr = (c_void_p * m)(*[t.handle for t in trees])
    st = pc_stats()
    _check(lib().pc_count_tree_batch(arr, m, ctypes.byref(bins.s),
                                     ctypes.byref(opts) if opts is not None else None,
                                     _stream_handle(stream), pc_, pw_, ctypes.byref(st)),
           "pc_count_tree_batch")
    del keep
    return counts, wcounts, st


def pc_aabb(xyz, stream=None):
    px, keep, n = _ptr(xyz, np.float64, 3)
    lo = (c_double * 3)()
    hi = (c_double * 3)()
    _check(lib().pc_aabb(px, n, _stream_handle(stream), lo, hi), "pc_aabb")
    del keep
    return np.array(lo[:]), np.array(hi[:])


def pc_stencil(cell, r_max: float, half: bool = False) -> np.ndarray:
    """Stencil rows {dy, dz, xlo, xhi} of the grid path (host-only)."""
    c = (c_double * 3)(*np.broadcast_to(np.asarray(cell, dtype=np.float64), (3,)))
    nr = c_int(0)
    lib().pc_stencil(c, float(r_max), int(bool(half)), 0, None, ctypes.byref(nr))
    rows = np.zeros((max(nr.value, 1), 4), dtype=np.int32)
    _check(lib().pc_stencil(c, float(r_max), int(bool(half)), nr.value,
                            rows.ctypes.data_as(POINTER(c_int)), ctypes.byref(nr)), "pc_stencil")
    return rows[:nr.value]


def pc_fp32_bands(bins: "Bins", cell, lo, hi, L=None, periodic: bool = False,
                  rmin: float = 0.0) -> dict:
    """The FP32 path's error bands and bin decisions for a count (host-only)."""
    def v3(a):
        return (c_double * 3)(*np.broadcast_to(np.asarray(a, dtype=np.float64), (3,)))
    out = (c_double * 19)()
    _check(lib().pc_fp32_bands(ctypes.byref(bins.s), v3(cell), v3(lo), v3(hi),
                               v3(L) if L is not None else None, int(bool(periodic)),
                               float(rmin), out), "pc_fp32_bands")
    keys = ("eps_a", "eps_b", "mu_A", "mu_B", "rcut", "fp32_ok", "lin", "r2cut",
            "lin_invA", "lin_offA", "lin_thrA", "lin_nB", "lin_mA", "lin_cB", "lin_norange",
            "lin_log", "lin_invB", "lin_thrB", "lin_mS")
    return dict(zip(keys, (float(v) for v in out)))


def pc_fp32_tables(bins: "Bins", cell, lo, hi, L=None, periodic: bool = False,
                   rmin: float = 0.0):
    """The FP32 path's lookup tables for a count (host-only): (entries as a
    float32 array of shape (n, 2), descriptor dict)."""
    def v3(a):
        return (c_double * 3)(*np.broadcast_to(np.asarray(a, dtype=np.float64), (3,)))
    args = (ctypes.byref(bins.s), v3(cell), v3(lo), v3(hi),
            v3(L) if L is not None else None, int(bool(periodic)), float(rmin))
    n = c_int(0)
    desc = (c_double * 7)()
    lib().pc_fp32_tables(*args, None, 0, ctypes.byref(n), desc)
    lut = np.zeros((max(n.value, 1), 2), dtype=np.float32)
    _check(lib().pc_fp32_tables(*args, lut.ctypes.data_as(POINTER(c_float)), n.value,
                                ctypes.byref(n), desc), "pc_fp32_tables")
    keys = ("a_off", "a_T", "a_inv", "b_off", "b_T", "b_inv", "mu_W")
    return lut[:n.value], dict(zip(keys, (float(v) for v in desc)))


def pc_suggest_cell_size(n: int, volume: float, r_max: float, mode: int = 0) -> float:
    return float(lib().pc_suggest_cell_size(int(n), float(volume), float(r_max), int(mode)))


# --------------------------------------------------------------------------
# convenience: build, count, free
# --------------------------------------------------------------------------

def count(x1, x2=None, *, w1=None, w2=None, box=None, periodic=False, mode="s", los="z",
          edges_a, edges_b=None, prec="f32", cell_size=0.0, ipt=0, priv=-1,
          rescue_capacity=0, weighted=None, stream=None, return_stats=False):
    """Auto (x2 None) or cross pair counts through the C ABI.

    Returns (counts, wcounts) like the oracle's ``count`` (wcounts None when
    unweighted), plus the pc_stats struct when return_stats is true.
    """
    bins = Bins(mode, los, edges_a, edges_b)
    if weighted is None:
        weighted = w1 is not None
    opts = make_opts(prec, cell_size, ipt, priv, rescue_capacity)
    if periodic:
        b = make_box(box, True)
    elif x2 is not None:
        lo1, hi1 = pc_aabb(x1, stream)
        lo2, hi2 = pc_aabb(x2, stream)
        lo, hi = np.minimum(lo1, lo2), np.maximum(hi1, hi2)
        hi = np.where(hi > lo, hi, lo + 1e-9 * (np.abs(lo) + 1.0))
        b = make_box(None, False, lo, hi)
    else:
        b = make_box(None, False)
    g1 = pc_build_grid(x1, w1 if weighted else None, box=b, r_max=bins.r_max, opts=opts,
                       stream=stream)
    try:
        if x2 is None:
            c, wc, st = pc_count_auto(g1, bins, opts, stream, weighted=weighted)
        else:
            g2 = pc_build_grid(x2, w2 if weighted else None, box=b, r_max=bins.r_max,
                               opts=make_opts(prec, g1.cell_size, ipt, priv, rescue_capacity),
                               stream=stream)
            try:
                c, wc, st = pc_count_cross(g1, g2, bins, opts, stream, weighted=weighted)
            finally:
                g2.free()
    finally:
        g1.free()
    if return_stats:
        return c, wc, st
    return c, wc


def count_tree(x1, x2=None, *, w1=None, w2=None, box=None, periodic=False, mode="s", los="z",
               edges_a, edges_b=None, n_leaf=32, list_cap=0, ipt=2, priv=-1, rescue_capacity=0,
               weighted=None, stream=None, return_stats=False):
    """Auto (x2 None) or cross pair counts through the k-d tree path (build
    the trees, count, free); same results as ``count``."""
    bins = Bins(mode, los, edges_a, edges_b)
    if weighted is None:
        weighted = w1 is not None
    opts = make_opts("f32", 0.0, ipt, priv, rescue_capacity)
    b = make_box(box, True) if periodic else make_box(None, False)
    t1 = pc_build_tree(x1, w1 if weighted else None, box=b, n_leaf=n_leaf, list_cap=list_cap,
                       stream=stream)
    try:
        if x2 is None:
            c, wc, st = pc_count_tree(t1, None, bins, opts, stream, weighted=weighted)
        else:
            t2 = pc_build_tree(x2, w2 if weighted else None, box=b, n_leaf=n_leaf,
                               list_cap=list_cap, stream=stream)
            try:
                c, wc, st = pc_count_tree(t1, t2, bins, opts, stream, weighted=weighted)
            finally:
                t2.free()
    finally:
        t1.free()
    if return_stats:
        return c, wc, st
    return c, wc
