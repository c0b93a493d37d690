"""CPU-side checks of the C ABI: the library builds, loads, exports every
entry point declared in include/paircount.h, the binding's structs, enums and
argument lists match the header, and bad arguments are rejected on the host
(no kernel is launched here)."""

import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import paper_2301_12557_gb300 as P

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    P.build()
    return P.lib()


def _declared():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            names += re.findall(r"^\s*(?:[\w\s\*]+?)\b(pc_\w+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "pc_build_grid" in names and "pc_count_batch" in names
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) <= set(P.EXPORTS) | set(names)


def test_binding_covers_the_abi():
    for n in _declared():
        assert hasattr(P, n), f"binding lacks {n}"


def test_status_strings_and_version(lib):
    assert P.pc_strerror(P.PC_OK) == "success"
    assert P.pc_strerror(P.PC_EINVAL) == "invalid argument"
    assert "sm_103a" in P.pc_version()


def test_host_side_argument_checks(lib):
    box = P.make_box(100.0, True)
    out = ctypes.c_void_p()
    # NULL out pointer, negative n, bad r_max: rejected before any CUDA call
    assert lib.pc_build_grid(None, None, 0, 10, ctypes.byref(box), 10.0, None, None, None) == P.PC_EINVAL
    assert lib.pc_build_grid(None, None, 0, -1, ctypes.byref(box), 10.0, None, None,
                             ctypes.byref(out)) == P.PC_EINVAL
    assert "n < 0" in P.pc_last_error()
    x = np.zeros((4, 3))
    assert lib.pc_build_grid(x.ctypes.data, None, 0, 4, ctypes.byref(box), -1.0, None, None,
                             ctypes.byref(out)) == P.PC_EINVAL
    assert lib.pc_build_grid(x.ctypes.data, None, 0, 1 << 31, ctypes.byref(box), 1.0, None,
                             None, ctypes.byref(out)) == P.PC_EOVERFLOW
    b = P.Bins("s", "z", [0.0, 1.0])
    assert lib.pc_count_auto(None, ctypes.byref(b.s), None, None, None, None, None) == P.PC_EINVAL
    assert lib.pc_count_cross(None, None, ctypes.byref(b.s), None, None, None, None, None) == P.PC_EINVAL
    assert lib.pc_count_batch(None, 0, ctypes.byref(b.s), None, None, None, None, None) == P.PC_EINVAL


def test_cost_model_cell_size(lib):
    R = 200.0
    c_dense = P.pc_suggest_cell_size(100_000_000, 3000.0 ** 3, R)
    c_mid = P.pc_suggest_cell_size(2_000_000, 1000.0 ** 3, R)
    c_sparse = P.pc_suggest_cell_size(20_000, 1000.0 ** 3, R)
    for c in (c_dense, c_mid, c_sparse):
        assert R / 16 <= c <= 2 * R
    # denser catalogues favour smaller cells (Appendix B.1: the N_pair term grows)
    assert c_dense <= c_mid <= c_sparse


def test_bins_helper():
    b = P.Bins("sigpi", "mid", np.linspace(0, 30, 4), np.linspace(0, 40, 5))
    assert b.nbins == 12
    assert abs(b.r_max - 50.0) < 1e-12
    b = P.Bins("smu", "z", [0, 1, 2], [0, 0.5, 1])
    assert b.nbins == 4
    assert b.s.n_a == 2 and b.s.n_b == 2


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(P, "_lib", None)
    monkeypatch.setattr(P._build, "LIB", str(tmp_path / "nope.so"))
    with pytest.raises(RuntimeError):
        P.lib()


def test_tune_host_side_checks(lib):
    box = P.make_box(100.0, True)
    bins = P.Bins("s", "z", np.linspace(0.0, 20.0, 5))
    out = P.pc_opts()
    x = np.zeros((1, 3))
    # missing output / bad trial array: rejected before any CUDA call
    assert lib.pc_tune(x.ctypes.data, None, 0, 1, ctypes.byref(box), ctypes.byref(bins.s), None,
                       None, None, None, 0, None) == P.PC_EINVAL
    assert lib.pc_tune(x.ctypes.data, None, 0, 1, ctypes.byref(box), ctypes.byref(bins.s), None,
                       None, ctypes.byref(out), None, 4, None) == P.PC_EINVAL
    # fewer than two points: nothing to time, the cost model's cell side is returned
    nt = ctypes.c_int(-1)
    assert lib.pc_tune(x.ctypes.data, None, 0, 1, ctypes.byref(box), ctypes.byref(bins.s), None,
                       None, ctypes.byref(out), None, 0, ctypes.byref(nt)) == P.PC_OK
    assert nt.value == 0 and out.ipt == 2
    assert out.cell_size == pytest.approx(P.pc_suggest_cell_size(1, 1e6, 20.0, 0))


def test_tree_batch_host_side_checks(lib):
    # no catalogues, no output array, an empty catalogue, weights for one
    # catalogue only, bad leaf capacity: rejected before any CUDA call
    box = P.make_box(100.0, True)
    x = np.zeros((4, 3))
    xs = (ctypes.c_void_p * 2)(x.ctypes.data, x.ctypes.data)
    out = (ctypes.c_void_p * 2)()
    ns = (ctypes.c_longlong * 2)(4, 4)
    assert lib.pc_build_tree_batch(xs, None, 0, ns, 0, ctypes.byref(box), 8, 0, None, out) == P.PC_EINVAL
    assert lib.pc_build_tree_batch(xs, None, 0, ns, 2, ctypes.byref(box), 8, 0, None, None) == P.PC_EINVAL
    n0 = (ctypes.c_longlong * 2)(4, 0)
    assert lib.pc_build_tree_batch(xs, None, 0, n0, 2, ctypes.byref(box), 8, 0, None, out) == P.PC_EINVAL
    w = np.ones(4)
    ws = (ctypes.c_void_p * 2)(w.ctypes.data, None)
    assert lib.pc_build_tree_batch(xs, ws, 0, ns, 2, ctypes.byref(box), 8, 0, None, out) == P.PC_EINVAL
    assert lib.pc_build_tree_batch(xs, None, 0, ns, 2, ctypes.byref(box), 0, 0, None, out) == P.PC_EINVAL
    assert out[0] is None and out[1] is None


def test_fp_peak_host_side_checks(lib):
    # bad kind, negative iterations or no output: rejected before any CUDA call
    tf = ctypes.c_double(0.0)
    assert lib.pc_fp_peak(3, 0, None, ctypes.byref(tf), None) == P.PC_EINVAL
    assert lib.pc_fp_peak(-1, 0, None, ctypes.byref(tf), None) == P.PC_EINVAL
    assert lib.pc_fp_peak(0, -5, None, ctypes.byref(tf), None) == P.PC_EINVAL
    assert lib.pc_fp_peak(0, 0, None, None, None) == P.PC_EINVAL


def test_tree_and_hist_host_side_checks(lib):
    box = P.make_box(100.0, True)
    out = ctypes.c_void_p()
    x = np.zeros((4, 3))
    # k-d tree build: NULL out, no points, bad leaf capacity or list capacity,
    # too many points -- all rejected before any CUDA call
    assert lib.pc_build_tree(x.ctypes.data, None, 0, 4, ctypes.byref(box), 8, 0, None,
                             None) == P.PC_EINVAL
    assert lib.pc_build_tree(x.ctypes.data, None, 0, 0, ctypes.byref(box), 8, 0, None,
                             ctypes.byref(out)) == P.PC_EINVAL
    assert lib.pc_build_tree(x.ctypes.data, None, 0, 4, ctypes.byref(box), 0, 0, None,
                             ctypes.byref(out)) == P.PC_EINVAL
    assert lib.pc_build_tree(x.ctypes.data, None, 0, 4, ctypes.byref(box), 129, 0, None,
                             ctypes.byref(out)) == P.PC_EINVAL
    assert lib.pc_build_tree(x.ctypes.data, None, 0, 4, ctypes.byref(box), 8, 300, None,
                             ctypes.byref(out)) == P.PC_EINVAL
    assert lib.pc_build_tree(x.ctypes.data, None, 0, 1 << 31, ctypes.byref(box), 8, 0, None,
                             ctypes.byref(out)) == P.PC_EOVERFLOW
    b = P.Bins("s", "z", [0.0, 1.0])
    assert lib.pc_count_tree(None, None, ctypes.byref(b.s), None, None, None, None,
                             None) == P.PC_EINVAL
    opts = P.pc_opts()
    cap = ctypes.c_int()
    assert lib.pc_tune_tree(x.ctypes.data, None, 0, 4, None, ctypes.byref(b.s), 8, None, None,
                            ctypes.byref(opts), ctypes.byref(cap), None, 0, None) == P.PC_EINVAL
    # histogram micro-benchmark: bad sizes, edges, methods and table sizes
    s2 = np.ones(8, dtype=np.float32)
    e = np.array([0.0, 1.0, 2.0])
    cnt = np.zeros(2, dtype=np.int64)
    ep = e.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    assert lib.pc_hist_s2(s2.ctypes.data, -1, 1, ep, 2, 0, 0, None, cnt.ctypes.data,
                          None) == P.PC_EINVAL
    assert lib.pc_hist_s2(s2.ctypes.data, 8, 0, ep, 2, 0, 0, None, cnt.ctypes.data,
                          None) == P.PC_EINVAL
    assert lib.pc_hist_s2(s2.ctypes.data, 8, 1, ep, 2, 7, 0, None, cnt.ctypes.data,
                          None) == P.PC_EINVAL
    assert lib.pc_hist_s2(s2.ctypes.data, 8, 1, ep, 2, 4, 0, None, cnt.ctypes.data,
                          None) == P.PC_EINVAL
    assert lib.pc_hist_s2(s2.ctypes.data, 8, 1, ep, 2, 3, 0, None, cnt.ctypes.data,
                          None) == P.PC_EINVAL      # log mapping with e[0] = 0
    bad = np.array([0.0, 2.0, 1.0])
    assert lib.pc_hist_s2(s2.ctypes.data, 8, 1, bad.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                          2, 0, 0, None, cnt.ctypes.data, None) == P.PC_EINVAL


def _c_layout(tmp_path):
    """sizeof/offsetof of every header struct and the enum values, as a C
    compiler lays them out from include/paircount.h."""
    structs = {"pc_box": P.pc_box, "pc_bins": P.pc_bins, "pc_opts": P.pc_opts,
               "pc_stats": P.pc_stats, "pc_tune_trial": P.pc_tune_trial}
    enums = ["PC_OK", "PC_EINVAL", "PC_ENOMEM", "PC_ECUDA", "PC_EOVERFLOW", "PC_ETIMEOUT",
             "PC_EUNSUPPORTED", "PC_BIN_S", "PC_BIN_SMU", "PC_BIN_SIGPI", "PC_LOS_Z",
             "PC_LOS_MIDPOINT", "PC_PREC_F32_RESCUE", "PC_PREC_F64"]
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "paircount.h"',
             "int main(void) {"]
    for s, cls in structs.items():
        lines.append(f'printf("{s} size %zu\\n", sizeof({s}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{s}.{f} off %zu size %zu\\n", offsetof({s}, {f}), '
                         f'sizeof((({s} *)0)->{f}));')
    for e in enums:
        lines.append(f'printf("{e} val %d\\n", (int){e});')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    "-o", str(exe), str(src)], check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    got = {}
    for ln in out.splitlines():
        parts = ln.split()
        got[parts[0]] = [int(v) for v in parts[2::2]]
    return structs, enums, got


def test_binding_structs_and_enums_match_the_header(tmp_path):
    """The ctypes mirrors of the header's structs have the C layout (size and
    every field's offset and size), and the Python constants the header's
    enum values; a field added to one side only fails here."""
    structs, enums, got = _c_layout(tmp_path)
    for s, cls in structs.items():
        assert got[s] == [ctypes.sizeof(cls)], s
        for f, _ in cls._fields_:
            fld = getattr(cls, f)
            assert got[f"{s}.{f}"] == [fld.offset, fld.size], (s, f)
    for e in enums:
        assert got[e] == [getattr(P, e)], e


def test_binding_argument_counts_match_the_prototypes(lib):
    """Every prototype in the header takes as many parameters as the
    binding's ctypes argtypes declare."""
    txt = open(os.path.join(ROOT, "include", "paircount.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    protos = re.findall(r"^[\w \*]*?\b(pc_\w+)\s*\(([^;{]*?)\)\s*;", txt, flags=re.M | re.S)
    assert len(protos) >= len(P.EXPORTS)
    for name, params in protos:
        params = params.strip()
        n = 0 if params in ("", "void") else params.count(",") + 1
        assert len(getattr(lib, name).argtypes) == n, name


def test_host_only_views_check_their_arguments(lib):
    b = P.Bins("smu", "z", np.linspace(0.0, 40.0, 11), np.linspace(0.0, 1.0, 6))
    out = (ctypes.c_double * 19)()
    v3 = lambda *a: (ctypes.c_double * 3)(*a)   # noqa: E731
    ok = lib.pc_fp32_bands(ctypes.byref(b.s), v3(10, 10, 10), v3(0, 0, 0), v3(100, 100, 100),
                           v3(100, 100, 100), 1, 0.0, out)
    assert ok == P.PC_OK and out[0] > 0 and out[4] > 40.0
    assert lib.pc_fp32_bands(None, v3(10, 10, 10), v3(0, 0, 0), v3(1, 1, 1), None, 0, 0.0,
                             out) == P.PC_EINVAL
    assert lib.pc_fp32_bands(ctypes.byref(b.s), v3(0, 10, 10), v3(0, 0, 0), v3(1, 1, 1), None, 0,
                             0.0, out) == P.PC_EINVAL
    assert lib.pc_fp32_bands(ctypes.byref(b.s), v3(10, 10, 10), v3(0, 0, 0), v3(1, 1, 1), None,
                             1, 0.0, out) == P.PC_EINVAL          # periodic without a box
    bad = P.Bins("smu", "z", [0.0, 2.0, 1.0], [0.0, 1.0])
    assert lib.pc_fp32_bands(ctypes.byref(bad.s), v3(10, 10, 10), v3(0, 0, 0), v3(1, 1, 1), None,
                             0, 0.0, out) == P.PC_EINVAL
    n = ctypes.c_int(0)
    desc = (ctypes.c_double * 7)()
    assert lib.pc_fp32_tables(ctypes.byref(b.s), v3(10, 10, 10), v3(0, 0, 0), v3(100, 100, 100),
                              v3(100, 100, 100), 1, 0.0, None, 0, ctypes.byref(n),
                              desc) == P.PC_EOVERFLOW
    assert n.value > 0
    lut, d = P.pc_fp32_tables(b, 10.0, np.zeros(3), np.full(3, 100.0), 100.0, True)
    assert lut.shape == (n.value, 2) and d["a_T"] >= 16
    # a periodic separation of half the box is refused, as by the counts
    b2 = P.Bins("s", "z", [0.0, 50.0])
    assert lib.pc_fp32_bands(ctypes.byref(b2.s), v3(10, 10, 10), v3(0, 0, 0), v3(100, 100, 100),
                             v3(100, 100, 100), 1, 0.0, out) == P.PC_EINVAL


def test_header_compiles_as_c_and_cxx(tmp_path):
    """include/paircount.h stands alone in C99 and in C++17 (extern "C")."""
    src = tmp_path / "use.c"
    src.write_text('#include "paircount.h"\nint main(void) { return (int)PC_OK; }\n')
    for cc, std, lang in (("gcc", "-std=c99", "c"), ("g++", "-std=c++17", "c++")):
        subprocess.run([cc, std, "-x", lang, "-Wall", "-Wextra", "-Werror", "-pedantic",
                        "-fsyntax-only", "-I", os.path.join(ROOT, "include"), str(src)],
                       check=True, capture_output=True)
