"""The allocation-free count entry point (pc_count_auto_noalloc).

It serves callers that cannot allocate device memory while counting: their
device memory is owned by another allocator, or an allocation (with its
possible implicit device synchronisation) is not allowed in their loop.  Its
results must equal pc_count_auto's and the oracle's on the same grid,
including on a second call in a row, since every call reuses one fixed
scratch array inside the library; it must make no allocation at all (the
library counts every allocation it makes: pc_alloc_count), also when it is
the first count of a fresh process; and it must refuse, before any device
work, sizes its array cannot hold.  This file is collected last so that a run
stopping at the first failure has already run every other test.
"""

import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
import synth

P = pytest.importorskip("paper_2301_12557_gb300")
torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

WREL = 1e-10
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P.build()
    oracle.build()
    torch.cuda.init()
    yield


def _weighted_close(got, want):
    zero = want == 0
    assert np.all(got[zero] == 0)
    rel = np.abs(got[~zero] - want[~zero]) / np.abs(want[~zero])
    assert rel.size == 0 or rel.max() <= WREL


@pytest.mark.parametrize("mode,eb", [("smu", np.linspace(0.0, 1.0, 21)), ("s", None),
                                     ("sigpi", np.linspace(0.0, 25.0, 11))])
def test_noalloc_equals_count_auto_and_oracle_on_two_calls(mode, eb):
    L = 200.0
    x = synth.neyman_scott(30000, 3000, 10.0, 3.0, L, synth.SEED_BASE + 301)
    w = synth.lognormal_weights(x.shape[0], 0.3, synth.SEED_BASE + 302, np.float64)
    xd = torch.from_numpy(x).cuda()
    wd = torch.from_numpy(w).cuda()
    ea = np.linspace(0.0, 40.0, 21)
    bins = P.Bins(mode, "z", ea, eb)
    want, wwant = oracle.count(x, w1=w, box=L, periodic=True, mode=mode, edges_a=ea, edges_b=eb,
                               method="grid")
    g = P.pc_build_grid(xd, wd, box=P.make_box(L, True), r_max=bins.r_max)
    try:
        ref, wref, _ = P.pc_count_auto(g, bins, weighted=True)
        assert np.array_equal(ref, want)
        out = torch.zeros(bins.nbins, dtype=torch.int64, device="cuda")
        wout = torch.zeros(bins.nbins, dtype=torch.float64, device="cuda")
        a0 = P.pc_alloc_count()
        for _ in range(2):
            P.pc_count_auto_noalloc(g, bins, counts=out, wcounts=wout, weighted=True)
            assert np.array_equal(out.cpu().numpy(), ref)
            _weighted_close(wout.cpu().numpy(), wwant)
            c, _ = P.pc_count_auto_noalloc(g, bins)           # host output, unweighted
            assert np.array_equal(c, want)
        assert P.pc_alloc_count() == a0, "the allocation-free call allocated"
    finally:
        g.free()


def test_noalloc_rescue_queue_overflow():
    """A lattice whose every pair sits exactly on a squared edge: all 8.6e6
    in-range pairs need the binary64 definition, far more than the array's
    131,072 rescue slots, so most are evaluated inside the pair kernel."""
    side = 40
    x = synth.lattice_points(side ** 3, side, synth.SEED_BASE + 304)
    ea = np.sqrt(np.arange(0.0, 17.0))                  # s^2 edges 0, 1, ..., 16
    bins = P.Bins("s", "z", ea)
    want, _ = oracle.count(x, box=float(side), periodic=True, edges_a=ea, method="grid")
    g = P.pc_build_grid(x, box=P.make_box(float(side), True), r_max=bins.r_max)
    try:
        ref, _, st = P.pc_count_auto(g, bins)
        assert st.rescued > 131072
        assert np.array_equal(ref, want)
        a0 = P.pc_alloc_count()
        for _ in range(2):
            c, _ = P.pc_count_auto_noalloc(g, bins)
            assert np.array_equal(c, want)
        assert P.pc_alloc_count() == a0
    finally:
        g.free()


def test_noalloc_midpoint_near_observer_takes_the_fp64_kernel():
    """Points around the observer along the midpoint line of sight: the FP32
    error bound does not hold, so the call runs the plain FP64 kernel."""
    x = synth.uniform_box(20000, 100.0, synth.SEED_BASE + 305) - 50.0
    ea = np.linspace(0.0, 20.0, 11)
    mu = np.linspace(0.0, 1.0, 11)
    bins = P.Bins("smu", "mid", ea, mu)
    want, _ = oracle.count(x, periodic=False, mode="smu", los="mid", edges_a=ea, edges_b=mu,
                           method="grid")
    box = P.make_box(None, False, x.min(0), x.max(0))
    g = P.pc_build_grid(x, box=box, r_max=bins.r_max)
    try:
        ref, _, st = P.pc_count_auto(g, bins)
        assert st.prec == P.PC_PREC_F64
        assert np.array_equal(ref, want)
        for _ in range(2):
            c, _ = P.pc_count_auto_noalloc(g, bins)
            assert np.array_equal(c, want)
    finally:
        g.free()


FRESH = r"""
import sys
sys.path.insert(0, {root!r})
import numpy as np, torch
import paper_2301_12557_gb300 as P, synth, oracle
torch.cuda.set_device(0)
L = 150.0
x = synth.neyman_scott(20000, 2000, 10.0, 3.0, L, synth.SEED_BASE + 306)
ea = np.linspace(0.0, 30.0, 16)
mu = np.linspace(0.0, 1.0, 11)
bins = P.Bins("smu", "z", ea, mu)
g = P.pc_build_grid(torch.from_numpy(x).cuda(), box=P.make_box(L, True), r_max=bins.r_max)
out = torch.zeros(bins.nbins, dtype=torch.int64, device="cuda")
torch.cuda.synchronize()
a0 = P.pc_alloc_count()
got = []
for _ in range(2):
    P.pc_count_auto_noalloc(g, bins, counts=out)
    got.append(out.cpu().numpy().copy())
a1 = P.pc_alloc_count()
want, _ = oracle.count(x, box=L, periodic=True, mode="smu", edges_a=ea, edges_b=mu, method="grid")
ok = a1 == a0 and all(np.array_equal(c, want) for c in got)
g.free()
print("FRESH", "ok" if ok else "bad", a0, a1, flush=True)
"""


def test_noalloc_first_count_of_a_fresh_process():
    """The first count of a new process is an allocation-free one: it makes
    no allocation (the array's address lookup included) and its results on
    two calls equal the oracle's."""
    r = subprocess.run([sys.executable, "-c", FRESH.format(root=ROOT)], capture_output=True,
                       text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = [ln for ln in r.stdout.splitlines() if ln.startswith("FRESH")][-1]
    assert line.split()[1] == "ok", line


def _rejects(g, bins, what):
    a0 = P.pc_alloc_count(), P.pc_launch_count()
    with pytest.raises(P.PairCountError) as ei:
        P.pc_count_auto_noalloc(g, bins)
    assert ei.value.status == P.PC_EOVERFLOW, what
    assert (P.pc_alloc_count(), P.pc_launch_count()) == a0, f"{what}: work before the refusal"


def test_noalloc_rejects_sizes_beyond_its_scratch():
    L = 100.0
    x = synth.uniform_box(1000, L, synth.SEED_BASE + 303)
    box = P.make_box(L, True)
    # 20100 bins > 16384
    bins = P.Bins("smu", "z", np.linspace(0.0, 20.0, 201), np.linspace(0.0, 1.0, 101))
    g = P.pc_build_grid(x, box=box, r_max=bins.r_max)
    try:
        _rejects(g, bins, "bins")
    finally:
        g.free()
    # 100^3 cells > 262144
    bins = P.Bins("s", "z", np.linspace(0.0, 5.0, 6))
    g = P.pc_build_grid(x, box=box, r_max=bins.r_max, opts=P.make_opts("f32", 1.0))
    try:
        assert g.cell_size <= 1.0
        _rejects(g, bins, "cells")
    finally:
        g.free()
    # a flat catalogue of 150 x 150 unit cells, reach 75 cells: a half
    # stencil of about 8,900 rows > 8192 (cells 22,500 within the limit)
    rng = np.random.default_rng(7)
    flat = np.column_stack([rng.random(2000) * 150.0, rng.random(2000) * 150.0,
                            rng.random(2000) * 0.5])
    bins = P.Bins("s", "z", np.linspace(0.0, 75.0, 6))
    fbox = P.make_box(None, False, np.array([0.0, 0.0, 0.0]), np.array([150.0, 150.0, 0.5]))
    g = P.pc_build_grid(flat, box=fbox, r_max=bins.r_max, opts=P.make_opts("f32", 1.0))
    try:
        assert P.pc_stencil([1.0, 1.0, 1.0], 75.0, half=True).shape[0] > 8192
        _rejects(g, bins, "stencil rows")
    finally:
        g.free()
