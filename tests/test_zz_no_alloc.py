"""The allocation-free count entry point (pc_count_auto_noalloc).

It serves callers that cannot allocate device memory while counting: their
device memory is owned by another allocator, or an allocation (with its
possible implicit device synchronisation) is not allowed in their loop.  Its
results must equal pc_count_auto's on the same grid, including on a second
call in a row, since every call reuses one fixed scratch array inside the
library.  This file is collected last so that a run stopping at the first
failure has already run every other test.
"""

import numpy as np
import pytest

import synth

P = pytest.importorskip("paper_2301_12557_gb300")
torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

WREL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P.build()
    torch.cuda.init()
    yield


def _weighted_close(got, want):
    zero = want == 0
    assert np.all(got[zero] == 0)
    rel = np.abs(got[~zero] - want[~zero]) / np.abs(want[~zero])
    assert rel.size == 0 or rel.max() <= WREL


@pytest.mark.parametrize("mode,eb", [("smu", np.linspace(0.0, 1.0, 21)), ("s", None),
                                     ("sigpi", np.linspace(0.0, 25.0, 11))])
def test_noalloc_equals_count_auto_on_two_calls(mode, eb):
    L = 200.0
    x = synth.neyman_scott(30000, 3000, 10.0, 3.0, L, synth.SEED_BASE + 301)
    w = synth.lognormal_weights(x.shape[0], 0.3, synth.SEED_BASE + 302, np.float64)
    xd = torch.from_numpy(x).cuda()
    wd = torch.from_numpy(w).cuda()
    bins = P.Bins(mode, "z", np.linspace(0.0, 40.0, 21), eb)
    g = P.pc_build_grid(xd, wd, box=P.make_box(L, True), r_max=bins.r_max)
    try:
        ref, wref, _ = P.pc_count_auto(g, bins, weighted=True)
        for _ in range(2):
            out = torch.zeros(bins.nbins, dtype=torch.int64, device="cuda")
            wout = torch.zeros(bins.nbins, dtype=torch.float64, device="cuda")
            P.pc_count_auto_noalloc(g, bins, counts=out, wcounts=wout, weighted=True)
            assert np.array_equal(out.cpu().numpy(), ref)
            _weighted_close(wout.cpu().numpy(), wref)
            c, _ = P.pc_count_auto_noalloc(g, bins)           # host output, unweighted
            assert np.array_equal(c, ref)
    finally:
        g.free()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    L = 100.0
    x = synth.uniform_box(1000, L, synth.SEED_BASE + 303)
    bins = P.Bins("smu", "z", np.linspace(0.0, 20.0, 201), np.linspace(0.0, 1.0, 101))
    g = P.pc_build_grid(x, box=P.make_box(L, True), r_max=bins.r_max)
    try:
        with pytest.raises(P.PairCountError) as ei:
            P.pc_count_auto_noalloc(g, bins)      # 20100 bins > 16384
        assert ei.value.status == P.PC_EOVERFLOW
    finally:
        g.free()
