"""GPU parity of the histogram-update micro-benchmark kernel (Sect. 3.2.4):
every update algorithm, and the lookup table at every size, gives the
oracle's histogram of the same squared separations exactly."""

import numpy as np
import pytest

import oracle
import synth

P = pytest.importorskip("paper_2301_12557_gb300")
torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P.build()
    torch.cuda.init()
    yield


R = 200.0
EDGES = {
    "lin20": np.linspace(0.0, R, 21),
    "lin200": np.linspace(0.0, R, 201),
    "log20": np.geomspace(0.1, R, 21),
    "log200": np.geomspace(0.1, R, 201),
    "irregular": np.concatenate([[0.0], np.sort(np.random.default_rng(3).uniform(0.5, R, 30)), [R]]),
    "integer": np.arange(0.0, R + 1.0, 10.0),
}


def _samples(edges, n=1 << 21, seed=11):
    s2 = synth.s2_samples(n, R, seed)
    E = (np.asarray(edges, dtype=np.float64) ** 2).astype(np.float32)
    ties = np.concatenate([E, np.nextafter(E, np.float32(0)), np.nextafter(E, np.float32(1e9))])
    return np.concatenate([s2, ties, np.float32([0.0, 1e-30, R * R, 5e4])]).astype(np.float32)


@pytest.mark.parametrize("name", list(EDGES))
def test_every_method_matches_the_oracle(name):
    edges = EDGES[name]
    s2 = _samples(edges)
    want = oracle.hist_s2(s2, edges)
    d = torch.from_numpy(s2).cuda()
    methods = [("bsearch", 0), ("reverse", 0), ("map_lin", 0)]
    if edges[0] > 0:
        methods.append(("map_log", 0))
    methods += [("lut", t) for t in (1, 2, 7, 100, 4096, 49152)]
    for m, t in methods:
        got, ms = P.pc_hist_s2(d, edges, m, table_size=t, repeat=3)
        assert np.array_equal(got, 3 * want), (name, m, t, np.nonzero(got != 3 * want)[0][:5])
        assert ms > 0


def test_host_inputs_and_device_outputs():
    edges = EDGES["log20"]
    s2 = _samples(edges, n=100000)
    out = torch.zeros(20, dtype=torch.int64, device="cuda")
    P.pc_hist_s2(s2, edges, "lut", table_size=1000, counts=out)
    assert np.array_equal(out.cpu().numpy(), oracle.hist_s2(s2, edges))
    got, _ = P.pc_hist_s2(s2[:0], edges, "bsearch")
    assert got.sum() == 0
    # a device view one sample in (not 16-byte aligned): the scalar loop
    d = torch.from_numpy(s2).cuda()
    got, _ = P.pc_hist_s2(d[1:], edges, "lut", table_size=512)
    assert np.array_equal(got, oracle.hist_s2(s2[1:], edges))
    got, _ = P.pc_hist_s2(d[3:], edges, "map_log")
    assert np.array_equal(got, oracle.hist_s2(s2[3:], edges))


def test_errors():
    s2 = np.ones(10, dtype=np.float32)
    with pytest.raises(P.PairCountError):
        P.pc_hist_s2(s2, [0.0, 1.0], "lut", table_size=0)
    with pytest.raises(P.PairCountError):
        P.pc_hist_s2(s2, [0.0, 1.0], "lut", table_size=49153)
    with pytest.raises(P.PairCountError):
        P.pc_hist_s2(s2, [0.0, 1.0], "map_log")
    with pytest.raises(P.PairCountError):
        P.pc_hist_s2(s2, [1.0, 0.5], "bsearch")
    with pytest.raises(P.PairCountError):
        P.pc_hist_s2(s2, [0.0, 1.0], 9)
