"""Pins for the oracle's squared-separation histogram and the App. C sampler
used by the histogram-update micro-benchmark (Sect. 3.2.4)."""

import numpy as np

import oracle
import synth


def _loop_hist(s2, edges):
    """The bin rule written out: bin k iff e_k^2 <= s2 < e_{k+1}^2."""
    E = [float(e) * float(e) for e in edges]
    h = [0] * (len(edges) - 1)
    for v in s2:
        v = float(v)
        for k in range(len(h)):
            if E[k] <= v < E[k + 1]:
                h[k] += 1
                break
    return np.array(h, dtype=np.int64)


def test_hist_equals_the_bin_rule_with_ties():
    rng = np.random.default_rng(1)
    edges = np.array([0.0, 1.0, 2.0, 2.5, 7.0, 10.0])
    E = (edges * edges).astype(np.float32)
    v = rng.uniform(0.0, 110.0, 3000).astype(np.float32)
    ties = np.concatenate([E, np.nextafter(E, np.float32(0)), np.nextafter(E, np.float32(200))])
    s2 = np.concatenate([v, ties]).astype(np.float32)
    got = oracle.hist_s2(s2, edges)
    assert got.tolist() == _loop_hist(s2, edges).tolist()
    # a sample exactly on an inner edge goes to the upper bin; the top edge is excluded
    one = oracle.hist_s2(np.array([4.0], dtype=np.float32), edges)
    assert one.tolist() == [0, 0, 1, 0, 0]
    assert oracle.hist_s2(np.array([100.0], dtype=np.float32), edges).sum() == 0


def test_sampler_follows_the_volume_distribution():
    """App. C: P(s < e) = (e / R)^3; every bin within 5 sigma of the
    multinomial expectation, for linear and logarithmic bins."""
    R, n = 200.0, 2_000_000
    s2 = synth.s2_samples(n, R, 5)
    assert s2.dtype == np.float32 and s2.min() >= 0 and s2.max() < R * R
    for edges in (np.linspace(0.0, R, 21), np.geomspace(0.1, R, 21)):
        h = oracle.hist_s2(s2, edges)
        p = np.diff((edges / R) ** 3)
        mu = n * p
        sig = np.sqrt(n * p * (1 - p))
        assert np.all(np.abs(h - mu) <= 5 * sig + 1), (h, mu)
