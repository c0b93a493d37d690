"""The integer weight-product path's error bound (CPU, emulated).

When every weight of a catalogue is a non-negative normal binary32 value (or
zero), its exponents span at most 8 binades, and the two catalogues' spans
add up to at most 12, the pair kernel accumulates each pair weight w_i w_j
(Sect. 2.5) as an integer.  The weight w = M 2^(e - 150) (M the 24-bit
significand, e the biased exponent) is packed as M 2^(8 - k), k = e_max - e
(below 2^32); the exact 64-bit product of two packed weights is
P = M_i M_j 2^(16 - k_i - k_j), and p = P >> 16 equals (M_i M_j) >> (k_i +
k_j) exactly (below 2^48).  Its three 16-bit pieces, bits 16-31, 32-47 and
48-63 of P, are added to three 32-bit lane counters (at most 2^16 products
between flushes, so no counter wraps), and a flush recombines each lane's
counters into the exact 64-bit sum, converts it to binary64 and multiplies it
by 2^(e_max,i + e_max,j - 300).  The truncation of one product is below
2^(k_i + k_j - 46) <= 2^-34 of it, so every bin's sum is within 2^-34
relative of the exact sum.  This test emulates the path on weights spanning
the allowed exponents and checks the bound against exact rational sums, and
that it is close to tight.
"""

from fractions import Fraction

import numpy as np

F32 = np.float32
WINT_LIMIT = 1 << 16


def _pack(w, emax, emin):
    """Packed weights M 2^(8 - k) (below 2^32), and M and k for the check."""
    assert emax - emin <= 8
    b = w.astype(F32).view(np.uint32).astype(np.int64)
    e = (b >> 23) & 0xFF
    m = np.where(e > 0, (b & 0x7FFFFF) | 0x800000, 0)
    k = np.where(e > 0, emax - e, 0)
    packed = [int(a) << int(8 - kk) if a else 0 for a, kk in zip(m, k)]
    assert max(packed, default=0) < 2 ** 32
    return packed, m, k


def _emulated_sum(wi, wj, ext_i, ext_j):
    """The kernel's integer accumulation of sum_i w_i wj_i (pairs given as two
    aligned arrays), flushed every WINT_LIMIT products, as binary64.  ext_* =
    (e_max, e_min) of each catalogue."""
    (emax_i, emin_i), (emax_j, emin_j) = ext_i, ext_j
    pi, mi, ki = _pack(wi, emax_i, emin_i)
    pj, mj, kj = _pack(wj, emax_j, emin_j)
    full = [a * b for a, b in zip(pi, pj)]              # the exact 64-bit products P
    assert max(full, default=0) < 2 ** 64
    prod = [q >> 16 for q in full]
    # the same integer as the significands' product shifted by both offsets
    assert prod == [(int(a) * int(b)) >> int(s) for a, b, s in zip(mi, mj, ki + kj)]
    assert max(prod, default=0) < 2 ** 48
    unit = 2.0 ** (emax_i + emax_j - 300)
    total = 0.0
    for s in range(0, len(prod), WINT_LIMIT):
        chunk = prod[s:s + WINT_LIMIT]
        pieces = full[s:s + WINT_LIMIT]                   # bits 16-31, 32-47, 48-63 of P
        lo = sum((q >> 16) & 0xFFFF for q in pieces)
        mid = sum((q >> 32) & 0xFFFF for q in pieces)
        hi = sum(q >> 48 for q in pieces)
        assert max(lo, mid, hi) < 2 ** 32          # three u32 plane counters
        acc = lo + (mid << 16) + (hi << 32)        # the flush's recombination
        assert acc == sum(chunk) and acc < 2 ** 64
        total += float(acc) * unit
    return total


def _weights(rng, n, e_lo, e_hi):
    """Binary32 weights with biased exponents in [e_lo, e_hi] and full
    significands (so truncations are as large as they get)."""
    e = rng.integers(e_lo, e_hi + 1, n)
    m = rng.integers(0x800000, 0x1000000, n)
    return (m.astype(np.float64) * 2.0 ** (e - 150)).astype(F32)


def test_integer_products_within_two_to_minus_34():
    rng = np.random.default_rng(5)
    for span_i, span_j in ((0, 0), (3, 3), (6, 6), (8, 4), (5, 7)):
        e0i, e0j = 120, 130
        wi = _weights(rng, 20000, e0i, e0i + span_i)
        wj = _weights(rng, 20000, e0j, e0j + span_j)
        got = _emulated_sum(wi, wj, (e0i + span_i, e0i), (e0j + span_j, e0j))
        exact = sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(wi, wj))
        rel = abs(Fraction(got) - exact) / exact
        assert rel < Fraction(1, 2 ** 34), (span_i, span_j, float(rel))
    # the adverse case: one weight of each catalogue sets the maxima 6 above
    # all the others, so nearly every product loses twelve bits; the sum's
    # error then comes within a small factor of the bound
    wi = _weights(rng, 20000, 120, 120)
    wj = _weights(rng, 20000, 130, 130)
    wi[0] = F32(2.0 ** (126 - 127))
    wj[0] = F32(2.0 ** (136 - 127))
    got = _emulated_sum(wi, wj, (126, 120), (136, 130))
    exact = sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(wi, wj))
    rel = abs(Fraction(got) - exact) / exact
    assert Fraction(1, 2 ** 38) < rel < Fraction(1, 2 ** 34), float(rel)


def test_single_pair_truncation_reaches_the_bound():
    """A pair whose exponents sit 6 below each maximum (k_i + k_j = 12), with
    significands near 2^23 whose product ends in twelve set bits
    ((2^23 + 4095)(2^23 + 4097) = -1 mod 2^12), loses just under 2^-34 of
    itself: the bound is tight."""
    emax_i = emax_j = 140
    e = 134
    wi = np.array([(2 ** 23 + 4095) * 2.0 ** (e - 150)], dtype=F32)
    wj = np.array([(2 ** 23 + 4097) * 2.0 ** (e - 150)], dtype=F32)
    got = _emulated_sum(wi, wj, (emax_i, e), (emax_j, e))
    exact = Fraction(float(wi[0])) * Fraction(float(wj[0]))
    rel = float(abs(Fraction(got) - exact) / exact)
    assert 2.0 ** -35 < rel < 2.0 ** -34


def test_planes_hold_the_flush_limit_of_largest_products():
    """The worst case between two flushes: 2^16 products of 2^48 - 1 each.
    No 32-bit plane counter wraps and the recombined sum is exact in 64 bits."""
    p = (1 << 48) - 1
    n = WINT_LIMIT
    lo, mid, hi = n * (p & 0xFFFF), n * ((p >> 16) & 0xFFFF), n * (p >> 32)
    assert max(lo, mid, hi) < 2 ** 32
    acc = lo + (mid << 16) + (hi << 32)
    assert acc == n * p < 2 ** 64
