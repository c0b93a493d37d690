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


# ---------------------------------------------------------------------------
# binary64 weights: integer products of the binary32 roundings plus the
# remainders' terms (stats.wsum == 3)
# ---------------------------------------------------------------------------
# A binary64 weight w is split into hi = fl32(w) (packed as above) and
# lo = fl32(w - hi), stored scaled as l = lo 2^(142 - e_max).  With
# wscale = 2^(e_max,i + e_max,j - 300) the unit of the accumulators,
# hi_i hi_j = P 2^-16 wscale and (hi_i lo_j + lo_i hi_j) / wscale =
# P_i l_j + l_i P_j (P the packed weights).  The kernel evaluates
# c = fl32(fma(pf_i, l_j, fl32(l_i pf_j))) (pf = fl32 of the packed weight),
# rounds it to the nearest integer k and accumulates
# V = ((P + 2^15) >> 16) + k < 2^49 in pieces of bits 0-15, 16-31 and 32-48
# (at most 2^15 products between flushes, so that no sum wraps).

def _f32(q: Fraction) -> Fraction:
    """Round a rational to the nearest binary32 value (ties to even)."""
    if q == 0:
        return Fraction(0)
    sgn = -1 if q < 0 else 1
    a = abs(q)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** e > a:
        e -= 1
    e = max(e, -126)                       # subnormals keep the spacing 2^-149
    scale = Fraction(2) ** (e - 23)
    m = a / scale
    n = m.numerator // m.denominator
    rem = m - n
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and n % 2 == 1):
        n += 1
    return sgn * n * scale


def _rne_int(q: Fraction) -> int:
    n = q.numerator // q.denominator
    rem = q - n
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and n % 2 == 1):
        n += 1
    return n


def _split64(w, emax):
    """(packed, pf, l) of binary64 weights: the kernel's per-point inputs."""
    hi = w.astype(F32)
    lo = (w - hi.astype(np.float64)).astype(F32)
    packed, _, _ = _pack(hi, emax, emax - 8)
    pf = [_f32(Fraction(p)) for p in packed]
    l = [_f32(Fraction(float(v)) * Fraction(2) ** (142 - emax)) for v in lo]
    return packed, pf, l


def _emulated_sum64(wi, wj, emax_i, emax_j):
    pi, pfi, li = _split64(wi, emax_i)
    pj, pfj, lj = _split64(wj, emax_j)
    vs = []
    for a, fa, la, b, fb, lb in zip(pi, pfi, li, pj, pfj, lj):
        t = _f32(la * fb)
        c = _f32(fa * lb + t)
        k = _rne_int(c)
        v = ((a * b + 2 ** 15) >> 16) + k
        assert 0 <= v < 2 ** 49
        vs.append(v)
    total = Fraction(0)
    for s in range(0, len(vs), WINT_LIMIT // 2):
        chunk = vs[s:s + WINT_LIMIT // 2]
        lo = sum(v & 0xFFFF for v in chunk)
        mid = sum((v >> 16) & 0xFFFF for v in chunk)
        hi = sum(v >> 32 for v in chunk)
        assert max(lo, mid, hi) < 2 ** 32                      # no u32 sum wraps
        total += lo + (mid << 16) + (hi << 32)
    return total * Fraction(2) ** (emax_i + emax_j - 300)


def _weights64(rng, n, e_lo, e_hi):
    """Binary64 weights with binary32 roundings in binades [e_lo, e_hi]
    (biased exponents) and full 53-bit significands."""
    e = rng.integers(e_lo, e_hi + 1, n)
    m = rng.integers(2 ** 52, 2 ** 53, n).astype(np.float64)
    w = m * np.exp2(e.astype(np.float64) - 127.0 - 52.0)
    # stay inside the binade after rounding to binary32
    return np.minimum(w, np.exp2(e.astype(np.float64) - 126.0) * (1.0 - 2.0 ** -25))


def test_binary64_remainders_within_two_to_minus_34():
    rng = np.random.default_rng(17)
    for span_i, span_j in ((0, 0), (3, 5), (6, 6), (8, 4)):
        e0i, e0j = 120, 131
        wi = _weights64(rng, 3000, e0i, e0i + span_i)
        wj = _weights64(rng, 3000, e0j, e0j + span_j)
        emax_i = int(max((wi.astype(F32).view(np.uint32) >> 23) & 0xFF))
        emax_j = int(max((wj.astype(F32).view(np.uint32) >> 23) & 0xFF))
        got = _emulated_sum64(wi, wj, emax_i, emax_j)
        exact = sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(wi, wj))
        rel = abs(got - exact) / exact
        assert rel < Fraction(1, 2 ** 34) * Fraction(1001, 1000), (span_i, span_j, float(rel))
    # without remainders (binary32 weights on both sides) the rounding of
    # P / 2^16 alone is left: half the truncation bound
    wi = _weights(rng, 3000, 120, 126).astype(np.float64)
    wj = _weights(rng, 3000, 130, 136).astype(np.float64)
    got = _emulated_sum64(wi, wj, 126, 136)
    exact = sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(wi, wj))
    assert abs(got - exact) / exact < Fraction(1, 2 ** 35)


def test_binary64_remainders_single_pair_bound():
    """Pairs whose binary32 roundings sit 6 binades below both maxima
    (products near 2^34 units, where the two roundings weigh most): every
    pair within 2^-34 (1 + 2^-10) of its exact product."""
    rng = np.random.default_rng(19)
    emax_i = emax_j = 140
    wi = _weights64(rng, 400, 134, 134)
    wj = _weights64(rng, 400, 134, 134)
    for a, b in zip(wi, wj):
        got = _emulated_sum64(np.array([a]), np.array([b]), emax_i, emax_j)
        exact = Fraction(float(a)) * Fraction(float(b))
        assert abs(got - exact) / exact < Fraction(1, 2 ** 34) * Fraction(1025, 1024)


def test_binary64_record_holds_its_flush_limit():
    """2^15 values of V just below 2^49 between two flushes: no u32 sum of
    the record wraps, and the recombination is exact."""
    v = 2 ** 49 - 1
    n = WINT_LIMIT // 2
    lo, mid, hi = n * (v & 0xFFFF), n * ((v >> 16) & 0xFFFF), n * (v >> 32)
    assert max(lo, mid, hi) < 2 ** 32
    assert lo + (mid << 16) + (hi << 32) == n * v


def test_fold_mode_totals_are_exact():
    """Fold mode (large histograms): at every product limit each lane copy's
    record, whose recombined sum stays below 2^64, is added with carry into a
    128-bit total held as two u64 words; the flush converts the total once.
    Over many folds of the largest sums the words carry, the total equals the
    exact integer sum, and the conversion (hi 2^64 + lo, each word rounded to
    binary64) stays within 2^-52 relative."""
    rng = np.random.default_rng(29)
    M64 = 2 ** 64
    lo = hi = 0
    exact = 0
    for _ in range(300):
        for _copy in range(2):
            n = WINT_LIMIT // 2
            v = int(rng.integers(2 ** 48, 2 ** 49))         # W == 3 products below 2^49
            words = (n * (v & 0xFFFF), n * ((v >> 16) & 0xFFFF), n * (v >> 32))
            assert max(words) < 2 ** 32
            t = words[0] + (words[1] << 16) + (words[2] << 32)
            assert t < M64 and t == n * v
            l1 = (lo + t) % M64                             # u64 add with carry
            hi += 1 if l1 < t else 0
            lo = l1
            exact += t
    assert hi > 0 and (hi << 64) + lo == exact
    w = Fraction(float(hi)) * M64 + Fraction(float(lo))
    assert abs(w - exact) / exact < Fraction(1, 2 ** 52)
