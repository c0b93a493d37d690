"""Planted mistakes in the oracle are caught by its pins.

Each case copies the oracle's C source, plants one plausible mistake (a
dropped periodic wrap, an edge or mu tie sent to the lower bin, a dropped
term, self pairs counted, a pair weight squared, weights summed without
compensation, sigma^2 left unclamped, the line of sight from the wrong
component or the wrong midpoint, a k-d tree that loses a child pair or prunes
without the periodic images, a median split off by one), compiles the copy,
loads it in place of the oracle and runs the pins of test_oracle_pins.py and
test_oracle_kdtree.py against it: at least one must fail.  The mutants live
in a temporary directory; the oracle's source is not touched.
"""

import ctypes
import os
import subprocess
import tempfile

import pytest

import oracle
import test_oracle_kdtree as K
import test_oracle_pins as T

SRC = os.path.join(os.path.dirname(oracle.__file__), "paircount_oracle.c")

MUTANTS = {
    "no_x_wrap": ("if (d0 > c->hL[0]) d0 -= c->L[0]; else if (d0 < -c->hL[0]) d0 += c->L[0];", ""),
    "edge_tie_low": ("if (v >= E[mid]) lo = mid; else hi = mid;",
                     "if (v > E[mid]) lo = mid; else hi = mid;"),
    "mu_tie_low": ("if (p2 >= t) lo = mid; else hi = mid;", "if (p2 > t) lo = mid; else hi = mid;"),
    "dropped_dz_term": ("double s2 = (d0 * d0 + d1 * d1) + d2 * d2;",
                        "double s2 = (d0 * d0 + d1 * d1);"),
    "self_pairs": ("int64_t j0 = jb->is_auto ? i + 1 : 0;", "int64_t j0 = jb->is_auto ? i : 0;"),
    "pi_from_dy": ("p2 = d2 * d2;", "p2 = d1 * d1;"),
    "midpoint_minus": ("double l0 = a[0] + b[0], l1 = a[1] + b[1], l2 = a[2] + b[2];",
                       "double l0 = a[0] - b[0], l1 = a[1] - b[1], l2 = a[2] - b[2];"),
    "tree_lost_child": ("st[top++] = (npair){2 * q.a + 1, 2 * q.a + 2};", ""),
    "tree_no_images": ("int ns = c->periodic ? 3 : 1;", "int ns = 1;"),
    "weight_square": ("jb->w1[i] * jb->w2[j]);", "jb->w1[i] * jb->w1[i]);"),
    "no_compensation": ("    if (fabs(*sum) >= fabs(v)) *comp += (*sum - t) + v;\n"
                        "    else *comp += (v - t) + *sum;\n", ""),
    "sigma_no_clamp": ("    if (q2 < 0.0) q2 = 0.0;\n", ""),
    "tree_median_off": ("int64_t nl = count / 2;", "int64_t nl = (count + 1) / 2;"),
}


def _pins():
    """The pins run against each mutant (fast ones; each raises on a miss)."""
    for case in T.LATTICE_CASES:
        yield lambda c=case: T.test_lattice_exact(*c)
    for case in T.LATTICE_CASES[::2]:
        yield lambda c=case: T.test_lattice_weighted_exact(*c)
    for method in ("brute", "kdtree"):
        yield lambda m=method: T.test_weighted_sums_are_the_exactly_rounded_sums(m)
    yield T.test_radial_pairs_have_zero_sigma
    yield T.test_cube_corner_golden
    yield T.test_midpoint_golden
    yield T.test_mu_closed_top_and_zero_separation
    yield T.test_periodic_wrap_and_canonical_form
    yield lambda: K.test_kdtree_properties(5000, 33)
    yield lambda: K.test_kdtree_properties(3001, 8)
    for mode, los, periodic, ea, eb in [("s", "z", True, [0, 1, 2, 3, 4], None),
                                        ("smu", "z", True, [0, 1, 2, 3, 4],
                                         [0, 0.25, 0.5, 0.75, 1])]:
        yield lambda a=(mode, los, periodic, ea, eb): K.test_dualtree_lattice_exact(*a)


@pytest.fixture(scope="module")
def tmpdir():
    with tempfile.TemporaryDirectory() as d:
        yield d


def _build(name, old, new, tmp):
    src = open(SRC).read()
    assert src.count(old) == 1, name
    path = os.path.join(tmp, f"{name}.c")
    with open(path, "w") as f:
        f.write(src.replace(old, new))
    so = os.path.join(tmp, f"{name}.so")
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                    "-pthread", "-o", so, path, "-lm"], check=True, capture_output=True)
    return oracle._configure(ctypes.CDLL(so))


def _failures(lib, monkeypatch):
    monkeypatch.setattr(oracle, "_lib", lib)
    failed = 0
    for pin in _pins():
        try:
            pin()
        except (AssertionError, ValueError):
            failed += 1
    return failed


def test_unmutated_copy_passes_every_pin(tmpdir, monkeypatch):
    old = "int64_t j0 = jb->is_auto ? i + 1 : 0;"
    assert _failures(_build("identity", old, old, tmpdir), monkeypatch) == 0


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name, tmpdir, monkeypatch):
    old, new = MUTANTS[name]
    assert _failures(_build(name, old, new, tmpdir), monkeypatch) > 0, \
        f"mutant {name} passes every pin"
