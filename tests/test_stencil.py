"""The grid path's neighbour-cell stencil (Sect. 2.1, Sect. 3.1), host-only.

Completeness against brute-force cell distances: a cell offset belongs to
the stencil exactly when the smallest distance between the two cells is
below the largest separation; the half stencil of an auto count keeps one of
each pair of opposite offsets.  The number of cells follows the paper's
cell-count model (App. B: N_inner ~ 4 pi / 3 L^-3 cells fully inside the
query range of a reference cell and N_edge ~ 8 pi L^-1.94 partly inside, L
the cell side over the separation) in its small-cell limit, within the
looseness of its fitted exponent.
"""

import itertools
import math

import pytest

P = pytest.importorskip("paper_2301_12557_gb300")


@pytest.fixture(scope="module")
def lib():
    P.build()
    return P.lib()


def _offsets(rows):
    out = set()
    for dy, dz, xlo, xhi in rows:
        for dx in range(xlo, xhi + 1):
            out.add((int(dx), int(dy), int(dz)))
    return out


def _brute(cell, r):
    """Offsets whose cells come within r of each other (and nothing within a
    relative 1e-9 of the boundary, where the stencil may be more inclusive)."""
    need, maybe = set(), set()
    k = [int(math.ceil(r / c)) + 1 for c in cell]
    for d in itertools.product(*[range(-kk, kk + 1) for kk in k]):
        m2 = sum((max(abs(di) - 1, 0) * c) ** 2 for di, c in zip(d, cell))
        if m2 < r * r * (1 - 1e-9):
            need.add(d)
        elif m2 < r * r * (1 + 1e-9):
            maybe.add(d)
    return need, maybe


CASES = [((10.0, 10.0, 10.0), 25.0), ((10.0, 10.0, 10.0), 20.0), ((7.0, 11.0, 13.0), 40.0),
         ((50.0, 50.0, 50.0), 200.0), ((84.09, 84.09, 84.09), 200.0), ((300.0, 300.0, 300.0), 200.0)]


@pytest.mark.parametrize("cell,r", CASES)
def test_full_stencil_is_exactly_the_cells_in_reach(lib, cell, r):
    full = _offsets(P.pc_stencil(cell, r, half=False))
    need, maybe = _brute(cell, r)
    assert need <= full
    assert full <= need | maybe


@pytest.mark.parametrize("cell,r", CASES)
def test_half_stencil_keeps_one_of_each_opposite_pair(lib, cell, r):
    full = _offsets(P.pc_stencil(cell, r, half=False))
    half = _offsets(P.pc_stencil(cell, r, half=True))
    mirror = {(-a, -b, -c) for a, b, c in half}
    assert not (half & mirror)
    assert (0, 0, 0) not in half
    assert half | mirror | {(0, 0, 0)} == full
    # rows of the half stencil reach equally far up and down in y and z
    rows = P.pc_stencil(cell, r, half=True)
    assert abs(int((rows[:, 0] > 0).sum()) - int((rows[:, 0] < 0).sum())) <= 2


@pytest.mark.parametrize("lhat,tol", [(0.1, 0.05), (0.2, 0.2), (0.25, 0.2)])
def test_cell_count_model(lib, lhat, tol):
    """The model's formulae hold in the small-cell limit: within 5 % at a
    cell of a tenth of the separation, 20 % at a fifth to a quarter."""
    r = 100.0
    c = lhat * r
    full = _offsets(P.pc_stencil((c, c, c), r, half=False))
    # a cell is fully inside the query range of the reference cell when its
    # farthest point lies within r of that cell: per axis |d| c
    inner = sum(1 for d in full if sum((abs(di) * c) ** 2 for di in d) < r * r)
    edge = len(full) - inner
    n_inner = 4 * math.pi / 3 * lhat ** -3
    n_edge = 8 * math.pi * lhat ** -1.94
    assert abs(inner - n_inner) <= tol * n_inner, (inner, n_inner)
    assert abs(edge - n_edge) <= tol * n_edge, (edge, n_edge)


def test_stencil_rejects_bad_arguments(lib):
    with pytest.raises(P.PairCountError):
        P.pc_stencil((10.0, 10.0, 0.0), 20.0)
    with pytest.raises(P.PairCountError):
        P.pc_stencil((10.0, 10.0, 10.0), -1.0)
