"""Pins of the cell-neighbour reduction of Table 1 (B = fac x the sum of A
over a cell's three neighbours) and of the cell numberings, to facts other
than the oracle:

* each numbering (structured, unstructured, Hilbert) is a bijection onto
  the storage indices;
* the neighbour table is the triangle adjacency of the patch: two cells are
  neighbours exactly when they share two nodes (brute force over the
  triangles' node sets), the relation is symmetric and alternates colours;
* A = 1 gives 3 fac; with integer fields the total of B is exactly
  3 fac times the total of A (every cell is a neighbour of three cells);
* the result does not depend on the numbering, bit for bit, once mapped
  back to (row, colour, column).
"""
import itertools

import numpy as np
import pytest

import oracle
from synth import cells

SIZES = [(4, 4), (5, 7), (8, 8), (3, 12)]


@pytest.mark.parametrize("numbering", cells.NUMBERINGS)
@pytest.mark.parametrize("nr,nc", SIZES)
def test_numbering_is_a_bijection(nr, nc, numbering):
    p = cells.storage_index(nr, nc, numbering).ravel()
    assert np.array_equal(np.sort(p), np.arange(2 * nr * nc))


@pytest.mark.parametrize("nr,nc", SIZES)
def test_table_is_the_triangle_adjacency(nr, nc):
    nb = cells.neighbours_rck(nr, nc)
    def nodes(r, k, c):
        up = [(r, c), (r, c + 1), (r + 1, c + 1)]
        dn = [(r, c), (r + 1, c + 1), (r + 1, c)]
        return frozenset(((a % nr), (b % nc)) for a, b in (up if k == 0 else dn))
    tri = {(r, k, c): nodes(r, k, c) for r in range(nr) for k in range(2) for c in range(nc)}
    for cell, ns in tri.items():
        # the cells sharing an edge (two nodes) with this one
        share = {o for o, ms in tri.items() if o != cell and len(ns & ms) == 2}
        listed = {tuple(x) for x in nb[cell[0], cell[1], cell[2]]}
        if nr >= 3 and nc >= 3:
            assert listed == share and len(listed) == 3
        for o in listed:
            assert o[1] == 1 - cell[1]
            assert cell in {tuple(x) for x in nb[o[0], o[1], o[2]]}


@pytest.mark.parametrize("numbering", cells.NUMBERINGS)
def test_table_counts(numbering):
    t = cells.c2c(6, 9, numbering)
    n = 2 * 6 * 9
    assert t.shape == (3, n) and t.dtype == np.int32
    assert np.all(np.bincount(t.ravel(), minlength=n) == 3)
    for s in range(n):
        assert len(set(t[:, s])) == 3


@pytest.mark.parametrize("numbering", cells.NUMBERINGS)
def test_constant_and_total(numbering):
    nr, nc, nz = 7, 10, 3
    t = cells.c2c(nr, nc, numbering)
    one = np.ones((nz, 2 * nr * nc))
    assert np.all(oracle.cells_sum(t, one, 0.5) == 1.5)
    A = cells.field(nr, nc, nz, seed=3, numbering=numbering, integer=True)
    B = oracle.cells_sum(t, A, 2.0)
    assert np.array_equal(B.sum(axis=1), 6.0 * A.sum(axis=1))


def test_numbering_invariance():
    nr, nc, nz = 8, 8, 4
    ref = None
    for numbering in cells.NUMBERINGS:
        perm = cells.storage_index(nr, nc, numbering).ravel()
        A = cells.field(nr, nc, nz, seed=5, numbering=numbering)
        B = oracle.cells_sum(cells.c2c(nr, nc, numbering), A, 0.7)
        C = oracle.cells_sum(cells.c2c(nr, nc, numbering), B, 1.3)
        got = C[:, perm]           # back to (r, colour, c) order
        if ref is None:
            ref = got
        assert np.array_equal(got, ref)


def test_hilbert_numbering_is_local():
    """Consecutive positions of the Hilbert numbering are lattice neighbours
    (distance 1 on a power-of-two square)."""
    n = 16
    p = cells.storage_index(n, n, "HN")[:, 0, :] // 2     # rank of each (r, c)
    pos = np.empty((n * n, 2), dtype=int)
    for r, c in itertools.product(range(n), range(n)):
        pos[p[r, c]] = (r, c)
    assert np.all(np.abs(np.diff(pos, axis=0)).sum(axis=1) == 1)


@pytest.mark.parametrize("numbering", cells.NUMBERINGS)
def test_delta_response_is_the_edge_neighbours(numbering):
    """A = 1 at one cell, 0 elsewhere: B = fac exactly at the cells that
    share an edge with it (found from the triangles' node sets) and 0
    elsewhere."""
    nr, nc = 5, 6
    perm = cells.storage_index(nr, nc, numbering)
    t = cells.c2c(nr, nc, numbering)
    def nodes(r, k, c):
        up = [(r, c), (r, c + 1), (r + 1, c + 1)]
        dn = [(r, c), (r + 1, c + 1), (r + 1, c)]
        return frozenset((a % nr, b % nc) for a, b in (up if k == 0 else dn))
    for cell in [(0, 0, 0), (2, 1, 3), (4, 1, 5), (3, 0, 0)]:
        A = np.zeros((1, 2 * nr * nc))
        A[0, perm[cell]] = 1.0
        B = oracle.cells_sum(t, A, 0.25)
        ns = nodes(*cell)
        want = np.zeros_like(B)
        for r in range(nr):
            for k in range(2):
                for c in range(nc):
                    if (r, k, c) != cell and len(nodes(r, k, c) & ns) == 2:
                        want[0, perm[r, k, c]] = 0.25
        assert np.array_equal(B, want)
