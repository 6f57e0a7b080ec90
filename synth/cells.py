"""Seeded inputs for the cell-neighbour reductions of Table 1 on the
periodic triangular patch of ``synth.octahedral``: the cells (triangles),
their three edge neighbours, and three numberings of the cells (Sec. 3.2).

Like the rest of ``synth`` it holds none of the operations' arithmetic.

Cells.  For nodes (r, c) of an nr x nc periodic patch the cells are the
upward triangles U(r, c) = (r, c), (r, c+1), (r+1, c+1) and the downward
triangles D(r, c) = (r, c), (r+1, c+1), (r+1, c): two colours (Fig. 10).
Each cell has three neighbours, the cells across its edges, in this order:

    U(r, c):  D(r-1, c), D(r, c+1), D(r, c)
    D(r, c):  U(r, c),   U(r+1, c), U(r, c-1)

(indices periodic).  Every cell is a neighbour of exactly three cells.

Numberings (storage index of each cell; fields are level-major
[nz][ncells] in that order):

    SN  structured: (row, colour, column) -> (2 r + colour) nc + c; colour 0
        upward, 1 downward (Fig. 10);
    UN  unstructured, as a mesh library without colours numbers a row: the
        two triangles of each column next to each other,
        r (2 nc) + 2 c + colour (Fig. 12);
    HN  along a Hilbert curve through the (r, c) positions (of the enclosing
        power-of-two square), the two triangles of a position consecutive.

``c2c(numbering)`` gives the neighbour table in a numbering's storage order,
structure-of-arrays [3][ncells] (int32), each cell's neighbours in the
order above.
"""
from __future__ import annotations

import numpy as np

DEFAULT_SEED = 1234
NUMBERINGS = ("SN", "UN", "HN")


def _hilbert_d(n: int, x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Position along the Hilbert curve of side n (a power of two) of the
    points (x, y) (the standard rotate-and-accumulate construction)."""
    x = x.astype(np.int64).copy()
    y = y.astype(np.int64).copy()
    d = np.zeros_like(x)
    s = n // 2
    while s > 0:
        rx = ((x & s) > 0).astype(np.int64)
        ry = ((y & s) > 0).astype(np.int64)
        d += s * s * ((3 * rx) ^ ry)
        # rotate the quadrant
        flip = ry == 0
        swap_x = np.where(flip & (rx == 1), s - 1 - x, x)
        swap_y = np.where(flip & (rx == 1), s - 1 - y, y)
        x = np.where(flip, swap_y, swap_x)
        y = np.where(flip, swap_x, swap_y)
        s //= 2
    return d


def storage_index(nr: int, nc: int, numbering: str) -> np.ndarray:
    """perm[r, colour, c] = storage index of cell (r, colour, c)."""
    R, K, C = np.meshgrid(np.arange(nr), np.arange(2), np.arange(nc), indexing="ij")
    if numbering == "SN":
        return (2 * R + K) * nc + C
    if numbering == "UN":
        return R * (2 * nc) + 2 * C + K
    if numbering == "HN":
        side = 1
        while side < max(nr, nc):
            side *= 2
        d = _hilbert_d(side, C[:, 0, :].ravel(), R[:, 0, :].ravel())  # position order
        rank = np.empty(nr * nc, dtype=np.int64)
        rank[np.argsort(d, kind="stable")] = np.arange(nr * nc)
        rank = rank.reshape(nr, nc)
        return 2 * rank[:, None, :] + K
    raise ValueError(numbering)


def neighbours_rck(nr: int, nc: int):
    """For every cell (r, colour, c): its three neighbours as (r, colour, c)
    triples, shape (nr, 2, nc, 3, 3)."""
    R, K, C = np.meshgrid(np.arange(nr), np.arange(2), np.arange(nc), indexing="ij")
    out = np.empty((nr, 2, nc, 3, 3), dtype=np.int64)
    up = K == 0
    # U(r,c): D(r-1,c), D(r,c+1), D(r,c);  D(r,c): U(r,c), U(r+1,c), U(r,c-1)
    dr = np.where(up[..., None], np.array([-1, 0, 0]), np.array([0, 1, 0]))
    dc = np.where(up[..., None], np.array([0, 1, 0]), np.array([0, 0, -1]))
    out[..., 0] = np.mod(R[..., None] + dr, nr)
    out[..., 1] = (1 - K)[..., None]
    out[..., 2] = np.mod(C[..., None] + dc, nc)
    return out


def c2c(nr: int, nc: int, numbering: str) -> np.ndarray:
    """Neighbour table [3][ncells] (int32) in the numbering's storage order."""
    perm = storage_index(nr, nc, numbering)
    nb = neighbours_rck(nr, nc)
    nbs = perm[nb[..., 0], nb[..., 1], nb[..., 2]]       # (nr, 2, nc, 3) storage ids
    t = np.empty((3, 2 * nr * nc), dtype=np.int32)
    for j in range(3):
        t[j, perm.ravel()] = nbs[..., j].ravel()
    return t


def field(nr: int, nc: int, nz: int, seed: int = DEFAULT_SEED, numbering: str = "SN",
          integer: bool = False) -> np.ndarray:
    """A seeded cell field [nz][ncells] in the numbering's storage order: the
    same values per cell (r, colour, c) whatever the numbering; with
    ``integer`` small integers (sums exact in any order)."""
    rng = np.random.default_rng(seed)
    vals = (rng.integers(-50, 50, size=(nz, nr, 2, nc)).astype(np.float64) if integer
            else rng.standard_normal((nz, nr, 2, nc)))
    perm = storage_index(nr, nc, numbering)
    out = np.empty((nz, 2 * nr * nc))
    out[:, perm.ravel()] = vals.reshape(nz, -1)
    return out
