"""Seeded inputs for the edge-based flux stages on a structured triangular
(octahedral-grid) patch: the upwind flux on edges, the vertical flux on
nodes, their divergence and the advance (Sec. 5, Listings 5, 7 and 8).

Like the rest of ``synth`` this module holds none of the scheme's
arithmetic, only the patch, its connectivity and the fields on it.

The patch.  nr x nc nodes on a triangular lattice, periodic in both
directions (a torus: the structure of one parallelogram of the octahedral
grid, Sec. 3.2, without its irregular corners).  Node (r, c) sits at
c e1 + r e2 with e1 at 0 and e2 at 120 degrees.  Every node owns the three
edges that leave it in the colours

    0: (r, c) -> (r, c+1)        (0 degrees)
    1: (r, c) -> (r+1, c)        (120 degrees)
    2: (r, c) -> (r+1, c+1)      (60 degrees)

so each node has six edges: its own three, on which it is the first node,
and three of its neighbours', on which it is the second.  Cells are the
upward triangles (r, c), (r, c+1), (r+1, c+1) and the downward triangles
(r, c), (r+1, c+1), (r+1, c): two colours, as in Fig. 10.

Structured numbering (Figs. 9 and 11): node (r, c) -> r nc + c; edge
(r, colour, c) -> (3 r + colour) nc + c.  Fields are level-major:

    pD   (nz, nr, nc)       nodes (vertices)
    vn   (nz, nr, 3, nc)    edges, (row, colour, column) within a level
    wn   (nz+1, nr, nc)     vertical faces: face k lies between levels k-1
                            and k; faces 0 and nz are the boundaries, whose
                            fluxes Listing 7 takes from the adjacent interior
                            face: their values are NaN and never read
    rho  (nz, nr, nc)       nodes, > 0
    vol  (nr, nc)           dual volume of each node (2D), > 0

Connectivity tables for indirect addressing (the oracle's view):

    e2n       (E, 2)  first and second node of every edge
    n2e       (N, 6)  the six edges of every node
    n2e_sign  (N, 6)  +1 where the node is the edge's first node, else -1

A positive vn moves mass from an edge's first node to its second.
"""
from __future__ import annotations

import dataclasses

import numpy as np

DEFAULT_SEED = 1234

# (dr, dc) of the second node of each colour's edge
EDGE_OFFSETS = ((0, 1), (1, 0), (1, 1))


@dataclasses.dataclass
class EdgeCase:
    nr: int
    nc: int
    nz: int
    pivbz: float
    pD: np.ndarray
    vn: np.ndarray
    wn: np.ndarray
    rho: np.ndarray
    vol: np.ndarray
    e2n: np.ndarray
    n2e: np.ndarray
    n2e_sign: np.ndarray
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def nnodes(self) -> int:
        return self.nr * self.nc

    @property
    def nedges(self) -> int:
        return 3 * self.nr * self.nc


def node_id(r, c, nr, nc):
    return (np.mod(r, nr)) * nc + np.mod(c, nc)


def edge_id(r, colour, c, nr, nc):
    return (3 * np.mod(r, nr) + colour) * nc + np.mod(c, nc)


def connectivity(nr: int, nc: int):
    """e2n, n2e, n2e_sign of the periodic patch in structured numbering."""
    R, C = np.meshgrid(np.arange(nr), np.arange(nc), indexing="ij")
    E = 3 * nr * nc
    e2n = np.empty((E, 2), dtype=np.int64)
    for col, (dr, dc) in enumerate(EDGE_OFFSETS):
        ids = edge_id(R, col, C, nr, nc).ravel()
        e2n[ids, 0] = node_id(R, C, nr, nc).ravel()
        e2n[ids, 1] = node_id(R + dr, C + dc, nr, nc).ravel()
    n2e = np.empty((nr * nc, 6), dtype=np.int64)
    sgn = np.empty((nr * nc, 6), dtype=np.float64)
    nid = node_id(R, C, nr, nc).ravel()
    for col, (dr, dc) in enumerate(EDGE_OFFSETS):
        n2e[nid, col] = edge_id(R, col, C, nr, nc).ravel()            # own edge
        sgn[nid, col] = 1.0
        n2e[nid, 3 + col] = edge_id(R - dr, col, C - dc, nr, nc).ravel()  # neighbour's
        sgn[nid, 3 + col] = -1.0
    return e2n, n2e, sgn


def _cell_stream_fluxes(chi_up, chi_dn, nr, nc):
    """Edge values chi(left cell) - chi(right cell) for a cell function chi:
    around every node they telescope, so their signed sum is zero."""
    up = lambda r, c: chi_up[np.mod(r, nr)][:, np.mod(c, nc)]
    dn = lambda r, c: chi_dn[np.mod(r, nr)][:, np.mod(c, nc)]
    r = np.arange(nr)
    c = np.arange(nc)
    out = np.empty((nr, 3, nc))
    # colour 0 (0 deg): left = upward (r, c), right = downward (r-1, c)
    out[:, 0, :] = up(r, c) - dn(r - 1, c)
    # colour 1 (120 deg): left = upward (r, c-1), right = downward (r, c)
    out[:, 1, :] = up(r, c - 1) - dn(r, c)
    # colour 2 (60 deg): left = downward (r, c), right = upward (r, c)
    out[:, 2, :] = dn(r, c) - up(r, c)
    return out


def _scale_to_courant(vn, wn, rho, vol, cmax, e2n_shape):
    """Scale vn and wn so that at every node-level the sum of the absolute
    values of its eight face values (six edges, two vertical faces; the
    boundary faces counted with their adjacent interior face) is at most
    cmax times vol * rho: the outflow then never exceeds the content."""
    nz, nr, _, nc = vn.shape
    a = np.abs(vn)
    s = a.sum(axis=2)                                    # own edges
    for col, (dr, dc) in enumerate(EDGE_OFFSETS):        # the neighbours' edges
        s = s + np.roll(np.roll(a[:, :, col, :], dr, axis=1), dc, axis=2)
    w = np.abs(wn.copy())
    w[0] = w[1] if nz > 1 else 0.0
    w[nz] = w[nz - 1] if nz > 1 else 0.0
    s = s + w[:-1] + w[1:]
    f = cmax / float(np.max(s / (vol[None] * rho)))
    return vn * f, wn * f


def edge_case(nr: int, nc: int, nz: int, seed: int = DEFAULT_SEED, pivbz: float = 0.0,
              cmax: float = 0.9, divergent: bool = True, psi_lo: float = 0.2) -> EdgeCase:
    """A seeded patch: pD = psi_lo + a Gaussian ridge + uniform noise; rho in
    [0.5, 1.5], vol in [0.8, 1.2]; vn and wn uniform random (divergent) or,
    with divergent=False, vn from a random cell function (zero divergence
    at every node) and wn = 0; scaled by _scale_to_courant."""
    if nz < 2:
        raise ValueError("nz >= 2: the vertical boundary fluxes come from an interior face")
    rng = np.random.default_rng(seed)
    e2n, n2e, sgn = connectivity(nr, nc)
    R, C = np.meshgrid(np.arange(nr), np.arange(nc), indexing="ij")
    ridge = np.exp(-((R - 0.4 * nr) ** 2 + (C - 0.6 * nc) ** 2) / (0.05 * (nr * nr + nc * nc)))
    pD = psi_lo + ridge[None] + 0.3 * rng.random((nz, nr, nc))
    rho = rng.uniform(0.5, 1.5, size=(nz, nr, nc))
    vol = rng.uniform(0.8, 1.2, size=(nr, nc))
    wn = np.zeros((nz + 1, nr, nc))
    if divergent:
        vn = rng.uniform(-1.0, 1.0, size=(nz, nr, 3, nc))
        wn[1:nz] = rng.uniform(-1.0, 1.0, size=(nz - 1, nr, nc))
    else:
        vn = np.stack([_cell_stream_fluxes(rng.uniform(-1, 1, (nr, nc)),
                                           rng.uniform(-1, 1, (nr, nc)), nr, nc)
                       for _ in range(nz)])
    vn, wn = _scale_to_courant(vn, wn, rho, vol, cmax, e2n.shape)
    wn[0] = np.nan
    wn[nz] = np.nan
    return EdgeCase(nr, nc, nz, float(pivbz), pD, vn, wn, rho, vol, e2n, n2e, sgn,
                    meta=dict(seed=seed, divergent=divergent))


def shift_case(nr: int, nc: int, nz: int, colour: int, seed: int = DEFAULT_SEED) -> EdgeCase:
    """Courant number exactly 1 along one edge colour: vn = vol * rho on that
    colour's edges (rho and vol constant per column so the edge's two nodes
    agree), 0 elsewhere, wn = 0; pD uniform in [1, 2)."""
    rng = np.random.default_rng(seed)
    e2n, n2e, sgn = connectivity(nr, nc)
    pD = rng.uniform(1.0, 2.0, size=(nz, nr, nc))
    rho = np.full((nz, nr, nc), 1.0)
    vol = np.full((nr, nc), 1.0)
    vn = np.zeros((nz, nr, 3, nc))
    vn[:, :, colour, :] = 1.0
    wn = np.zeros((nz + 1, nr, nc))
    wn[0] = np.nan
    wn[nz] = np.nan
    return EdgeCase(nr, nc, nz, 0.0, pD, vn, wn, rho, vol, e2n, n2e, sgn,
                    meta=dict(seed=seed, colour=colour))
