"""Pins of the oracle's edge-based flux stages (upwind flux on edges,
vertical upwind flux, flux divergence, advance: Sec. 5, Listings 5, 7, 8)
and of the patch generator, to facts other than the oracle itself:

* the connectivity of the periodic triangular patch (six distinct edges per
  node, every edge in exactly two nodes' lists with opposite signs);
* exact mass conservation with closed vertical boundaries (pivbz = 0);
* with pivbz = 1 (boundary flux = the adjacent interior face's) a uniform
  field in a uniform vertical flow passes through unchanged, while with
  pivbz = 0 the closed ends fill and drain by the closed-form amounts;
* Courant number 1 along each edge colour, both signs: an exact shift;
* the textbook upwind amplification factor on a Fourier mode along a colour;
* constant preservation in a flow with zero divergence at every node;
* positivity below Courant number 1;
* the same answer, bit for bit, under a random renumbering of nodes and
  edges (the oracle reads the mesh only through its tables).
"""
import numpy as np
import pytest

import oracle
from synth import octahedral as octa


def test_connectivity_of_the_periodic_patch():
    for nr, nc in [(3, 4), (5, 7), (8, 8)]:
        e2n, n2e, sgn = octa.connectivity(nr, nc)
        N, E = nr * nc, 3 * nr * nc
        assert e2n.shape == (E, 2) and n2e.shape == (N, 6)
        for n in range(N):
            assert len(set(n2e[n])) == 6
            for j in range(6):
                e = n2e[n, j]
                assert e2n[e, 0 if sgn[n, j] > 0 else 1] == n
        count = np.zeros(E, dtype=int)
        for n in range(N):
            for j in range(6):
                count[n2e[n, j]] += 1
        assert np.all(count == 2)
        # the second node of colour c's edge at (r, col) is (r, col) + offset_c
        for col, (dr, dc) in enumerate(octa.EDGE_OFFSETS):
            e = octa.edge_id(1, col, 2, nr, nc)
            assert e2n[e, 1] == octa.node_id(1 + dr, 2 + dc, nr, nc)


@pytest.mark.parametrize("divergent", [True, False])
def test_mass_conservation_closed(divergent):
    c = octa.edge_case(9, 11, 6, seed=3, pivbz=0.0, divergent=divergent)
    m0 = oracle.edge_mass(c, c.pD)
    p = oracle.edge_run(c, nsteps=5)
    assert abs(oracle.edge_mass(c, p) - m0) <= 1e-14 * m0


@pytest.mark.parametrize("pivbz", [0.0, 1.0])
def test_uniform_vertical_flow_through_the_boundaries(pivbz):
    """pD = 2, W = w on every interior face, no horizontal flow, vol rho = 1:
    every interior fluz is 2w.  With pivbz = 1 the boundary faces carry 2w
    too and nothing changes; with pivbz = 0 the bottom level loses 2w and
    the top level gains it, the others stay."""
    c = octa.edge_case(4, 5, 5, seed=1, pivbz=pivbz)
    c.pD[:] = 2.0
    c.vn[:] = 0.0
    c.wn[1:c.nz] = 0.25
    c.rho[:] = 1.0
    c.vol[:] = 1.0
    p = oracle.edge_run(c)
    if pivbz == 1.0:
        assert np.array_equal(p, c.pD)
    else:
        assert np.all(p[0] == 2.0 - 0.5) and np.all(p[-1] == 2.0 + 0.5)
        assert np.all(p[1:-1] == 2.0)


@pytest.mark.parametrize("colour", [0, 1, 2])
@pytest.mark.parametrize("sign", [1, -1])
def test_courant_one_shift_along_each_colour(colour, sign):
    c = octa.shift_case(6, 7, 3, colour, seed=colour)
    c.vn *= sign
    p = oracle.edge_run(c, nsteps=2)
    dr, dc = octa.EDGE_OFFSETS[colour]
    expect = np.roll(np.roll(c.pD, 2 * sign * dr, axis=1), 2 * sign * dc, axis=2)
    assert np.array_equal(p, expect)


@pytest.mark.parametrize("colour", [0, 1, 2])
@pytest.mark.parametrize("C", [0.3, -0.6])
def test_upwind_symbol_on_a_fourier_mode(colour, C):
    """vn = C vol rho on one colour: along that colour the step is the 1D
    upwind scheme, whose amplification factor is 1 - |C| + |C| e^{-i s theta}
    (s the sign of C) for a mode exp(i theta m) that one step along the
    colour moves by theta: m = c for colour 0 (0, 1), m = r for colour 1
    (1, 0) and for colour 2 (1, 1)."""
    n = 12
    c = octa.shift_case(n, n, 2, colour, seed=2)
    c.vn *= C
    theta = 2 * np.pi * 3 / n
    R, Cc = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    m = Cc if colour == 0 else R
    c.pD[:] = 1.0 + 0.5 * np.cos(theta * m)[None]
    p = oracle.edge_run(c)
    s = 1.0 if C > 0 else -1.0
    a = abs(C)
    amp = 1 - a + a * np.exp(-1j * s * theta)
    expect = 1.0 + 0.5 * np.real(amp * np.exp(1j * theta * m))
    assert np.max(np.abs(p - expect[None])) <= 1e-14


def test_constant_preservation_in_nondivergent_flow():
    c = octa.edge_case(10, 9, 4, seed=8, divergent=False)
    c.pD[:] = 1.7
    p = oracle.edge_run(c, nsteps=10)
    assert np.max(np.abs(p - 1.7)) <= 1e-14


@pytest.mark.parametrize("pivbz", [0.0, 1.0])
def test_positivity_below_courant_one(pivbz):
    c = octa.edge_case(12, 10, 6, seed=5, pivbz=pivbz, cmax=0.95, psi_lo=0.0)
    c.pD[c.pD < 0.5] = 0.0
    p = c.pD
    for _ in range(6):
        p = oracle.edge_run(c, pD=p)
        assert p.min() >= 0.0


def test_renumbering_gives_the_same_answer():
    """Relabel nodes and edges by random permutations (an unstructured
    numbering of the same mesh): the advanced field, mapped back, is equal
    bit for bit."""
    c = octa.edge_case(7, 9, 4, seed=11, pivbz=1.0)
    ref = oracle.edge_run(c, nsteps=2)
    rng = np.random.default_rng(0)
    N, E = c.nnodes, c.nedges
    pn = rng.permutation(N)          # new id of node n
    pe = rng.permutation(E)          # new id of edge e
    inv_n = np.argsort(pn)
    inv_e = np.argsort(pe)
    u = octa.EdgeCase(c.nr, c.nc, c.nz, c.pivbz,
                      c.pD.reshape(c.nz, N)[:, inv_n],
                      c.vn.reshape(c.nz, E)[:, inv_e],
                      c.wn.reshape(c.nz + 1, N)[:, inv_n],
                      c.rho.reshape(c.nz, N)[:, inv_n],
                      c.vol.reshape(N)[inv_n],
                      pn[c.e2n[inv_e]], pe[c.n2e[inv_n]], c.n2e_sign[inv_n])
    got = oracle.edge_run(u, nsteps=2)
    assert np.array_equal(got[:, pn], ref.reshape(c.nz, N))


@pytest.mark.parametrize("sign", [1, -1])
def test_vertical_courant_one_shift_with_closed_ends(sign):
    """W = +-1 on every interior face, vol rho = 1, pD in [1, 2): each level
    takes its upwind neighbour's value; the closed end the flow runs into
    keeps its own value plus its neighbour's, the one it leaves empties."""
    c = octa.shift_case(4, 5, 5, 0, seed=9)
    c.vn[:] = 0.0
    c.wn[1:c.nz] = float(sign)
    p = oracle.edge_run(c)
    q = c.pD
    if sign > 0:
        assert np.array_equal(p[1:-1], q[:-2])
        assert np.array_equal(p[-1], q[-1] + q[-2]) and np.all(p[0] == 0.0)
    else:
        assert np.array_equal(p[1:-1], q[2:])
        assert np.array_equal(p[0], q[0] + q[1]) and np.all(p[-1] == 0.0)


def test_open_boundaries_copy_the_adjacent_face():
    """pD = 1, vol rho = 1, W_k = k/10 on the interior faces, pivbz = 1:
    every interior fluz equals W_k, the boundary faces copy their neighbour,
    so level k changes by -(W_{k+1} - W_k) inside and not at all at the two
    ends."""
    c = octa.edge_case(3, 4, 6, seed=2, pivbz=1.0)
    c.pD[:] = 1.0
    c.vn[:] = 0.0
    c.rho[:] = 1.0
    c.vol[:] = 1.0
    W = np.arange(c.nz + 1) / 10.0
    c.wn[1:c.nz] = W[1:c.nz, None, None]
    p = oracle.edge_run(c)
    assert np.all(p[0] == 1.0) and np.all(p[-1] == 1.0)
    for k in range(1, c.nz - 1):
        assert np.all(p[k] == 1.0 - (W[k + 1] - W[k]))
