"""Pins of the CPU oracle to facts other than the oracle itself.

Each test fixes part of the oracle against a closed form, an invariant of the
scheme, an exact special case, a limit the modified-equation analysis gives,
a convergence order, or a numpy library routine, so that a dropped term, a
wrong sign or index, or a transposed operand fails at least one of them.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from synth import pad, interior

H = 2


def _run(c, iord=None, nonosc=None, nsteps=1, h=H, **kw):
    P = [pad(x, h) for x in (c.psi, c.u, c.v, c.w, c.g)]
    return oracle.run(*P, h=h, iord=c.iord if iord is None else iord,
                      nonosc=c.nonosc if nonosc is None else nonosc, nsteps=nsteps, **kw)


def _const_fields(nx, ny, nz, psi, cx=0.0, cy=0.0, cz=0.0, g=1.0):
    shp = (nz, ny, nx)
    G = np.full(shp, g)
    return synth.Case("c", nx, ny, nz, np.asarray(psi, dtype=np.float64).reshape(shp),
                      np.full(shp, cx * g), np.full(shp, cy * g), np.full(shp, cz * g), G)


# ----------------------------------------------------------------- halos --

def test_halo_fill_matches_numpy_pad():
    """Periodic i-j halo with edge-copied k halo equals numpy.pad(wrap/edge)."""
    rng = np.random.default_rng(5)
    for (nx, ny, nz, h) in [(7, 5, 3, 2), (4, 9, 1, 2), (3, 3, 2, 3)]:
        a = rng.standard_normal((nz, ny, nx))
        f = pad(a, h, fill=np.nan)
        oracle.fill_halo(f, h, kind=0)
        ref = np.pad(np.pad(a, ((0, 0), (h, h), (h, h)), mode="wrap"), ((h, h), (0, 0), (0, 0)),
                     mode="edge")
        assert np.array_equal(f, ref)
        w = pad(a, h, fill=np.nan)
        oracle.fill_halo(w, h, kind=1)
        refw = ref.copy()
        refw[:h] = 0.0
        refw[h + nz - 1:] = 0.0      # the top face k = nz-1/2 and beyond carry no flux
        assert np.array_equal(w, refw)


def test_halo_fill_periodic_k_matches_numpy_pad():
    """With a periodic vertical boundary both field kinds wrap in all three
    directions (numpy.pad(wrap)); no face is closed."""
    rng = np.random.default_rng(6)
    for (nx, ny, nz, h) in [(7, 5, 3, 2), (4, 9, 1, 2), (3, 3, 2, 3)]:
        a = rng.standard_normal((nz, ny, nx))
        ref = np.pad(a, h, mode="wrap")
        for kind in (0, 1):
            f = pad(a, h, fill=np.nan)
            oracle.fill_halo(f, h, kind=kind, kbc=1)
            assert np.array_equal(f, ref)


# ------------------------------------------------ donor cell: Fourier pins --

def _upwind_symbol(c, theta):
    """Amplification factor of the first-order upwind scheme for Courant c."""
    cp, cm = max(c, 0.0), min(c, 0.0)
    return 1.0 - cp * (1.0 - np.exp(-1j * theta)) - cm * (np.exp(1j * theta) - 1.0)


@pytest.mark.parametrize("c,g", [(0.3, 1.0), (-0.45, 1.0), (0.7, 2.0), (-0.2, 0.5)])
@pytest.mark.parametrize("axis", ["x", "y"])
def test_donor_cell_fourier_1d(c, g, axis):
    """Donor cell on a Fourier mode with constant Courant number c = U/G
    multiplies it by the textbook upwind symbol (Listings 4/5 flux)."""
    n = 48
    for m in (1, 3, 7, 23):
        th = 2 * np.pi * m / n
        idx = np.arange(n)
        a = 1.0 - 0.5j
        psi1d = 2.0 + np.real(a * np.exp(1j * th * idx))
        if axis == "x":
            case = _const_fields(n, 1, 1, psi1d[None, None, :], cx=c, g=g)
        else:
            case = _const_fields(1, n, 1, psi1d[None, :, None], cy=c, g=g)
        out = interior(_run(case, iord=1, nonosc=0), H).ravel()
        expect = 2.0 + np.real(a * _upwind_symbol(c, th) * np.exp(1j * th * idx))
        assert np.max(np.abs(out - expect)) < 1e-14


def test_donor_cell_fourier_2d():
    """Constant (cx, cy): the 2D donor-cell symbol is the sum of the 1D ones."""
    n = 32
    idx = np.arange(n)
    for (cx, cy, mx, my) in [(0.3, 0.2, 1, 2), (-0.25, 0.4, 5, 3), (0.1, -0.6, 4, 11)]:
        tx, ty = 2 * np.pi * mx / n, 2 * np.pi * my / n
        mode = np.exp(1j * (tx * idx[None, :] + ty * idx[:, None]))
        psi = 3.0 + np.real(mode)
        case = _const_fields(n, n, 1, psi[None], cx=cx, cy=cy)
        out = interior(_run(case, iord=1, nonosc=0), H)[0]
        sym = 1.0 - (1 - _upwind_symbol(cx, tx)) - (1 - _upwind_symbol(cy, ty))
        expect = 3.0 + np.real(sym * mode)
        assert np.max(np.abs(out - expect)) < 1e-14


# ------------------------------------ antidiffusive pass: linearised symbol --

def test_mpdata_linearised_symbol_1d():
    """Small perturbation delta on a large background B: one iord=2 step
    acts on a Fourier mode like upwind followed by the antidiffusive
    correction 1 + (|c| - c^2)(1 - cos theta), up to O(delta^2 / B)."""
    n = 40
    idx = np.arange(n)
    for c, g in [(0.3, 1.0), (-0.6, 1.0), (0.45, 1.7)]:
        errs = []
        for B in (1e3, 1e4, 1e5):
            worst = 0.0
            for m in (1, 4, 9):
                th = 2 * np.pi * m / n
                psi = B + np.cos(th * idx)
                case = _const_fields(n, 1, 1, psi[None, None, :], cx=c, g=g)
                out = interior(_run(case, iord=2, nonosc=0), H).ravel()
                s1 = _upwind_symbol(c, th)
                s2 = 1.0 + (abs(c) - c * c) * (1.0 - np.cos(th))
                expect = B + np.real(s1 * s2 * np.exp(1j * th * idx))
                worst = max(worst, np.max(np.abs(out - expect)))
            errs.append(worst)
        # the mismatch is the O(delta^2/B) nonlinearity: it falls ~10x per decade of B
        assert errs[2] < 2e-4, errs
        assert errs[1] / errs[2] > 5 and errs[0] / errs[1] > 5, errs


# -------------------------------------------------- conservation / invariants --

@pytest.mark.parametrize("iord,nonosc", [(1, 0), (2, 0), (2, 1), (3, 1)])
def test_mass_conservation(iord, nonosc):
    """sum psi G is conserved (periodic i-j, zero-flux k) in divergent flow."""
    c = synth.random_case(11, 9, 6, seed=7, cmax=0.3)
    P = [pad(x, H) for x in (c.psi, c.u, c.v, c.w, c.g)]
    m0 = oracle.mass(P[0], P[4], H)
    out = oracle.run(*P, h=H, iord=iord, nonosc=nonosc, nsteps=5)
    m1 = oracle.mass(out, P[4], H)
    assert abs(m1 - m0) <= 1e-14 * abs(m0)
    # a non-trivial flow: the field did change
    assert np.max(np.abs(interior(out, H) - c.psi)) > 1e-3


@pytest.mark.parametrize("nz", [1, 5])
def test_constant_preservation(nz):
    """A constant field stays constant in discretely non-divergent flow
    (G-weighted continuity), limiter on, after 100 steps."""
    c = synth.nondivergent_case(12, 10, nz, seed=3, cmax=0.45, const=1.7)
    out = _run(c, iord=2, nonosc=1, nsteps=100)
    assert np.max(np.abs(interior(out, H) - 1.7)) <= 1e-14 * 1.7 * 10


@pytest.mark.parametrize("iord,nonosc", [(1, 0), (2, 0), (2, 1), (3, 1)])
@pytest.mark.parametrize("axis,sign", [("x", 1), ("x", -1), ("y", 1), ("y", -1)])
def test_courant_one_shift_horizontal(iord, nonosc, axis, sign):
    """Courant number exactly 1 (G = 1) moves psi by one cell per step,
    bit for bit, for any number of corrective passes and with the limiter."""
    c = synth.uniform_shift_case(9, 7, 3, axis, sign, seed=11)
    out = interior(_run(c, iord=iord, nonosc=nonosc, nsteps=3), H)
    ax = {"x": 2, "y": 1}[axis]
    assert np.array_equal(out, np.roll(c.psi, 3 * sign, axis=ax))


@pytest.mark.parametrize("iord,nonosc", [(1, 0), (2, 1)])
def test_courant_one_shift_vertical_zero_flux(iord, nonosc):
    """W = +1 on interior faces, 0 on the bottom/top faces (pivbz = 0,
    Listing 7): levels shift up by one, the bottom level empties and the top
    level accumulates what arrives; exactly."""
    c = synth.uniform_shift_case(5, 4, 6, "z", 1, seed=2)
    out = interior(_run(c, iord=iord, nonosc=nonosc, nsteps=1), H)
    p = c.psi
    assert np.array_equal(out[1:-1], p[:-2])
    assert np.array_equal(out[0], np.zeros_like(p[0]))
    assert np.array_equal(out[-1], p[-1] + p[-2])


@pytest.mark.parametrize("iord,nonosc", [(1, 0), (2, 0), (2, 1), (3, 1)])
@pytest.mark.parametrize("sign", [1, -1])
def test_courant_one_shift_vertical_periodic(iord, nonosc, sign):
    """Periodic k, W = +-1 on every face: the levels roll by one per step,
    bit for bit, the top level wrapping to the bottom."""
    c = synth.uniform_shift_case(5, 4, 6, "z", sign, seed=2, kbc=1)
    P = [pad(x, H) for x in (c.psi, c.u, c.v, c.w, c.g)]
    out = interior(oracle.run(*P, h=H, iord=iord, nonosc=nonosc, nsteps=3, kbc=1), H)
    assert np.array_equal(out, np.roll(c.psi, 3 * sign, axis=0))


@pytest.mark.parametrize("iord,nonosc", [(1, 0), (2, 1), (3, 1)])
def test_mass_conservation_periodic_k(iord, nonosc):
    """Periodic k with flux through the top face: sum psi G is conserved."""
    c = synth.random_case(11, 9, 6, seed=8, cmax=0.3, kbc=1)
    assert np.max(np.abs(c.w[-1])) > 0.01  # the top face carries flux
    P = [pad(x, H) for x in (c.psi, c.u, c.v, c.w, c.g)]
    m0 = oracle.mass(P[0], P[4], H)
    out = oracle.run(*P, h=H, iord=iord, nonosc=nonosc, nsteps=5, kbc=1)
    assert abs(oracle.mass(out, P[4], H) - m0) <= 1e-14 * abs(m0)
    assert np.max(np.abs(interior(out, H) - c.psi)) > 1e-3


@pytest.mark.parametrize("nz", [1, 4])
def test_constant_preservation_periodic_k(nz):
    """Periodic k, discretely non-divergent flow with flux through every
    vertical face: a constant stays constant (limiter on, 100 steps)."""
    c = synth.nondivergent_case(12, 10, nz, seed=4, cmax=0.45, const=1.7, kbc=1)
    P = [pad(x, H) for x in (c.psi, c.u, c.v, c.w, c.g)]
    out = oracle.run(*P, h=H, iord=2, nonosc=1, nsteps=100, kbc=1)
    assert np.max(np.abs(interior(out, H) - 1.7)) <= 1e-14 * 1.7 * 10


# --------------------------------------------------- pseudo-velocity limit --

def _taylor_fields(n, nz, gvar):
    """Smooth psi, velocities and G sampled at their staggered positions."""
    d = 2 * np.pi / n
    ii = np.arange(n) * d
    kk = np.arange(nz) * d
    half = d / 2

    def grid(ox=0.0, oy=0.0, oz=0.0):
        Z, Y, X = np.meshgrid(kk + oz, ii + oy, ii + ox, indexing="ij")
        return X, Y, Z

    gf = (lambda X, Y, Z: 1.2 + 0.3 * np.sin(X) * np.cos(Y)) if gvar else (lambda X, Y, Z: 1.6 + 0 * X)
    uf = lambda X, Y, Z: gf(X, Y, Z) * (0.3 + 0.1 * np.sin(X + 2 * Y) * np.cos(Z))
    vf = lambda X, Y, Z: gf(X, Y, Z) * (-0.2 + 0.1 * np.cos(2 * X - Y + Z))
    wf = lambda X, Y, Z: gf(X, Y, Z) * (0.15 + 0.05 * np.sin(X - Y) * np.sin(2 * Z))
    psif = lambda X, Y, Z: np.exp(np.sin(X) + np.cos(Y) + 0.5 * np.sin(Z))
    # log-derivatives of psi
    lx = lambda X, Y, Z: np.cos(X)
    ly = lambda X, Y, Z: -np.sin(Y)
    lz = lambda X, Y, Z: 0.5 * np.cos(Z)
    c = grid()
    fields = dict(psi=psif(*c), g=gf(*c), u=uf(*grid(ox=half)), v=vf(*grid(oy=half)),
                  w=wf(*grid(oz=half)))
    fields["w"][-1] = 0.0

    def limit(face):
        """Continuous antidiffusive velocity at the centre of each face."""
        X, Y, Z = grid(**{dict(u="ox", v="oy", w="oz")[face]: half})
        G = gf(X, Y, Z)
        vel = dict(u=uf(X, Y, Z), v=vf(X, Y, Z), w=wf(X, Y, Z))
        der = dict(u=lx(X, Y, Z), v=ly(X, Y, Z), w=lz(X, Y, Z))
        a = vel[face]
        others = [o for o in "uvw" if o != face]
        cross = sum(vel[o] * half * der[o] for o in others)
        return (np.abs(a) - a * a / G) * half * der[face] - a * cross / G

    return fields, limit


@pytest.mark.parametrize("gvar", [False, True])
def test_pseudo_velocity_taylor_limit(gvar):
    """The pseudo-velocity tends to the modified-equation antidiffusive
    velocity of donor cell (Smolarkiewicz 1984), here with smoothly varying
    U, V, W and G sampled at their staggered positions:
      Ut -> (|U| - U^2/G) dx/2 psi_x/psi - U (V dy/2 psi_y/psi + W dz/2 psi_z/psi)/G
    with absolute error O(dx^3) (relative O(dx^2)).  A factor slip, a
    misplaced average or a wrong face of G leaves an O(dx) relative error
    and breaks the observed order."""
    errs = {"u": [], "v": [], "w": []}
    for n in (16, 32, 64):
        nz = n // 2
        f, limit = _taylor_fields(n, nz, gvar)
        P = [pad(f[k], H) for k in ("psi", "u", "v", "w", "g")]
        got = dict(zip("uvw", (interior(a, H) for a in oracle.pseudo_velocity(*P, h=H))))
        ks = slice(2, nz - 3)
        for face in "uvw":
            errs[face].append(np.max(np.abs(got[face] - limit(face))[ks]))
    for key, e in errs.items():
        orders = [math.log2(e[i] / e[i + 1]) for i in range(len(e) - 1)]
        assert min(orders) > 2.6, (key, e, orders)


# --------------------------------------------- limiter: monotone, positive --

def test_limiter_monotone_rotating_cone():
    """With the limiter, no new extrema: every step stays inside the
    previous step's global range, and inside the local bounds the limiter
    forms; without it the same data overshoots."""
    c = synth.rotation_2d(64, seed=1234)
    P = [pad(x, H) for x in (c.psi, c.u, c.v, c.w, c.g)]
    psi = P[0]
    for s in range(40):
        lo, hi = interior(psi, H).min(), interior(psi, H).max()
        nxt, st = oracle.run(psi, *P[1:], h=H, iord=2, nonosc=1, stages=True)
        ni = interior(nxt, H)
        tol = 4 * np.finfo(float).eps * hi
        assert ni.min() >= lo - tol and ni.max() <= hi + tol
        assert np.all(ni <= interior(st["mx"], H) + tol)
        assert np.all(ni >= interior(st["mn"], H) - tol)
        psi = nxt
    unl = oracle.run(*P, h=H, iord=2, nonosc=0, nsteps=40)
    ui = interior(unl, H)
    assert ui.max() > c.psi.max() + 1e-3 or ui.min() < c.psi.min() - 1e-3


def test_limiter_monotone_step_3d():
    """3D lat-lon case (Gaussian + step, G = cos(lat)): monotone with the
    limiter, overshoot without."""
    c = synth.latlon_3d(40, 32, 10, seed=9)
    lo, hi = c.psi.min(), c.psi.max()
    out = interior(_run(c, iord=2, nonosc=1, nsteps=10), H)
    assert out.min() >= lo - 1e-15 and out.max() <= hi + 4e-16 * hi
    unl = interior(_run(c, iord=2, nonosc=0, nsteps=10), H)
    assert unl.max() > hi + 1e-4 or unl.min() < lo - 1e-4


@pytest.mark.parametrize("nonosc", [0, 1])
def test_positivity(nonosc):
    """psi >= 0 (with exact zeros) stays non-negative when the outflow
    Courant sum is at most 1 (positive-definite scheme)."""
    c = synth.random_case(13, 11, 5, seed=21, cmax=0.3)
    c.psi[c.psi < 0.4] = 0.0
    out = interior(_run(c, iord=2, nonosc=nonosc, nsteps=10), H)
    assert out.min() >= 0.0


# ------------------------------------------------------ convergence order --

def _translation(n, cx=0.25, cy=0.25):
    T = int(round(n / cx))
    x = (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(x, x, indexing="xy")
    psi = 2 + np.sin(2 * np.pi * X) * np.sin(2 * np.pi * Y)
    return _const_fields(n, n, 1, psi[None], cx=cx, cy=cy), T


@pytest.mark.parametrize("iord,nonosc,lo,hi", [(1, 0, 0.4, 1.1), (2, 0, 1.9, 2.3),
                                                 (2, 1, 1.9, 2.3), (3, 0, 2.6, 3.3)])
def test_convergence_order(iord, nonosc, lo, hi):
    """Smooth field translated diagonally (|Cx| + |Cy| = 0.5) for one period;
    the exact solution is the initial field.  Donor cell converges at first
    order, one corrective pass at second, two at third."""
    errs = []
    for n in (16, 32, 64):
        case, T = _translation(n)
        out = interior(_run(case, iord=iord, nonosc=nonosc, nsteps=T), H)[0]
        errs.append(np.sqrt(np.mean((out - case.psi[0]) ** 2)))
    order = math.log2(errs[1] / errs[2])
    assert lo <= order <= hi, (errs, order)


# ------------------------------------------------------------ Table 2 pin --

def test_table2_access_counts():
    """The paper's main-memory access count (Table 2) with its node and edge
    counts: the counting method of the traffic model."""
    import bench
    rows = {}
    with open(__import__("os").path.join(__import__("os").path.dirname(__file__), "golden",
                                         "table2_accesses.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split("=")
                rows[k.strip()] = int(v)
    nodes, edges = rows["nodes"], rows["edges"]
    assert bench.table2_accesses(nodes, edges, fused=False) == rows["without_fusion"]
    assert bench.table2_accesses(nodes, edges, fused=True) == rows["with_fusion"]


# ------------------------------------------------- tangent-linear model --

def test_tlm_matches_central_differences():
    """The dual-number tangent-linear model agrees with central differences
    of the forward step (directions chosen to cross no branch)."""
    c = synth.random_case(8, 7, 4, seed=31, cmax=0.25, psi_lo=0.5, psi_hi=1.5)
    rng = np.random.default_rng(32)
    P = [pad(x, H) for x in (c.psi, c.u, c.v, c.w, c.g)]
    d = [pad(rng.standard_normal(c.psi.shape), H) for _ in range(4)]
    d[3][H + c.nz - 1] = 0.0
    for nonosc in (0, 1):
        base, tl = oracle.tlm(*P, *d, h=H, iord=2, nonosc=nonosc, nsteps=2)
        eps = 1e-6
        plus = oracle.run(*(p + eps * q for p, q in zip(P[:4], d)), P[4], h=H, iord=2,
                          nonosc=nonosc, nsteps=2)
        minus = oracle.run(*(p - eps * q for p, q in zip(P[:4], d)), P[4], h=H, iord=2,
                           nonosc=nonosc, nsteps=2)
        fd = (plus - minus) / (2 * eps)
        ti, fi = interior(tl, H), interior(fd, H)
        assert np.max(np.abs(ti - fi)) <= 1e-6 * np.max(np.abs(ti))
        assert np.array_equal(interior(base, H), interior(oracle.run(*P, h=H, iord=2,
                                                                     nonosc=nonosc, nsteps=2), H))


@pytest.mark.parametrize("c", [0.4, -0.4, 0.15, -0.7])
@pytest.mark.parametrize("axis", ["x", "y", "z"])
def test_limiter_inactive_on_smooth_monotone_data(axis, c):
    """On smooth data the non-oscillatory bounds never bind: every beta is
    at least 1, so the limited step equals the unlimited one bit for bit
    (x, y: a well-resolved sine, everywhere; z: a monotone profile, away
    from the closed top and bottom).  Bounds drawn from too small a
    neighbourhood would bind here."""
    n = 64
    if axis == "z":
        nz = 24
        psi = (2.0 + (np.arange(nz) + 0.5) / nz)[:, None, None] * np.ones((nz, 3, 4))
        shp = psi.shape
        u, v, w = np.zeros(shp), np.zeros(shp), np.full(shp, c)
        w[-1] = 0.0
        sl = (slice(3, nz - 3),)
    else:
        p1 = 2.0 + np.sin(2 * np.pi * np.arange(n) / n)
        psi = p1[None, None, :] * np.ones((1, 3, 1)) if axis == "x" else p1[None, :, None] * np.ones((1, 1, 3))
        shp = psi.shape
        u = np.full(shp, c) if axis == "x" else np.zeros(shp)
        v = np.full(shp, c) if axis == "y" else np.zeros(shp)
        w = np.zeros(shp)
        sl = (slice(None),)
    P = [pad(a, H) for a in (psi, u, v, w, np.ones(shp))]
    lim = interior(oracle.run(*P, h=H, iord=2, nonosc=1), H)
    unl = interior(oracle.run(*P, h=H, iord=2, nonosc=0), H)
    assert np.array_equal(lim[sl], unl[sl])
    assert not np.array_equal(unl, psi)


# ---------------------------------------------------------------- adjoint --

def _inner(a, b, h=H):
    return float(np.sum(interior(a, h) * interior(b, h)))


@pytest.mark.parametrize("iord,nonosc,nsteps,kbc", [
    (1, 0, 1, 0), (2, 0, 1, 0), (2, 1, 1, 0), (2, 1, 3, 0), (2, 0, 3, 0), (3, 0, 1, 0),
    (3, 1, 1, 0), (3, 1, 2, 0), (4, 1, 1, 0), (1, 0, 1, 1), (2, 1, 2, 1), (3, 1, 1, 1)])
def test_adjoint_dot_product_against_tlm(iord, nonosc, nsteps, kbc):
    """<L dx, dy> = <dx, L^T dy> with L the dual-number tangent-linear model
    (an independent derivative of the forward code) and L^T the hand-written
    reverse mode, to 1e-12 relative (kbc 1: periodic k, open top face)."""
    c = synth.random_case(9, 8, 5, seed=41, cmax=0.25, psi_lo=0.2, psi_hi=1.5, kbc=kbc)
    rng = np.random.default_rng(42)
    P = [pad(x, H) for x in (c.psi, c.u, c.v, c.w, c.g)]
    dx = [pad(rng.standard_normal(c.psi.shape), H) for _ in range(4)]
    dy = pad(rng.standard_normal(c.psi.shape), H)
    _, tl = oracle.tlm(*P, *dx, h=H, iord=iord, nonosc=nonosc, nsteps=nsteps, kbc=kbc)
    lhs = _inner(tl, dy)
    pb, ub, vb, wb = oracle.adjoint(*P, dy, h=H, iord=iord, nonosc=nonosc, nsteps=nsteps,
                                    kbc=kbc)
    rhs = _inner(dx[0], pb) + _inner(dx[1], ub) + _inner(dx[2], vb) + _inner(dx[3], wb)
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1e-30), (lhs, rhs)


def test_adjoint_dot_product_on_rotating_cone():
    """The same identity on the cone configuration: exact ties (flat
    background, zero velocities outside the rotation radius) exercise the
    branch rules shared by the tangent and the adjoint."""
    c = synth.rotation_2d(24, radius_frac=0.4, cone_radius=4.0, cone_offset=5.0)
    rng = np.random.default_rng(7)
    P = [pad(x, H) for x in (c.psi, c.u, c.v, c.w, c.g)]
    dx = [pad(rng.standard_normal(c.psi.shape), H) for _ in range(4)]
    dx[3][:] = 0.0
    dy = pad(rng.standard_normal(c.psi.shape), H)
    _, tl = oracle.tlm(*P, *dx, h=H, iord=2, nonosc=1, nsteps=4)
    pb, ub, vb, wb = oracle.adjoint(*P, dy, h=H, iord=2, nonosc=1, nsteps=4)
    lhs = _inner(tl, dy)
    rhs = _inner(dx[0], pb) + _inner(dx[1], ub) + _inner(dx[2], vb)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


@pytest.mark.parametrize("iord", [2, 3])
def test_adjoint_gradient_matches_central_differences(iord):
    """dJ/dx from the reverse mode against central differences of
    J = sum (psi_T - psi_obs)^2 G, in random directions of psi_0 and of the
    Courant fields (relative error <= 1e-6, h = 1e-6 |x|)."""
    c = synth.random_case(8, 7, 4, seed=51, cmax=0.25, psi_lo=0.3, psi_hi=1.4)
    rng = np.random.default_rng(52)
    P = [pad(x, H) for x in (c.psi, c.u, c.v, c.w, c.g)]
    obs = P[0] + pad(0.05 * rng.standard_normal(c.psi.shape), H)

    def J(p, u, v, w):
        out = oracle.run(p, u, v, w, P[4], h=H, iord=iord, nonosc=1, nsteps=3)
        return float(np.sum(interior((out - obs) ** 2 * P[4], H)))

    out = oracle.run(*P, h=H, iord=iord, nonosc=1, nsteps=3)
    dJ = 2.0 * (out - obs) * P[4]
    pb, ub, vb, wb = oracle.adjoint(*P, dJ, h=H, iord=iord, nonosc=1, nsteps=3)
    grads = [pb, ub, vb, wb]
    for trial in range(6):
        d = [pad(rng.standard_normal(c.psi.shape), H) for _ in range(4)]
        d[3][H + c.nz - 1] = 0.0
        x = P[:4]
        eps = 1e-6 * max(np.max(np.abs(interior(a, H))) for a in x)
        jp = J(*(a + eps * b for a, b in zip(x, d)))
        jm = J(*(a - eps * b for a, b in zip(x, d)))
        fd = (jp - jm) / (2 * eps)
        an = sum(_inner(gr, dd) for gr, dd in zip(grads, d))
        assert abs(fd - an) <= 1e-6 * abs(an), (trial, fd, an)
