"""Pins of the oracle's corrective-pass options to facts other than the
oracle: DFL (the divergent-flow term), ABS (signed fields) and IGA (the
infinite gauge).

* DFL: second-order convergence in divergent flows against exact solutions
  by characteristics (1D along each axis, G constant and varying; 2D
  separable flows), where the basic scheme falls to first order; no effect
  in a discretely non-divergent flow; exact mass conservation.
* IGA: the basic scheme applied to psi + c, minus c, tends to IGA as 1/c;
  IGA is linear in psi and gauge invariant; second order on a signed wave;
  no new extrema with the limiter on a signed step.
* ABS: equal, bit for bit, to the basic scheme where psi >= 0; odd in psi,
  bit for bit; converges on a signed wave; no new extrema with the limiter
  on a signed step, where the basic scheme blows up.
"""
import numpy as np
import pytest

import oracle
import synth
from synth import interior, pad

H = 2
DFL, ABS, IGA = oracle.DFL, oracle.ABS, oracle.IGA


def _run(psi, u, v, w, g, nsteps=1, opts=0, iord=2, nonosc=0, kbc=0):
    P = [pad(x, H) for x in (psi, u, v, w, g)]
    return interior(oracle.run(*P, h=H, iord=iord, nonosc=nonosc, nsteps=nsteps, kbc=kbc,
                               opts=opts), H)


def _orders(errs):
    return [float(np.log2(errs[i] / errs[i + 1])) for i in range(len(errs) - 1)]


def _foot(x, vel, t, m=400):
    """Foot X of the characteristic dX/ds = vel(X) through x at time t
    (classical RK4 backwards in m steps: local error ~ (t/m)^5, far below
    the errors measured here)."""
    X = np.array(x, dtype=np.float64)
    ds = t / m
    for _ in range(m):
        k1 = -vel(X)
        k2 = -vel(X + 0.5 * ds * k1)
        k3 = -vel(X + 0.5 * ds * k2)
        k4 = -vel(X + ds * k3)
        X = X + ds / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
    return X


# ------------------------------------------------------ divergent flow --

C0, AMP, TEND = 0.4, 0.5, 0.6


def _axis_fields(n, axis, Uf, Gc, psi):
    """1D data along one axis of a 3D grid (the other extents 1)."""
    shp = {"x": (1, 1, n), "y": (1, n, 1), "z": (n, 1, 1)}[axis]
    z = np.zeros(shp)
    vel = {"x": 0, "y": 1, "z": 2}[axis]
    f = [z, z, z]
    f[vel] = Uf.reshape(shp)
    return psi.reshape(shp), f[0], f[1], f[2], Gc.reshape(shp)


def _dfl_errors_1d(axis, opts, gvar, ns):
    b = 0.3 if gvar else 0.0
    Ucont = lambda x: C0 * (1 + AMP * np.sin(2 * np.pi * x))
    Gcont = lambda x: 1 + b * np.cos(2 * np.pi * x)
    ucont = lambda x: Ucont(x) / Gcont(x)
    psi0 = lambda x: 0.5 + np.exp(-((np.mod(x, 1.0) - 0.5) / 0.12) ** 2)
    errs = []
    for n in ns:
        xc = (np.arange(n) + 0.5) / n
        xf = (np.arange(n) + 1.0) / n
        nsteps = int(round(TEND * n))
        t = nsteps / n  # dt = dx: Courant number U/G is the speed in cells per step
        got = _run(*_axis_fields(n, axis, Ucont(xf), Gcont(xc), psi0(xc)), nsteps=nsteps,
                   opts=opts, kbc=1 if axis == "z" else 0).ravel()
        X = _foot(xc, ucont, t)
        # G psi u is constant along a characteristic of the steady flow
        exact = Gcont(X) * psi0(X) * ucont(X) / ucont(xc) / Gcont(xc)
        errs.append(float(np.sqrt(np.mean((got - exact) ** 2))))
    return errs


@pytest.mark.parametrize("gvar", [False, True])
@pytest.mark.parametrize("axis", ["x", "y", "z"])
def test_dfl_restores_second_order_in_divergent_flow(axis, gvar):
    """Steady divergent flow U = 0.4 (1 + 0.5 sin 2 pi x) (and G = 1 + 0.3
    cos 2 pi x), refined at fixed Courant number against the exact solution:
    with the term the order is 2, without it it decays towards 1 (the
    donor cell's divergence error is left uncancelled).  The z case runs
    with periodic k."""
    ns = (128, 256, 512)
    with_term = _orders(_dfl_errors_1d(axis, DFL, gvar, ns))
    without = _orders(_dfl_errors_1d(axis, 0, gvar, ns))
    assert min(with_term) >= 1.9, with_term
    assert without[-1] <= 1.3, without


def _dfl_errors_2d(plane, opts, ns):
    """Separable divergent flow in the x-y or x-z plane, G = 1: u(x), v(y)
    (or w(z)); the exact solution is psi0 at the feet of the two 1D
    characteristics times u(X) v(Y) / (u(x) v(y))."""
    c0 = 0.3
    ua = lambda x: c0 * (1 + AMP * np.sin(2 * np.pi * x))
    va = lambda y: c0 * (1 + AMP * np.cos(2 * np.pi * y))
    psi0 = lambda x, y: 0.5 + np.exp(-((np.mod(x, 1) - 0.5) ** 2 + (np.mod(y, 1) - 0.4) ** 2)
                                     / 0.15 ** 2)
    errs = []
    for n in ns:
        c = (np.arange(n) + 0.5) / n
        f = (np.arange(n) + 1.0) / n
        nsteps = int(round(TEND * n))
        t = nsteps / n
        Y2, X2 = np.meshgrid(c, c, indexing="ij")   # [second axis][x]
        U = np.broadcast_to(ua(f)[None, :], (n, n))
        V = np.broadcast_to(va(f)[:, None], (n, n))
        zero = np.zeros((n, n))
        if plane == "xy":
            shp = (1, n, n)
            fields = (psi0(X2, Y2), U, V, zero, np.ones((n, n)))
            kbc = 0
        else:
            shp = (n, 1, n)
            fields = (psi0(X2, Y2), U, zero, V, np.ones((n, n)))
            kbc = 1
        got = _run(*[np.ascontiguousarray(a).reshape(shp) for a in fields], nsteps=nsteps,
                   opts=opts, kbc=kbc).reshape(n, n)
        Xf, Yf = _foot(c, ua, t)[None, :], _foot(c, va, t)[:, None]  # separable flow
        exact = psi0(Xf, Yf) * ua(Xf) * va(Yf) / (ua(X2) * va(Y2))
        errs.append(float(np.sqrt(np.mean((got - exact) ** 2))))
    return errs


def check_dfl_2d(plane, ns=(32, 64, 128)):
    with_term = _orders(_dfl_errors_2d(plane, DFL, ns))
    without = _orders(_dfl_errors_2d(plane, 0, ns))
    assert with_term[-1] >= 1.85, with_term
    assert without[-1] <= 1.6, without


@pytest.mark.parametrize("plane", ["xy", "xz"])
def test_dfl_second_order_in_2d_divergent_flow(plane):
    """The divergence of every face's two cells includes the cross
    directions' Courant differences: a 2D separable divergent flow converges
    at second order with the term only."""
    check_dfl_2d(plane)


@pytest.mark.parametrize("nonosc", [0, 1])
def test_dfl_vanishes_in_nondivergent_flow(nonosc):
    """In a discretely non-divergent flow every cell's divergence is zero to
    rounding: the term changes the step by rounding only."""
    c = synth.nondivergent_case(14, 11, 6, seed=8, const=None)
    a = _run(c.psi, c.u, c.v, c.w, c.g, nsteps=3, opts=DFL, nonosc=nonosc)
    b = _run(c.psi, c.u, c.v, c.w, c.g, nsteps=3, opts=0, nonosc=nonosc)
    assert np.max(np.abs(a - b)) <= 1e-13 * np.max(np.abs(b))
    assert np.max(np.abs(a - b)) > 0.0 or nonosc  # the term is evaluated


@pytest.mark.parametrize("opts", [DFL, DFL | ABS])
@pytest.mark.parametrize("kbc", [0, 1])
def test_variant_mass_conservation(opts, kbc):
    """The options change face fluxes only: mass is conserved to rounding in
    a divergent random flow."""
    c = synth.random_case(13, 9, 5, seed=41, cmax=0.25, kbc=kbc)
    for nonosc in (0, 1):
        out = _run(c.psi, c.u, c.v, c.w, c.g, nsteps=4, opts=opts, nonosc=nonosc, kbc=kbc)
        m0 = float(np.sum(c.psi * c.g))
        assert abs(float(np.sum(out * c.g)) - m0) <= 1e-13 * m0


# ------------------------------------------------------- infinite gauge --

@pytest.mark.parametrize("nonosc", [0, 1])
def test_iga_is_the_limit_of_a_growing_gauge(nonosc):
    """basic(psi + c) - c -> IGA(psi) as c grows, with error proportional to
    1/c (non-divergent flow, so the donor pass keeps the constant exactly):
    the pseudo-flux limits cA -> (psi_R - psi_L)/2 and cB -> N/8 are the
    scheme's own."""
    c = synth.nondivergent_case(12, 10, 6, seed=3, const=None, cmax=0.4)
    iga = _run(c.psi, c.u, c.v, c.w, c.g, opts=IGA, nonosc=nonosc)
    base = _run(c.psi, c.u, c.v, c.w, c.g, nonosc=nonosc)
    errs = []
    for cc in (1e3, 1e4, 1e5):
        got = _run(c.psi + cc, c.u, c.v, c.w, c.g, nonosc=nonosc) - cc
        errs.append(float(np.max(np.abs(got - iga))))
    assert 9.5 <= errs[0] / errs[1] <= 10.5, errs
    assert 9.0 <= errs[1] / errs[2] <= 11.0, errs
    assert errs[2] <= 2e-5 * np.max(np.abs(base - iga)), errs


def test_iga_is_linear_and_gauge_invariant():
    c = synth.nondivergent_case(12, 10, 6, seed=4, const=None, cmax=0.4)
    rng = np.random.default_rng(12)
    p2 = rng.standard_normal(c.psi.shape)
    run = lambda p, nonosc=0: _run(p, c.u, c.v, c.w, c.g, nsteps=2, opts=IGA, nonosc=nonosc)
    a, b = run(c.psi), run(p2)
    assert np.max(np.abs(run(2.0 * c.psi - 3.0 * p2) - (2.0 * a - 3.0 * b))) <= 1e-13
    for nonosc in (0, 1):
        ref = run(c.psi, nonosc)
        assert np.max(np.abs(run(c.psi + 7.0, nonosc) - 7.0 - ref)) <= 1e-13


def _wave_errors(opts, axis, ns, C=0.4):
    """A signed sine translated by a constant Courant number C along one axis
    for half the domain; exact solution the shifted sine."""
    errs = []
    for n in ns:
        x = (np.arange(n) + 0.5) / n
        nsteps = int(n * 0.5 / C)
        fields = _axis_fields(n, axis, np.full(n, C), np.ones(n), np.sin(2 * np.pi * x))
        got = _run(*fields, nsteps=nsteps, opts=opts, kbc=1 if axis == "z" else 0).ravel()
        exact = np.sin(2 * np.pi * (x - nsteps * C / n))
        errs.append(float(np.sqrt(np.mean((got - exact) ** 2))))
    return errs


@pytest.mark.parametrize("axis", ["x", "y", "z"])
def test_iga_second_order_on_signed_wave(axis):
    o = _orders(_wave_errors(IGA, axis, (32, 64, 128, 256)))
    assert min(o) >= 1.9, o


def _signed_step(nx, ny, nz):
    i = np.arange(nx)[None, None, :]
    j = np.arange(ny)[None, :, None]
    inside = (i > nx // 4) & (i < 3 * nx // 4) & (j > ny // 4) & (j < 3 * ny // 4)
    return np.where(inside, 1.0, -1.0) * np.ones((nz, 1, 1))


@pytest.mark.parametrize("opts", [IGA, ABS])
def test_limited_signed_step_makes_no_new_extrema(opts):
    """A signed step (+1 inside, -1 outside) in a non-divergent flow, 30
    limited steps: every step stays within [-1, 1] and within the local
    bounds of the previous state."""
    c = synth.nondivergent_case(32, 28, 4, seed=5, const=None, cmax=0.4)
    p = _signed_step(32, 28, 4)
    for _ in range(30):
        nxt = _run(p, c.u, c.v, c.w, c.g, opts=opts, nonosc=1)
        assert nxt.max() <= 1.0 + 4e-16 and nxt.min() >= -1.0 - 4e-16
        p = nxt


def test_basic_scheme_blows_up_on_the_signed_step():
    """What the signed-field options are for: the basic scheme's A ratio has
    psi_R + psi_L in its denominator, which vanishes across a sign change."""
    c = synth.nondivergent_case(32, 28, 4, seed=5, const=None, cmax=0.4)
    p = _signed_step(32, 28, 4)
    worst = 0.0
    for _ in range(30):
        p = _run(p, c.u, c.v, c.w, c.g, opts=0, nonosc=1)
        worst = max(worst, float(np.nanmax(np.abs(p))))
    assert not worst <= 1.5


# -------------------------------------------------------- signed fields --

@pytest.mark.parametrize("iord,nonosc", [(2, 0), (2, 1), (3, 0), (3, 1)])
def test_abs_equals_basic_for_nonnegative_fields(iord, nonosc):
    c = synth.random_case(13, 11, 5, seed=4, cmax=0.3)
    a = _run(c.psi, c.u, c.v, c.w, c.g, nsteps=2, opts=ABS, iord=iord, nonosc=nonosc)
    b = _run(c.psi, c.u, c.v, c.w, c.g, nsteps=2, opts=0, iord=iord, nonosc=nonosc)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("iord,nonosc", [(2, 0), (2, 1), (3, 0), (3, 1)])
@pytest.mark.parametrize("kbc", [0, 1])
def test_abs_is_odd_in_psi(iord, nonosc, kbc):
    """|psi| makes the pseudo-velocities even in psi and the fluxes odd; the
    limiter's bounds and betas swap roles under psi -> -psi, and taking the
    factors by the flux's direction makes the limited step odd too: bit
    for bit."""
    c = synth.random_case(13, 11, 5, seed=6, cmax=0.3, kbc=kbc)
    p = np.random.default_rng(7).uniform(-1.0, 1.0, c.psi.shape)
    a = _run(p, c.u, c.v, c.w, c.g, nsteps=2, opts=ABS, iord=iord, nonosc=nonosc, kbc=kbc)
    b = _run(-p, c.u, c.v, c.w, c.g, nsteps=2, opts=ABS, iord=iord, nonosc=nonosc, kbc=kbc)
    assert np.array_equal(a, -b)


def test_abs_converges_on_signed_wave():
    """Away from its zero crossings the signed variant is the basic scheme;
    at them A and B saturate at +-1, so on a sine the error falls at first
    order (where the basic scheme does not converge at all)."""
    errs = _wave_errors(ABS, "x", (32, 64, 128, 256))
    o = _orders(errs)
    assert min(o) >= 0.85, o
    assert errs[-1] <= 0.015
