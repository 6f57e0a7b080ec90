"""GPU parity with a periodic vertical boundary (k_bc = MPDATA_K_PERIODIC):
the k neighbours of the levels 0 and nz-1 are each other, and every
vertical face, the one above level nz-1 included, carries flux.  The
library against the oracle run with kbc = 1 on the same seeded inputs:
forward steps (both kernels, both precisions, every scheme), the halo
fill, mass conservation with flux through the top face, the exact vertical
shift at Courant number 1, and the adjoint (direct and through autograd).
Tolerances are those of the zero-flux tests: the periodic boundary
changes which neighbours enter a formula, not the formulas."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import rel_err, rounded_inputs, run_library, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KP = 1
F64_TOL = 1e-12
F32_TOL = 2e-5
ADJ_TOL = 1e-11
H = 2
VARIANTS = {"fused": 0, "staged": 1}

# nz = 1 and 2 make a level its own (or its only) vertical neighbour; the
# others span several tiles with ragged edges and, for nz >= 9, several
# level chunks of the fused kernel
SHAPES = [(5, 7, 1), (13, 11, 2), (9, 8, 3), (37, 29, 9), (16, 16, 4), (70, 12, 5), (33, 17, 40)]
SCHEMES = [(1, 0), (2, 0), (2, 1), (3, 0), (3, 1)]


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_06094_b300 import build
    build.build()


def _oracle(case, iord, nonosc, nsteps):
    P = [synth.pad(x, case.halo) for x in (case.psi, case.u, case.v, case.w, case.g)]
    return oracle.run(*P, h=case.halo, iord=iord, nonosc=nonosc, nsteps=nsteps, kbc=KP)


def _wrap_all(inner, h):
    return np.pad(inner, ((h, h), (h, h), (h, h)), mode="wrap")


@pytest.mark.parametrize("variant", list(VARIANTS))
@pytest.mark.parametrize("shape", SHAPES, ids=[f"{a}x{b}x{c}" for a, b, c in SHAPES])
@pytest.mark.parametrize("iord,nonosc", SCHEMES)
def test_periodic_k_f64_parity(shape, iord, nonosc, variant):
    nx, ny, nz = shape
    c = synth.random_case(nx, ny, nz, seed=nx * 1000 + ny * 10 + nz + 7, cmax=0.3, kbc=KP)
    for nsteps in (1, 3):
        ref = _oracle(c, iord, nonosc, nsteps)
        got = run_library(c, torch.float64, iord, nonosc, nsteps, variant=VARIANTS[variant],
                          k_bc=KP)
        assert rel_err(got, ref) <= F64_TOL * nsteps, (shape, nsteps)
        # the result's halo is the periodic image of its interior in i, j and k
        assert np.array_equal(got, _wrap_all(synth.interior(got, c.halo), c.halo))


@pytest.mark.parametrize("variant", list(VARIANTS))
@pytest.mark.parametrize("shape", [(13, 11, 2), (37, 29, 9), (16, 16, 1), (40, 20, 33)])
@pytest.mark.parametrize("iord,nonosc", [(1, 0), (2, 0), (2, 1), (3, 1)])
def test_periodic_k_f32_against_f64_oracle(shape, iord, nonosc, variant):
    nx, ny, nz = shape
    c = rounded_inputs(synth.random_case(nx, ny, nz, seed=98, cmax=0.3, kbc=KP), torch.float32)
    ref = _oracle(c, iord, nonosc, 2)
    got = run_library(c, torch.float32, iord, nonosc, 2, variant=VARIANTS[variant], k_bc=KP)
    assert rel_err(got, ref) <= 2 * F32_TOL


def test_periodic_k_latlon_256_f64():
    """The 3D FP64 grid at full size (256x256x64) with the lat-lon flow and a
    vertical velocity that crosses the top face: both kernels, 2 steps."""
    c = synth.latlon_3d(256, 256, 64)
    rng = np.random.default_rng(64)
    c.w = 0.1 * np.cos(2 * np.pi * (np.arange(64)[:, None, None] + 1.0) / 64) \
        * (1.0 + 0.2 * rng.random(c.w.shape))
    s = synth.outflow_courant_max(c.u, c.v, c.w, c.g, KP)
    if s > 0.98:
        c.u, c.v, c.w = (x * (0.98 / s) for x in (c.u, c.v, c.w))
    assert np.abs(c.w[-1]).max() > 0.01
    ref = _oracle(c, 2, 1, 2)
    for v in VARIANTS.values():
        got = run_library(c, torch.float64, 2, 1, 2, variant=v, k_bc=KP)
        assert rel_err(got, ref) <= 2 * F64_TOL, v


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("nz", [1, 2, 5])
def test_periodic_k_fill_halo(kind, nz):
    """Both halo kinds wrap in k (no closed faces): against the oracle's fill
    and numpy's wrap padding."""
    from paper_1908_06094_b300 import MPDATA
    rng = np.random.default_rng(nz + 10 * kind)
    nx, ny = 11, 6
    a = rng.standard_normal((nz, ny, nx))
    m = MPDATA(nx, ny, nz, halo=H, dtype=torch.float64, k_bc=KP)
    f = to_dev(synth.pad(a, H, fill=7.0), torch.float64)
    m.fill_halo(f, kind)
    ref = synth.pad(a, H)
    oracle.fill_halo(ref, H, kind=kind, kbc=KP)
    got = f.cpu().numpy()
    assert np.array_equal(got, ref)
    assert np.array_equal(got, _wrap_all(a, H))
    m.close()


@pytest.mark.parametrize("variant", list(VARIANTS))
@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-14), (torch.float32, 1e-6)])
def test_periodic_k_mass_conserved(dtype, tol, variant):
    """With every vertical face open the mass still only moves between cells:
    drift over 20 steps within the zero-flux bounds, for a flow whose W
    through the top face is not zero."""
    from paper_1908_06094_b300 import MPDATA
    c = rounded_inputs(synth.nondivergent_case(48, 40, 12, seed=21, kbc=KP), dtype)
    assert np.abs(c.w[-1]).max() > 0.01
    m = MPDATA(c.nx, c.ny, c.nz, halo=H, iord=2, nonoscillatory=True, dtype=dtype,
               variant=VARIANTS[variant], k_bc=KP)
    d = [to_dev(synth.pad(x, H), dtype) for x in (c.psi, c.u, c.v, c.w, c.g)]
    m0 = m.mass(d[0], d[4]).item()
    m.step(*d, nsteps=20)
    m1 = m.mass(d[0], d[4]).item()
    assert abs(m1 - m0) <= tol * abs(m0)
    m.close()


@pytest.mark.parametrize("sign", [1, -1])
def test_periodic_k_courant_one_vertical_roll(sign):
    """W = +-1 on every face, G = 1: each step rolls the field one level,
    through the top face back to the bottom, exactly."""
    c = synth.uniform_shift_case(6, 5, 7, "z", sign, seed=5, kbc=KP)
    for v in VARIANTS.values():
        got = synth.interior(run_library(c, torch.float64, 2, 1, 3, variant=v, k_bc=KP), c.halo)
        assert np.array_equal(got, np.roll(c.psi, 3 * sign, axis=0)), v


def _gpu_adjoint(c, iord, nonosc, nsteps, dy, dtype, variant):
    from paper_1908_06094_b300 import MPDATA, _capi
    m = MPDATA(c.nx, c.ny, c.nz, halo=H, iord=iord, nonoscillatory=nonosc, dtype=dtype,
               k_bc=KP)
    m.set_variant(VARIANTS[variant])
    d = [to_dev(synth.pad(x, H), dtype) for x in (c.psi, c.u, c.v, c.w, c.g)]
    states = [d[0].clone()]
    for _ in range(nsteps - 1):
        nxt = torch.empty_like(states[-1])
        m.step_out(states[-1], nxt, *d[1:])
        states.append(nxt)
    pb = to_dev(dy, dtype)
    ub, vb, wb = (torch.zeros_like(d[0]) for _ in range(3))
    for s in reversed(range(nsteps)):
        _capi.mpdata_adjoint_step(m._ctx, states[s].data_ptr(), d[1].data_ptr(), d[2].data_ptr(),
                                  d[3].data_ptr(), d[4].data_ptr(), pb.data_ptr(), ub.data_ptr(),
                                  vb.data_ptr(), wb.data_ptr())
    torch.cuda.synchronize()
    out = [t.double().cpu().numpy() for t in (pb, ub, vb, wb)]
    m.close()
    return out


def _adj_errors(got, ref):
    """max |gpu - oracle| of each adjoint over the interior, relative to
    max |oracle| of that field, but never to less than 1e-2 of the largest
    adjoint: with nz = 1 the one vertical face joins a cell to itself, its
    flux leaves and enters the same cell, and without the limiter W's
    adjoint is zero up to the rounding of the terms that cancel."""
    g = [synth.interior(a, H) for a in got]
    r = [synth.interior(b, H) for b in ref]
    scale = max(float(np.abs(b).max()) for b in r)
    return [float(np.abs(a - b).max()) / max(float(np.abs(b).max()), 1e-2 * scale)
            for a, b in zip(g, r)]


@pytest.mark.parametrize("shape", [(9, 8, 1), (9, 8, 2), (21, 13, 7), (37, 30, 3)])
@pytest.mark.parametrize("iord,nonosc", [(1, 0), (2, 0), (2, 1), (3, 1)])
@pytest.mark.parametrize("variant", ["staged", "fused"])
def test_periodic_k_adjoint_f64(shape, iord, nonosc, variant):
    nx, ny, nz = shape
    c = synth.random_case(nx, ny, nz, seed=nx + 100 * nz + 1, cmax=0.25, psi_lo=0.2,
                          psi_hi=1.5, kbc=KP)
    rng = np.random.default_rng(15)
    dy = synth.pad(rng.standard_normal(c.psi.shape), H)
    P = [synth.pad(x, H) for x in (c.psi, c.u, c.v, c.w, c.g)]
    ref = oracle.adjoint(*P, dy, h=H, iord=iord, nonosc=nonosc, nsteps=2, kbc=KP)
    got = _gpu_adjoint(c, iord, nonosc, 2, dy, torch.float64, variant)
    for name, err in zip(("psi_bar", "u_bar", "v_bar", "w_bar"), _adj_errors(got, ref)):
        assert err <= 2 * ADJ_TOL, (name, err)


@pytest.mark.parametrize("shape", [(9, 8, 1), (9, 8, 2), (40, 35, 6)])
@pytest.mark.parametrize("iord,nonosc", [(1, 0), (2, 1), (3, 1)])
@pytest.mark.parametrize("variant", ["fused", "staged"])
def test_periodic_k_adjoint_f32(shape, iord, nonosc, variant):
    nx, ny, nz = shape
    c = synth.random_case(nx, ny, nz, seed=5 + nx + nz, cmax=0.25, psi_lo=0.2, psi_hi=1.5,
                          kbc=KP)
    for k in ("psi", "u", "v", "w", "g"):
        setattr(c, k, getattr(c, k).astype(np.float32).astype(np.float64))
    rng = np.random.default_rng(16)
    dy = synth.pad(rng.standard_normal(c.psi.shape), H).astype(np.float32).astype(np.float64)
    P = [synth.pad(x, H) for x in (c.psi, c.u, c.v, c.w, c.g)]
    ref = oracle.adjoint(*P, dy, h=H, iord=iord, nonosc=nonosc, nsteps=2, kbc=KP)
    got = _gpu_adjoint(c, iord, nonosc, 2, dy, torch.float32, variant)
    for err in _adj_errors(got, ref):
        assert err <= 2e-4


def test_periodic_k_autograd_against_oracle():
    """The differentiable run (5 steps, checkpoints every 2) with periodic k
    against the oracle adjoint of the same steps."""
    from paper_1908_06094_b300 import MPDATA, mpdata_run
    c = synth.random_case(21, 13, 6, seed=19, cmax=0.25, psi_lo=0.2, psi_hi=1.5, kbc=KP)
    m = MPDATA(c.nx, c.ny, c.nz, halo=H, iord=2, nonoscillatory=True, dtype=torch.float64,
               k_bc=KP)
    P = [synth.pad(x, H) for x in (c.psi, c.u, c.v, c.w, c.g)]
    rng = np.random.default_rng(20)
    dy = synth.pad(rng.standard_normal(c.psi.shape), H)
    x = [to_dev(a, torch.float64).requires_grad_(True) for a in P[:4]]
    out = mpdata_run(m, *x, to_dev(P[4], torch.float64), 5, 2)
    torch.sum(out * to_dev(dy, torch.float64)).backward()
    ref = oracle.adjoint(*P, dy, h=H, iord=2, nonosc=1, nsteps=5, kbc=KP)
    for a, b in zip([t.grad.cpu().numpy() for t in x], ref):
        assert rel_err(synth.interior(a, H), synth.interior(b, H)) <= 5 * ADJ_TOL
    m.close()
