"""GPU parity of the corrective-pass options against the oracle run with the
same options on the same seeded inputs: DFL (divergent-flow term), ABS
(signed fields), DFL | ABS and IGA (infinite gauge); both precisions, both
vertical boundaries, with and without the limiter, iord 2 and 3 (IGA: 2),
ragged tiles and single levels.  The signed-field options run on fields of
both signs, DFL alone on a positive one (the basic scheme's domain).
Tolerances are the basic scheme's: the options add terms of the same kind
(a few rounded operations each) to the formulas."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import rel_err, rounded_inputs, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F64_TOL = 1e-12
F32_TOL = 2e-5
H = 2
OPTS = {"dfl": oracle.DFL, "abs": oracle.ABS, "dfl+abs": oracle.DFL | oracle.ABS,
        "iga": oracle.IGA}
SHAPES = [(13, 11, 6), (37, 29, 9), (16, 16, 1), (9, 8, 2)]


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_06094_b300 import build
    build.build()


def _case(opts, shape, seed, kbc):
    nx, ny, nz = shape
    c = synth.random_case(nx, ny, nz, seed=seed, cmax=0.3, kbc=kbc)
    if opts & (oracle.ABS | oracle.IGA):
        c.psi = np.random.default_rng(seed + 1).uniform(-1.0, 1.0, c.psi.shape)
    return c


def _gpu(c, dtype, iord, nonosc, opts, nsteps, kbc, variant=None):
    from paper_1908_06094_b300 import MPDATA
    m = MPDATA(c.nx, c.ny, c.nz, halo=H, iord=iord, nonoscillatory=nonosc, dtype=dtype,
               k_bc=kbc, options=opts, variant=variant)
    d = [to_dev(synth.pad(x, H, fill=np.nan), dtype) for x in (c.psi, c.u, c.v, c.w, c.g)]
    m.step(*d, nsteps=nsteps)
    torch.cuda.synchronize()
    out = d[0].double().cpu().numpy()
    m.close()
    return out


def _oracle(c, iord, nonosc, opts, nsteps, kbc):
    P = [synth.pad(x, H) for x in (c.psi, c.u, c.v, c.w, c.g)]
    return oracle.run(*P, h=H, iord=iord, nonosc=nonosc, nsteps=nsteps, kbc=kbc, opts=opts)


def _schemes(name):
    return [(2, 0), (2, 1)] if name == "iga" else [(2, 0), (2, 1), (3, 0), (3, 1)]


CASES = [(n, s, io, no, kbc) for n in OPTS for s in SHAPES for (io, no) in _schemes(n)
         for kbc in (0, 1)]


@pytest.mark.parametrize("name,shape,iord,nonosc,kbc", CASES,
                         ids=[f"{n}-{a}x{b}x{c}-i{io}n{no}-k{kb}"
                              for n, (a, b, c), io, no, kb in CASES])
def test_variant_f64_parity(name, shape, iord, nonosc, kbc):
    opts = OPTS[name]
    c = _case(opts, shape, seed=sum(shape) * 7 + iord, kbc=kbc)
    for nsteps in (1, 3):
        ref = _oracle(c, iord, nonosc, opts, nsteps, kbc)
        got = _gpu(c, torch.float64, iord, nonosc, opts, nsteps, kbc)
        assert rel_err(got, ref) <= F64_TOL * nsteps, nsteps


@pytest.mark.parametrize("variant", ["fused", "staged"])
@pytest.mark.parametrize("name", list(OPTS))
@pytest.mark.parametrize("shape", [(37, 29, 9), (16, 16, 1), (70, 40, 20)])
@pytest.mark.parametrize("nonosc", [0, 1])
@pytest.mark.parametrize("kbc", [0, 1])
def test_variant_f32_against_f64_oracle(name, shape, nonosc, kbc, variant):
    """FP32 options on the fused kernel (the FP32 default) and the staged
    ones, both vertical boundaries; (70, 40, 20) splits the fused kernel's
    levels into chunks."""
    opts = OPTS[name]
    c = rounded_inputs(_case(opts, shape, seed=55, kbc=kbc), torch.float32)
    ref = _oracle(c, 2, nonosc, opts, 2, kbc)
    got = _gpu(c, torch.float32, 2, nonosc, opts, 2, kbc, {"fused": 0, "staged": 1}[variant])
    assert rel_err(got, ref) <= 2 * F32_TOL


@pytest.mark.parametrize("name", ["dfl", "iga"])
def test_variant_full_size_f64(name):
    """The 3D FP64 grid (256x256x64) with a divergent random flow (DFL) or a
    signed field (IGA), limiter on: one step."""
    opts = OPTS[name]
    c = _case(opts, (256, 256, 64), seed=1234, kbc=0)
    ref = _oracle(c, 2, 1, opts, 1, 0)
    got = _gpu(c, torch.float64, 2, 1, opts, 1, 0)
    assert rel_err(got, ref) <= F64_TOL


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-13), (torch.float32, 1e-6)])
@pytest.mark.parametrize("name", ["dfl", "dfl+abs"])
def test_variant_mass_conserved(name, dtype, tol):
    """The options change face fluxes only: mass drift over 20 steps in a
    divergent flow within the basic scheme's bounds."""
    from paper_1908_06094_b300 import MPDATA
    c = rounded_inputs(synth.random_case(48, 40, 12, seed=3, cmax=0.25), dtype)
    m = MPDATA(c.nx, c.ny, c.nz, halo=H, dtype=dtype, options=OPTS[name])
    d = [to_dev(synth.pad(x, H), dtype) for x in (c.psi, c.u, c.v, c.w, c.g)]
    m0 = m.mass(d[0], d[4]).item()
    m.step(*d, nsteps=20)
    assert abs(m.mass(d[0], d[4]).item() - m0) <= tol * abs(m0)
    m.close()


def test_option_errors_on_device():
    """Unknown bits, IGA with another option or iord 3 are refused and leave
    the options unchanged; with options set the adjoint calls are refused."""
    from paper_1908_06094_b300 import _capi
    L = _capi.lib
    ctx = _capi.mpdata_init(8, 8, 4, 2, 2, 1, _capi.MPDATA_F64)
    assert L.mpdata_set_options(ctx, 8) == _capi.MPDATA_EINVAL
    assert L.mpdata_set_options(ctx, _capi.MPDATA_OPT_IGA | _capi.MPDATA_OPT_DFL) == \
        _capi.MPDATA_EINVAL
    assert L.mpdata_set_options(ctx, _capi.MPDATA_OPT_IGA | _capi.MPDATA_OPT_ABS) == \
        _capi.MPDATA_EINVAL
    assert _capi.mpdata_get_options(ctx) == 0
    _capi.mpdata_set_options(ctx, _capi.MPDATA_OPT_DFL)
    assert _capi.mpdata_get_options(ctx) == _capi.MPDATA_OPT_DFL
    t = torch.zeros(12 * 12 * 8, dtype=torch.float64, device="cuda")
    p = t.data_ptr()
    assert L.mpdata_adjoint_step(ctx, p, p, p, p, p, p, p, p, p) == _capi.MPDATA_EINVAL
    assert L.mpdata_step_tape(ctx, p, p + 8, p, p, p, p, p) == _capi.MPDATA_EINVAL
    _capi.mpdata_destroy(ctx)
    ctx3 = _capi.mpdata_init(8, 8, 4, 2, 3, 1, _capi.MPDATA_F64)
    assert L.mpdata_set_options(ctx3, _capi.MPDATA_OPT_IGA) == _capi.MPDATA_EINVAL
    _capi.mpdata_destroy(ctx3)


def test_fp32_options_run_the_fused_kernel():
    """With an option set an FP32 context still steps with one launch."""
    from paper_1908_06094_b300 import MPDATA, _capi
    c = synth.random_case(40, 36, 10, seed=7)
    for name, o in OPTS.items():
        m = MPDATA(c.nx, c.ny, c.nz, halo=H, dtype=torch.float32, options=o)
        d = [to_dev(synth.pad(x, H), torch.float32) for x in (c.psi, c.u, c.v, c.w, c.g)]
        out = torch.empty_like(d[0])
        n0 = _capi.mpdata_launch_count(m._ctx)
        m.step_out(d[0], out, *d[1:])
        assert _capi.mpdata_launch_count(m._ctx) - n0 == 1, name
        m.close()


def test_options_off_again_restores_the_basic_step():
    """Options set and cleared: the step is bitwise the basic scheme's again
    (the fused kernel comes back for FP32)."""
    from paper_1908_06094_b300 import MPDATA, _capi
    c = synth.random_case(40, 36, 10, seed=77)
    for dt in (torch.float64, torch.float32):
        m = MPDATA(c.nx, c.ny, c.nz, halo=H, dtype=dt)
        d = [to_dev(synth.pad(x, H), dt) for x in (c.psi, c.u, c.v, c.w, c.g)]
        a = torch.empty_like(d[0])
        b = torch.empty_like(d[0])
        m.step_out(d[0], a, *d[1:])
        _capi.mpdata_set_options(m._ctx, _capi.MPDATA_OPT_DFL)
        _capi.mpdata_set_options(m._ctx, 0)
        m.step_out(d[0], b, *d[1:])
        assert torch.equal(a, b)
        m.close()


def _gpu_h(c, opts, h, nsteps, kbc):
    from paper_1908_06094_b300 import MPDATA
    m = MPDATA(c.nx, c.ny, c.nz, halo=h, iord=2, nonoscillatory=True, dtype=torch.float32,
               k_bc=kbc, options=opts, variant=0)
    d = [to_dev(synth.pad(x, h, fill=np.nan), torch.float32) for x in (c.psi, c.u, c.v, c.w, c.g)]
    m.step(*d, nsteps=nsteps)
    torch.cuda.synchronize()
    out = synth.interior(d[0].double().cpu().numpy(), h)
    m.close()
    return out


@pytest.mark.parametrize("kbc", [0, 1], ids=["zeroflux", "periodic_k"])
@pytest.mark.parametrize("shape", [(40, 29, 9), (64, 26, 5)])
@pytest.mark.parametrize("name", list(OPTS))
def test_options_two_column_kernel_same_bits(name, shape, kbc):
    """FP32 with the limiter and an option runs the two-column kernel where
    nx and the halo are even: bit for bit the one-column kernel (halo 3) on
    the same interior, 3 steps, and within the tolerance of the oracle."""
    opts = OPTS[name]
    c = rounded_inputs(_case(opts, shape, 91 + shape[0], kbc), torch.float32)
    a = _gpu_h(c, opts, 2, 3, kbc)
    b = _gpu_h(c, opts, 3, 3, kbc)
    assert np.array_equal(a, b), int(np.count_nonzero(a != b))
    ref = synth.interior(_oracle(c, 2, 1, opts, 3, kbc), H)
    assert rel_err(a, ref) <= 3 * F32_TOL
