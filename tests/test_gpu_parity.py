"""GPU parity: the CUDA library, called through its C ABI, against the CPU
oracle on the same seeded inputs.

Tolerances (max |gpu - oracle| / max |oracle|):
* FP64: 1e-12 per step.  The kernels and the oracle evaluate the same
  formulas in a different order and the GPU contracts to FMA, so single
  results differ by a few ulps; every ratio in the step is bounded by the
  scheme (|A|, |B| <= 1, limiter factors in [0, 1]) so those differences
  stay within a few hundred ulps of max|psi| per step.
* FP32 (against the FP64 oracle run on the FP32-rounded inputs): 2e-5 per
  step, i.e. ~170 FP32 ulps of max|psi|: about 35 rounded operations feed
  one output through the chain donor cell -> pseudo-velocity -> beta ->
  limited flux -> advance, each at most 0.5 ulp relative to its operand,
  and the limiter's ratios can amplify the rounding of psimax - psi by up
  to the (bounded) flux ratio.  The measured errors stay below 1e-5.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth
from gpu_util import rel_err, rounded_inputs, run_library, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F64_TOL = 1e-12
F32_TOL = 2e-5

SHAPES = [(5, 7, 3), (13, 11, 6), (37, 29, 9), (1, 9, 4), (9, 1, 4), (16, 16, 1), (33, 17, 2),
          (70, 12, 5)]
SCHEMES = [(1, 0), (2, 0), (2, 1), (3, 0), (3, 1)]


def _oracle(case, iord, nonosc, nsteps, h=None):
    h = case.halo if h is None else h
    P = [synth.pad(x, h) for x in (case.psi, case.u, case.v, case.w, case.g)]
    return oracle.run(*P, h=h, iord=iord, nonosc=nonosc, nsteps=nsteps)


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_06094_b300 import build
    build.build()


VARIANTS = {"fused": 0, "staged": 1}


@pytest.mark.parametrize("variant", list(VARIANTS))
@pytest.mark.parametrize("shape", SHAPES, ids=[f"{a}x{b}x{c}" for a, b, c in SHAPES])
@pytest.mark.parametrize("iord,nonosc", SCHEMES)
def test_f64_parity_small(shape, iord, nonosc, variant):
    nx, ny, nz = shape
    c = synth.random_case(nx, ny, nz, seed=nx * 1000 + ny * 10 + nz, cmax=0.3)
    for nsteps in (1, 3):
        ref = _oracle(c, iord, nonosc, nsteps)
        got = run_library(c, torch.float64, iord, nonosc, nsteps, variant=VARIANTS[variant])
        assert rel_err(got, ref) <= F64_TOL * nsteps, (shape, nsteps)
        # the halo of the result is the periodic/edge-copy image of its interior
        inner = synth.interior(got, c.halo)
        h = c.halo
        ref_halo = np.pad(np.pad(inner, ((0, 0), (h, h), (h, h)), mode="wrap"),
                          ((h, h), (0, 0), (0, 0)), mode="edge")
        assert np.array_equal(got, ref_halo)


@pytest.mark.parametrize("variant", list(VARIANTS))
@pytest.mark.parametrize("shape", [(13, 11, 6), (37, 29, 9), (16, 16, 1)])
@pytest.mark.parametrize("iord,nonosc", [(1, 0), (2, 0), (2, 1), (3, 1)])
def test_f32_against_f64_oracle(shape, iord, nonosc, variant):
    nx, ny, nz = shape
    c = rounded_inputs(synth.random_case(nx, ny, nz, seed=99, cmax=0.3), torch.float32)
    ref = _oracle(c, iord, nonosc, 2)
    got = run_library(c, torch.float32, iord, nonosc, 2, variant=VARIANTS[variant])
    assert rel_err(got, ref) <= 2 * F32_TOL


def test_rotating_cone_100_steps_f64():
    """The 2D configuration (64x64, cone on background 1), all 100 steps."""
    c = synth.rotation_2d(64)
    ref = _oracle(c, 2, 1, c.steps)
    got = run_library(c, torch.float64, 2, 1, c.steps)
    assert rel_err(got, ref) <= F64_TOL * c.steps


def test_latlon_256_full_field_f64():
    """The 3D FP64 configuration at full size (256x256x64, halo 2) in the
    launch configuration the benchmark times (fused kernel, k split into
    chunks): full-field comparison after 1 and 4 steps, both variants."""
    c = synth.latlon_3d(256, 256, 64)
    for nsteps in (1, 4):
        ref = _oracle(c, 2, 1, nsteps)
        for v in VARIANTS.values():
            got = run_library(c, torch.float64, 2, 1, nsteps, variant=v)
            assert rel_err(got, ref) <= F64_TOL * nsteps, (nsteps, v)


@pytest.mark.parametrize("nz", [9, 40, 64])
def test_fused_k_chunk_restart(nz):
    """Few columns and many levels: the fused kernel splits k into chunks
    that each rebuild their first planes' intermediates."""
    c = synth.random_case(37, 20, nz, seed=nz, cmax=0.3)
    ref = _oracle(c, 2, 1, 2)
    got = run_library(c, torch.float64, 2, 1, 2, variant=0)
    assert rel_err(got, ref) <= 2 * F64_TOL


def test_out_of_place_step_equals_in_place():
    from paper_1908_06094_b300 import MPDATA
    c = synth.random_case(40, 36, 10, seed=77)
    for dt in (torch.float64, torch.float32):
        for variant in VARIANTS.values():
            m = MPDATA(c.nx, c.ny, c.nz, halo=2, dtype=dt, variant=variant)
            d = [to_dev(synth.pad(x, 2), dt) for x in (c.psi, c.u, c.v, c.w, c.g)]
            psi_in = d[0].clone()
            out = torch.full_like(d[0], float("nan"))
            m.step_out(psi_in, out, *d[1:])
            m.step(*d, nsteps=1)
            assert torch.equal(out, d[0])
            assert torch.equal(psi_in, to_dev(synth.pad(c.psi, 2), dt))  # input untouched
            m.close()


def test_fused_and_staged_agree_and_conserve():
    from paper_1908_06094_b300 import MPDATA
    c = synth.latlon_3d(64, 48, 12)
    outs = []
    for variant in VARIANTS.values():
        m = MPDATA(c.nx, c.ny, c.nz, halo=2, dtype=torch.float64, variant=variant)
        d = [to_dev(synth.pad(x, 2), torch.float64) for x in (c.psi, c.u, c.v, c.w, c.g)]
        m0 = m.mass(d[0], d[4]).item()
        m.step(*d, nsteps=7)
        assert abs(m.mass(d[0], d[4]).item() - m0) <= 1e-14 * m0
        outs.append(d[0].cpu().numpy())
        m.close()
    assert rel_err(outs[0], outs[1]) <= 7 * F64_TOL


def test_latlon_512_f32_full_field():
    """The 3D FP32 configuration at full size (512x512x128): one step against
    the FP64 oracle on the same FP32-rounded inputs."""
    c = rounded_inputs(synth.latlon_3d(512, 512, 128), torch.float32)
    ref = _oracle(c, 2, 1, 1)
    got = run_library(c, torch.float32, 2, 1, 1)
    err = rel_err(got, ref)
    assert err <= F32_TOL, err


def test_courant_one_shift_bitwise_f64():
    """U = 1, G = 1: the GPU step is an exact shift, like the oracle's."""
    c = synth.uniform_shift_case(19, 10, 4, "x", 1, seed=4)
    got = synth.interior(run_library(c, torch.float64, 2, 1, 3), c.halo)
    assert np.array_equal(got, np.roll(c.psi, 3, axis=2))
    c = synth.uniform_shift_case(6, 5, 7, "z", 1, seed=5)
    got = synth.interior(run_library(c, torch.float64, 2, 1, 1), c.halo)
    assert np.array_equal(got[1:-1], c.psi[:-2])
    assert np.array_equal(got[-1], c.psi[-1] + c.psi[-2])


def test_mass_kernel_parity_and_determinism():
    from paper_1908_06094_b300 import MPDATA
    for dtype, tol in ((torch.float64, 1e-13), (torch.float32, 1e-13)):
        c = rounded_inputs(synth.random_case(45, 33, 7, seed=8), dtype)
        m = MPDATA(c.nx, c.ny, c.nz, halo=2, dtype=dtype)
        P = [synth.pad(x, 2, fill=np.nan) for x in (c.psi, c.g)]
        d = [to_dev(x, dtype) for x in P]
        a = m.mass(*d).item()
        b = m.mass(*d).item()
        ref = oracle.mass(np.nan_to_num(P[0]), np.nan_to_num(P[1]), 2)
        assert a == b
        assert abs(a - ref) <= tol * abs(ref)
        m.close()


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-14), (torch.float32, 1e-6)])
def test_mass_conserved_on_gpu(dtype, tol):
    """Mass drift over 20 steps of the lat-lon flow (FP32 target: <= 1e-6)."""
    from paper_1908_06094_b300 import MPDATA
    c = rounded_inputs(synth.latlon_3d(96, 80, 16), dtype)
    m = MPDATA(c.nx, c.ny, c.nz, halo=2, iord=2, nonoscillatory=True, dtype=dtype)
    d = [to_dev(synth.pad(x, 2), dtype) for x in (c.psi, c.u, c.v, c.w, c.g)]
    m0 = m.mass(d[0], d[4]).item()
    m.step(*d, nsteps=20)
    m1 = m.mass(d[0], d[4]).item()
    assert abs(m1 - m0) <= tol * abs(m0)
    m.close()


def test_zero_steps_and_host_call():
    from paper_1908_06094_b300 import MPDATA
    c = synth.random_case(21, 13, 5, seed=12)
    m = MPDATA(c.nx, c.ny, c.nz, halo=2, dtype=torch.float64)
    P = [synth.pad(x, 2) for x in (c.psi, c.u, c.v, c.w, c.g)]
    d = [to_dev(x, torch.float64) for x in P]
    before = d[0].clone()
    m.step(*d, nsteps=0)
    assert torch.equal(before, d[0])
    m.step(*d, nsteps=2)
    host = [torch.from_numpy(x.copy()).pin_memory() for x in P]
    m.step_host(*host, nsteps=2)
    assert torch.equal(host[0], d[0].cpu())
    m.close()


def test_fill_halo_matches_numpy():
    from paper_1908_06094_b300 import MPDATA, _capi
    rng = np.random.default_rng(3)
    nx, ny, nz, h = 11, 6, 4, 2
    a = rng.standard_normal((nz, ny, nx))
    m = MPDATA(nx, ny, nz, halo=h, dtype=torch.float64)
    for kind in (_capi.MPDATA_HALO_CELL, _capi.MPDATA_HALO_WFACE):
        f = to_dev(synth.pad(a, h, fill=7.0), torch.float64)
        m.fill_halo(f, kind)
        ref = synth.pad(a, h)
        oracle.fill_halo(ref, h, kind=kind)
        assert np.array_equal(f.cpu().numpy(), ref)
    m.close()


def test_error_paths_on_device():
    from paper_1908_06094_b300 import _capi
    L = _capi.lib
    ctx = _capi.mpdata_init(8, 8, 4, 2, 2, 1, _capi.MPDATA_F64)
    t = torch.zeros(12 * 12 * 8 + 1, dtype=torch.float64, device="cuda")
    p = t.data_ptr()
    assert L.mpdata_step(ctx, p + 8, p, p, p, p, 1) == _capi.MPDATA_EALIGN
    assert L.mpdata_step(ctx, None, p, p, p, p, 1) == _capi.MPDATA_EINVAL
    assert L.mpdata_step(ctx, p, p, p, p, p, -1) == _capi.MPDATA_EINVAL
    assert L.mpdata_fill_halo(ctx, p, 5) == _capi.MPDATA_EINVAL
    assert L.mpdata_profile_read(ctx, 99, ctypes.byref(ctypes.c_double()),
                                 ctypes.byref(ctypes.c_int())) == _capi.MPDATA_EINVAL
    _capi.mpdata_destroy(ctx)


def test_profile_and_launch_count():
    from paper_1908_06094_b300 import MPDATA, _capi
    c = synth.random_case(40, 24, 6, seed=2)
    m = MPDATA(c.nx, c.ny, c.nz, halo=2, dtype=torch.float64)
    d = [to_dev(synth.pad(x, 2), torch.float64) for x in (c.psi, c.u, c.v, c.w, c.g)]
    n0 = _capi.mpdata_launch_count(m._ctx)
    _capi.mpdata_profile(m._ctx, True)
    m.step(*d, nsteps=3)
    n1 = _capi.mpdata_launch_count(m._ctx)
    assert n1 > n0
    tot = 0
    for name, sid in _capi.STAGES.items():
        ms, k = _capi.mpdata_profile_read(m._ctx, sid)
        assert ms >= 0.0
        tot += k
    assert tot == n1 - n0
    _capi.mpdata_profile(m._ctx, False)
    m.close()


def _exact_mass(psi, g):
    """sum of the interior products psi*G, each rounded once, summed exactly."""
    import math
    return math.fsum((np.asarray(psi, dtype=np.float64) * np.asarray(g, dtype=np.float64)).ravel())


def test_latlon_256_f64_fifty_steps():
    """The 3D FP64 configuration run for its 50 steps: the FP64 error stays
    within the per-step bound times the step count, and mass is conserved."""
    c = synth.latlon_3d(256, 256, 64)
    ref = _oracle(c, 2, 1, 50)
    got = run_library(c, torch.float64, 2, 1, 50)
    assert rel_err(got, ref) <= 50 * F64_TOL
    # mass: the products psi*G summed exactly (a running sum of 4.2M terms
    # would itself be off by ~1e-13 relative)
    m0 = _exact_mass(c.psi, c.g)
    assert abs(_exact_mass(synth.interior(got, c.halo), c.g) - m0) <= 1e-13 * m0


def test_latlon_512_f32_five_steps_error_and_drift():
    """The 3D FP32 configuration over 5 steps against the FP64 oracle on the
    same FP32-rounded inputs: max-abs and L2 errors relative to max |psi|
    and the mass drift (FP64 sums of the FP32 fields)."""
    c = rounded_inputs(synth.latlon_3d(512, 512, 128), torch.float32)
    ref = _oracle(c, 2, 1, 5)
    got = run_library(c, torch.float32, 2, 1, 5)
    h = c.halo
    gi, ri = synth.interior(got, h), synth.interior(ref, h)
    scale = float(np.abs(ri).max())
    max_abs = float(np.abs(gi - ri).max()) / scale
    l2 = float(np.sqrt(np.mean((gi - ri) ** 2))) / scale
    assert max_abs <= 5 * F32_TOL, max_abs
    assert l2 <= 5 * F32_TOL / 10, l2
    m0 = _exact_mass(c.psi, c.g)
    assert abs(_exact_mass(gi, c.g) - m0) <= 1e-6 * m0


@pytest.mark.parametrize("variant", list(VARIANTS))
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("iord,h", [(1, 1), (2, 3), (2, 4), (5, 2), (8, 3)])
@pytest.mark.parametrize("nonosc", [0, 1])
def test_iord_and_halo_range(iord, h, nonosc, dtype, variant):
    """The documented ranges beyond the defaults: the donor cell alone with a
    one-cell halo, deeper halos (the output's halo filled to its depth) and
    up to eight passes."""
    c = synth.random_case(23, 17, 6, seed=iord * 10 + h, cmax=0.25)
    if dtype == torch.float32:
        c = rounded_inputs(c, dtype)
    ref = _oracle(c, iord, nonosc, 2, h=h)
    got = run_library(c, dtype, iord, nonosc, 2, h=h, variant=VARIANTS[variant])
    tol = (F64_TOL if dtype == torch.float64 else F32_TOL) * 2 * max(1, iord - 1)
    assert rel_err(got, ref) <= tol
    inner = synth.interior(got, h)
    ref_halo = np.pad(np.pad(inner, ((0, 0), (h, h), (h, h)), mode="wrap"),
                      ((h, h), (0, 0), (0, 0)), mode="edge")
    assert np.array_equal(got, ref_halo)


SMALL_2D = [(64, 64, 1), (37, 29, 1), (128, 128, 1), (8, 12, 1), (129, 120, 1), (130, 128, 1),
            (5, 7, 1), (4, 4, 1)]


@pytest.mark.parametrize("kbc", [0, 1], ids=["zeroflux", "periodic_k"])
@pytest.mark.parametrize("nonosc", [0, 1])
@pytest.mark.parametrize("shape", SMALL_2D, ids=[f"{a}x{b}x{c}" for a, b, c in SMALL_2D])
def test_f64_one_level_grid_default_step(shape, nonosc, kbc):
    """FP64 on one level: the default step (the one-kernel step on 8 x 4
    tiles up to 64 x 64 columns, 8 x 8 up to 128 x 128, the staged kernels
    above) against the oracle and against the staged kernels, 1 and 5
    steps, the halo of the result filled."""
    nx, ny, nz = shape
    c = synth.random_case(nx, ny, nz, seed=nx * 7 + ny, cmax=0.4, kbc=kbc)
    P = [synth.pad(x, c.halo) for x in (c.psi, c.u, c.v, c.w, c.g)]
    for nsteps in (1, 5):
        ref = oracle.run(*P, h=c.halo, iord=2, nonosc=nonosc, nsteps=nsteps, kbc=kbc)
        got = run_library(c, torch.float64, 2, nonosc, nsteps, k_bc=kbc)
        staged = run_library(c, torch.float64, 2, nonosc, nsteps, variant=1, k_bc=kbc)
        assert rel_err(got, ref) <= F64_TOL * nsteps, nsteps
        assert rel_err(got, staged) <= F64_TOL * nsteps, nsteps
        ref_halo = ref.copy()
        oracle.fill_halo(ref_halo, c.halo, kind=0, kbc=kbc)
        h = c.halo
        assert rel_err(got[:h], ref_halo[:h]) <= F64_TOL * nsteps
        assert rel_err(got[:, :h], ref_halo[:, :h]) <= F64_TOL * nsteps


@pytest.mark.parametrize("halo", [3, 4])
def test_f64_one_level_grid_wider_halo(halo):
    """The small one-level path with a halo of 3 or 4: the oracle's result,
    the halo of the output included."""
    c = synth.random_case(30, 22, 1, seed=77, cmax=0.4)
    P = [synth.pad(x, halo) for x in (c.psi, c.u, c.v, c.w, c.g)]
    ref = oracle.run(*P, h=halo, iord=2, nonosc=1, nsteps=4)
    got = run_library(c, torch.float64, 2, 1, 4, h=halo)
    oracle.fill_halo(ref, halo, kind=0, kbc=0)
    assert rel_err(got, ref) <= F64_TOL * 4
