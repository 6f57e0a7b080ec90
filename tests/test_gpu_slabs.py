"""The i-j slab decomposition on one GPU: the library's halo pack/unpack
kernels, and px x py slabs stepped with one exchange before each step
against the undivided domain.

A slab's step is the one-kernel step reading its exchanged halo, so after
any number of steps the gathered slabs must equal, bit for bit, the
undivided domain stepped by the same kernel (variant fused); both must
match the oracle within the step tolerances (FP64 1e-12, FP32 2e-5 per
step against the oracle on the FP32-rounded inputs)."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import rounded_inputs, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F64_TOL, F32_TOL = 1e-12, 2e-5


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_06094_b300 import build
    build.build()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_pack_unpack_strips(dtype):
    """The strips a slab packs are its interior edge values, and unpacking a
    neighbour's strips (x phase, then y phase) reproduces the periodic
    padding of the undivided domain, corners included."""
    from paper_1908_06094_b300 import SlabDecomposition
    NX, NY, nz, h = 23, 17, 4, 3
    rng = np.random.default_rng(4)
    glob = rng.random((nz, NY, NX))
    for px, py in ((1, 1), (2, 1), (2, 3)):
        dec = SlabDecomposition(NX, NY, nz, px, py, halo=h, dtype=dtype)
        fields = dec.scatter(glob)
        torch.cuda.synchronize()
        wrapped = np.pad(glob.astype(np.float32).astype(np.float64) if dtype == torch.float32
                         else glob, ((0, 0), (h, h), (h, h)), mode="wrap")
        for (i0, nx, j0, ny), f in zip(dec.ext, fields):
            got = f[h:h + nz].double().cpu().numpy()
            want = wrapped[:, j0:j0 + ny + 2 * h, i0:i0 + nx + 2 * h]
            assert np.array_equal(got, want), (px, py, i0, j0)
        dec.close()


def _case_fields(c, dtype, h):
    return [to_dev(synth.pad(x, h, fill=np.nan), dtype) for x in (c.psi, c.u, c.v, c.w, c.g)]


def _run_slabs(c, px, py, dtype, nsteps, h=3):
    from paper_1908_06094_b300 import SlabDecomposition
    dec = SlabDecomposition(c.nx, c.ny, c.nz, px, py, halo=h, dtype=dtype)
    f = [dec.scatter(x) for x in (c.psi, c.u, c.v, c.w, c.g)]
    m0 = dec.mass(f[0], f[4]).item()
    dec.step(*f, nsteps=nsteps)
    out = dec.gather(f[0]).double().cpu().numpy()
    m1 = dec.mass(f[0], f[4]).item()
    dec.close()
    return out, m0, m1


def _run_whole(c, dtype, nsteps, h=3):
    from paper_1908_06094_b300 import MPDATA
    m = MPDATA(c.nx, c.ny, c.nz, halo=h, dtype=dtype, variant=0)
    d = _case_fields(c, dtype, h)
    m.step(*d, nsteps=nsteps)
    torch.cuda.synchronize()
    out = synth.interior(d[0].double().cpu().numpy(), h)
    m.close()
    return out


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("px,py", [(2, 1), (2, 2)])
def test_slabs_equal_the_undivided_step_full_size(dtype, px, py):
    """The 3D configuration's grid (256x256x64) in 2 and 4 slabs, 5 steps:
    bit for bit the undivided one-kernel step; the domain's mass conserved."""
    c = rounded_inputs(synth.latlon_3d(256, 256, 64), dtype)
    got, m0, m1 = _run_slabs(c, px, py, dtype, 5)
    whole = _run_whole(c, dtype, 5)
    assert np.array_equal(got, whole)
    assert abs(m1 - m0) <= (1e-14 if dtype == torch.float64 else 1e-6) * abs(m0)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("px,py,shape", [(3, 2, (50, 41, 7)), (1, 3, (19, 30, 5)),
                                         (4, 1, (37, 12, 9)), (4, 3, (12, 9, 4))])
def test_uneven_slabs_against_the_oracle(dtype, px, py, shape):
    """Uneven slab sizes (a ragged split) and slabs as narrow as their
    halo (12 x 9 in 4 x 3: every slab 3 x 3), 3 steps: equal to the
    undivided step and within the step tolerance of the oracle."""
    nx, ny, nz = shape
    c = rounded_inputs(synth.random_case(nx, ny, nz, seed=nx + ny, cmax=0.3), dtype)
    got, _, _ = _run_slabs(c, px, py, dtype, 3)
    assert np.array_equal(got, _run_whole(c, dtype, 3))
    P = [synth.pad(x, 2) for x in (c.psi, c.u, c.v, c.w, c.g)]
    ref = synth.interior(oracle.run(*P, h=2, iord=2, nonosc=1, nsteps=3), 2)
    tol = 3 * (F64_TOL if dtype == torch.float64 else F32_TOL)
    assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) <= tol


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_slabs_periodic_k(dtype):
    """Slabs of a domain periodic in k as well (2 x 2, 3 steps): equal to the
    undivided periodic-k step bit for bit, and within the step tolerance of
    the oracle run periodic in k."""
    from paper_1908_06094_b300 import MPDATA, SlabDecomposition, _capi as C
    c = rounded_inputs(synth.random_case(41, 30, 9, seed=8, cmax=0.3, kbc=1), dtype)
    h = 3
    dec = SlabDecomposition(c.nx, c.ny, c.nz, 2, 2, halo=h, dtype=dtype,
                            k_bc=C.MPDATA_K_PERIODIC)
    f = [dec.scatter(x) for x in (c.psi, c.u, c.v, c.w, c.g)]
    dec.step(*f, nsteps=3)
    got = dec.gather(f[0]).double().cpu().numpy()
    dec.close()
    m = MPDATA(c.nx, c.ny, c.nz, halo=h, dtype=dtype, variant=0, k_bc=C.MPDATA_K_PERIODIC)
    d = _case_fields(c, dtype, h)
    m.step(*d, nsteps=3)
    torch.cuda.synchronize()
    whole = synth.interior(d[0].double().cpu().numpy(), h)
    m.close()
    assert np.array_equal(got, whole)
    P = [synth.pad(x, 2) for x in (c.psi, c.u, c.v, c.w, c.g)]
    ref = synth.interior(oracle.run(*P, h=2, iord=2, nonosc=1, nsteps=3, kbc=1), 2)
    tol = 3 * (F64_TOL if dtype == torch.float64 else F32_TOL)
    assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) <= tol


def test_slab_refusals():
    """A slab context refuses what would read its halo as periodic."""
    from paper_1908_06094_b300 import MPDATA, _capi as C
    m = MPDATA(16, 16, 4, halo=2, dtype=torch.float64)
    with pytest.raises(C.MPDATAError):
        C.mpdata_set_ij_boundary(m._ctx, C.MPDATA_IJ_HALO)     # halo < 3
    m.close()
    m = MPDATA(16, 16, 4, halo=3, iord=3, dtype=torch.float64)
    with pytest.raises(C.MPDATAError):
        C.mpdata_set_ij_boundary(m._ctx, C.MPDATA_IJ_HALO)     # iord != 2
    m.close()
    m = MPDATA(16, 16, 4, halo=3, dtype=torch.float64)
    C.mpdata_set_ij_boundary(m._ctx, C.MPDATA_IJ_HALO)
    f = torch.zeros(m.shape, dtype=torch.float64, device="cuda")
    with pytest.raises(C.MPDATAError):
        m.fill_halo(f)
    with pytest.raises(C.MPDATAError):
        C.mpdata_set_options(m._ctx, C.MPDATA_OPT_DFL)
    with pytest.raises(C.MPDATAError):
        C.mpdata_adjoint_step(m._ctx, *[f.data_ptr()] * 9)
    C.mpdata_set_ij_boundary(m._ctx, C.MPDATA_IJ_PERIODIC)   # back to the whole domain
    m.fill_halo(f)
    m.close()
