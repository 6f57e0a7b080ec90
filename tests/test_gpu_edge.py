"""GPU parity of the edge-based flux stages (structured numbering, direct
access: fused and staged kernels) against the oracle, which walks the
connectivity tables of the same patch.

Tolerances (max |gpu - oracle| / max |oracle|): FP64 1e-13 per step -- a
node-level is eight products, their sum and one division, each a few ulps
apart between the two sides (FMA contraction, the reciprocal); FP32 against
the FP64 oracle on FP32-rounded inputs 4e-6 per step: the eight terms are
at most the Courant bound times pD each, so their FP32 rounding stays
below ~1e-6 of max pD, plus the division's."""
import ctypes

import numpy as np
import pytest

import oracle
from gpu_util import rel_err, to_dev
from synth import octahedral as octa

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

VARIANTS = {"fused": 0, "staged": 1}


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_06094_b300 import build
    build.build()


def _gpu(c, dtype, variant, nsteps=1, width=0):
    from paper_1908_06094_b300 import EdgeMPDATA
    e = EdgeMPDATA(c.nr, c.nc, c.nz, dtype=dtype, pivbz=c.pivbz, variant=VARIANTS[variant])
    e.set_width(width)
    f = {k: to_dev(getattr(c, k), dtype) for k in ("vn", "wn", "rho", "vol")}
    a = to_dev(c.pD, dtype)
    b = torch.full_like(a, float("nan"))
    for _ in range(nsteps):
        e.step(a, b, f["vn"], f["wn"], f["rho"], f["vol"])
        a, b = b, a
    torch.cuda.synchronize()
    out = a.double().cpu().numpy()
    e.close()
    return out


def _rounded(c):
    for k in ("pD", "vn", "wn", "rho", "vol"):
        setattr(c, k, getattr(c, k).astype(np.float32).astype(np.float64))
    c.pivbz = float(np.float32(c.pivbz))
    return c


SHAPES = [(9, 11, 6), (37, 29, 5), (3, 4, 2), (1, 5, 3), (6, 1, 4), (17, 70, 9)]


@pytest.mark.parametrize("variant", list(VARIANTS))
@pytest.mark.parametrize("shape", SHAPES, ids=[f"{a}x{b}x{c}" for a, b, c in SHAPES])
@pytest.mark.parametrize("pivbz", [0.0, 1.0, 0.5])
def test_edge_f64_parity(shape, pivbz, variant):
    nr, nc, nz = shape
    c = octa.edge_case(nr, nc, nz, seed=nr * 100 + nc + nz, pivbz=pivbz)
    for nsteps in (1, 3):
        ref = oracle.edge_run(c, nsteps=nsteps)
        got = _gpu(c, torch.float64, variant, nsteps)
        assert rel_err(got, ref) <= 1e-13 * nsteps, nsteps


@pytest.mark.parametrize("width", [1, 4])
@pytest.mark.parametrize("shape", [(13, 40, 2), (9, 4, 3), (5, 8, 5), (37, 132, 9)],
                         ids=["13x40x2", "9x4x3", "5x8x5", "37x132x9"])
@pytest.mark.parametrize("pivbz", [0.0, 0.7])
def test_edge_fused_f32_widths(width, shape, pivbz):
    """The FP32 fused kernel with one node per thread and with four (rows
    read as 16-byte vectors; nc a multiple of 4, down to a single vector
    whose two end columns wrap onto each other)."""
    nr, nc, nz = shape
    c = _rounded(octa.edge_case(nr, nc, nz, seed=nz + nc, pivbz=pivbz))
    ref = oracle.edge_run(c, nsteps=2)
    got = _gpu(c, torch.float32, "fused", 2, width)
    assert rel_err(got, ref) <= 2 * 4e-6


@pytest.mark.parametrize("variant", list(VARIANTS))
@pytest.mark.parametrize("shape", [(37, 29, 5), (17, 70, 9)])
@pytest.mark.parametrize("pivbz", [0.0, 1.0])
def test_edge_f32_against_f64_oracle(shape, pivbz, variant):
    nr, nc, nz = shape
    c = _rounded(octa.edge_case(nr, nc, nz, seed=7, pivbz=pivbz))
    ref = oracle.edge_run(c, nsteps=2)
    got = _gpu(c, torch.float32, variant, 2)
    assert rel_err(got, ref) <= 2 * 4e-6


@pytest.mark.parametrize("variant", list(VARIANTS))
def test_edge_full_size_f64(variant):
    """The paper's global grid size (71424 nodes, 80 levels) as a 279 x 256
    patch, both organisations, one step, open boundaries (pivbz = 1)."""
    c = octa.edge_case(279, 256, 80, seed=1234, pivbz=1.0)
    ref = oracle.edge_run(c)
    got = _gpu(c, torch.float64, variant)
    assert rel_err(got, ref) <= 1e-13


@pytest.mark.parametrize("variant", list(VARIANTS))
@pytest.mark.parametrize("colour", [0, 1, 2])
def test_edge_courant_one_shift_bitwise(colour, variant):
    c = octa.shift_case(6, 7, 3, colour, seed=colour)
    got = _gpu(c, torch.float64, variant, 2)
    dr, dc = octa.EDGE_OFFSETS[colour]
    assert np.array_equal(got, np.roll(np.roll(c.pD, 2 * dr, axis=1), 2 * dc, axis=2))


@pytest.mark.parametrize("variant", list(VARIANTS))
@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-13), (torch.float32, 1e-6)])
def test_edge_mass_conserved_closed(dtype, tol, variant):
    c = octa.edge_case(40, 36, 8, seed=2, pivbz=0.0)
    if dtype == torch.float32:
        c = _rounded(c)
    m0 = oracle.edge_mass(c, c.pD)
    got = _gpu(c, dtype, variant, 10)
    assert abs(oracle.edge_mass(c, got) - m0) <= tol * m0


def test_edge_error_paths():
    from paper_1908_06094_b300 import _capi
    L = _capi.lib
    out = ctypes.c_void_p()
    assert L.mpdata_edge_init(ctypes.byref(out), 4, 4, 1, 0, 0.0, None) == _capi.MPDATA_EINVAL
    assert L.mpdata_edge_init(ctypes.byref(out), 0, 4, 3, 0, 0.0, None) == _capi.MPDATA_EINVAL
    assert L.mpdata_edge_init(ctypes.byref(out), 4, 4, 3, 5, 0.0, None) == _capi.MPDATA_EINVAL
    assert L.mpdata_edge_init(ctypes.byref(out), 4, 4, 3, 0, float("nan"), None) == \
        _capi.MPDATA_EINVAL
    assert L.mpdata_edge_init(ctypes.byref(out), 4, 4, 3, 0, 0.0, None) == _capi.MPDATA_OK
    e = out.value
    # inputs of the 4 x 4 x 3 patch (vn, the largest, has 144 values), a
    # separate output
    t = torch.ones(4 * 4 * 3 * 4 + 8, dtype=torch.float64, device="cuda")
    o = torch.zeros(4 * 4 * 3, dtype=torch.float64, device="cuda")
    p, q = t.data_ptr(), o.data_ptr()
    assert L.mpdata_edge_step(e, p, p, p, p, p, p) == _capi.MPDATA_EINVAL
    assert L.mpdata_edge_step(e, p, q + 8, p, p, p, p) == _capi.MPDATA_EALIGN
    assert L.mpdata_edge_step(e, None, q, p, p, p, p) == _capi.MPDATA_EINVAL
    assert L.mpdata_edge_set_variant(e, 7) == _capi.MPDATA_EINVAL
    assert L.mpdata_edge_set_width(e, 3) == _capi.MPDATA_EINVAL
    assert L.mpdata_edge_set_width(e, 4) == _capi.MPDATA_EINVAL  # FP64 context
    n0 = L.mpdata_edge_launch_count(e)
    assert L.mpdata_edge_set_variant(e, 1) == _capi.MPDATA_OK
    assert L.mpdata_edge_step(e, p, q, p, p, p, p) == _capi.MPDATA_OK
    torch.cuda.synchronize()
    assert L.mpdata_edge_launch_count(e) == n0 + 4
    L.mpdata_edge_destroy(e)
