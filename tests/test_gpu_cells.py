"""GPU parity of the cell-neighbour reduction (Table 1): direct access in
structured numbering and indirect access through the structured,
unstructured and Hilbert tables, against the oracle's table-driven sum.
The sum of three values times fac in the same order on both sides is the
same rounding: FP64 results are compared bit for bit; FP32 ones too, on
small-integer fields whose sums are exact."""
import ctypes

import numpy as np
import pytest

import oracle
from gpu_util import to_dev
from synth import cells

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SCHEMES = [("SN", "direct"), ("SN", "indirect"), ("UN", "indirect"), ("HN", "indirect")]


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_06094_b300 import build
    build.build()


def _make(nr, nc, nz, dtype, numbering, access):
    from paper_1908_06094_b300 import CellsReduction
    if access == "direct":
        return CellsReduction(nz, dtype=dtype, nr=nr, nc=nc)
    return CellsReduction(nz, dtype=dtype, table=cells.c2c(nr, nc, numbering))


@pytest.mark.parametrize("numbering,access", SCHEMES)
@pytest.mark.parametrize("shape", [(4, 4, 3), (5, 7, 1), (16, 16, 80), (33, 70, 9), (1, 3, 2),
                                   (128, 128, 80)],
                         ids=["4x4x3", "5x7x1", "16x16x80", "33x70x9", "1x3x2", "128x128x80"])
def test_cells_sum_f64_bitwise(shape, numbering, access):
    nr, nc, nz = shape
    A = cells.field(nr, nc, nz, seed=nr + nc + nz, numbering=numbering)
    t = cells.c2c(nr, nc, numbering)
    ref1 = oracle.cells_sum(t, A, 0.7)
    ref2 = oracle.cells_sum(t, ref1, 1.3)
    red = _make(nr, nc, nz, torch.float64, numbering, access)
    a = to_dev(A, torch.float64)
    b = torch.full_like(a, float("nan"))
    c = torch.full_like(a, float("nan"))
    red.sum(a, b, 0.7)
    red.sum(b, c, 1.3)
    torch.cuda.synchronize()
    assert np.array_equal(b.cpu().numpy(), ref1)
    assert np.array_equal(c.cpu().numpy(), ref2)
    red.close()


@pytest.mark.parametrize("numbering,access", SCHEMES)
def test_cells_sum_f32_exact_on_integers(numbering, access):
    nr, nc, nz = 24, 36, 7
    A = cells.field(nr, nc, nz, seed=9, numbering=numbering, integer=True)
    ref = oracle.cells_sum(cells.c2c(nr, nc, numbering), A, 0.5)
    red = _make(nr, nc, nz, torch.float32, numbering, access)
    a = to_dev(A, torch.float32)
    b = torch.empty_like(a)
    red.sum(a, b, 0.5)
    torch.cuda.synchronize()
    assert np.array_equal(b.double().cpu().numpy(), ref)
    red.close()


def test_cells_error_paths():
    from paper_1908_06094_b300 import _capi
    L = _capi.lib
    out = ctypes.c_void_p()
    t = cells.c2c(4, 4, "UN")
    bad = t.copy()
    bad[1, 5] = 32                     # one past the last cell
    IP = ctypes.POINTER(ctypes.c_int)
    assert L.mpdata_cells_init(ctypes.byref(out), 32, 3, 0, bad.ctypes.data_as(IP), 0, 0,
                               None) == _capi.MPDATA_EINVAL
    bad[1, 5] = -1
    assert L.mpdata_cells_init(ctypes.byref(out), 32, 3, 0, bad.ctypes.data_as(IP), 0, 0,
                               None) == _capi.MPDATA_EINVAL
    assert L.mpdata_cells_init(ctypes.byref(out), 30, 3, 0, None, 4, 4, None) == \
        _capi.MPDATA_EINVAL            # direct access needs ncells = 2 nr nc
    assert L.mpdata_cells_init(ctypes.byref(out), 32, 0, 0, None, 4, 4, None) == \
        _capi.MPDATA_EINVAL
    assert L.mpdata_cells_init(ctypes.byref(out), 32, 3, 0, None, 4, 4, None) == _capi.MPDATA_OK
    c = out.value
    a = torch.zeros(3 * 32 + 4, dtype=torch.float64, device="cuda")
    b = torch.zeros(3 * 32, dtype=torch.float64, device="cuda")
    assert L.mpdata_cells_sum(c, a.data_ptr(), a.data_ptr(), 1.0) == _capi.MPDATA_EINVAL
    assert L.mpdata_cells_sum(c, a.data_ptr() + 8, b.data_ptr(), 1.0) == _capi.MPDATA_EALIGN
    assert L.mpdata_cells_sum(c, None, b.data_ptr(), 1.0) == _capi.MPDATA_EINVAL
    n0 = L.mpdata_cells_launch_count(c)
    assert L.mpdata_cells_sum(c, a.data_ptr(), b.data_ptr(), 1.0) == _capi.MPDATA_OK
    torch.cuda.synchronize()
    assert L.mpdata_cells_launch_count(c) == n0 + 1
    L.mpdata_cells_destroy(c)
