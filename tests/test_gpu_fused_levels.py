"""The one-kernel step's level bookkeeping: the march runs its levels in a
guarded form near the bottom, the top and the start of each k-chunk, and in
a steady form (plane guards and boundary tests compiled out) in between,
with 32-bit element offsets when the field has fewer than 2^31 elements.
These cases sweep the number of levels across the boundaries of the steady
range (none, one, a few, many), with grids of few column tiles (so the
k-chunking cost model splits k into many chunks, each with its own guarded
start) and of several tiles with ragged edges, both vertical boundaries,
against the FP64 oracle on the FP32-rounded inputs and against the staged
kernels; and the results' halos, written by the kernel itself."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import rel_err, rounded_inputs, run_library

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F32_TOL = 2e-5
F64_TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_06094_b300 import build
    build.build()


def _oracle(c, nsteps, kbc):
    P = [synth.pad(x, 2) for x in (c.psi, c.u, c.v, c.w, c.g)]
    return oracle.run(*P, h=2, iord=2, nonosc=1, nsteps=nsteps, kbc=kbc)


@pytest.mark.parametrize("kbc", [0, 1], ids=["zeroflux", "periodic_k"])
@pytest.mark.parametrize("nz", [1, 2, 3, 5, 6, 7, 8, 11, 17, 33, 70])
@pytest.mark.parametrize("nxy", [(20, 9), (70, 37)], ids=["one_tile", "ragged_tiles"])
def test_fused_levels_against_oracle(nz, nxy, kbc):
    nx, ny = nxy
    if kbc == 1 and nz < 2:
        pytest.skip("periodic k needs two levels")
    c = synth.random_case(nx, ny, nz, seed=nz * 7 + nx, cmax=0.3, kbc=kbc)
    for dt, tol in ((torch.float32, F32_TOL), (torch.float64, F64_TOL)):
        cc = rounded_inputs(c, dt)
        ref = _oracle(cc, 2, kbc)
        fused = run_library(cc, dt, 2, 1, 2, variant=0, k_bc=kbc)
        assert rel_err(fused, ref) <= 2 * tol, (dt, nz)
        if dt == torch.float32:
            staged = run_library(cc, dt, 2, 1, 2, variant=1, k_bc=kbc)
            assert rel_err(fused, staged) <= 4 * tol, nz
        # the halo the kernel writes is the periodic / edge-copy image
        h = 2
        inner = synth.interior(fused, h)
        want = np.pad(inner, ((0, 0), (h, h), (h, h)), mode="wrap")
        want = np.pad(want, ((h, h), (0, 0), (0, 0)), mode="wrap" if kbc else "edge")
        assert np.array_equal(fused, want), (dt, nz)


@pytest.mark.parametrize("kbc", [0, 1], ids=["zeroflux", "periodic_k"])
@pytest.mark.parametrize("nonosc", [1, 0], ids=["limited", "unlimited"])
@pytest.mark.parametrize("shape", [(64, 48, 12), (70, 37, 9), (34, 25, 3), (96, 50, 1), (8, 6, 5)])
def test_two_column_kernel_same_bits(shape, nonosc, kbc):
    """The FP32 step takes the two-column kernel (packed f32x2 arithmetic)
    where nx and the halo are even, the one-column kernel otherwise (both
    vertical boundaries).  Every
    lane of the two-column kernel performs the one-column kernel's
    explicitly rounded operations in the same order, so the interiors must
    agree bit for bit: halo 2 (two-column) against halo 3 (one-column) on
    the same interior, 3 steps, over ragged tiles (ny not a multiple of the
    tile's 24 rows), short columns and grids narrower than one tile; and
    both within the step tolerance of the oracle."""
    nx, ny, nz = shape
    if kbc == 1 and nz < 2:
        pytest.skip("periodic k needs two levels")
    c = rounded_inputs(synth.random_case(nx, ny, nz, seed=nx + 3 * ny, cmax=0.3, kbc=kbc),
                       torch.float32)
    a = synth.interior(run_library(c, torch.float32, 2, nonosc, 3, h=2, variant=0, k_bc=kbc), 2)
    b = synth.interior(run_library(c, torch.float32, 2, nonosc, 3, h=3, variant=0, k_bc=kbc), 3)
    assert np.array_equal(a, b), int(np.count_nonzero(a != b))
    P = [synth.pad(x, 2) for x in (c.psi, c.u, c.v, c.w, c.g)]
    ref = synth.interior(oracle.run(*P, h=2, iord=2, nonosc=nonosc, nsteps=3, kbc=kbc), 2)
    assert rel_err(a, ref) <= 3 * F32_TOL
