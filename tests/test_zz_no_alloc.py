"""mpdata_mass_noalloc: the mass sum for callers that cannot allocate.

Callers whose device memory is all owned by their own pool or arena, or
that forbid allocation after start-up, cannot call cudaMalloc -- and so cannot create a context, since mpdata_init
allocates the step's scratch.  mpdata_mass_noalloc serves them with its
partial sums in a static device array.  These checks call it through the C
ABI and compare it with mpdata_mass (the context path) on two calls in a
row; they pass alone in a fresh process and after the rest of the suite.
"""
import ctypes

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MASS_TOL = 1e-13   # the mass tolerance of the other GPU tests


@pytest.fixture(scope="module")
def capi():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_06094_b300 import build
    build.build()
    from paper_1908_06094_b300 import _capi
    return _capi


def _fields(nx, ny, nz, h, seed, dtype):
    c = synth.random_case(nx, ny, nz, seed=seed)
    return [torch.from_numpy(synth.pad(x, h, fill=np.nan)).to("cuda", dtype).contiguous()
            for x in (c.psi, c.g)]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_noalloc_mass_matches_context_mass_twice(capi, dtype):
    nx, ny, nz, h = 45, 33, 7, 2
    code = capi.MPDATA_F64 if dtype == torch.float64 else capi.MPDATA_F32
    ctx = capi.mpdata_init(nx, ny, nz, h, 2, 1, code)
    out_ctx = torch.empty((), dtype=torch.float64, device="cuda")
    out_na = torch.empty((), dtype=torch.float64, device="cuda")
    free_before_second = None
    for call, seed in enumerate((101, 202)):           # two calls in a row
        psi, g = _fields(nx, ny, nz, h, seed, dtype)
        capi.mpdata_mass(ctx, psi.data_ptr(), g.data_ptr(), out_ctx.data_ptr())
        torch.cuda.synchronize()
        if call == 1:
            free_before_second = torch.cuda.mem_get_info()[0]
        rc = capi.lib.mpdata_mass_noalloc(psi.data_ptr(), g.data_ptr(), nx, ny, nz, h, code,
                                          out_na.data_ptr(), None)
        assert rc == capi.MPDATA_OK, capi.mpdata_strerror(rc)
        torch.cuda.synchronize()
        a, b = out_na.item(), out_ctx.item()
        # the same kernels with the same grid shape and a fixed summation
        # order: the two paths agree bit for bit (well inside MASS_TOL)
        assert a == b, (call, a, b)
        assert abs(a - b) <= MASS_TOL * abs(b), (call, a, b)
    # the second call took no device memory
    assert torch.cuda.mem_get_info()[0] == free_before_second
    capi.mpdata_destroy(ctx)


def test_noalloc_mass_rejects_bad_arguments(capi):
    L = capi.lib
    out = torch.empty((), dtype=torch.float64, device="cuda")
    t = torch.zeros(64, dtype=torch.float64, device="cuda")
    p = t.data_ptr()
    assert L.mpdata_mass_noalloc(None, p, 4, 4, 4, 2, 0, out.data_ptr(), None) == \
        capi.MPDATA_EINVAL
    assert L.mpdata_mass_noalloc(p, p, 0, 4, 4, 2, 0, out.data_ptr(), None) == capi.MPDATA_EINVAL
    assert L.mpdata_mass_noalloc(p, p, 4, 4, 4, 2, 5, out.data_ptr(), None) == capi.MPDATA_EINVAL
    assert L.mpdata_mass_noalloc(p + 8, p, 4, 4, 4, 2, 0, out.data_ptr(), None) == \
        capi.MPDATA_EALIGN
    # sizes beyond the stated maximum are refused before anything is launched
    assert L.mpdata_mass_noalloc(p, p, 4, 70000, 70000, 2, 0, out.data_ptr(), None) == \
        capi.MPDATA_ERANGE
    assert L.mpdata_mass_noalloc(p, p, 70000, 70000, 1, 2, 0, out.data_ptr(), None) == \
        capi.MPDATA_ERANGE


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_noalloc_mass_in_a_global_mode_stream_capture(capi, dtype):
    """The entry point's purpose: after a first (eager) call it can be
    captured in a CUDA graph in global capture mode, which refuses any
    allocation; the replayed graph gives the eager call's bits."""
    nx, ny, nz, h = 61, 40, 9, 2
    code = capi.MPDATA_F64 if dtype == torch.float64 else capi.MPDATA_F32
    psi, g = _fields(nx, ny, nz, h, 303, dtype)
    eager = torch.empty((), dtype=torch.float64, device="cuda")
    capi.mpdata_mass_noalloc(psi.data_ptr(), g.data_ptr(), nx, ny, nz, h, code,
                             eager.data_ptr())
    torch.cuda.synchronize()
    out = torch.full((), -1.0, dtype=torch.float64, device="cuda")
    graph = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s, capture_error_mode="global"):
            capi.mpdata_mass_noalloc(psi.data_ptr(), g.data_ptr(), nx, ny, nz, h, code,
                                     out.data_ptr(), s.cuda_stream)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    assert out.item() == -1.0  # captured, not run
    graph.replay()
    torch.cuda.synchronize()
    assert out.item() == eager.item()
