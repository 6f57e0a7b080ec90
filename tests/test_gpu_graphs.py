"""The library's calls are asynchronous on the caller's stream, allocate
nothing after their first use and never synchronise, so a sequence of them
can be captured in a CUDA graph and replayed.  Each test captures calls on
torch's capture stream and checks that replaying the graph gives, bit for
bit, what the same calls give when run eagerly."""
import numpy as np
import pytest

import synth
from gpu_util import to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_06094_b300 import build
    build.build()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("nsteps", [1, 2, 3])
def test_step_and_mass_replay(dtype, nsteps):
    """nsteps in-place steps (the fused FP32 path ends odd counts with a
    device copy-back) and the mass reduction, captured once and replayed
    three times, against nine eager calls."""
    from paper_1908_06094_b300 import MPDATA
    c = synth.latlon_3d(64, 48, 12, seed=3)
    m = MPDATA(c.nx, c.ny, c.nz, halo=2, dtype=dtype)
    d = [to_dev(synth.pad(x, 2), dtype) for x in (c.psi, c.u, c.v, c.w, c.g)]
    eager = d[0].clone()
    for _ in range(3):
        m.step(eager, *d[1:], nsteps=nsteps)
    mass_eager = m.mass(eager, d[4]).item()
    psi = d[0].clone()
    mass_out = torch.empty((), dtype=torch.float64, device="cuda")
    m.step(psi.clone(), *d[1:], nsteps=nsteps)  # first use outside the capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            m.step(psi, *d[1:], nsteps=nsteps)
            m.mass(psi, d[4], out=mass_out)
    torch.cuda.current_stream().wait_stream(s)
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    assert torch.equal(psi, eager)
    assert mass_out.item() == mass_eager
    m.close()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_adjoint_step_replay(dtype):
    """The reverse step after one eager call (which allocates its scratch)."""
    from paper_1908_06094_b300 import MPDATA, _capi
    c = synth.random_case(33, 20, 7, seed=17, cmax=0.25, psi_lo=0.2, psi_hi=1.5)
    m = MPDATA(c.nx, c.ny, c.nz, halo=2, dtype=dtype)
    d = [to_dev(synth.pad(x, 2), dtype) for x in (c.psi, c.u, c.v, c.w, c.g)]
    dy = to_dev(synth.pad(np.random.default_rng(3).standard_normal(c.psi.shape), 2), dtype)

    def adjoint(pb, bars):
        _capi.mpdata_adjoint_step(m._ctx, d[0].data_ptr(), *[t.data_ptr() for t in d[1:]],
                                  pb.data_ptr(), *[t.data_ptr() for t in bars])

    m._sync_stream()
    pb_e, bars_e = dy.clone(), [torch.zeros_like(d[0]) for _ in range(3)]
    adjoint(pb_e, bars_e)
    torch.cuda.synchronize()
    pb, bars = dy.clone(), [torch.zeros_like(d[0]) for _ in range(3)]
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            m._sync_stream()
            adjoint(pb, bars)
    torch.cuda.current_stream().wait_stream(s)
    g.replay()
    torch.cuda.synchronize()
    tol = 0.0 if dtype == torch.float64 else 1e-6
    for a, b in zip([pb] + bars, [pb_e] + bars_e):
        # FP32 reverse sums some adjoints with atomic adds (order may differ)
        assert float((a - b).abs().max()) <= tol * float(b.abs().max()) + (
            1e-12 if dtype == torch.float64 else 0.0)
    m.close()


def test_edge_step_and_cells_sum_replay():
    from paper_1908_06094_b300 import CellsReduction, EdgeMPDATA
    from synth import cells, octahedral as octa
    c = octa.edge_case(40, 64, 6, seed=2, pivbz=1.0)
    f = {k: to_dev(getattr(c, k), torch.float32) for k in ("pD", "vn", "wn", "rho", "vol")}
    e = EdgeMPDATA(c.nr, c.nc, c.nz, dtype=torch.float32, pivbz=1.0)
    red = CellsReduction(5, dtype=torch.float32, table=cells.c2c(8, 8, "HN"))
    A = to_dev(cells.field(8, 8, 5, seed=1, numbering="HN"), torch.float32)
    # eager
    a, b = f["pD"].clone(), torch.empty_like(f["pD"])
    for _ in range(2):
        e.step(a, b, f["vn"], f["wn"], f["rho"], f["vol"])
        a, b = b, a
    B_e = torch.empty_like(A)
    red.sum(A, B_e, 0.5)
    torch.cuda.synchronize()
    # captured
    x, y = f["pD"].clone(), torch.empty_like(f["pD"])
    B = torch.empty_like(A)
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            e.step(x, y, f["vn"], f["wn"], f["rho"], f["vol"])
            e.step(y, x, f["vn"], f["wn"], f["rho"], f["vol"])
            red.sum(A, B, 0.5)
    torch.cuda.current_stream().wait_stream(s)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(x, a)
    assert torch.equal(B, B_e)
    e.close()
    red.close()
