"""The pipelined HOST-buffer steps (mpdata_step_host_async / mpdata_host_wait):
a stream of independent problems from page-locked host memory, two in
flight, gives for every problem exactly what the device-buffer step gives
on the same inputs."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_06094_b300 import build
    build.build()


def _host(x, dt):
    return torch.from_numpy(np.ascontiguousarray(x)).to(dt).pin_memory()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("nsteps", [1, 2])
def test_stream_of_problems_equals_device_steps(dtype, nsteps):
    from paper_1908_06094_b300 import MPDATA
    nx, ny, nz, h = 40, 33, 6, 2
    m = MPDATA(nx, ny, nz, halo=h, dtype=dtype)
    ref = MPDATA(nx, ny, nz, halo=h, dtype=dtype)
    cases = [synth.random_case(nx, ny, nz, seed=s, cmax=0.3) for s in range(5)]
    ins, outs, fields = [], [], []
    for c in cases:
        P = [synth.pad(x, h) for x in (c.psi, c.u, c.v, c.w, c.g)]
        fields.append([_host(x, dtype) for x in P])
        outs.append(torch.empty_like(fields[-1][0]).pin_memory())
    for f, o in zip(fields, outs):       # every problem enqueued before any wait
        m.step_host_async(f[0], o, *f[1:], nsteps=nsteps)
    m.host_wait()
    for f, o in zip(fields, outs):
        d = [x.cuda() for x in f]
        ref.step(*d, nsteps=nsteps)
        torch.cuda.synchronize()
        assert torch.equal(o, d[0].cpu())
    # the result may overwrite the input buffer
    f = fields[0]
    keep = f[0].clone()
    m.step_host_async(f[0], f[0], *f[1:], nsteps=nsteps)
    m.host_wait()
    d = [keep.cuda()] + [x.cuda() for x in f[1:]]
    ref.step(*d, nsteps=nsteps)
    torch.cuda.synchronize()
    assert torch.equal(f[0], d[0].cpu())
    m.close()
    ref.close()


def test_zero_steps_copies_through():
    """nsteps = 0: the problem's psi comes back unchanged."""
    from paper_1908_06094_b300 import MPDATA
    c = synth.random_case(17, 13, 3, seed=3)
    P = [synth.pad(x, 2) for x in (c.psi, c.u, c.v, c.w, c.g)]
    f = [_host(x, torch.float64) for x in P]
    out = torch.empty_like(f[0]).pin_memory()
    m = MPDATA(17, 13, 3, halo=2, dtype=torch.float64)
    m.step_host_async(f[0], out, *f[1:], nsteps=0)
    m.host_wait()
    assert torch.equal(out, f[0])
    m.close()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("shape", [(40, 33, 6), (37, 29, 1), (64, 64, 1)])
def test_interior_host_arrays_equal_device_steps(dtype, shape):
    """mpdata_step_host_interior_async: host arrays of the interior alone
    (no halo crosses the host link) give, problem by problem, the interior
    of what the device-buffer step gives; the result may overwrite the
    input."""
    from paper_1908_06094_b300 import MPDATA
    nx, ny, nz = shape
    h = 2
    m = MPDATA(nx, ny, nz, halo=h, dtype=dtype)
    ref = MPDATA(nx, ny, nz, halo=h, dtype=dtype)
    cases = [synth.random_case(nx, ny, nz, seed=40 + s, cmax=0.3) for s in range(3)]
    fields = [[_host(x, dtype) for x in (c.psi, c.u, c.v, c.w, c.g)] for c in cases]
    outs = [torch.empty_like(f[0]).pin_memory() for f in fields]
    for f, o in zip(fields, outs):
        m.step_host_interior_async(f[0], o, *f[1:], nsteps=2)
    m.step_host_interior_async(fields[0][0], fields[0][0], *fields[0][1:], nsteps=2)
    m.host_wait()
    for q, (c, o) in enumerate(zip(cases, outs)):
        d = [torch.from_numpy(synth.pad(x, h)).to("cuda", dtype).contiguous()
             for x in (c.psi, c.u, c.v, c.w, c.g)]
        ref.step(*d, nsteps=2)
        torch.cuda.synchronize()
        want = torch.from_numpy(np.ascontiguousarray(
            synth.interior(d[0].cpu().numpy(), h)))
        assert torch.equal(o, want), q
        if q == 0:
            assert torch.equal(fields[0][0], want)
    m.close()
    ref.close()
