"""GPU adjoint: the library's reverse-mode step against the oracle's
hand-written adjoint, against central differences of the GPU forward, and
through torch.autograd with checkpointing.

Tolerance against the oracle adjoint: 1e-11 relative (max-abs over the
field / max-abs of the oracle) per step in FP64.  The reverse chain has
about twice the rounded operations of the forward step and the forward
intermediates it differentiates at are the GPU's own (within 1e-12 of the
oracle's), and the cases are random fields without exact ties, so both
sides take the same branches.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import rel_err, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ADJ_TOL = 1e-11
H = 2


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_06094_b300 import build
    build.build()


VARIANTS = {"fused": 0, "staged": 1, "auto": 2}


def _gpu_adjoint(c, iord, nonosc, nsteps, dy, dtype=torch.float64, variant="auto"):
    """The adjoint of nsteps steps through the C ABI.  variant chooses the
    kernels of the forward and taped steps (fused / staged / auto)."""
    from paper_1908_06094_b300 import MPDATA, _capi
    m = MPDATA(c.nx, c.ny, c.nz, halo=H, iord=iord, nonoscillatory=nonosc, dtype=dtype)
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


@pytest.mark.parametrize("shape", [(9, 8, 5), (21, 13, 7), (37, 30, 3)])
@pytest.mark.parametrize("iord,nonosc", [(1, 0), (2, 0), (2, 1), (3, 0), (3, 1), (4, 1)])
@pytest.mark.parametrize("nsteps", [1, 3])
@pytest.mark.parametrize("variant", ["staged", "fused"])
def test_adjoint_parity_f64(shape, iord, nonosc, nsteps, variant):
    """FP64 adjoint against the oracle's, with the taped forward on the staged
    kernels (the FP64 default) and on the fused kernel."""
    nx, ny, nz = shape
    c = synth.random_case(nx, ny, nz, seed=nx + 100 * nz, cmax=0.25, psi_lo=0.2, psi_hi=1.5)
    rng = np.random.default_rng(5)
    dy = synth.pad(rng.standard_normal(c.psi.shape), H)
    P = [synth.pad(x, H) for x in (c.psi, c.u, c.v, c.w, c.g)]
    ref = oracle.adjoint(*P, dy, h=H, iord=iord, nonosc=nonosc, nsteps=nsteps)
    got = _gpu_adjoint(c, iord, nonosc, nsteps, dy, variant=variant)
    for name, a, b in zip(("psi_bar", "u_bar", "v_bar", "w_bar"), got, ref):
        err = rel_err(synth.interior(a, H), synth.interior(b, H))
        assert err <= ADJ_TOL * nsteps, (name, err)


@pytest.mark.parametrize("shape", [(9, 8, 5), (21, 13, 7), (40, 35, 6)])
@pytest.mark.parametrize("iord,nonosc", [(1, 0), (2, 0), (2, 1), (3, 1)])
@pytest.mark.parametrize("variant", ["fused", "staged"])
def test_adjoint_parity_f32_against_f64_oracle(shape, iord, nonosc, variant):
    """FP32 adjoint on FP32-rounded inputs against the FP64 oracle adjoint,
    with the taped forward on the fused kernel (the FP32 default) and on the
    staged kernels; tiles are ragged in i and j."""
    nx, ny, nz = shape
    c = synth.random_case(nx, ny, nz, seed=3 + nx, cmax=0.25, psi_lo=0.2, psi_hi=1.5)
    for k in ("psi", "u", "v", "w", "g"):
        setattr(c, k, getattr(c, k).astype(np.float32).astype(np.float64))
    rng = np.random.default_rng(6)
    dy = synth.pad(rng.standard_normal(c.psi.shape), H).astype(np.float32).astype(np.float64)
    P = [synth.pad(x, H) for x in (c.psi, c.u, c.v, c.w, c.g)]
    ref = oracle.adjoint(*P, dy, h=H, iord=iord, nonosc=nonosc, nsteps=2)
    got = _gpu_adjoint(c, iord, nonosc, 2, dy, dtype=torch.float32, variant=variant)
    for a, b in zip(got, ref):
        assert rel_err(synth.interior(a, H), synth.interior(b, H)) <= 2e-4


def test_gpu_gradient_matches_central_differences_f64():
    """<grad J, d> from the GPU adjoint against central differences of the
    GPU forward (J = sum (psi_T - obs)^2 G, 4 steps, checkpoint every 2).
    The step h = 1e-8 |x| keeps the chance that +-h straddles a min/max kink
    of the limiter negligible on this grid; the FD rounding error is then
    ~1e-16 J / h, well under the 1e-5 tolerance."""
    from paper_1908_06094_b300 import MPDATA, mpdata_run
    c = synth.random_case(12, 10, 5, seed=9, cmax=0.25, psi_lo=0.3, psi_hi=1.4)
    m = MPDATA(c.nx, c.ny, c.nz, halo=H, dtype=torch.float64)
    base = [to_dev(synth.pad(x, H), torch.float64) for x in (c.psi, c.u, c.v, c.w, c.g)]
    rng = np.random.default_rng(10)
    obs = base[0] + to_dev(synth.pad(0.05 * rng.standard_normal(c.psi.shape), H), torch.float64)
    mask = to_dev(synth.pad(np.ones(c.psi.shape), H), torch.float64)

    def J(p, u, v, w):
        out = mpdata_run(m, p, u, v, w, base[4], 4, 2)
        return torch.sum((out - obs) ** 2 * base[4] * mask)

    x = [t.clone().requires_grad_(True) for t in base[:4]]
    J(*x).backward()
    for trial in range(4):
        d = [to_dev(synth.pad(rng.standard_normal(c.psi.shape), H), torch.float64) for _ in range(4)]
        d[3][H + c.nz - 1] = 0.0
        eps = 1e-8 * max(float(t.abs().max()) for t in base[:4])
        with torch.no_grad():
            jp = J(*(a + eps * b for a, b in zip(base[:4], d))).item()
            jm = J(*(a - eps * b for a, b in zip(base[:4], d))).item()
        fd = (jp - jm) / (2 * eps)
        an = sum(float(torch.sum(xx.grad * dd)) for xx, dd in zip(x, d))
        assert abs(fd - an) <= 1e-5 * abs(an), (trial, fd, an)
    m.close()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("ckpt", [1, 2, 3, 4, 5, 20])
def test_checkpointing_does_not_change_the_gradient(ckpt, dtype):
    """10 steps with checkpoints every ckpt steps (3 and 4 leave a short last
    segment; 20 tapes the whole run in the forward pass) against ckpt 10.
    The steps are the same kernels on the same inputs; only the atomic adds
    of the reverse may sum in another order."""
    from paper_1908_06094_b300 import MPDATA, mpdata_run
    c = synth.latlon_3d(40, 32, 8, seed=4)
    m = MPDATA(c.nx, c.ny, c.nz, halo=H, dtype=dtype)
    base = [to_dev(synth.pad(x, H), dtype) for x in (c.psi, c.u, c.v, c.w, c.g)]
    x = [t.clone().requires_grad_(True) for t in base[:4]]
    out = mpdata_run(m, *x, base[4], 10, ckpt)
    torch.sum(out * out).backward()
    grads = [t.grad.cpu().double().numpy() for t in x]
    x2 = [t.clone().requires_grad_(True) for t in base[:4]]
    out2 = mpdata_run(m, *x2, base[4], 10, 10)
    torch.sum(out2 * out2).backward()
    tol = 1e-12 if dtype == torch.float64 else 1e-5
    for a, b in zip(grads, [t.grad.cpu().double().numpy() for t in x2]):
        assert rel_err(a, b) <= tol
    m.close()


def test_autograd_iord3_against_oracle():
    """The differentiable run at iord 3 (two corrective passes per step,
    tapes of two blocks, checkpoints every 2 of 5 steps) against the oracle
    adjoint of the same steps."""
    from paper_1908_06094_b300 import MPDATA, mpdata_run
    c = synth.random_case(21, 13, 7, seed=9, cmax=0.25, psi_lo=0.2, psi_hi=1.5)
    m = MPDATA(c.nx, c.ny, c.nz, halo=H, iord=3, nonoscillatory=True, dtype=torch.float64)
    P = [synth.pad(x, H) for x in (c.psi, c.u, c.v, c.w, c.g)]
    rng = np.random.default_rng(10)
    dy = synth.pad(rng.standard_normal(c.psi.shape), H)
    x = [to_dev(a, torch.float64).requires_grad_(True) for a in P[:4]]
    out = mpdata_run(m, *x, to_dev(P[4], torch.float64), 5, 2)
    torch.sum(out * to_dev(dy, torch.float64)).backward()
    ref = oracle.adjoint(*P, dy, h=H, iord=3, nonosc=1, nsteps=5)
    for a, b in zip([t.grad.cpu().numpy() for t in x], ref):
        assert rel_err(synth.interior(a, H), synth.interior(b, H)) <= 5 * ADJ_TOL
    m.close()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_forward_output_is_the_same_with_and_without_gradient(dtype):
    """With a gradient wanted the forward pass runs its last segment as taped
    steps; the taped kernels only add stores, so the output is bitwise the
    output of the plain steps."""
    from paper_1908_06094_b300 import MPDATA, mpdata_run
    c = synth.latlon_3d(40, 32, 8, seed=5)
    m = MPDATA(c.nx, c.ny, c.nz, halo=H, dtype=dtype)
    base = [to_dev(synth.pad(x, H), dtype) for x in (c.psi, c.u, c.v, c.w, c.g)]
    plain = mpdata_run(m, *base[:4], base[4], 7, 3)
    x = [t.clone().requires_grad_(True) for t in base[:4]]
    taped = mpdata_run(m, *x, base[4], 7, 3)
    assert torch.equal(plain, taped.detach())
    m.close()


def test_c5_adjoint_full_size_against_oracle():
    """The adjoint configuration's grid (256x256x64, lat-lon flow), 2 steps,
    FP64: GPU gradient of J w.r.t. psi_0 and U, V, W against the oracle."""
    c = synth.latlon_3d(256, 256, 64)
    rng = np.random.default_rng(1235)
    dy = synth.pad(rng.standard_normal(c.psi.shape), H)
    P = [synth.pad(x, H) for x in (c.psi, c.u, c.v, c.w, c.g)]
    ref = oracle.adjoint(*P, dy, h=H, iord=2, nonosc=1, nsteps=2)
    got = _gpu_adjoint(c, 2, 1, 2, dy)
    for name, a, b in zip(("psi_bar", "u_bar", "v_bar", "w_bar"), got, ref):
        err = rel_err(synth.interior(a, H), synth.interior(b, H))
        assert err <= 2 * ADJ_TOL, (name, err)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_taped_adjoint_equals_recomputing_adjoint(dtype):
    """mpdata_adjoint_step_tape on a tape recorded by mpdata_step_tape gives
    the same adjoint as mpdata_adjoint_step (which records its own tape)."""
    from paper_1908_06094_b300 import MPDATA, _capi
    c = synth.random_case(33, 20, 7, seed=17, cmax=0.25, psi_lo=0.2, psi_hi=1.5)
    m = MPDATA(c.nx, c.ny, c.nz, halo=H, dtype=dtype)
    d = [to_dev(synth.pad(x, H), dtype) for x in (c.psi, c.u, c.v, c.w, c.g)]
    rng = np.random.default_rng(3)
    dy = to_dev(synth.pad(rng.standard_normal(c.psi.shape), H), dtype)
    tape = torch.empty(_capi.mpdata_tape_bytes(m._ctx), dtype=torch.uint8, device="cuda")
    out = torch.empty_like(d[0])
    _capi.mpdata_step_tape(m._ctx, d[0].data_ptr(), out.data_ptr(), *[t.data_ptr() for t in d[1:]],
                           tape.data_ptr())
    res = []
    for taped in (True, False):
        pb = dy.clone()
        bars = [torch.zeros_like(d[0]) for _ in range(3)]
        if taped:
            _capi.mpdata_adjoint_step_tape(m._ctx, tape.data_ptr(), d[0].data_ptr(),
                                           *[t.data_ptr() for t in d[1:]], pb.data_ptr(),
                                           *[t.data_ptr() for t in bars])
        else:
            _capi.mpdata_adjoint_step(m._ctx, d[0].data_ptr(), *[t.data_ptr() for t in d[1:]],
                                      pb.data_ptr(), *[t.data_ptr() for t in bars])
        torch.cuda.synchronize()
        res.append([pb.double().cpu().numpy()] + [t.double().cpu().numpy() for t in bars])
    tol = 1e-13 if dtype == torch.float64 else 1e-5
    for a, b in zip(*res):
        assert rel_err(a, b) <= tol
    # the taped step's output equals the ordinary step's
    ref = torch.empty_like(d[0])
    m.set_variant(1)
    m.step_out(d[0], ref, *d[1:])
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    m.close()
