"""The FP32 step keeps the limiter's guarantees (Smolarkiewicz & Grabowski
1990): no new extrema, every value inside the local bounds the limiter was
built from, and a non-negative field stays non-negative.

The limiter's ratios beta-up = (psimax - psi) G/(in + eps) and beta-down =
(psi - psimin) G/(out + eps) are formed in FP32.  Where psi sits at a bound,
psimax - psi is a difference of nearly equal numbers; these checks show
whether that cancellation breaks monotonicity in FP32 on the configurations'
data.

Per step, from the FP32 field psi^n that the GPU holds (exact in FP64):
* local: psi^(n+1) in [psimin, psimax] +- tol, where the bounds are the ones
  the FP64 oracle forms on the same inputs (the 7-point neighbourhood of
  psi^n and of its donor-cell field psi^1);
* global, in non-divergent flow: min psi^n - tol <= psi^(n+1) <= max psi^n
  + tol.  (In a divergent flow psi is a density that convergence may raise
  above max psi^n -- already the donor-cell field psi^1 does -- so there the
  local bounds, which include psi^1, are the guarantee.)
* positivity: psi^(n+1) >= 0 exactly where psi^n >= 0 everywhere.
tol = 8 FP32 ulps of max |psi|, the FP32 tolerance of these properties.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import rounded_inputs, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_06094_b300 import build
    build.build()


def _tol(psi):
    return 8.0 * float(np.spacing(np.float32(np.max(np.abs(psi)))))


def _march(c, nsteps, local_every=1, variant=None, h=2, nondivergent=True):
    """Advance the FP32-rounded case step by step on the GPU; check the
    properties after every step (local bounds every local_every steps, the
    global ones in non-divergent flow only).  Returns the worst excursions
    seen (in units of tol)."""
    from paper_1908_06094_b300 import MPDATA
    c = rounded_inputs(c, torch.float32)
    m = MPDATA(c.nx, c.ny, c.nz, halo=h, iord=2, nonoscillatory=True, dtype=torch.float32,
               variant=variant)
    P = [synth.pad(x, h) for x in (c.psi, c.u, c.v, c.w, c.g)]
    d = [to_dev(x, torch.float32) for x in P]
    worst = {"global": 0.0, "local": 0.0}
    nonneg = bool(np.min(c.psi) >= 0.0)
    for n in range(nsteps):
        cur = d[0].double().cpu().numpy()       # psi^n as the GPU holds it
        inner = synth.interior(cur, h)
        lo_g, hi_g = float(inner.min()), float(inner.max())
        tol = _tol(inner)
        m.step(*d, nsteps=1)
        torch.cuda.synchronize()
        new = synth.interior(d[0].double().cpu().numpy(), h)
        if nondivergent:
            worst["global"] = max(worst["global"], (lo_g - new.min()) / tol,
                                  (new.max() - hi_g) / tol)
            assert new.min() >= lo_g - tol, (n, new.min(), lo_g)
            assert new.max() <= hi_g + tol, (n, new.max(), hi_g)
        if nonneg:
            assert new.min() >= 0.0, (n, new.min())
        if n % local_every == 0:
            _, st = oracle.run(cur, *P[1:], h=h, iord=2, nonosc=1, nsteps=1, stages=True)
            mx, mn = synth.interior(st["mx"], h), synth.interior(st["mn"], h)
            over = np.max(new - mx) / tol
            under = np.max(mn - new) / tol
            worst["local"] = max(worst["local"], over, under)
            assert over <= 1.0 and under <= 1.0, (n, over, under)
    m.close()
    return worst


@pytest.mark.parametrize("variant", [0, 1], ids=["fused", "staged"])
def test_rotating_cone_fp32_monotone(variant):
    """The 2D configuration (cone of height 4 on background 1, 64x64,
    max Courant 0.5), all 100 steps, local bounds every step."""
    c = synth.rotation_2d(64)
    _march(c, c.steps, variant=variant)


@pytest.mark.parametrize("variant", [0, 1], ids=["fused", "staged"])
def test_latlon_gaussian_and_step_fp32_monotone(variant):
    """The 3D lat-lon case (Gaussian + step on background 0, deformational
    flow with weak w, which is divergent) on a 96x64x12 grid, 20 steps:
    local bounds and positivity."""
    c = synth.latlon_3d(96, 64, 12, seed=5)
    _march(c, 20, variant=variant, nondivergent=False)


@pytest.mark.parametrize("variant", [0, 1], ids=["fused", "staged"])
def test_latlon_horizontal_flow_fp32_no_new_extrema(variant):
    """The same case without w: the corner-stream-function flow is
    non-divergent, so no step may raise the maximum or lower the minimum."""
    c = synth.latlon_3d(96, 64, 12, seed=5)
    c.w = np.zeros_like(c.w)
    _march(c, 20, variant=variant)


def _zero_region_case(nx, ny, nz, seed):
    """Lat-lon flow carrying a tracer with exact zeros over most of the
    domain: a +1 box and a cone of height 3 on background 0."""
    c = synth.latlon_3d(nx, ny, nz, seed=seed)
    i = np.arange(nx)[None, None, :]
    j = np.arange(ny)[None, :, None]
    box = ((i >= nx // 8) & (i < nx // 3) & (j >= ny // 3) & (j < 2 * ny // 3)).astype(float)
    r = np.sqrt((i - 0.6 * nx) ** 2 + (j - 0.5 * ny) ** 2)
    cone = 3.0 * np.maximum(0.0, 1.0 - r / (0.12 * nx))
    c.psi = np.broadcast_to(box + cone, (nz, ny, nx)).copy()
    return c


@pytest.mark.parametrize("variant", [0, 1], ids=["fused", "staged"])
def test_exact_zeros_stay_non_negative_fp32(variant):
    """Positivity with exact zeros: no value of the FP32 step goes below 0."""
    c = _zero_region_case(80, 64, 8, seed=9)
    assert np.count_nonzero(c.psi == 0.0) > c.psi.size // 2
    _march(c, 30, variant=variant, nondivergent=False)


def test_fp32_configuration_full_size_monotone():
    """The FP32 configuration's grid (512x512x128, halo 2) in the launch the
    benchmark times (the fused kernel), over the configuration's 100 steps:
    positivity on every step, and the local bounds against the oracle on
    the first and the last step.  Then the same grid with the horizontal
    (non-divergent) flow alone: no new extrema on any of 100 steps."""
    from paper_1908_06094_b300 import MPDATA
    c = rounded_inputs(synth.latlon_3d(512, 512, 128), torch.float32)
    h = 2
    ip = (slice(h, -h),) * 3
    for nondiv in (False, True):
        w = np.zeros_like(c.w) if nondiv else c.w
        P = [synth.pad(x, h) for x in (c.psi, c.u, c.v, w, c.g)]
        d = [to_dev(x, torch.float32) for x in P]
        m = MPDATA(c.nx, c.ny, c.nz, halo=h, dtype=torch.float32)
        lo, hi = float(c.psi.min()), float(c.psi.max())
        tol = _tol(c.psi)
        assert lo >= 0.0
        for n in range(100):
            local = not nondiv and n in (0, 99)
            if local:
                cur = d[0].double().cpu().numpy()
                _, st = oracle.run(cur, *P[1:], h=h, iord=2, nonosc=1, nsteps=1, stages=True)
                mx = torch.from_numpy(np.ascontiguousarray(st["mx"][ip])).cuda()
                mn = torch.from_numpy(np.ascontiguousarray(st["mn"][ip])).cuda()
                del st
            m.step(*d, nsteps=1)
            new = d[0][ip].double()
            if local:
                assert float((new - mx).max()) <= tol, n
                assert float((mn - new).max()) <= tol, n
            nmin, nmax = float(new.min()), float(new.max())
            assert nmin >= 0.0, (n, nmin)
            if nondiv:
                assert lo - tol <= nmin and nmax <= hi + tol, (n, nmin, nmax)
            lo, hi = nmin, nmax
        m.close()
