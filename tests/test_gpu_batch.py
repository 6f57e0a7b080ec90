"""Batched persistent step: every tracer of every domain against the
single-domain fused kernel (bit for bit: the same per-cell arithmetic in a
different tile/chunk decomposition) and against the oracle."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

H = 2
DIMS = [(33, 17, 6), (40, 40, 4), (64, 20, 9), (16, 48, 3), (8, 8, 2), (70, 33, 12)]


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_06094_b300 import build
    build.build()


def _make(dtype, ntr=3, seed=0):
    rng = np.random.default_rng(seed)
    doms, cases = [], []
    for q, (nx, ny, nz) in enumerate(DIMS):
        c = synth.random_case(nx, ny, nz, seed=seed + q, cmax=0.25)
        psi = np.stack([rng.uniform(0.0, 1.0, size=c.psi.shape) for _ in range(ntr)])
        c.psi = psi
        if dtype == torch.float32:
            for k in ("psi", "u", "v", "w", "g"):
                setattr(c, k, getattr(c, k).astype(np.float32).astype(np.float64))
        d = dict(psi=torch.from_numpy(synth.pad(c.psi, H)).to("cuda", dtype).contiguous(), halo=H)
        for k in ("u", "v", "w", "g"):
            d[k] = torch.from_numpy(synth.pad(getattr(c, k), H)).to("cuda", dtype).contiguous()
        doms.append(d)
        cases.append(c)
    return doms, cases


def _single(d, tr, nsteps, dtype):
    from paper_1908_06094_b300 import MPDATA
    nz, ny, nx = (s - 2 * H for s in d["u"].shape)
    m = MPDATA(nx, ny, nz, halo=H, dtype=dtype, variant=0)
    a = d["psi"][tr].clone()
    b = torch.empty_like(a)
    for _ in range(nsteps):
        m.step_out(a, b, d["u"], d["v"], d["w"], d["g"])
        a, b = b, a
    torch.cuda.synchronize()
    m.close()
    return a


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("graph", [False, True])
@pytest.mark.parametrize("shape,kchunk", [(0, 0), (1, 4), (2, 2), (4, 0), (5, 4)])
def test_batch_matches_single_domain_bitwise(dtype, graph, shape, kchunk):
    """Shapes 4 and 5 (FP32) advance two tracers per item (an odd tracer
    count leaves the last pair with one)."""
    from paper_1908_06094_b300 import MPDATABatch
    if dtype == torch.float64 and shape > 2:
        pytest.skip("FP64 has three shapes")
    doms, cases = _make(dtype)
    ref = [[_single(d, t, 3, dtype) for t in range(3)] for d in doms]
    b = MPDATABatch(doms)
    b.set_config(shape, kchunk)
    b.step(3, graph=graph)
    torch.cuda.synchronize()
    for i in range(len(doms)):
        for t in range(3):
            assert torch.equal(b.state(i)[t], ref[i][t]), (i, t)
    b.close()


def test_batch_against_oracle_f64():
    from paper_1908_06094_b300 import MPDATABatch
    doms, cases = _make(torch.float64, ntr=2, seed=5)
    b = MPDATABatch(doms)
    b.step(2, graph=True)
    torch.cuda.synchronize()
    for i, c in enumerate(cases):
        for t in range(2):
            P = [synth.pad(x, H) for x in (c.psi[t], c.u, c.v, c.w, c.g)]
            ref = oracle.run(*P, h=H, iord=2, nonosc=1, nsteps=2)
            assert rel_err(b.state(i)[t].cpu().numpy(), ref) <= 2e-12, (i, t)
    b.close()


def test_batch_autotune_keeps_results(tmp_path):
    from paper_1908_06094_b300 import MPDATABatch
    doms, _ = _make(torch.float32, seed=9)
    ref = [[_single(d, t, 2, torch.float32) for t in range(3)] for d in doms]
    b = MPDATABatch(doms)
    cache = str(tmp_path / "tune.json")
    cfg = b.autotune(reps=2, cache=cache)
    assert not cfg["cached"] and cfg["items"] > 0
    b.step(2, graph=True)
    torch.cuda.synchronize()
    for i in range(len(doms)):
        for t in range(3):
            assert torch.equal(b.state(i)[t], ref[i][t])
    cfg2 = b.autotune(reps=2, cache=cache)
    assert cfg2["cached"] and cfg2["shape"] == cfg["shape"]
    b.close()


def test_batched_configuration_full_size_sampled():
    """The batched configuration (64 log-uniform domains x 8 tracers, FP32):
    one graph-replayed step; two domains x two tracers checked against the
    FP64 oracle on the FP32-rounded inputs."""
    from paper_1908_06094_b300 import MPDATABatch
    cases = synth.batched_domains(64, 8, seed=1234)
    doms = []
    for c in cases:
        d = dict(psi=torch.from_numpy(synth.pad(c.psi, H)).to("cuda", torch.float32).contiguous(),
                 halo=H)
        for k in ("u", "v", "w", "g"):
            d[k] = torch.from_numpy(synth.pad(getattr(c, k), H)).to("cuda", torch.float32).contiguous()
        doms.append(d)
    b = MPDATABatch(doms)
    b.step(1, graph=True)
    torch.cuda.synchronize()
    for i in (0, 37):
        c = cases[i]
        for t in (0, 7):
            P = [synth.pad(x, H).astype(np.float32).astype(np.float64)
                 for x in (c.psi[t], c.u, c.v, c.w, c.g)]
            ref = oracle.run(*P, h=H, iord=2, nonosc=1, nsteps=1)
            assert rel_err(b.state(i)[t].double().cpu().numpy(), ref) <= 2e-5, (i, t)
    b.close()
