"""bench.py's modes besides the default line, run as the driver would run
them (a subprocess, one JSON line on stdout): the slab-decomposition mode
on one GPU (the slab wraps onto itself) and the reference arm."""
import json
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_06094_b300 import build
    build.build()


def _run(*args):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT,
                         capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    return json.loads(out.stdout.strip().splitlines()[-1])


def test_slab_mode_one_gpu():
    d = _run("--decomp", "slab", "--steps", "3", "--warmup", "3")
    assert d["n_gpus"] == 1 and d["value"] > 0 and d["gpu_launches"] > 0
    assert d["config"]["parallelism"] == "slabs 1x1"
    # the decomposed domain conserves mass like the undivided one
    assert d["mass_drift_rel"] < 1e-13


def test_reference_arm_prints_the_same_config():
    ours = _run("--steps", "3", "--warmup", "3", "--no-extras")
    ref = _run("--impl", "reference", "--steps", "3", "--warmup", "3")
    assert ref["impl"] == "reference"
    assert ref["config"] == ours["config"]
    assert (ref["metric"], ref["unit"], ref["higher_is_better"]) == \
        (ours["metric"], ours["unit"], ours["higher_is_better"])
