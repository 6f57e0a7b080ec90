"""Host-side logic of bench.py's N > 1 mode on CPU processes (gloo): the
ranks run independent replicas (weak scaling, no data-path collective), the
job's throughput is the units of all ranks over the slowest rank's time,
and only rank 0 of the reference arm does any work."""
import argparse
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out_dir):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=ws)
    try:
        # rank r took 10 (r + 1) ms for 100 (r + 1) units
        value, ms = bench.job_throughput(10.0 * (rank + 1), 100.0 * (rank + 1), ws, "cpu")
        dist.barrier()
        with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
            f.write(f"{value!r} {ms!r}\n")
    finally:
        dist.destroy_process_group()


def test_job_throughput_two_gloo_ranks(tmp_path):
    ws = 2
    mp.start_processes(_rank_main, args=(ws, _free_port(), str(tmp_path)), nprocs=ws,
                       start_method="spawn")
    for r in range(ws):
        value, ms = (float(x) for x in (tmp_path / f"r{r}.txt").read_text().split())
        # slowest rank 20 ms, units 100 + 200
        assert ms == 20.0
        assert value == pytest.approx(300.0 / 0.020)


def test_job_throughput_one_rank_needs_no_process_group():
    value, ms = bench.job_throughput(4.0, 50.0, 1)
    assert (value, ms) == (50.0 / 0.004, 4.0)


def test_replicas_are_distinct_problems_of_one_size():
    import synth
    a = synth.latlon_3d(16, 12, 4, seed=bench.replica_seed(0))
    b = synth.latlon_3d(16, 12, 4, seed=bench.replica_seed(1))
    assert a.psi.shape == b.psi.shape
    assert bench.replica_seed(0) != bench.replica_seed(1)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")
    args = argparse.Namespace(steps=3, warmup=3, gpus=2, cpu_seconds=1.0)
    assert bench.run_reference(args, "latlon256_f64") is None


class _FakeNVML:
    """Stands in for pynvml: SM clock 1900 MHz of 2032, power cap active."""
    NVML_CLOCK_SM = 1
    nvmlClocksEventReasonHwSlowdown = 0x8
    nvmlClocksEventReasonHwThermalSlowdown = 0x40
    nvmlClocksEventReasonSwThermalSlowdown = 0x20
    nvmlClocksEventReasonSwPowerCap = 0x4

    def nvmlInit(self):
        pass

    def nvmlDeviceGetHandleByIndex(self, i):
        return ("gpu", i)

    def nvmlDeviceGetClockInfo(self, h, kind):
        return 1900

    def nvmlDeviceGetMaxClockInfo(self, h, kind):
        return 2032

    def nvmlDeviceGetCurrentClocksEventReasons(self, h):
        return 0x4 | 0x1   # power cap, and a bit the summary does not report


def test_clock_sampler_reads_nvml_during_the_region():
    import time
    s = bench.ClockSampler(0, period_s=0.002, nvml=_FakeNVML())
    t0 = time.time()
    time.sleep(0.05)
    t1 = time.time()
    s.stop()
    out = s.summary(t0, t1)
    assert out["source"] == "nvml" and out["samples"] >= 5
    assert out["sm_mhz"] == 1900.0 and out["sm_max_mhz"] == 2032.0
    assert out["reasons"] == ["sw_power_cap"]


def test_clock_sampler_without_a_gpu_reports_nothing():
    class NoNVML(_FakeNVML):
        def nvmlInit(self):
            raise RuntimeError("no driver")
    s = bench.ClockSampler(0, nvml=NoNVML())
    s.stop()
    assert s.summary(0.0, 1e18) is None or s.source == "nvidia-smi"
