"""MPDATA step benchmark: grid-point updates per second on one B300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload latlon256_f64|latlon512_f32] [--no-extras]

A step is one MPDATA time step (donor cell + iord-1 limited corrective
passes, halo of the result included) plus the FP64 mass reduction, on the
3D lat-lon configuration: 256x256x64, halo 2, FP64, iord 2, non-oscillatory,
G = cos(lat), deformational flow with weak w, Gaussian + step tracer
(synthetic, seeded).  Inputs are resident in HBM when timing starts; the
five input fields (5 x 36.8 MB) exceed the 126 MB L2, so no flush is used.

Under torchrun each rank advances its own replica of the workload (the
configurations are independent problems; no data-path collective), the
timed region is bracketed by a barrier and device syncs, and the slowest
rank's time is used: value = total updates of all ranks / max time.

--impl reference times the CPU oracle (plain FP64 C++, OpenMP over k) on the
host cores on the same workload, as the comparison arm.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "MPDATA grid-point updates/s"
UNIT = "updates/s"

WORKLOADS = {
    "latlon256_f64": dict(nx=256, ny=256, nz=64, halo=2, dtype="f64", iord=2, nonosc=1,
                          config_steps=50),
    "latlon512_f32": dict(nx=512, ny=512, nz=128, halo=2, dtype="f32", iord=2, nonosc=1,
                          config_steps=100),
}

# Algorithmic words per interior point moved by each kernel stage (reads +
# writes of whole fields the stage must touch; neighbour re-reads are not
# counted).  The whole step needs 6 (read psi, U, V, W, G; write psi).
STAGE_WORDS = {
    "donor": 7,      # psi, U, V, W -> fx, fy, fz
    "advance": 6,    # psi, fx, fy, fz, G -> psi'
    "pseudo": 8,     # psi1, U, V, W, G -> Ut, Vt, Wt
    "beta": 8,       # psi^n, psi1, Ut, Vt, Wt, G -> beta_up, beta_down
    "limit": 9,      # psi1, Ut, Vt, Wt, beta x2 -> fx, fy, fz
    "mass": 2,       # psi, G
    "halo": 0,
    "fused": 6,      # psi^n, U, V, W, G -> psi^(n+1) (+ its halo images, a perimeter)
    "fused_donor": 6,  # psi^n, U, V, W, G -> psi1
}
STEP_WORDS = 6

# Algorithmic floating-point operations per interior point of each stage,
# counted from the formulas (each +, -, *, / is one; min, max and |x| are
# not counted).  Per face of the pseudo-velocity: G_face 2, A 4, each B 9,
# each cross average 4, the combination 10 -> 42; three faces -> 126.
STAGE_FLOPS = {
    "donor": 9,      # three "+" face fluxes (2 mul + 1 add each)
    "advance": 7,    # 5 adds, 1 division, 1 subtraction
    "pseudo": 126,
    "beta": 36,      # six fluxes (18), in/out sums (10), two betas (8)
    "limit": 18,     # three limited velocities (9) and their fluxes (9)
    "mass": 2,
    "halo": 0,
    "fused": 212,    # the whole step: 25 + 126 + 36 + 18 + 7
    "fused_donor": 25,
}
STEP_FLOPS = 212

# The FP64 staged step assigns part of the limiter's work to another kernel:
# its pseudo-velocity kernel also forms the donor fluxes of the pseudo-
# velocities on the three "+" faces (9 flops, 3 words written), the beta
# kernel reads those fluxes instead of forming the six of its faces (its
# in/out sums and betas remain: 18 flops), and the limiter reads them with
# Ut, Vt, Wt and the betas and scales them in place (11 words).
STAGE_FLOPS_F64 = dict(STAGE_FLOPS, pseudo=126 + 9, beta=18)
STAGE_WORDS_F64 = dict(STAGE_WORDS, pseudo=8 + 3, limit=11)

# FP64 peak of the B300 from its unit count and clock: 2 FP64 FMA lanes per
# SM per clock (ncu: sm__sass_thread_inst_executed_op_dfma_pred_on
# peak_sustained = 2) x 148 SMs x 2.032 GHz x 2 flops per FMA.  Reported
# beside the rate the FP64 FMA probe measures in the same run, which is the
# roofline's denominator.
FP64_PEAK_GFLOPS = 2 * 148 * 2.032 * 2


def measure_fp64_peak(dev, blocks=148 * 16, iters=4096, reps=5):
    """The device's FP64 FMA rate (GFLOP/s): the library's probe kernel
    (8 independent FMA chains per thread, 2368 x 256 threads), timed with
    CUDA events on the launching stream after 3 warm-up launches; best of
    reps launches."""
    import torch
    from paper_1908_06094_b300 import _capi
    out = torch.zeros(1, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(3):
        _capi.mpdata_probe_fp64_fma(out.data_ptr(), blocks, iters, stream.cuda_stream)
    torch.cuda.synchronize(dev)
    best = 0.0
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        flops = _capi.mpdata_probe_fp64_fma(out.data_ptr(), blocks, iters, stream.cuda_stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        best = max(best, flops / (e0.elapsed_time(e1) / 1e3) / 1e9)
    return best


def _fp64_instructions(stage: str, workload: str):
    """FP64 instructions per interior point of a stage (or of the whole step,
    stage "step") from a committed ncu opcode count, only if it was taken on
    the current kernel sources (same source hash as in dram_traffic.txt)."""
    path = os.path.join(ROOT, "profiles", "fp64_instructions.txt")
    try:
        for line in open(path):
            if line.startswith("#") or not line.strip():
                continue
            st, wl, h, n = line.split()[:4]
            if st == stage and wl == workload and h == _source_hash(None if st == "step" else st):
                return float(n)
    except OSError:
        pass
    return None


def table2_accesses(nodes: int, edges: int, fused: bool) -> int:
    """Main-memory accesses per vertical plane for the MPDATA fluxes with the
    counting of Table 2: unfused 1 r + 1 w per edge and 7 r + 3 w per node;
    fused 4 r + 1 w per node."""
    return nodes * (4 + 1) if fused else edges * (1 + 1) + nodes * (7 + 3)


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


# ------------------------------------------------------------------ clocks --

class _CtypesNVML:
    """The few read-only NVML calls the sampler uses, through the driver's
    libnvidia-ml (for hosts without the pynvml module)."""
    NVML_CLOCK_SM = 1
    # clock-event reason bits of the NVML API
    nvmlClocksEventReasonSwPowerCap = 0x4
    nvmlClocksEventReasonHwSlowdown = 0x8
    nvmlClocksEventReasonSwThermalSlowdown = 0x20
    nvmlClocksEventReasonHwThermalSlowdown = 0x40

    def __init__(self):
        import ctypes
        self._c = ctypes
        self._lib = ctypes.CDLL("libnvidia-ml.so.1")

    def _ok(self, rc, what):
        if rc != 0:
            raise RuntimeError(f"{what}: NVML error {rc}")

    def nvmlInit(self):
        self._ok(self._lib.nvmlInit_v2(), "nvmlInit")

    def nvmlDeviceGetHandleByIndex(self, i):
        h = self._c.c_void_p()
        self._ok(self._lib.nvmlDeviceGetHandleByIndex_v2(self._c.c_uint(i), self._c.byref(h)),
                 "handle")
        return h

    def _uint(self, fn, h, *args):
        v = self._c.c_uint()
        self._ok(fn(h, *args, self._c.byref(v)), fn.__name__)
        return v.value

    def nvmlDeviceGetClockInfo(self, h, kind):
        return self._uint(self._lib.nvmlDeviceGetClockInfo, h, self._c.c_int(kind))

    def nvmlDeviceGetMaxClockInfo(self, h, kind):
        return self._uint(self._lib.nvmlDeviceGetMaxClockInfo, h, self._c.c_int(kind))

    def nvmlDeviceGetCurrentClocksEventReasons(self, h):
        v = self._c.c_ulonglong()
        self._ok(self._lib.nvmlDeviceGetCurrentClocksThrottleReasons(h, self._c.byref(v)),
                 "reasons")
        return v.value


class ClockSampler:
    """SM clock and clock-event (throttle) samples during a timed region,
    stamped with the host clock.  Read-only queries: NVML every 5 ms (the
    timed regions are tens of milliseconds), else nvidia-smi every 100 ms."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, index: int, period_s: float = 0.005, nvml=None):
        self.samples = []  # (host time, sm MHz, max sm MHz, [4 reason flags])
        self.proc = None
        self._stop = threading.Event()
        self.source = None
        try:
            if nvml is None:
                try:
                    import pynvml as nvml
                except ImportError:
                    nvml = _CtypesNVML()
            nvml.nvmlInit()
            h = nvml.nvmlDeviceGetHandleByIndex(index)
            self._nvml, self._h = nvml, h
            self._bits = [nvml.nvmlClocksEventReasonHwSlowdown,
                          nvml.nvmlClocksEventReasonHwThermalSlowdown,
                          nvml.nvmlClocksEventReasonSwThermalSlowdown,
                          nvml.nvmlClocksEventReasonSwPowerCap]
            self.source = "nvml"
            self.t = threading.Thread(target=self._poll, args=(period_s,), daemon=True)
            self.t.start()
            return
        except Exception:
            self.source = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.source = "nvidia-smi"
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _poll(self, period_s):
        n, h = self._nvml, self._h
        while not self._stop.is_set():
            try:
                sm = n.nvmlDeviceGetClockInfo(h, n.NVML_CLOCK_SM)
                mx = n.nvmlDeviceGetMaxClockInfo(h, n.NVML_CLOCK_SM)
                r = n.nvmlDeviceGetCurrentClocksEventReasons(h)
                self.samples.append((time.time(), float(sm), float(mx),
                                     [bool(r & b) for b in self._bits]))
            except Exception:
                pass
            self._stop.wait(period_s)

    def _read(self):
        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                self.samples.append((time.time(), num(parts[0]), num(parts[1]),
                                     [parts[4 + q].lower() == "active" for q in range(4)]))

    def stop(self):
        self._stop.set()
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self, t0: float, t1: float):
        rows = [x for x in self.samples if t0 <= x[0] <= t1]
        if not rows:   # region shorter than the sampling period: take the nearest
            rows = [x for x in self.samples if t0 - 0.25 <= x[0] <= t1 + 0.25]
        if not rows:
            return None
        sm = [x[1] for x in rows if x[1] is not None]
        mx = [x[2] for x in rows if x[2] is not None]
        reasons = sorted({self.NAMES[q] for x in rows for q in range(4) if x[3][q]})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "source": self.source}


# -------------------------------------------------------------- our arm --

def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def replica_seed(rank: int) -> int:
    """The seed of a rank's replica: every rank advances its own synthetic
    problem of the same size (weak scaling, no data-path collective)."""
    return 1234 + rank


def job_throughput(ms_local: float, units_local: float, ws: int, device=None):
    """Whole-job throughput over ws ranks: the units all ranks processed over
    the slowest rank's time (ms), with the time and the units reduced across
    the process group (MAX and SUM) when ws > 1.  Returns (units/s, ms)."""
    if ws > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([ms_local, units_local], dtype=torch.float64, device=device)
        mx = t[:1].clone()
        dist.all_reduce(mx, op=dist.ReduceOp.MAX)
        sm = t[1:].clone()
        dist.all_reduce(sm, op=dist.ReduceOp.SUM)
        ms_local, units_local = float(mx.item()), float(sm.item())
    return units_local / (ms_local / 1e3), ms_local


# The sources a stage's dominant kernel is built and launched from: a DRAM
# figure taken with ncu stays valid while these files are unchanged.
STAGE_SOURCES = {
    "pseudo": ("march.cuh", "grid.cuh"),                # FP64 k-marching pseudo-velocity
    "fused": ("fusedx.cuh", "fused2.cuh", "grid.cuh", "capi.cu"),  # FP32 fused step (+ its chunking)
    "edge": ("edge.cuh", "edge.cu", "grid.cuh"),        # edge-based flux stages
}


def _source_hash(stage=None):
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1908_06094_b300", "csrc")
    files = STAGE_SOURCES.get(stage) or sorted(os.listdir(csrc))
    for fn in files:
        with open(os.path.join(csrc, fn), "rb") as f:
            h.update(fn.encode())
            h.update(f.read())
    return h.hexdigest()[:16]


def _traffic_from_profiles(stage: str, workload: str, src_hash: str):
    """DRAM bytes per launch of a stage from a committed ncu summary, only if
    it was taken on the current kernel sources (same source hash)."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    try:
        for line in open(path):
            if line.startswith("#") or not line.strip():
                continue
            st, wl, h, b = line.split()[:4]
            if st == stage and wl == workload and h == src_hash:
                return float(b)
    except OSError:
        pass
    return None


def _oracle_sample(call, units_per_call: float, seconds: float, unit: str, sample: str):
    """The CPU oracle as it stands, timed on the host cores: call() repeated
    until ``seconds`` have passed (at least once); units/s."""
    t0 = time.perf_counter()
    k = 0
    while True:
        call()
        k += 1
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    return {"value": units_per_call * k / dt, "unit": unit, "cores": os.cpu_count() or 1,
            "kind": "oracle", "sample": f"{k} x {sample}"}


def _oracle_rate(wl, seconds: float, psi, fields, h):
    """Updates/s of the CPU oracle on the full workload grid, stepping until
    ``seconds`` have passed (at least one step)."""
    import oracle
    n = wl["nx"] * wl["ny"] * wl["nz"]
    cur = psi
    steps = 0
    t0 = time.perf_counter()
    while True:
        cur = oracle.run(cur, *fields, h=h, iord=wl["iord"], nonosc=wl["nonosc"], nsteps=1)
        steps += 1
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    return steps * n / dt, steps


def bench_config(wl_name: str, ws: int, variant=None) -> dict:
    """The workload description both arms print (same keys, same values)."""
    wl = WORKLOADS[wl_name]
    esize = 8 if wl["dtype"] == "f64" else 4
    h = wl["halo"]
    field_mb = esize * (wl["nx"] + 2 * h) * (wl["ny"] + 2 * h) * (wl["nz"] + 2 * h) / 1e6
    return {"workload": f"latlon_3d {wl['nx']}x{wl['ny']}x{wl['nz']} halo {h} "
                        f"{wl['dtype']} iord={wl['iord']} nonoscillatory",
            "nx": wl["nx"], "ny": wl["ny"], "nz": wl["nz"], "halo": h,
            "iord": wl["iord"], "nonoscillatory": wl["nonosc"],
            "step": "one MPDATA step + FP64 mass reduction",
            "l2": "no flush: the 5 input fields (%.0f MB) exceed the 126 MB L2" % (5 * field_mb),
            "variant": {0: "fused", 1: "staged", 2: "auto"}.get(variant, "auto"),
            "parallelism": f"replicas x{ws}"}


def run_ours(args, wl_name):
    import numpy as np
    import torch
    import synth

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)

    from paper_1908_06094_b300 import MPDATA, _capi

    wl = WORKLOADS[wl_name]
    dt = torch.float64 if wl["dtype"] == "f64" else torch.float32
    h = wl["halo"]
    case = synth.latlon_3d(wl["nx"], wl["ny"], wl["nz"], seed=replica_seed(rank))
    padded = [synth.pad(x, h) for x in (case.psi, case.u, case.v, case.w, case.g)]
    if dt == torch.float32:
        padded = [x.astype(np.float32) for x in padded]
    d = [torch.from_numpy(x).to(dev).contiguous() for x in padded]
    m = MPDATA(wl["nx"], wl["ny"], wl["nz"], halo=h, iord=wl["iord"],
               nonoscillatory=wl["nonosc"], dtype=dt, device=dev)
    if args.variant is not None:
        m.set_variant(args.variant)
    mass_out = torch.empty((), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    npts = wl["nx"] * wl["ny"] * wl["nz"]

    # the state double-buffered (mpdata_step_out), as a caller keeps it: the
    # one-kernel step cannot run in place, and mpdata_step with nsteps = 1
    # would add a copy back into psi
    state = [d[0], torch.empty_like(d[0])]

    def step():
        m.step_out(state[0], state[1], *d[1:])
        state.reverse()
        m.mass(state[0], d[4], out=mass_out)

    m0 = m.mass(d[0], d[4]).item()
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)

    sampler = ClockSampler(dev.index or 0) if rank == 0 else None
    time.sleep(0.3 if sampler else 0.0)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    launches0 = _capi.mpdata_launch_count(m._ctx)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    wall0 = time.time()
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    wall1 = time.time()
    if ws > 1:
        torch.distributed.barrier()
    ms = ev0.elapsed_time(ev1)
    launches = _capi.mpdata_launch_count(m._ctx) - launches0
    m1 = mass_out.item()
    value, ms = job_throughput(ms, npts * args.steps, ws, dev)
    clocks = None
    if sampler:
        sampler.stop()
        clocks = sampler.summary(wall0, wall1)
    # the same K steps timed 4 more times (median of 5 beside the headline),
    # then once more with CUDA events around every launch for the per-kernel
    # durations of the roofline; neither pass is part of the headline
    repeat_ms = [ms]
    for _ in range(4 if rank == 0 else 0):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        repeat_ms.append(e0.elapsed_time(e1))
    stage_ms = {}
    prof_ms = None
    if rank == 0:
        _capi.mpdata_profile(m._ctx, True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        prof_ms = e0.elapsed_time(e1)
        for name, sid in _capi.STAGES.items():
            t, k = _capi.mpdata_profile_read(m._ctx, sid)
            if k:
                stage_ms[name] = (t, k)
        _capi.mpdata_profile(m._ctx, False)

    out = None
    if rank == 0:
        hbm, peak_kind = _peaks()
        dom = max(stage_ms, key=lambda s: stage_ms[s][0]) if stage_ms else None
        esize = 8 if dt == torch.float64 else 4
        roof = None
        if dom:
            t, k = stage_ms[dom]
            per_launch_ms = t / k
            src = _source_hash(dom)
            traffic = _traffic_from_profiles(dom, wl_name, src)
            share = {s_: round(v[0] / sum(x[0] for x in stage_ms.values()), 4)
                     for s_, v in stage_ms.items()}
            if dt == torch.float64:
                # FP64 on the B300 runs at 1/64 of FP32: these kernels are bound by
                # the FP64 pipe, not by HBM.  The denominator is the FP64 FMA rate
                # the probe kernel measures on this device in this run.
                fp64_peak = measure_fp64_peak(dev)
                flops = STAGE_FLOPS_F64[dom] * npts
                achieved = flops / (per_launch_ms / 1e3) / 1e9
                roof = {"bound": "alu", "kernel": dom, "achieved": round(achieved, 1),
                        "peak": round(fp64_peak, 1), "unit": "GFLOP/s (FP64)",
                        "frac": round(achieved / fp64_peak, 4), "traffic": traffic,
                        "algorithmic_flops": flops,
                        "hbm_frac": round(STAGE_WORDS_F64[dom] * esize * npts /
                                          (per_launch_ms / 1e3) / 1e9 / hbm, 4),
                        "launch_ms": round(per_launch_ms, 5),
                        "peak_source": "measured in this run: FP64 FMA probe kernel "
                                       "(mpdata_probe_fp64_fma), best of 5",
                        "peak_derived": round(FP64_PEAK_GFLOPS, 1),
                        "frac_of_derived": round(achieved / FP64_PEAK_GFLOPS, 4),
                        "stage_share": share}
                # the whole step's floor on the FP64 pipe: its FP64 instructions per
                # point (ncu opcode counts on the current sources) at the probe's
                # instruction rate (one FMA = one instruction = 2 flops)
                ninst = _fp64_instructions("step", wl_name)
                if ninst:
                    floor_ms = ninst * npts / (fp64_peak / 2 * 1e9) * 1e3
                    roof["fp64_pipe_floor"] = {
                        "instructions_per_point": ninst, "ms_per_step": round(floor_ms, 4),
                        "step_over_floor": round((ms / args.steps) / floor_ms, 3)}
            else:
                bytes_launch = STAGE_WORDS[dom] * esize * npts
                achieved = bytes_launch / (per_launch_ms / 1e3) / 1e9
                roof = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1),
                        "peak": hbm, "unit": "GB/s", "frac": round(achieved / hbm, 4),
                        "traffic": traffic, "algorithmic_bytes": bytes_launch,
                        "launch_ms": round(per_launch_ms, 5),
                        "peak_source": peak_kind + " (MEASURED_PEAKS hbm_gbs)",
                        "stage_share": share}
        step_bytes = STEP_WORDS * esize * npts
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": wl["dtype"],
            "data": "synthetic (seeded lat-lon deformational flow, Gaussian + step tracer)",
            "config": bench_config(wl_name, ws, args.variant),
            "hbm_roofline_frac_step": round(value / ws * step_bytes / npts / 1e9 / hbm, 4),
            "fp64_alu_frac_step": (round(value / ws * STEP_FLOPS / 1e9 / roof["peak"], 4)
                                   if dt == torch.float64 and roof else None),
            "repeats": {"runs": len(repeat_ms), "ms_per_step_median":
                        round(statistics.median(repeat_ms) / args.steps, 5),
                        "ms_per_step_all": [round(x / args.steps, 5) for x in repeat_ms]},
            "profiled_pass": {"ms_per_step": round(prof_ms / args.steps, 5) if prof_ms else None,
                              "what": "the same K steps with CUDA events around every "
                                      "launch (per-kernel durations); outside the timed "
                                      "region"},
            "roofline": roof,
            "gpu_launches": launches,
            "mass_drift_rel": abs(m1 - m0) / abs(m0) if m0 else None,
            "clocks": clocks,
        }
    # end-to-end through the HOST-buffer C calls: every step copies its
    # psi, U, V, W, G from page-locked host memory and its result back
    if rank == 0 and not args.no_extras:
        host = [torch.from_numpy(x.copy()).pin_memory() for x in padded]
        outs = [torch.empty_like(host[0]).pin_memory() for _ in range(2)]
        k = max(3, min(args.steps, 20))
        fb = padded[0].nbytes
        # (a) the pipelined calls: a stream of k one-step problems, two in
        # flight (copies of one overlap the step of another)
        for q in range(3):
            m.step_host_async(host[0], outs[q % 2], *host[1:], nsteps=1)
        m.host_wait()
        t0 = time.perf_counter()
        for q in range(k):
            m.step_host_async(host[0], outs[q % 2], *host[1:], nsteps=1)
        m.host_wait()
        e2e_s = time.perf_counter() - t0
        # (c) the same with host arrays of the interior alone: the halo,
        # which the step neither reads nor needs from the host, stays off the
        # host link
        ihost = [torch.from_numpy(np.ascontiguousarray(synth.interior(x, h))).pin_memory()
                 for x in padded]
        iouts = [torch.empty_like(ihost[0]).pin_memory() for _ in range(2)]
        ib = ihost[0].numel() * ihost[0].element_size()
        for q in range(3):
            m.step_host_interior_async(ihost[0], iouts[q % 2], *ihost[1:], nsteps=1)
        m.host_wait()
        t0 = time.perf_counter()
        for q in range(k):
            m.step_host_interior_async(ihost[0], iouts[q % 2], *ihost[1:], nsteps=1)
        m.host_wait()
        e2e_i_s = time.perf_counter() - t0
        # (b) the blocking call, one problem at a time
        hs = [x.clone().pin_memory() for x in host]
        m.step_host(*hs, nsteps=1)
        t0 = time.perf_counter()
        for _ in range(k):
            m.step_host(*hs, nsteps=1)
        ser_s = time.perf_counter() - t0
        out["e2e"] = {"value": npts * k / e2e_i_s, "unit": UNIT, "h2d_bytes_per_step": 5 * ib,
                      "d2h_bytes_per_step": ib, "steps": k,
                      "path": "mpdata_step_host_interior_async + mpdata_host_wait: per step, "
                              "pinned host psi,U,V,W,G interiors -> device, 1 step, psi "
                              "interior -> host; two steps in flight",
                      "padded_host": {"value": npts * k / e2e_s, "h2d_bytes_per_step": 5 * fb,
                                      "d2h_bytes_per_step": fb,
                                      "path": "mpdata_step_host_async (padded host fields)"},
                      "blocking_call": {"value": npts * k / ser_s,
                                        "path": "mpdata_step_host, one step per call"}}
        # CPU baseline: the oracle as it stands, all host cores, bounded sample
        ncores = os.cpu_count() or 1
        cpu_rate, cpu_steps = _oracle_rate(wl, args.cpu_seconds, padded[0].astype("float64"),
                                           [x.astype("float64") for x in padded[1:]], h)
        out["adjoint"] = {"f64": measure_adjoint(dev, torch.float64, cpu_seconds=3.0),
                          "f32": measure_adjoint(dev, torch.float32)}
        out["batched"] = measure_batched(dev)
        out["fp32"] = measure_config(dev, "latlon512_f32")
        out["rotation_2d"] = measure_rotation_2d(dev)
        out["options"] = measure_options(dev)
        out["octahedral_edge"] = measure_edge(dev)
        out["table1_cells"] = measure_cells(dev)
        out["cpu_baseline"] = {"value": cpu_rate, "unit": UNIT, "cores": ncores,
                               "kind": "oracle",
                               "sample": f"{cpu_steps} full steps of the same workload "
                                         f"(OMP_NUM_THREADS={os.environ.get('OMP_NUM_THREADS', ncores)})"}
    m.close()
    if ws > 1:
        torch.distributed.destroy_process_group()
    return out


def slab_grid_shape(ws: int):
    """px x py = ws with px >= py as close to square as possible."""
    py = max(d for d in range(1, int(ws ** 0.5) + 1) if ws % d == 0)
    return ws // py, py


def run_slab(args, wl_name):
    """The workload as an i-j decomposed domain: each of the N ranks owns one
    nx x ny x nz slab of a (px nx) x (py ny) x nz domain (weak scaling), the
    slabs exchange psi's halo (depth 3, torch.distributed send/recv, NCCL)
    before every one-kernel step, and the domain's mass is one FP64
    all-reduce per step.  With N = 1 the single slab wraps onto itself (no
    messages: its halo strips are packed and unpacked locally)."""
    import numpy as np
    import torch
    import synth
    from paper_1908_06094_b300 import _capi
    from paper_1908_06094_b300.slabs import SlabRank

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)
    wl = WORKLOADS[wl_name]
    dt = torch.float64 if wl["dtype"] == "f64" else torch.float32
    px, py = slab_grid_shape(ws)
    NX, NY, nz, h = px * wl["nx"], py * wl["ny"], wl["nz"], 3
    case = synth.latlon_3d(NX, NY, nz, seed=1234)
    sl = SlabRank(NX, NY, nz, px, py, rank, halo=h, dtype=dt, device=dev) if ws > 1 else \
        SlabRank(NX, NY, nz, 1, 1, 0, halo=h, dtype=dt, device=dev)
    i0, nx, j0, ny = sl.i0, sl.nx, sl.j0, sl.ny
    f = []
    for x in (case.psi, case.u, case.v, case.w, case.g):
        t = torch.full(sl.s.m.shape, float("nan"), dtype=dt, device=dev)
        t[h:h + nz, h:h + ny, h:h + nx] = torch.from_numpy(
            np.ascontiguousarray(x[:, j0:j0 + ny, i0:i0 + nx])).to(dev, dt)
        f.append(t)
    for t in f[1:]:
        sl.exchange(t)
    cur = [f[0], torch.empty_like(f[0])]
    npts = nx * ny * nz

    def step():
        sl.exchange(cur[0])
        sl.s.m.step_out(cur[0], cur[1], *f[1:])
        cur.reverse()
        return sl.mass(cur[0], f[4])

    m0 = float(step())
    for _ in range(args.warmup):
        step()
    stream = torch.cuda.current_stream(dev)
    torch.cuda.synchronize(dev)
    if ws > 1:
        torch.distributed.barrier()
    launches0 = _capi.mpdata_launch_count(sl.s.m._ctx)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        mass = step()
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    if ws > 1:
        torch.distributed.barrier()
    ms = ev0.elapsed_time(ev1)
    launches = _capi.mpdata_launch_count(sl.s.m._ctx) - launches0
    m1 = float(mass)
    value, ms = job_throughput(ms, npts * args.steps, ws, dev)
    out = None
    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": wl["dtype"],
               "data": "synthetic (seeded lat-lon deformational flow, Gaussian + step tracer)",
               "config": dict(bench_config(wl_name, ws, 0), halo=h,
                              parallelism=f"slabs {px}x{py}",
                              domain=f"{NX}x{NY}x{nz}",
                              step="halo exchange + one-kernel MPDATA step + FP64 mass "
                                   "all-reduce"),
               "gpu_launches": launches,
               "mass_drift_rel": abs(m1 - m0) / abs(m0) if m0 else None}
    sl.close()
    if ws > 1:
        torch.distributed.destroy_process_group()
    return out


def measure_config(dev, wl_name, variant=None, steps=30, warmup=3):
    """Another configuration measured the same way as the headline (device
    resident inputs, CUDA events on the launching stream): value, then a
    separate pass with per-launch events for the roofline of its dominant
    kernel.  For FP32, the error of the configuration's full step count
    (100) against the FP64 step from the same FP32-rounded inputs."""
    import numpy as np
    import torch
    import synth
    from paper_1908_06094_b300 import MPDATA, _capi
    wl = WORKLOADS[wl_name]
    dt = torch.float64 if wl["dtype"] == "f64" else torch.float32
    h = wl["halo"]
    c = synth.latlon_3d(wl["nx"], wl["ny"], wl["nz"], seed=1234)
    padded = [synth.pad(x, h) for x in (c.psi, c.u, c.v, c.w, c.g)]
    d = [torch.from_numpy(x).to(dev, dt).contiguous() for x in padded]
    m = MPDATA(wl["nx"], wl["ny"], wl["nz"], halo=h, dtype=dt, device=dev)
    if variant is not None:
        m.set_variant(variant)
    npts = wl["nx"] * wl["ny"] * wl["nz"]
    out_mass = torch.empty((), dtype=torch.float64, device=dev)
    m0 = m.mass(d[0], d[4]).item()
    # the state double-buffered, as a caller of mpdata_step_out keeps it (a
    # one-kernel step cannot run in place: mpdata_step with nsteps = 1 would
    # add a copy back into psi)
    st_ = [d[0], torch.empty_like(d[0])]

    def one_step():
        m.step_out(st_[0], st_[1], *d[1:])
        st_.reverse()
    for _ in range(warmup):
        one_step()
    stream = torch.cuda.current_stream(dev)
    torch.cuda.synchronize(dev)

    def timed(profile):
        if profile:
            _capi.mpdata_profile(m._ctx, True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            one_step()
            m.mass(st_[0], d[4], out=out_mass)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1)
    ms = timed(False)
    ms_prof = timed(True)
    st = {n: _capi.mpdata_profile_read(m._ctx, sid) for n, sid in _capi.STAGES.items()}
    st = {n: v for n, v in st.items() if v[1]}
    _capi.mpdata_profile(m._ctx, False)
    m1 = out_mass.item()
    m.close()
    err = None
    if dt == torch.float32:
        # error norms of the configuration's 100 FP32 steps against 100 FP64
        # steps (the FP64 step is parity-tested against the oracle to 1e-12
        # per step) from the same FP32-rounded inputs, relative to max |psi|;
        # mass drift of each run over the 100 steps
        nsteps = wl["config_steps"]
        d64 = [x.double() for x in d]
        d32 = [x.clone() for x in d]
        m64 = MPDATA(wl["nx"], wl["ny"], wl["nz"], halo=h, dtype=torch.float64, device=dev)
        m32 = MPDATA(wl["nx"], wl["ny"], wl["nz"], halo=h, dtype=torch.float32, device=dev)
        d64[0] = torch.from_numpy(padded[0]).to(dev, torch.float32).double()
        d32[0] = d64[0].float()
        mass64_0 = m64.mass(d64[0], d64[4]).item()
        mass32_0 = m32.mass(d32[0], d32[4]).item()
        m64.step(*d64, nsteps=nsteps)
        m32.step(*d32, nsteps=nsteps)
        mass64 = m64.mass(d64[0], d64[4]).item()
        mass32 = m32.mass(d32[0], d32[4]).item()
        diff = (d32[0].double() - d64[0])[h:-h, h:-h, h:-h]
        scale = float(d64[0][h:-h, h:-h, h:-h].abs().max())
        err = {"steps": nsteps, "max_abs_rel": float(diff.abs().max()) / scale,
               "l2_rel": float(diff.pow(2).mean().sqrt()) / scale,
               "mass_drift_rel_f32": abs(mass32 - mass32_0) / abs(mass32_0),
               "mass_drift_rel_f64": abs(mass64 - mass64_0) / abs(mass64_0),
               "mass_f32_vs_f64_rel": abs(mass32 - mass64) / abs(mass64),
               "reference": "the FP64 step on the same FP32-rounded inputs"}
        m64.close()
        m32.close()
    hbm, _ = _peaks()
    esize = 8 if dt == torch.float64 else 4
    dom = max(st, key=lambda n: st[n][0])
    per = st[dom][0] / st[dom][1]
    gbs = STAGE_WORDS[dom] * esize * npts / (per / 1e3) / 1e9
    value = npts * steps / (ms / 1e3)
    return {"workload": f"latlon_3d {wl['nx']}x{wl['ny']}x{wl['nz']} {wl['dtype']}",
            "value": value, "unit": UNIT, "ms_per_step": ms / steps,
            "profiled_ms_per_step": ms_prof / steps, "dtype": wl["dtype"],
            "hbm_roofline_frac_step": round(value * STEP_WORDS * esize / 1e9 / hbm, 4),
            "mass_drift_rel_after_steps": abs(m1 - m0) / abs(m0),
            "error_vs_f64": err,
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": round(gbs, 1), "peak": hbm,
                         "unit": "GB/s", "frac": round(gbs / hbm, 4),
                         "traffic": _traffic_from_profiles(dom, wl_name, _source_hash(dom)),
                         "algorithmic_bytes": STAGE_WORDS[dom] * esize * npts,
                         "launch_ms": round(per, 5)}}


def measure_rotation_2d(dev, nsteps=100, reps=5):
    """The 2D configuration: 64x64 periodic, one level, FP64, iord 2 with the
    limiter, G = 1, solid-body rotation of a cone (max Courant 0.5), 100
    steps.  Latency-bound (4096 points), so the unit is microseconds per step:
    the 100 steps issued as plain calls, and replayed from one captured CUDA
    graph; median of reps runs each.  The oracle runs the same 100 steps on
    the host cores."""
    import torch
    import synth
    import oracle
    from paper_1908_06094_b300 import MPDATA
    c = synth.rotation_2d(64, seed=1234)
    h = 2
    P = [synth.pad(x, h) for x in (c.psi, c.u, c.v, c.w, c.g)]
    d = [torch.from_numpy(x).to(dev).contiguous() for x in P]
    m = MPDATA(c.nx, c.ny, c.nz, halo=h, iord=2, nonoscillatory=True, dtype=torch.float64,
               device=dev)
    stream = torch.cuda.current_stream(dev)
    psi = d[0].clone()
    m.step(psi, *d[1:], nsteps=3)
    torch.cuda.synchronize(dev)

    def run_plain():
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(nsteps):
            m.step(psi, *d[1:], nsteps=1)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1)
    plain = sorted(run_plain() for _ in range(reps))[reps // 2]
    # one graph of the 100 steps
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream(dev)
    s.wait_stream(stream)
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            for _ in range(nsteps):
                m.step(psi, *d[1:], nsteps=1)
    stream.wait_stream(s)
    g.replay()
    torch.cuda.synchronize(dev)

    def run_graph():
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.replay()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1)
    graph = sorted(run_graph() for _ in range(reps))[reps // 2]
    # the same 100 steps as one call (the library alternates its own buffers,
    # with no copy back between steps), captured and replayed the same way
    g100 = torch.cuda.CUDAGraph()
    s.wait_stream(stream)
    with torch.cuda.stream(s):
        with torch.cuda.graph(g100, stream=s):
            m.step(psi, *d[1:], nsteps=nsteps)
    stream.wait_stream(s)
    g100.replay()
    torch.cuda.synchronize(dev)

    def run_graph100():
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g100.replay()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1)
    graph100 = sorted(run_graph100() for _ in range(reps))[reps // 2]
    psi.copy_(d[0])
    g100.replay()
    torch.cuda.synchronize(dev)
    one_call = psi.clone()
    # parity of the 100 graph-replayed steps from the initial field
    psi.copy_(d[0])
    g.replay()
    torch.cuda.synchronize(dev)
    ref = oracle.run(*P, h=h, iord=2, nonosc=1, nsteps=nsteps)
    got = psi.cpu().numpy()
    err = float(abs(got - ref)[h:-h, h:-h, h:-h].max() / abs(ref[h:-h, h:-h, h:-h]).max())
    m.close()
    t0 = time.perf_counter()
    oracle.run(*P, h=h, iord=2, nonosc=1, nsteps=nsteps)
    cpu_s = time.perf_counter() - t0
    npts = c.nx * c.ny * c.nz
    return {"workload": "rotation_2d 64x64x1 f64 iord=2 nonoscillatory, 100 steps",
            "unit": "us/step", "higher_is_better": False,
            "us_per_step_plain": round(plain / nsteps * 1e3, 2),
            "us_per_step_graph": round(graph / nsteps * 1e3, 2),
            "us_per_step_one_call_graph": round(graph100 / nsteps * 1e3, 2),
            "one_call_equals_single_steps": bool(torch.equal(one_call, psi)),
            "value": round(graph / nsteps * 1e3, 2),
            "updates_per_s_graph": npts * nsteps / (graph / 1e3),
            "max_rel_err_vs_oracle_after_100_steps": err,
            "cpu_baseline": {"value": round(cpu_s / nsteps * 1e6, 2), "unit": "us/step",
                             "cores": os.cpu_count() or 1, "kind": "oracle",
                             "sample": "the same 100 steps"}}


def measure_options(dev, steps=20, warmup=3):
    """The corrective-pass options (DFL, ABS, IGA) on both workloads, measured
    like the headline (device-resident inputs, CUDA events, per-stage event
    timing), against the basic step of the same context shape.  ABS and IGA
    advance a signed tracer (the lat-lon tracer minus 1/2)."""
    import torch
    import synth
    from paper_1908_06094_b300 import MPDATA, _capi
    opts = {"basic": 0, "dfl": _capi.MPDATA_OPT_DFL, "abs": _capi.MPDATA_OPT_ABS,
            "iga": _capi.MPDATA_OPT_IGA}
    res = {}
    for wl_name in ("latlon256_f64", "latlon512_f32"):
        wl = WORKLOADS[wl_name]
        dt = torch.float64 if wl["dtype"] == "f64" else torch.float32
        h = wl["halo"]
        c = synth.latlon_3d(wl["nx"], wl["ny"], wl["nz"], seed=1234)
        d = [torch.from_numpy(synth.pad(x, h)).to(dev, dt).contiguous()
             for x in (c.psi, c.u, c.v, c.w, c.g)]
        signed = d[0] - 0.5
        npts = wl["nx"] * wl["ny"] * wl["nz"]
        stream = torch.cuda.current_stream(dev)
        row = {}
        for name, o in opts.items():
            m = MPDATA(wl["nx"], wl["ny"], wl["nz"], halo=h, dtype=dt, device=dev, options=o)
            psi = (signed if o & (_capi.MPDATA_OPT_ABS | _capi.MPDATA_OPT_IGA) else d[0]).clone()
            m.step(psi, *d[1:], nsteps=warmup)
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                m.step(psi, *d[1:], nsteps=1)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms = e0.elapsed_time(e1) / steps
            # the stage split from a few more steps with per-launch events
            _capi.mpdata_profile(m._ctx, True)
            m.step(psi, *d[1:], nsteps=5)
            torch.cuda.synchronize(dev)
            st = {n: _capi.mpdata_profile_read(m._ctx, sid) for n, sid in _capi.STAGES.items()}
            _capi.mpdata_profile(m._ctx, False)
            m.close()
            row[name] = {"value": npts / (ms / 1e3), "unit": UNIT, "ms_per_step": round(ms, 4),
                         "stage_ms_per_step": {n: round(v[0] / 5, 4)
                                               for n, v in st.items() if v[1]}}
        for name in opts:
            row[name]["vs_basic_time"] = round(row[name]["ms_per_step"] /
                                               row["basic"]["ms_per_step"], 3)
        res[wl_name] = row
    # the oracle with each option, on the FP64 grid (host cores)
    import oracle
    wl = WORKLOADS["latlon256_f64"]
    c = synth.latlon_3d(wl["nx"], wl["ny"], wl["nz"], seed=1234)
    P = [synth.pad(x, 2) for x in (c.psi, c.u, c.v, c.w, c.g)]
    npts = wl["nx"] * wl["ny"] * wl["nz"]
    res["cpu_baseline"] = {
        name: _oracle_sample(
            lambda o=o: oracle.run(P[0] - (0.5 if o & (oracle.ABS | oracle.IGA) else 0.0),
                                   *P[1:], h=2, iord=2, nonosc=1, opts=o), npts, 1.5,
            UNIT, f"one step of latlon_3d {wl['nx']}x{wl['ny']}x{wl['nz']}")
        for name, o in (("dfl", oracle.DFL), ("abs", oracle.ABS), ("iga", oracle.IGA))}
    return res


def measure_adjoint(dev, dtype, nsteps=20, ckpt=5, reps=2, cpu_seconds=0.0):
    """Forward and backward (recompute + adjoint) time of nsteps steps with
    checkpointing, on the 256x256x64 lat-lon case (the adjoint config)."""
    import numpy as np
    import torch
    import synth
    from paper_1908_06094_b300 import MPDATA, mpdata_run
    c = synth.latlon_3d(256, 256, 64, seed=1234)
    h = 2
    padded = [synth.pad(x, h) for x in (c.psi, c.u, c.v, c.w, c.g)]
    d = [torch.from_numpy(x).to(dev, dtype).contiguous() for x in padded]
    rng = np.random.default_rng(1235)
    obs = d[0] + torch.from_numpy(synth.pad(0.01 * rng.standard_normal(c.psi.shape), h)).to(dev, dtype)
    m = MPDATA(c.nx, c.ny, c.nz, halo=h, dtype=dtype, device=dev)
    stream = torch.cuda.current_stream(dev)
    best = None
    for r in range(reps + 1):
        x = [t.clone().requires_grad_(True) for t in d[:4]]
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        torch.cuda.synchronize(dev)
        e0.record(stream)
        out = mpdata_run(m, *x, d[4], nsteps, ckpt)
        e1.record(stream)
        loss = torch.sum((out - obs) ** 2 * d[4])
        loss.backward()
        e2.record(stream)
        torch.cuda.synchronize(dev)
        f, b = e0.elapsed_time(e1), e1.elapsed_time(e2)
        if r > 0 and (best is None or f + b < best[0] + best[1]):
            best = (f, b)
    m.close()
    out = {"fwd_ms": round(best[0], 3), "bwd_ms": round(best[1], 3),
           "ratio": round(best[1] / best[0], 3), "steps": nsteps, "ckpt": ckpt,
           "grid": "256x256x64", "backward": "recompute per segment + adjoint steps"}
    if cpu_seconds > 0:
        import oracle
        dy = synth.pad(rng.standard_normal(c.psi.shape), h)
        npts = c.nx * c.ny * c.nz
        out["cpu_baseline"] = _oracle_sample(
            lambda: oracle.adjoint(*padded, dy, h=h, iord=2, nonosc=1, nsteps=1), npts,
            cpu_seconds, "reverse-step cell-updates/s (GPU: steps x cells / bwd time)",
            "one reverse step of the same grid (forward recomputed)")
        out["value_gpu"] = nsteps * npts / (best[1] / 1e3)
    return out


def measure_batched(dev, steps=20, warmup=3, config=None):
    """Batched configuration: 64 domains (log-uniform 32x32x16..256x256x64)
    x 8 tracers, FP32, iord 2 with the limiter, one graph-replayed persistent
    launch per step, tile shape and chunk autotuned (or config = (shape,
    kchunk) given).  Unit: tracer-updates/s."""
    import torch
    import synth
    from paper_1908_06094_b300 import MPDATABatch
    hbm, _ = _peaks()
    cases = synth.batched_domains(64, 8, seed=1234)
    h = 2
    doms = []
    for c in cases:
        d = dict(psi=torch.from_numpy(synth.pad(c.psi, h)).to(dev, torch.float32).contiguous(),
                 halo=h)
        for k in ("u", "v", "w", "g"):
            d[k] = torch.from_numpy(synth.pad(getattr(c, k), h)).to(dev, torch.float32).contiguous()
        doms.append(d)
    b = MPDATABatch(doms)
    if config is None:
        cfg = b.autotune(reps=3)
    else:
        b.set_config(*config)
        cfg = dict(b.config(), cached=False, given=True)
    b.step(warmup, graph=True)
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    b.step(steps, graph=True)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1)
    n = b.npoints
    value = n * steps / (ms / 1e3)
    b.close()
    gbs = value * 10 / 1e9
    # the oracle on the batch's tracers, domain by domain (FP64, host cores)
    import oracle

    def one_pass():
        for c in cases:
            P = [synth.pad(getattr(c, k), h) for k in ("u", "v", "w", "g")]
            oracle.run(synth.pad(c.psi[0], h), *P, h=h, iord=2, nonosc=1, nsteps=1)
    tracer_pts_per_pass = sum(c.nx * c.ny * c.nz for c in cases)
    cpu = _oracle_sample(one_pass, tracer_pts_per_pass, 3.0, "tracer-point updates/s",
                         "one step of the first tracer of each of the 64 domains")
    return {"metric": "tracer-point updates/s", "value": value, "ms_per_step": ms / steps,
            "tracer_points": n, "domains": 64, "tracers": 8, "dtype": "f32",
            "config": cfg, "launches_per_step": 1,
            "roofline": {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm, "unit": "GB/s",
                         "frac": round(gbs / hbm, 4),
                         "algorithmic_bytes_per_update": 10},
            "cpu_baseline": cpu}


# --------------------------------------------------------- reference arm --

def run_reference(args, wl_name):
    ws, rank, _ = _dist()
    if rank != 0:
        return None
    import numpy as np
    import oracle
    import synth
    wl = WORKLOADS[wl_name]
    h = wl["halo"]
    case = synth.latlon_3d(wl["nx"], wl["ny"], wl["nz"], seed=1234)
    P = [synth.pad(x, h) for x in (case.psi, case.u, case.v, case.w, case.g)]
    if wl["dtype"] == "f32":
        P = [x.astype(np.float32).astype(np.float64) for x in P]
    npts = wl["nx"] * wl["ny"] * wl["nz"]
    # each step is a bounded sample of the workload: the full grid if one
    # oracle step is short, else a slab of levels
    nz_s = wl["nz"]
    t0 = time.perf_counter()
    oracle.run(*P, h=h, iord=wl["iord"], nonosc=wl["nonosc"], nsteps=1)
    one = time.perf_counter() - t0
    budget = 120.0 / max(1, args.steps + args.warmup)
    if one > budget:
        nz_s = max(2, int(wl["nz"] * budget / one))
        case = synth.latlon_3d(wl["nx"], wl["ny"], wl["nz"], seed=1234)
        P = [synth.pad(x[:nz_s], h) for x in (case.psi, case.u, case.v, case.w, case.g)]
        P[3][h + nz_s - 1] = 0.0
    cur = P[0]
    for _ in range(args.warmup):
        cur = oracle.run(cur, *P[1:], h=h, iord=wl["iord"], nonosc=wl["nonosc"], nsteps=1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        cur = oracle.run(cur, *P[1:], h=h, iord=wl["iord"], nonosc=wl["nonosc"], nsteps=1)
    el = time.perf_counter() - t0
    n_s = wl["nx"] * wl["ny"] * nz_s
    value = n_s * args.steps / el
    ncores = os.cpu_count() or 1
    sample = (f"{'full grid' if nz_s == wl['nz'] else f'{nz_s}-level slab'} "
              f"{wl['nx']}x{wl['ny']}x{nz_s}, one step per bench step")
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded)",
            "config": bench_config(wl_name, ws, args.variant),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": ncores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


# The paper's own workload for its flux stages (Sec. 5, Listings 5-9): the
# global grid of Table 2 / Fig. 14 (71424 nodes, 80 levels) as a periodic
# 279 x 256 triangular patch, open vertical boundaries.
EDGE_SHAPE = (279, 256, 80)
# words moved per node-level (Table 2's counting, every 3D field counted,
# 2D fields ignored): fused reads pD, 3 vn, W, rho and writes pD; staged
# adds the edge fluxes (3 w + 3 r), the vertical fluxes (1 w + 1 r), the
# divergence (1 w + 1 r) and the second and third reads of pD
EDGE_WORDS = {"fused": 7, "staged": 19}
# FP64 pipe operations per node-level of the fused kernel: 1 DMUL + 5 DFMA
# (edge fluxes), 2 DMUL (vertical fluxes), 2 DADD, 1 DMUL (vol rho), the
# reciprocal (3 DFMA after the hardware seed) and the final DFMA
EDGE_FP64_OPS = 15


def _edge_case():
    from synth import octahedral as octa
    nr, nc, nz = EDGE_SHAPE
    return octa.edge_case(nr, nc, nz, seed=1234, pivbz=1.0)


def measure_edge(dev, reps=20, cpu_seconds=5.0):
    """The edge-based flux stages on the 71424 x 80 patch, both dtypes, both
    organisations: median of reps launches with L2 flushed before each
    (CUDA events on the launching stream).  Units: node-level updates/s."""
    import torch
    from paper_1908_06094_b300 import EdgeMPDATA
    import oracle
    hbm, _ = _peaks()
    c = _edge_case()
    nr, nc, nz = EDGE_SHAPE
    npts = nr * nc * nz
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    res = {"workload": f"periodic triangular patch {nr}x{nc} nodes (71424), {nz} levels, pivbz 1",
           "unit": "node-level updates/s", "l2": "flushed (256 MB write) before each launch"}
    for dt in (torch.float64, torch.float32):
        name = "f64" if dt == torch.float64 else "f32"
        esize = 8 if dt == torch.float64 else 4
        f = {k: torch.from_numpy(getattr(c, k)).to(dev, dt).contiguous()
             for k in ("pD", "vn", "wn", "rho", "vol")}
        outb = torch.empty_like(f["pD"])
        row = {}
        for var, vname in ((0, "fused"), (1, "staged")):
            e = EdgeMPDATA(nr, nc, nz, dtype=dt, pivbz=1.0, variant=var, device=dev)
            for _ in range(3):
                e.step(f["pD"], outb, f["vn"], f["wn"], f["rho"], f["vol"])
            torch.cuda.synchronize(dev)
            ts = []
            for _ in range(reps):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                e.step(f["pD"], outb, f["vn"], f["wn"], f["rho"], f["vol"])
                e1.record(stream)
                torch.cuda.synchronize(dev)
                ts.append(e0.elapsed_time(e1))
            ts.sort()
            ms = ts[len(ts) // 2]
            algo = EDGE_WORDS[vname] * esize * npts
            gbs = algo / (ms / 1e3) / 1e9
            r = {"value": npts / (ms / 1e3), "ms": round(ms, 5), "launches": 1 if var == 0 else 4,
                 "algorithmic_bytes": algo, "achieved_gbs": round(gbs, 1),
                 "hbm_frac": round(gbs / hbm, 4)}
            if var == 0:
                r["width"] = e.width()
                src = _source_hash("edge")
                r["traffic"] = _traffic_from_profiles(f"edge_fused_{name}", "octa71424x80", src)
                if dt == torch.float64:
                    ach = EDGE_FP64_OPS * npts / (ms / 1e3) / 1e9
                    r["fp64_ops_frac"] = round(ach / (FP64_PEAK_GFLOPS / 2), 4)
            else:
                r["traffic"] = _traffic_from_profiles(f"edge_staged_{name}", "octa71424x80",
                                                      _source_hash("edge"))
            row[vname] = r
            e.close()
        row["staged_over_fused_time"] = round(row["staged"]["ms"] / row["fused"]["ms"], 3)
        res[name] = row
    N, E = nr * nc, 3 * nr * nc
    res["table2_accesses_per_plane"] = {"without_fusion": 2 * E + 10 * N, "with_fusion": 5 * N,
                                        "ratio": round((2 * E + 10 * N) / (5 * N), 3)}
    # the oracle (the same stages through the connectivity tables), host cores
    t0 = time.perf_counter()
    k = 0
    while True:
        oracle.edge_run(c, nsteps=1)
        k += 1
        if time.perf_counter() - t0 >= cpu_seconds:
            break
    res["cpu_baseline"] = {"value": npts * k / (time.perf_counter() - t0),
                           "unit": "node-level updates/s", "cores": os.cpu_count() or 1,
                           "kind": "oracle", "sample": f"{k} full steps of the same patch"}
    return res


def measure_cells(dev, reps=15):
    """Table 1 on the B300: the cell-neighbour sum B = sum of A over the
    three edge neighbours, and the two-stage operator (B = fac1 x sum A,
    C = fac2 x sum B: two launches), under structured numbering with direct
    access (SN DA) and with its table (SN IA), a mesh library's numbering
    through its table (UN IA) and a Hilbert numbering (HN IA).  Bandwidth =
    required transfer / time as in Table 1, the required transfer being
    each launch's input and output fields (2 words per cell-level per
    launch); median of reps with L2 flushed before each.  The paper's patch
    (128 x 128 x 80 nodes) holds 21 MB per FP64 field, inside the B300's
    126 MB L2, so a 512 x 512 x 80 patch (335 MB per field) is measured
    too."""
    import torch
    from paper_1908_06094_b300 import CellsReduction
    from synth import cells
    hbm, _ = _peaks()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    res = {"unit": "GB/s (required transfer / time)", "l2": "flushed before each measurement",
           "paper_p100_gbs": {"SN DA": [211, 226], "SN IA": [270, 269], "UN IA": [130, 135],
                              "HN IA": [256, 240]}}
    for (nr, nc, nz) in ((128, 128, 80), (512, 512, 80)):
        for dt in (torch.float64, torch.float32):
            esize = 8 if dt == torch.float64 else 4
            n = 2 * nr * nc * nz
            row = {}
            for numbering, access in (("SN", "direct"), ("SN", "indirect"), ("UN", "indirect"),
                                      ("HN", "indirect")):
                if access == "direct":
                    red = CellsReduction(nz, dtype=dt, nr=nr, nc=nc, device=dev)
                else:
                    red = CellsReduction(nz, dtype=dt, table=cells.c2c(nr, nc, numbering),
                                         device=dev)
                A = torch.from_numpy(cells.field(nr, nc, nz, seed=1, numbering=numbering)).to(
                    dev, dt).contiguous()
                B = torch.empty_like(A)
                Cf = torch.empty_like(A)
                out = {}
                for op in ("sum", "two_stage"):
                    def run():
                        red.sum(A, B, 1.0)
                        if op == "two_stage":
                            red.sum(B, Cf, 0.5)
                    for _ in range(3):
                        run()
                    ts = []
                    for _ in range(reps):
                        flush.zero_()
                        e0 = torch.cuda.Event(enable_timing=True)
                        e1 = torch.cuda.Event(enable_timing=True)
                        e0.record(stream)
                        run()
                        e1.record(stream)
                        torch.cuda.synchronize(dev)
                        ts.append(e0.elapsed_time(e1))
                    ts.sort()
                    ms = ts[len(ts) // 2]
                    words = 2 if op == "sum" else 4
                    out[op] = {"us": round(ms * 1e3, 2),
                               "gbs": round(words * esize * n / (ms / 1e3) / 1e9, 1)}
                row[f"{numbering} {'DA' if access == 'direct' else 'IA'}"] = out
                red.close()
            res[f"{nr}x{nc}x{nz}_{'f64' if esize == 8 else 'f32'}"] = row
    res["hbm_peak_gbs"] = hbm
    # the oracle's table-driven sum, host cores, on the larger patch
    import oracle
    nr, nc, nz = 512, 512, 80
    t = cells.c2c(nr, nc, "SN")
    A = cells.field(nr, nc, nz, seed=1)
    res["cpu_baseline"] = _oracle_sample(lambda: oracle.cells_sum(t, A, 1.0), 2 * nr * nc * nz,
                                         2.0, "cell-level updates/s",
                                         "the sum on the 512x512x80 patch, SN table")
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="latlon256_f64", choices=sorted(WORKLOADS))
    ap.add_argument("--variant", type=int, default=None, help="0 fused, 1 staged, 2 auto (default)")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the e2e and CPU-baseline legs")
    ap.add_argument("--decomp", default="replicas", choices=["replicas", "slab"],
                    help="N > 1: independent replicas (default) or one i-j decomposed "
                         "domain with a halo exchange")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.impl == "reference":
        out = run_reference(args, args.workload)
    elif args.decomp == "slab":
        out = run_slab(args, args.workload)
    else:
        out = run_ours(args, args.workload)
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
