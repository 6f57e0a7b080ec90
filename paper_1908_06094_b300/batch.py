"""Batched MPDATA: many independent domains, several tracers each, one
persistent graph-captured launch per step (torch front end of the
mpdata_batch_* C calls)."""
from __future__ import annotations

import hashlib
import json
import os

import torch

from . import _capi as C

_DT = {torch.float64: C.MPDATA_F64, torch.float32: C.MPDATA_F32}


class MPDATABatch:
    """domains: list of dicts with keys psi (tensor [ntracers, nz+2h, ny+2h,
    nx+2h]), u, v, w, g (padded tensors [nz+2h, ny+2h, nx+2h]) and halo.
    The batch owns a second tracer buffer per domain and steps ping-pong;
    ``state(d)`` is the current tracer tensor of domain d."""

    def __init__(self, domains, nonoscillatory=True, device=None):
        if not domains:
            raise ValueError("empty batch")
        self.dtype = domains[0]["psi"].dtype
        if self.dtype not in _DT:
            raise TypeError("float64 or float32 tracers")
        self.device = torch.device(device) if device is not None else domains[0]["psi"].device
        self.stream = torch.cuda.Stream(device=self.device)  # capture needs its own stream
        self.doms, descs = [], []
        for d in domains:
            psi = d["psi"]
            h = int(d["halo"])
            ntr, pz, py, px = psi.shape
            nz, ny, nx = pz - 2 * h, py - 2 * h, px - 2 * h
            for k in ("u", "v", "w", "g"):
                t = d[k]
                if t.dtype != self.dtype or tuple(t.shape) != (pz, py, px) or not t.is_contiguous():
                    raise ValueError(f"domain field {k}: expected {(pz, py, px)} {self.dtype}")
            if not psi.is_contiguous():
                raise ValueError("psi must be contiguous")
            other = torch.empty_like(psi)
            self.doms.append(dict(a=psi, b=other, u=d["u"], v=d["v"], w=d["w"], g=d["g"],
                                  nx=nx, ny=ny, nz=nz, h=h, ntr=ntr))
            descs.append(C.mpdata_domain_desc(nx, ny, nz, h, ntr, psi.data_ptr(), other.data_ptr(),
                                              d["u"].data_ptr(), d["v"].data_ptr(),
                                              d["w"].data_ptr(), d["g"].data_ptr()))
        with torch.cuda.device(self.device):
            self._b = C.mpdata_batch_init(descs, int(bool(nonoscillatory)), _DT[self.dtype],
                                          self.stream.cuda_stream)
        self.cur = 0  # 0: state in the "a" buffers

    def close(self):
        if getattr(self, "_b", None):
            C.mpdata_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def npoints(self):
        return sum(d["nx"] * d["ny"] * d["nz"] * d["ntr"] for d in self.doms)

    def state(self, i):
        d = self.doms[i]
        return d["a"] if self.cur == 0 else d["b"]

    def step(self, nsteps: int = 1, graph: bool = True):
        """nsteps steps of every tracer (ordered after the current stream)."""
        cs = torch.cuda.current_stream(self.device)
        self.stream.wait_stream(cs)
        for _ in range(nsteps):
            C.mpdata_batch_step(self._b, self.cur, graph)
            self.cur ^= 1
        cs.wait_stream(self.stream)

    def config(self):
        return C.mpdata_batch_get_config(self._b)

    def set_config(self, shape, kchunk):
        C.mpdata_batch_set_config(self._b, shape, kchunk)

    def signature(self):
        """Shape class of the batch: dtype, domain count, tracer count and
        the sorted grid sizes (the tuned configuration depends on nothing else)."""
        dims = sorted((d["nx"], d["ny"], d["nz"], d["ntr"]) for d in self.doms)
        key = json.dumps([str(self.dtype), dims, torch.cuda.get_device_name(self.device)])
        return hashlib.sha256(key.encode()).hexdigest()[:16]

    def autotune(self, reps: int = 3, cache: str | None = None):
        """Pick the fastest tile shape and level-chunk length (timed in the
        library), cached per shape class in the JSON file ``cache``.  Tuning
        runs steps, so it saves and restores the tracer state."""
        sig = self.signature()
        table = {}
        if cache and os.path.exists(cache):
            with open(cache) as f:
                table = json.load(f)
        if sig in table:
            cfg = table[sig]
            self.set_config(cfg["shape"], cfg["kchunk"])
            return dict(cfg, cached=True)
        saved = [self.state(i).clone() for i in range(len(self.doms))]
        torch.cuda.synchronize(self.device)
        ms = C.mpdata_batch_autotune(self._b, reps)
        torch.cuda.synchronize(self.device)
        for i, s in enumerate(saved):
            self.doms[i]["a"].copy_(s)
        self.cur = 0
        cfg = dict(self.config(), ms_per_step=ms)
        if cache:
            table[sig] = cfg
            os.makedirs(os.path.dirname(os.path.abspath(cache)), exist_ok=True)
            with open(cache, "w") as f:
                json.dump(table, f, indent=1)
        return dict(cfg, cached=False)
