"""torch-tensor front end of the C ABI: checks shapes/dtypes/devices and
passes raw device pointers and the current CUDA stream.  No arithmetic."""
from __future__ import annotations

import torch

from . import _capi as C

_DT = {torch.float64: C.MPDATA_F64, torch.float32: C.MPDATA_F32}


def padded_shape(nx: int, ny: int, nz: int, h: int):
    return (nz + 2 * h, ny + 2 * h, nx + 2 * h)


class MPDATA:
    """One grid's MPDATA context (owns the library scratch of one step).

    Fields are C-contiguous CUDA tensors of shape padded_shape(nx, ny, nz, h)
    and this context's dtype; U, V, W are G-weighted Courant numbers on the
    faces i+1/2, j+1/2, k+1/2.
    """

    def __init__(self, nx, ny, nz, halo=2, iord=2, nonoscillatory=True,
                 dtype=torch.float64, device=None, variant=None, k_bc=C.MPDATA_K_ZEROFLUX,
                 options=0):
        if dtype not in _DT:
            raise TypeError(f"dtype must be float64 or float32, got {dtype}")
        self.nx, self.ny, self.nz, self.h = nx, ny, nz, halo
        self.iord, self.nonosc, self.dtype = iord, int(bool(nonoscillatory)), dtype
        self.device = torch.device(device if device is not None else "cuda")
        with torch.cuda.device(self.device):
            stream = torch.cuda.current_stream(self.device).cuda_stream
            self._ctx = C.mpdata_init(nx, ny, nz, halo, iord, self.nonosc, _DT[dtype], k_bc,
                                      stream)
        if variant is not None:
            C.mpdata_set_variant(self._ctx, variant)
        if options:
            try:
                C.mpdata_set_options(self._ctx, options)
            except Exception:
                self.close()
                raise
        self.shape = padded_shape(nx, ny, nz, halo)
        self._k_bc, self._variant = k_bc, variant
        self._shadow = None

    def shadow(self) -> "MPDATA":
        """A second context of the same grid and scheme (its own scratch),
        created on first use: calls on another stream that must not share
        this context's scratch (the adjoint's recomputed segments) use it."""
        if self._shadow is None:
            opts = C.mpdata_get_options(self._ctx)
            self._shadow = MPDATA(self.nx, self.ny, self.nz, halo=self.h, iord=self.iord,
                                  nonoscillatory=self.nonosc, dtype=self.dtype,
                                  device=self.device, variant=self._variant, k_bc=self._k_bc,
                                  options=opts)
        return self._shadow

    def close(self):
        if getattr(self, "_shadow", None) is not None:
            self._shadow.close()
            self._shadow = None
        if getattr(self, "_ctx", None):
            C.mpdata_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _ptr(self, t: torch.Tensor, name: str) -> int:
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise TypeError(f"{name} must be a CUDA tensor")
        if t.dtype != self.dtype or tuple(t.shape) != self.shape or not t.is_contiguous():
            raise ValueError(f"{name}: expected contiguous {self.dtype} tensor of shape "
                             f"{self.shape}, got {t.dtype} {tuple(t.shape)}")
        if t.device != self.device and not (self.device.index is None and t.device.type == "cuda"):
            raise ValueError(f"{name} is on {t.device}, context on {self.device}")
        return t.data_ptr()

    def _sync_stream(self):
        C.mpdata_set_stream(self._ctx, torch.cuda.current_stream(self.device).cuda_stream)

    def set_variant(self, variant: int):
        C.mpdata_set_variant(self._ctx, variant)
        self._variant = variant
        if self._shadow is not None:
            C.mpdata_set_variant(self._shadow._ctx, variant)

    def step(self, psi, u, v, w, g, nsteps: int = 1):
        """Advance psi in place by nsteps steps (asynchronous, current stream)."""
        self._sync_stream()
        C.mpdata_step(self._ctx, self._ptr(psi, "psi"), self._ptr(u, "u"), self._ptr(v, "v"),
                      self._ptr(w, "w"), self._ptr(g, "g"), nsteps)
        return psi

    def step_out(self, psi_in, psi_out, u, v, w, g):
        """One step psi_out = step(psi_in) (distinct tensors; current stream)."""
        self._sync_stream()
        C.mpdata_step_out(self._ctx, self._ptr(psi_in, "psi_in"), self._ptr(psi_out, "psi_out"),
                          self._ptr(u, "u"), self._ptr(v, "v"), self._ptr(w, "w"),
                          self._ptr(g, "g"))
        return psi_out

    def fill_halo(self, f, kind: int = C.MPDATA_HALO_CELL):
        self._sync_stream()
        C.mpdata_fill_halo(self._ctx, self._ptr(f, "field"), kind)
        return f

    def mass(self, psi, g, out=None):
        """sum psi*G over the interior as a 0-d float64 CUDA tensor (no sync)."""
        self._sync_stream()
        if out is None:
            out = torch.empty((), dtype=torch.float64, device=psi.device)
        C.mpdata_mass(self._ctx, self._ptr(psi, "psi"), self._ptr(g, "g"), out.data_ptr())
        return out

    def step_host(self, psi_h, u_h, v_h, w_h, g_h, nsteps: int = 1):
        """HOST-buffer variant: tensors on the CPU (pinned for speed); psi_h
        is overwritten with the result; returns after the stream finished."""
        for name, t in (("psi", psi_h), ("u", u_h), ("v", v_h), ("w", w_h), ("g", g_h)):
            if t.is_cuda or t.dtype != self.dtype or tuple(t.shape) != self.shape \
                    or not t.is_contiguous():
                raise ValueError(f"{name}: expected a contiguous CPU {self.dtype} tensor of "
                                 f"shape {self.shape}")
        self._sync_stream()
        C.mpdata_step_host(self._ctx, psi_h.data_ptr(), u_h.data_ptr(), v_h.data_ptr(),
                           w_h.data_ptr(), g_h.data_ptr(), nsteps)
        return psi_h

    def step_host_async(self, psi_in_h, psi_out_h, u_h, v_h, w_h, g_h, nsteps: int = 1):
        """Pipelined HOST-buffer steps (one problem of a stream): enqueues the
        copies in, nsteps steps and the copy of the result into psi_out_h,
        and returns at once; call host_wait() before touching the buffers.
        CPU tensors, pinned for the copies to overlap."""
        for name, t in (("psi_in", psi_in_h), ("psi_out", psi_out_h), ("u", u_h), ("v", v_h),
                        ("w", w_h), ("g", g_h)):
            if t.is_cuda or t.dtype != self.dtype or tuple(t.shape) != self.shape \
                    or not t.is_contiguous():
                raise ValueError(f"{name}: expected a contiguous CPU {self.dtype} tensor of "
                                 f"shape {self.shape}")
        self._sync_stream()
        C.mpdata_step_host_async(self._ctx, psi_in_h.data_ptr(), psi_out_h.data_ptr(),
                                 u_h.data_ptr(), v_h.data_ptr(), w_h.data_ptr(), g_h.data_ptr(),
                                 nsteps)
        return psi_out_h

    def step_host_interior_async(self, psi_in_h, psi_out_h, u_h, v_h, w_h, g_h,
                                 nsteps: int = 1):
        """step_host_async for CPU tensors of the interior alone, shape
        (nz, ny, nx): only the interior crosses the host link, and psi_out_h
        receives the interior of the result."""
        shape = (self.nz, self.ny, self.nx)
        for name, t in (("psi_in", psi_in_h), ("psi_out", psi_out_h), ("u", u_h), ("v", v_h),
                        ("w", w_h), ("g", g_h)):
            if t.is_cuda or t.dtype != self.dtype or tuple(t.shape) != shape \
                    or not t.is_contiguous():
                raise ValueError(f"{name}: expected a contiguous CPU {self.dtype} tensor of "
                                 f"shape {shape}")
        self._sync_stream()
        C.mpdata_step_host_interior_async(self._ctx, psi_in_h.data_ptr(), psi_out_h.data_ptr(),
                                          u_h.data_ptr(), v_h.data_ptr(), w_h.data_ptr(),
                                          g_h.data_ptr(), nsteps)
        return psi_out_h

    def host_wait(self):
        """Wait for every problem enqueued by step_host_async or
        step_host_interior_async."""
        C.mpdata_host_wait(self._ctx)
