"""Edge-based flux stages on a structured triangular (octahedral-grid) patch:
torch front end of the mpdata_edge_* C calls.  Shapes and dtypes are
checked here; every stage runs in the library's kernels."""
from __future__ import annotations

import ctypes

import torch

from . import _capi as C

_DT = {torch.float64: C.MPDATA_F64, torch.float32: C.MPDATA_F32}


class EdgeMPDATA:
    """One patch of nr x nc nodes (periodic) and nz >= 2 levels.

    Fields (C-contiguous CUDA tensors of the context's dtype):
    pD, rho (nz, nr, nc); vn (nz, nr, 3, nc); wn (nz+1, nr, nc); vol (nr, nc).
    ``variant``: MPDATA_FUSED (default) or MPDATA_STAGED.
    """

    def __init__(self, nr, nc, nz, dtype=torch.float64, pivbz=0.0, variant=None, device=None):
        if dtype not in _DT:
            raise TypeError(f"dtype must be float64 or float32, got {dtype}")
        self.nr, self.nc, self.nz, self.dtype = nr, nc, nz, dtype
        self.device = torch.device(device if device is not None else "cuda")
        self.shapes = {"pD": (nz, nr, nc), "rho": (nz, nr, nc), "vn": (nz, nr, 3, nc),
                       "wn": (nz + 1, nr, nc), "vol": (nr, nc)}
        out = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            stream = torch.cuda.current_stream(self.device).cuda_stream
            rc = C.lib.mpdata_edge_init(ctypes.byref(out), nr, nc, nz, _DT[dtype], float(pivbz),
                                        stream)
        C._check(rc, "mpdata_edge_init")
        self._e = out.value
        if variant is not None:
            self.set_variant(variant)

    def _ptr(self, t, name, shape_key=None):
        shp = self.shapes[shape_key or name]
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise TypeError(f"{name} must be a CUDA tensor")
        if t.dtype != self.dtype or tuple(t.shape) != shp or not t.is_contiguous():
            raise ValueError(f"{name}: expected contiguous {self.dtype} {shp}, "
                             f"got {t.dtype} {tuple(t.shape)}")
        return t.data_ptr()

    def _rc(self, rc, where):
        if rc != C.MPDATA_OK:
            detail = C.lib.mpdata_edge_last_error_string(self._e).decode()
            raise C.MPDATAError(rc, where, detail)

    def set_variant(self, variant: int):
        self._rc(C.lib.mpdata_edge_set_variant(self._e, variant), "mpdata_edge_set_variant")

    def step(self, pD_in, pD_out, vn, wn, rho, vol):
        """pD_out = one application of the four stages to pD_in (current stream)."""
        self._rc(C.lib.mpdata_edge_set_stream(
            self._e, torch.cuda.current_stream(self.device).cuda_stream), "set_stream")
        self._rc(C.lib.mpdata_edge_step(
            self._e, self._ptr(pD_in, "pD_in", "pD"), self._ptr(pD_out, "pD_out", "pD"),
            self._ptr(vn, "vn"), self._ptr(wn, "wn"), self._ptr(rho, "rho"),
            self._ptr(vol, "vol")), "mpdata_edge_step")
        return pD_out

    def set_width(self, width: int):
        """Nodes per thread of the fused kernel: 1 or 4 (0: the default)."""
        self._rc(C.lib.mpdata_edge_set_width(self._e, width), "mpdata_edge_set_width")

    def width(self) -> int:
        out = ctypes.c_int()
        self._rc(C.lib.mpdata_edge_get_width(self._e, ctypes.byref(out)), "get_width")
        return out.value

    def launch_count(self) -> int:
        return C.lib.mpdata_edge_launch_count(self._e)

    def close(self):
        if getattr(self, "_e", None):
            C.lib.mpdata_edge_destroy(self._e)
            self._e = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
