"""Cell-neighbour reduction of Table 1: torch front end of the
mpdata_cells_* C calls (argument marshalling only)."""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _capi as C

_DT = {torch.float64: C.MPDATA_F64, torch.float32: C.MPDATA_F32}


class CellsReduction:
    """B = fac x the sum of A over each cell's three edge neighbours.

    ``table`` (numpy int32 [3][ncells]) selects indirect access in its
    numbering; without it the cells are those of a periodic nr x nc patch
    in structured numbering, reached by direct access.  Fields are CUDA
    tensors [nz][ncells] of the context's dtype."""

    def __init__(self, nz, dtype=torch.float64, table=None, nr=0, nc=0, device=None):
        if dtype not in _DT:
            raise TypeError(f"dtype must be float64 or float32, got {dtype}")
        self.dtype = dtype
        self.device = torch.device(device if device is not None else "cuda")
        if table is not None:
            t = np.ascontiguousarray(table, dtype=np.int32)
            if t.ndim != 2 or t.shape[0] != 3:
                raise ValueError("table: [3][ncells] int32")
            ncells = t.shape[1]
            tp = t.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        else:
            ncells, tp = 2 * nr * nc, None
        self.shape = (nz, ncells)
        out = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            stream = torch.cuda.current_stream(self.device).cuda_stream
            rc = C.lib.mpdata_cells_init(ctypes.byref(out), ncells, nz, _DT[dtype], tp, nr, nc,
                                         stream)
        C._check(rc, "mpdata_cells_init")
        self._c = out.value

    def _ptr(self, t, name):
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise TypeError(f"{name} must be a CUDA tensor")
        if t.dtype != self.dtype or tuple(t.shape) != self.shape or not t.is_contiguous():
            raise ValueError(f"{name}: expected contiguous {self.dtype} {self.shape}")
        return t.data_ptr()

    def sum(self, A, B, fac: float = 1.0):
        """B = fac x neighbour sum of A (current stream); returns B."""
        C.lib.mpdata_cells_set_stream(self._c, torch.cuda.current_stream(self.device).cuda_stream)
        rc = C.lib.mpdata_cells_sum(self._c, self._ptr(A, "A"), self._ptr(B, "B"), float(fac))
        if rc != C.MPDATA_OK:
            raise C.MPDATAError(rc, "mpdata_cells_sum",
                                C.lib.mpdata_cells_last_error_string(self._c).decode())
        return B

    def close(self):
        if getattr(self, "_c", None):
            C.lib.mpdata_cells_destroy(self._c)
            self._c = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
