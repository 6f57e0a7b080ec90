"""B300-native MPDATA step: a C-ABI CUDA library (libmpdata_b300.so) and a
thin Python binding over it.

* ``_capi``   -- ctypes binding, one function per C entry point;
* ``MPDATA``  -- the same calls taking torch CUDA tensors (pointer and stream
  marshalling only: every step of the method runs in the library's kernels);
* ``MPDATABatch`` -- many domains x tracers in one persistent launch;
* ``EdgeMPDATA`` -- the edge-based flux stages on a triangular patch;
* ``CellsReduction`` -- the cell-neighbour reduction of Table 1;
* ``MPDATAFunction`` / ``mpdata_run`` -- autograd over the forward and
  adjoint steps with checkpoint-and-recompute;
* ``SlabDecomposition`` / ``SlabRank`` -- an i-j decomposed domain with the
  halo exchange (all slabs on one device, or one slab per process).

The library is loaded on first use of either; a missing or unloadable
library raises ImportError (there is no fallback path).
"""
import importlib

__all__ = ["_capi", "MPDATA", "padded_shape", "MPDATAFunction", "mpdata_run", "MPDATABatch",
           "EdgeMPDATA", "CellsReduction", "SlabDecomposition", "SlabRank"]


def __getattr__(name):
    if name == "_capi":
        return importlib.import_module("._capi", __name__)
    if name in ("MPDATA", "padded_shape"):
        mod = importlib.import_module(".mpdata", __name__)
        return getattr(mod, name)
    if name == "CellsReduction":
        return importlib.import_module(".cells", __name__).CellsReduction
    if name == "EdgeMPDATA":
        return importlib.import_module(".edge", __name__).EdgeMPDATA
    if name == "MPDATABatch":
        return importlib.import_module(".batch", __name__).MPDATABatch
    if name in ("SlabDecomposition", "SlabRank"):
        return getattr(importlib.import_module(".slabs", __name__), name)
    if name in ("MPDATAFunction", "mpdata_run"):
        mod = importlib.import_module(".autograd", __name__)
        return getattr(mod, name)
    raise AttributeError(name)
