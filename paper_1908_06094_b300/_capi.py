"""ctypes binding of libmpdata_b300.so: the C ABI of include/mpdata.h, one
Python function per C function, same names, argument marshalling only.

There is no fallback: if the library is missing or does not load, importing
this module raises.  Build it with ``python -m paper_1908_06094_b300.build``.
"""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libmpdata_b300.so")

MPDATA_OK = 0
MPDATA_EINVAL = -1
MPDATA_ENOMEM = -2
MPDATA_ECUDA = -3
MPDATA_EALIGN = -4
MPDATA_EDEVICE = -5
MPDATA_ERANGE = -6
MPDATA_F64 = 0
MPDATA_F32 = 1
MPDATA_K_ZEROFLUX = 0
MPDATA_K_PERIODIC = 1
MPDATA_HALO_CELL = 0
MPDATA_HALO_WFACE = 1
MPDATA_FUSED = 0
MPDATA_STAGED = 1
MPDATA_AUTO = 2
MPDATA_OPT_DFL = 1
MPDATA_OPT_ABS = 2
MPDATA_OPT_IGA = 4

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libmpdata_b300.so not built (expected at {LIB_PATH}); "
                      "run `python -m paper_1908_06094_b300.build`")

lib = ctypes.CDLL(LIB_PATH)

_c = ctypes.c_void_p
_i = ctypes.c_int
_ctxpp = ctypes.POINTER(ctypes.c_void_p)

class mpdata_domain_desc(ctypes.Structure):
    """struct mpdata_domain_desc of include/mpdata.h."""
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("halo", ctypes.c_int), ("ntracers", ctypes.c_int),
                ("psi_a", ctypes.c_void_p), ("psi_b", ctypes.c_void_p),
                ("u", ctypes.c_void_p), ("v", ctypes.c_void_p), ("w", ctypes.c_void_p),
                ("g", ctypes.c_void_p)]


_dp = ctypes.POINTER(mpdata_domain_desc)
_ip = ctypes.POINTER(ctypes.c_int)

# symbol -> (restype, argtypes); the list is the ABI that include/mpdata.h declares
SIGNATURES = {
    "mpdata_init": (_i, [_ctxpp, _i, _i, _i, _i, _i, _i, _i, _i, _c]),
    "mpdata_set_stream": (_i, [_c, _c]),
    "mpdata_set_variant": (_i, [_c, _i]),
    "mpdata_set_options": (_i, [_c, _i]),
    "mpdata_edge_init": (_i, [_ctxpp, _i, _i, _i, _i, ctypes.c_double, _c]),
    "mpdata_edge_set_stream": (_i, [_c, _c]),
    "mpdata_edge_set_variant": (_i, [_c, _i]),
    "mpdata_edge_step": (_i, [_c, _c, _c, _c, _c, _c, _c]),
    "mpdata_edge_set_width": (_i, [_c, _i]),
    "mpdata_edge_get_width": (_i, [_c, _ip]),
    "mpdata_edge_launch_count": (ctypes.c_longlong, [_c]),
    "mpdata_edge_last_error_string": (ctypes.c_char_p, [_c]),
    "mpdata_edge_destroy": (None, [_c]),
    "mpdata_cells_init": (_i, [_ctxpp, ctypes.c_longlong, _i, _i, _ip, _i, _i, _c]),
    "mpdata_cells_set_stream": (_i, [_c, _c]),
    "mpdata_cells_sum": (_i, [_c, _c, _c, ctypes.c_double]),
    "mpdata_cells_launch_count": (ctypes.c_longlong, [_c]),
    "mpdata_cells_last_error_string": (ctypes.c_char_p, [_c]),
    "mpdata_cells_destroy": (None, [_c]),
    "mpdata_get_options": (_i, [_c, _ip]),
    "mpdata_step": (_i, [_c, _c, _c, _c, _c, _c, _i]),
    "mpdata_step_out": (_i, [_c, _c, _c, _c, _c, _c, _c]),
    "mpdata_step_host": (_i, [_c, _c, _c, _c, _c, _c, _i]),
    "mpdata_step_host_async": (_i, [_c, _c, _c, _c, _c, _c, _c, _i]),
    "mpdata_step_host_interior_async": (_i, [_c, _c, _c, _c, _c, _c, _c, _i]),
    "mpdata_host_wait": (_i, [_c]),
    "mpdata_fill_halo": (_i, [_c, _c, _i]),
    "mpdata_adjoint_step": (_i, [_c] * 10),
    "mpdata_fold_halo_adjoint": (_i, [_c, _c]),
    "mpdata_tape_bytes": (_i, [_c, ctypes.POINTER(ctypes.c_size_t)]),
    "mpdata_step_tape": (_i, [_c] * 8),
    "mpdata_adjoint_step_tape": (_i, [_c] * 11),
    "mpdata_mass": (_i, [_c, _c, _c, _c]),
    "mpdata_destroy": (None, [_c]),
    "mpdata_strerror": (ctypes.c_char_p, [_i]),
    "mpdata_last_error_string": (ctypes.c_char_p, [_c]),
    "mpdata_version": (_i, []),
    "mpdata_launch_count": (ctypes.c_longlong, [_c]),
    "mpdata_batch_init": (_i, [_ctxpp, _dp, _i, _i, _i, _c]),
    "mpdata_batch_step": (_i, [_c, _i, _i]),
    "mpdata_batch_set_config": (_i, [_c, _i, _i]),
    "mpdata_batch_get_config": (_i, [_c, _ip, _ip, _ip, _ip, _ip,
                                     ctypes.POINTER(ctypes.c_longlong)]),
    "mpdata_batch_autotune": (_i, [_c, _i, ctypes.POINTER(ctypes.c_double)]),
    "mpdata_batch_launch_count": (ctypes.c_longlong, [_c]),
    "mpdata_batch_last_error_string": (ctypes.c_char_p, [_c]),
    "mpdata_batch_destroy": (None, [_c]),
    "mpdata_mass_noalloc": (_i, [_c, _c, _i, _i, _i, _i, _i, _c, _c]),
    "mpdata_probe_fp64_fma": (_i, [_c, _i, _i, _c, ctypes.POINTER(ctypes.c_double)]),
    "mpdata_set_ij_boundary": (_i, [_c, _i]),
    "mpdata_halo_strip_elems": (_i, [_c, _i, ctypes.POINTER(ctypes.c_longlong)]),
    "mpdata_halo_pack": (_i, [_c, _c, _i, _c]),
    "mpdata_halo_unpack": (_i, [_c, _c, _i, _c]),
    "mpdata_profile": (_i, [_c, _i]),
    "mpdata_profile_read": (_i, [_c, _i, ctypes.POINTER(ctypes.c_double),
                                 ctypes.POINTER(ctypes.c_int)]),
}

STAGES = {"halo": 0, "donor": 1, "advance": 2, "pseudo": 3, "beta": 4, "limit": 5, "mass": 6,
          "fused": 7, "fused_donor": 8, "exchange": 9}
MPDATA_IJ_PERIODIC = 0
MPDATA_IJ_HALO = 1

for _name, (_res, _args) in SIGNATURES.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args


class MPDATAError(RuntimeError):
    def __init__(self, code: int, where: str, detail: str = ""):
        self.code = code
        msg = f"{where}: {mpdata_strerror(code)} ({code})"
        if detail:
            msg += f": {detail}"
        super().__init__(msg)


def _check(rc: int, where: str, ctx=None) -> None:
    if rc != MPDATA_OK:
        detail = mpdata_last_error_string(ctx) if (ctx and rc == MPDATA_ECUDA) else ""
        raise MPDATAError(rc, where, detail)


def mpdata_strerror(code: int) -> str:
    return lib.mpdata_strerror(code).decode()


def mpdata_last_error_string(ctx) -> str:
    return lib.mpdata_last_error_string(ctx).decode()


def mpdata_version() -> int:
    return lib.mpdata_version()


def mpdata_init(nx, ny, nz, halo, iord, nonoscillatory, dtype, k_bc=MPDATA_K_ZEROFLUX,
                cuda_stream=0):
    """Returns an opaque context handle (int); raises MPDATAError on failure."""
    out = ctypes.c_void_p()
    rc = lib.mpdata_init(ctypes.byref(out), nx, ny, nz, halo, iord, nonoscillatory, dtype, k_bc,
                         cuda_stream)
    _check(rc, "mpdata_init")
    return out.value


def mpdata_set_stream(ctx, cuda_stream):
    _check(lib.mpdata_set_stream(ctx, cuda_stream), "mpdata_set_stream", ctx)


def mpdata_set_variant(ctx, variant):
    _check(lib.mpdata_set_variant(ctx, variant), "mpdata_set_variant", ctx)


def mpdata_set_options(ctx, opts):
    _check(lib.mpdata_set_options(ctx, opts), "mpdata_set_options", ctx)


def mpdata_get_options(ctx) -> int:
    out = ctypes.c_int()
    _check(lib.mpdata_get_options(ctx, ctypes.byref(out)), "mpdata_get_options", ctx)
    return out.value


def mpdata_step(ctx, psi, u, v, w, g, nsteps):
    _check(lib.mpdata_step(ctx, psi, u, v, w, g, nsteps), "mpdata_step", ctx)


def mpdata_step_out(ctx, psi_in, psi_out, u, v, w, g):
    _check(lib.mpdata_step_out(ctx, psi_in, psi_out, u, v, w, g), "mpdata_step_out", ctx)


def mpdata_step_host(ctx, psi_h, u_h, v_h, w_h, g_h, nsteps):
    _check(lib.mpdata_step_host(ctx, psi_h, u_h, v_h, w_h, g_h, nsteps), "mpdata_step_host", ctx)


def mpdata_fill_halo(ctx, field, kind):
    _check(lib.mpdata_fill_halo(ctx, field, kind), "mpdata_fill_halo", ctx)


def mpdata_mass(ctx, psi, g, out_dev):
    _check(lib.mpdata_mass(ctx, psi, g, out_dev), "mpdata_mass", ctx)


def mpdata_destroy(ctx):
    lib.mpdata_destroy(ctx)


def mpdata_launch_count(ctx) -> int:
    return lib.mpdata_launch_count(ctx)


def mpdata_profile(ctx, enable: bool):
    _check(lib.mpdata_profile(ctx, int(bool(enable))), "mpdata_profile", ctx)


def mpdata_profile_read(ctx, stage: int):
    """(total ms, timed launches) of one stage since profiling was enabled."""
    ms = ctypes.c_double()
    n = ctypes.c_int()
    _check(lib.mpdata_profile_read(ctx, stage, ctypes.byref(ms), ctypes.byref(n)),
           "mpdata_profile_read", ctx)
    return ms.value, n.value


def mpdata_mass_noalloc(psi, g, nx, ny, nz, halo, dtype, out_dev, cuda_stream=0):
    """Context-free mass sum that allocates nothing (see include/mpdata.h)."""
    _check(lib.mpdata_mass_noalloc(psi, g, nx, ny, nz, halo, dtype, out_dev, cuda_stream),
           "mpdata_mass_noalloc")


def mpdata_adjoint_step(ctx, psi_n, u, v, w, g, psi_bar, u_bar, v_bar, w_bar):
    _check(lib.mpdata_adjoint_step(ctx, psi_n, u, v, w, g, psi_bar, u_bar, v_bar, w_bar),
           "mpdata_adjoint_step", ctx)


def mpdata_fold_halo_adjoint(ctx, field):
    _check(lib.mpdata_fold_halo_adjoint(ctx, field), "mpdata_fold_halo_adjoint", ctx)


def _bcheck(rc, where, b=None):
    if rc != MPDATA_OK:
        detail = lib.mpdata_batch_last_error_string(b).decode() if (b and rc == MPDATA_ECUDA) else ""
        raise MPDATAError(rc, where, detail)


def mpdata_batch_init(descs, nonoscillatory, dtype, cuda_stream=0):
    arr = (mpdata_domain_desc * len(descs))(*descs)
    out = ctypes.c_void_p()
    _bcheck(lib.mpdata_batch_init(ctypes.byref(out), arr, len(descs), nonoscillatory, dtype,
                                  cuda_stream), "mpdata_batch_init")
    return out.value


def mpdata_batch_step(b, direction, use_graph):
    _bcheck(lib.mpdata_batch_step(b, direction, int(bool(use_graph))), "mpdata_batch_step", b)


def mpdata_batch_set_config(b, shape, kchunk_levels):
    _bcheck(lib.mpdata_batch_set_config(b, shape, kchunk_levels), "mpdata_batch_set_config", b)


def mpdata_batch_get_config(b):
    v = [ctypes.c_int() for _ in range(5)]
    items = ctypes.c_longlong()
    _bcheck(lib.mpdata_batch_get_config(b, *[ctypes.byref(x) for x in v], ctypes.byref(items)),
            "mpdata_batch_get_config", b)
    return dict(shape=v[0].value, kchunk=v[1].value, tile_x=v[2].value, tile_y=v[3].value,
                threads=v[4].value, items=items.value)


def mpdata_batch_autotune(b, reps):
    ms = ctypes.c_double()
    _bcheck(lib.mpdata_batch_autotune(b, reps, ctypes.byref(ms)), "mpdata_batch_autotune", b)
    return ms.value


def mpdata_batch_launch_count(b):
    return lib.mpdata_batch_launch_count(b)


def mpdata_batch_destroy(b):
    lib.mpdata_batch_destroy(b)


def mpdata_tape_bytes(ctx) -> int:
    n = ctypes.c_size_t()
    _check(lib.mpdata_tape_bytes(ctx, ctypes.byref(n)), "mpdata_tape_bytes", ctx)
    return n.value


def mpdata_step_tape(ctx, psi_in, psi_out, u, v, w, g, tape):
    _check(lib.mpdata_step_tape(ctx, psi_in, psi_out, u, v, w, g, tape), "mpdata_step_tape", ctx)


def mpdata_adjoint_step_tape(ctx, tape, psi_n, u, v, w, g, psi_bar, u_bar, v_bar, w_bar):
    _check(lib.mpdata_adjoint_step_tape(ctx, tape, psi_n, u, v, w, g, psi_bar, u_bar, v_bar,
                                        w_bar), "mpdata_adjoint_step_tape", ctx)


def mpdata_probe_fp64_fma(out_dev, blocks, iters, cuda_stream=0) -> float:
    """Launch the FP64 FMA-rate probe; returns the launch's flop count."""
    flops = ctypes.c_double()
    _check(lib.mpdata_probe_fp64_fma(out_dev, blocks, iters, cuda_stream, ctypes.byref(flops)),
           "mpdata_probe_fp64_fma")
    return flops.value


def mpdata_set_ij_boundary(ctx, mode):
    _check(lib.mpdata_set_ij_boundary(ctx, mode), "mpdata_set_ij_boundary", ctx)


def mpdata_halo_strip_elems(ctx, face) -> int:
    n = ctypes.c_longlong()
    _check(lib.mpdata_halo_strip_elems(ctx, face, ctypes.byref(n)), "mpdata_halo_strip_elems",
           ctx)
    return n.value


def mpdata_halo_pack(ctx, field, face, buf):
    _check(lib.mpdata_halo_pack(ctx, field, face, buf), "mpdata_halo_pack", ctx)


def mpdata_halo_unpack(ctx, buf, face, field):
    _check(lib.mpdata_halo_unpack(ctx, buf, face, field), "mpdata_halo_unpack", ctx)


def mpdata_step_host_async(ctx, psi_in_h, psi_out_h, u_h, v_h, w_h, g_h, nsteps):
    _check(lib.mpdata_step_host_async(ctx, psi_in_h, psi_out_h, u_h, v_h, w_h, g_h, nsteps),
           "mpdata_step_host_async", ctx)


def mpdata_step_host_interior_async(ctx, psi_in_h, psi_out_h, u_h, v_h, w_h, g_h, nsteps):
    _check(lib.mpdata_step_host_interior_async(ctx, psi_in_h, psi_out_h, u_h, v_h, w_h, g_h,
                                               nsteps),
           "mpdata_step_host_interior_async", ctx)


def mpdata_host_wait(ctx):
    _check(lib.mpdata_host_wait(ctx), "mpdata_host_wait", ctx)
