"""MPDATA oracle: test infrastructure only.

A plain FP64 CPU implementation of one MPDATA step (``mpdata_oracle.cpp``),
loaded through ctypes.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg use it; the library under test never imports it,
and it imports nothing from the library.

All arrays are float64, C-contiguous, halo-padded [nz+2h][ny+2h][nx+2h].
Inputs are read at interior points only; outputs are padded with their halos
filled (periodic in i and j, edge copy in k).  ``kbc``: the vertical
boundary, 0 zero-flux (closed top and bottom faces) or 1 periodic in k.

Parity pins live in ``tests/test_oracle_pins.py``.  Parity unpinned: the exact
values of the limited iord=2 field beyond what those invariants and closed
forms fix (the paper prints no worked example).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mpdata_oracle.cpp")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

_D = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False, src: str = _SRC, out: str = _LIB) -> str:
    """Compile the oracle with g++ (-O2, no FMA contraction, OpenMP)."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        tmp = out + f".tmp{os.getpid()}"
        cmd = ["g++", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-std=c++17",
               "-shared", "-fPIC", src, "-o", tmp]
        subprocess.check_call(cmd)
        os.replace(tmp, out)
    return out


def _bind(path):
    lib = ctypes.CDLL(path)
    I = ctypes.c_int
    lib.orc_fill_halo.argtypes = [I, I, I, I, I, I, _D]
    lib.orc_run.argtypes = [I] * 9 + [_D] * 6 + [_D] * 11
    lib.orc_pseudo_velocity.argtypes = [I, I, I, I, I] + [_D] * 8
    lib.orc_mass.argtypes = [I, I, I, I, _D, _D]
    lib.orc_mass.restype = ctypes.c_double
    lib.orc_tlm.argtypes = [I, I, I, I, I, I, I, I] + [_D] * 11
    lib.orc_adjoint.argtypes = [I, I, I, I, I, I, I, I] + [_D] * 9
    L = ctypes.c_long
    _L = ctypes.POINTER(ctypes.c_long)
    lib.orc_edge_run.argtypes = [L, L, I, I, _L, _L, _D, _D, _D, _D, _D, ctypes.c_double, _D]
    lib.orc_cells_sum.argtypes = [L, I, ctypes.POINTER(ctypes.c_int), _D, ctypes.c_double, _D]
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(build())
    return _lib


def use_library(path: str):
    """Point this module at another build of the oracle source (used by the
    mutation tests, which compile deliberately broken copies); returns the
    previous library so it can be restored."""
    global _lib
    prev = _load()
    with _lock:
        _lib = _bind(path)
    return prev


def restore_library(lib):
    global _lib
    with _lock:
        _lib = lib


def _p(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def _dims(a, h):
    nz, ny, nx = (s - 2 * h for s in a.shape[-3:])
    return nx, ny, nz


def fill_halo(f: np.ndarray, h: int, kind: int = 0, kbc: int = 0) -> np.ndarray:
    """Fill the halo of a padded field in place (kind 1: vertical faces)."""
    nx, ny, nz = _dims(f, h)
    _load().orc_fill_halo(nx, ny, nz, h, kbc, kind, _p(f))
    return f


DFL, ABS, IGA = 1, 2, 4  # option flags of the corrective passes


def run(psi, u, v, w, g, h: int, iord: int = 2, nonosc: int = 1, nsteps: int = 1,
        stages: bool = False, kbc: int = 0, opts: int = 0):
    """nsteps MPDATA steps.  Returns psi^(n+nsteps) (padded), and with
    ``stages`` also a dict of the last corrective pass's intermediates.
    opts: DFL (divergent-flow term), ABS (signed fields), IGA (infinite
    gauge), or'ed."""
    nx, ny, nz = _dims(psi, h)
    arrs = [np.ascontiguousarray(x, dtype=np.float64) for x in (psi, u, v, w, g)]
    out = np.zeros_like(arrs[0])
    names = ["psi1", "ut", "vt", "wt", "mx", "mn", "bu", "bd", "ul", "vl", "wl"]
    st = {k: np.zeros_like(arrs[0]) for k in names} if stages else {}
    _load().orc_run(nx, ny, nz, h, kbc, iord, nonosc, opts, nsteps, *[_p(a) for a in arrs], _p(out),
                    *[_p(st.get(k)) for k in names])
    return (out, st) if stages else out


def pseudo_velocity(psi, u, v, w, g, h: int, kbc: int = 0):
    """Antidiffusive pseudo-velocities (Ut, Vt, Wt) of field psi."""
    nx, ny, nz = _dims(psi, h)
    arrs = [np.ascontiguousarray(x, dtype=np.float64) for x in (psi, u, v, w, g)]
    ut, vt, wt = (np.zeros_like(arrs[0]) for _ in range(3))
    _load().orc_pseudo_velocity(nx, ny, nz, h, kbc, *[_p(a) for a in arrs], _p(ut), _p(vt),
                                _p(wt))
    return ut, vt, wt


def mass(psi, g, h: int) -> float:
    """sum over the interior of psi * G, in (k, j, i) order."""
    nx, ny, nz = _dims(psi, h)
    return float(_load().orc_mass(nx, ny, nz, h, _p(np.ascontiguousarray(psi, dtype=np.float64)),
                                  _p(np.ascontiguousarray(g, dtype=np.float64))))


def tlm(psi, u, v, w, g, dpsi, du, dv, dw, h: int, iord: int = 2, nonosc: int = 1,
        nsteps: int = 1, kbc: int = 0):
    """Tangent-linear model: (psi_out, dpsi_out) along direction (dpsi, dU, dV, dW)."""
    nx, ny, nz = _dims(psi, h)
    arrs = [np.ascontiguousarray(x, dtype=np.float64) for x in (psi, u, v, w, g, dpsi, du, dv, dw)]
    out = np.zeros_like(arrs[0])
    dout = np.zeros_like(arrs[0])
    _load().orc_tlm(nx, ny, nz, h, kbc, iord, nonosc, nsteps, *[_p(a) for a in arrs], _p(out),
                    _p(dout))
    return out, dout


def adjoint(psi, u, v, w, g, psib, h: int, iord: int = 2, nonosc: int = 1, nsteps: int = 1,
            kbc: int = 0):
    """Reverse mode of nsteps steps.  psib: dJ/dpsi_T (padded, interior used).
    Returns (dJ/dpsi_0, dJ/dU, dJ/dV, dJ/dW), padded with zero halos."""
    nx, ny, nz = _dims(psi, h)
    arrs = [np.ascontiguousarray(x, dtype=np.float64) for x in (psi, u, v, w, g)]
    pb = np.array(psib, dtype=np.float64, order="C", copy=True)
    ub, vb, wb = (np.zeros_like(arrs[0]) for _ in range(3))
    _load().orc_adjoint(nx, ny, nz, h, kbc, iord, nonosc, nsteps, *[_p(a) for a in arrs], _p(pb),
                        _p(ub), _p(vb), _p(wb))
    inner = np.zeros_like(pb)
    sl = (slice(h, h + nz), slice(h, h + ny), slice(h, h + nx))
    inner[sl] = pb[sl]
    return inner, ub, vb, wb


def edge_run(case, nsteps: int = 1, pD=None):
    """nsteps applications of the edge-based flux stages on an
    ``synth.octahedral.EdgeCase`` through its connectivity tables; returns
    the new pD (nz, nr, nc).  ``pD`` overrides the case's initial field."""
    p = np.array(case.pD if pD is None else pD, dtype=np.float64, order="C", copy=True)
    N, E, nz = case.nnodes, case.nedges, case.nz
    arr = lambda a: np.ascontiguousarray(a, dtype=np.float64)
    idx = lambda a: np.ascontiguousarray(a, dtype=np.int64)
    e2n, n2e = idx(case.e2n), idx(case.n2e)
    sgn, vn, wn, rho, vol = (arr(x) for x in (case.n2e_sign, case.vn, case.wn, case.rho,
                                               case.vol))
    Lp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_long))
    _load().orc_edge_run(N, E, nz, nsteps, Lp(e2n), Lp(n2e), _p(sgn), _p(vn), _p(wn), _p(rho),
                         _p(vol), float(case.pivbz), _p(p))
    return p


def edge_mass(case, pD) -> float:
    """sum over nodes and levels of vol * rho * pD."""
    return float(np.sum(case.vol[None] * case.rho * pD))


def cells_sum(table, A, fac: float = 1.0):
    """B = fac * (sum of A over each cell's three neighbours), table [3][ncells]
    (int32), A [nz][ncells]."""
    t = np.ascontiguousarray(table, dtype=np.int32)
    a = np.ascontiguousarray(A, dtype=np.float64)
    out = np.empty_like(a)
    _load().orc_cells_sum(a.shape[1], a.shape[0], t.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                          _p(a), float(fac), _p(out))
    return out
