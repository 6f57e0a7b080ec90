"""Helpers shared by the GPU tests: run the library on numpy inputs through
the C ABI and compare with the oracle."""
import numpy as np

import synth


def to_dev(a, dtype):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype).contiguous()


def run_library(case, dtype, iord=None, nonosc=None, nsteps=1, h=None, variant=None,
                psi=None, halo_fill=np.nan, k_bc=0):
    """Advance case.psi by nsteps on the GPU; returns the padded result (float64)."""
    import torch
    from paper_1908_06094_b300 import MPDATA
    h = case.halo if h is None else h
    iord = case.iord if iord is None else iord
    nonosc = case.nonosc if nonosc is None else nonosc
    m = MPDATA(case.nx, case.ny, case.nz, halo=h, iord=iord, nonoscillatory=nonosc,
               dtype=dtype, variant=variant, k_bc=k_bc)
    P = [synth.pad(x, h, fill=halo_fill) for x in (case.psi if psi is None else psi,
                                                   case.u, case.v, case.w, case.g)]
    d = [to_dev(x, dtype) for x in P]
    m.step(*d, nsteps=nsteps)
    torch.cuda.synchronize()
    out = d[0].double().cpu().numpy()
    m.close()
    return out


def rounded_inputs(case, dtype):
    """The case with its fields rounded to the kernel's storage precision."""
    import torch
    if dtype == torch.float64:
        return case
    import copy
    c = copy.copy(case)
    for k in ("psi", "u", "v", "w", "g"):
        setattr(c, k, getattr(case, k).astype(np.float32).astype(np.float64))
    return c


def rel_err(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))
