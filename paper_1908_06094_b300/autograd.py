"""Differentiable MPDATA: torch.autograd.Function over the library's forward
and adjoint steps, with checkpoint-and-recompute.

forward(psi0, U, V, W, G, nsteps) runs nsteps steps and keeps psi every
``ckpt`` steps; backward walks the segments in reverse, recomputes each
segment's states from its checkpoint (library forward steps), then applies
the library's adjoint step to each state in reverse order.  Memory: about
nsteps/ckpt + ckpt fields.  G is not differentiated.  Every step of both
passes runs in the library's kernels; this module only orders the calls.
"""
from __future__ import annotations

import torch

from . import _capi as C
from .mpdata import MPDATA


class MPDATAFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, psi0, u, v, w, g, model: MPDATA, nsteps: int, ckpt: int):
        if ckpt < 1:
            raise ValueError("ckpt must be >= 1")
        ckpts = [psi0.detach().contiguous().clone()]
        cur = ckpts[0].clone()
        nxt = torch.empty_like(cur)
        for s in range(nsteps):
            model.step_out(cur, nxt, u, v, w, g)
            cur, nxt = nxt, cur
            if (s + 1) % ckpt == 0 and s + 1 < nsteps:
                ckpts.append(cur.clone())
        ctx.model, ctx.nsteps, ctx.ckpt = model, nsteps, ckpt
        ctx.save_for_backward(u, v, w, g, *ckpts)
        return cur

    @staticmethod
    def backward(ctx, grad_out):
        u, v, w, g, *ckpts = ctx.saved_tensors
        m, nsteps, ckpt = ctx.model, ctx.nsteps, ctx.ckpt
        m._sync_stream()
        psib = grad_out.contiguous().clone()
        # the output's halo holds copies of interior values
        C.mpdata_fold_halo_adjoint(m._ctx, m._ptr(psib, "grad"))
        ub, vb, wb = torch.zeros_like(u), torch.zeros_like(v), torch.zeros_like(w)
        nseg = len(ckpts)
        for seg in reversed(range(nseg)):
            start = seg * ckpt
            end = min(start + ckpt, nsteps)
            states = [ckpts[seg]]
            for _ in range(start, end - 1):
                nxt = torch.empty_like(states[-1])
                m.step_out(states[-1], nxt, u, v, w, g)
                states.append(nxt)
            for s in reversed(range(end - start)):
                C.mpdata_adjoint_step(m._ctx, m._ptr(states[s], "state"), m._ptr(u, "u"),
                                      m._ptr(v, "v"), m._ptr(w, "w"), m._ptr(g, "g"),
                                      m._ptr(psib, "psi_bar"), m._ptr(ub, "u_bar"),
                                      m._ptr(vb, "v_bar"), m._ptr(wb, "w_bar"))
        return psib, ub, vb, wb, None, None, None, None


def mpdata_run(model: MPDATA, psi0, u, v, w, g, nsteps: int, ckpt: int = 5):
    """psi after nsteps steps, differentiable in psi0, U, V, W."""
    return MPDATAFunction.apply(psi0, u, v, w, g, model, nsteps, ckpt)
