"""Differentiable MPDATA: torch.autograd.Function over the library's forward
and adjoint steps, with checkpoint-and-recompute.

forward(psi0, U, V, W, G, nsteps) runs nsteps steps and keeps psi every
``ckpt`` steps; backward walks the segments in reverse, re-runs each
segment once from its checkpoint with taped library steps (each keeping
its intermediates), then applies the library's taped adjoint step to each
step in reverse order; the re-run of a segment overlaps, on a second stream
and context, with the adjoint steps of the segment after it.  The last segment, which backward needs first, is
taped already by the forward pass (when a gradient is wanted), so it is
never re-run -- the segment schedule of checkpoint_sequential.  Memory:
nsteps/ckpt checkpoints plus two sets of ckpt states and tapes (11 fields
each).  G is
not differentiated.  Every step of both passes runs in the library's
kernels; this module only orders the calls.
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
        # the last segment [last, nsteps) is run taped when backward will follow
        taped = nsteps > 0 and any(ctx.needs_input_grad[:4])
        last = ((nsteps - 1) // ckpt) * ckpt if nsteps > 0 else 0
        tapes, states = _buffers(model, u, ckpts[0], min(ckpt, nsteps)) if taped else ([], [])
        P = lambda t, name: model._ptr(t, name)  # noqa: E731
        for s in range(nsteps):
            if taped and s >= last:
                i = s - last
                if i == 0:
                    states[0].copy_(cur)
                model._sync_stream()
                C.mpdata_step_tape(model._ctx, P(states[i], "state"), P(states[i + 1], "state"),
                                   P(u, "u"), P(v, "v"), P(w, "w"), P(g, "g"),
                                   tapes[i].data_ptr())
                cur = states[i + 1]
            else:
                model.step_out(cur, nxt, u, v, w, g)
                cur, nxt = nxt, cur
            if (s + 1) % ckpt == 0 and s + 1 < nsteps:
                ckpts.append(cur.clone())
        ctx.model, ctx.nsteps, ctx.ckpt = model, nsteps, ckpt
        ctx.tapes, ctx.states, ctx.taped = tapes, states, taped
        ctx.save_for_backward(u, v, w, g, *ckpts)
        # states are reused by backward for the other segments: return a copy
        return cur.clone() if taped else cur

    @staticmethod
    def backward(ctx, grad_out):
        u, v, w, g, *ckpts = ctx.saved_tensors
        m, nsteps, ckpt = ctx.model, ctx.nsteps, ctx.ckpt
        m._sync_stream()
        main = torch.cuda.current_stream(m.device)
        psib = grad_out.contiguous().clone()
        # the output's halo holds copies of interior values
        C.mpdata_fold_halo_adjoint(m._ctx, m._ptr(psib, "grad"))
        ub, vb, wb = torch.zeros_like(u), torch.zeros_like(v), torch.zeros_like(w)
        nseg = len(ckpts)
        seglen = min(ckpt, nsteps)
        # Two sets of tapes and states: while the main stream runs the
        # adjoint steps of segment k from one set, a side stream records
        # segment k-1 into the other (with a second context of the same
        # grid, so the two share no scratch).  Segment k-1's adjoint steps
        # wait for its recording; a set is recorded into again only after
        # the adjoint steps that read it have run.
        sets = [(ctx.tapes, ctx.states) if ctx.taped else _buffers(m, u, ckpts[0], seglen)]
        if nseg > 1:
            sets.append(_buffers(m, u, ckpts[0], seglen))
        rec = m.shadow() if nseg > 1 else None
        if rec is not None:
            C.mpdata_set_options(rec._ctx, C.mpdata_get_options(m._ctx))
        side = torch.cuda.Stream(m.device) if nseg > 1 else None
        ready = main.record_event()   # checkpoints and buffers are ready
        free = [ready, ready]         # when each set may be recorded into
        recorded = {}

        def record(seg, which, model, stream):
            tapes, states = sets[which]
            start = seg * ckpt
            P = lambda t, name: model._ptr(t, name)  # noqa: E731
            with torch.cuda.stream(stream):
                model._sync_stream()
                states[0].copy_(ckpts[seg])
                for s in range(min(start + ckpt, nsteps) - start):
                    C.mpdata_step_tape(model._ctx, P(states[s], "state"),
                                       P(states[s + 1], "state"), P(u, "u"), P(v, "v"),
                                       P(w, "w"), P(g, "g"), tapes[s].data_ptr())
            return stream.record_event()

        if not ctx.taped:  # the forward pass did not tape the last segment
            recorded[nseg - 1] = record(nseg - 1, 0, m, main)
        P = lambda t, name: m._ptr(t, name)  # noqa: E731
        for seg in reversed(range(nseg)):
            which = (nseg - 1 - seg) % 2
            if seg - 1 >= 0:  # record the next segment meanwhile, on the side stream
                side.wait_event(free[1 - which])
                recorded[seg - 1] = record(seg - 1, 1 - which, rec, side)
            if seg in recorded:
                main.wait_event(recorded[seg])
            m._sync_stream()
            tapes, states = sets[which]
            start = seg * ckpt
            for s in reversed(range(min(start + ckpt, nsteps) - start)):
                C.mpdata_adjoint_step_tape(m._ctx, tapes[s].data_ptr(), P(states[s], "state"),
                                           P(u, "u"), P(v, "v"), P(w, "w"), P(g, "g"),
                                           P(psib, "psi_bar"), P(ub, "u_bar"), P(vb, "v_bar"),
                                           P(wb, "w_bar"))
            free[which] = main.record_event()
        if side is not None:
            main.wait_stream(side)
        ctx.tapes = ctx.states = None
        return psib, ub, vb, wb, None, None, None, None


def _buffers(model: MPDATA, like_field, like_state, seglen: int):
    """Tapes and states of one segment of seglen steps."""
    nbytes = C.mpdata_tape_bytes(model._ctx)
    tapes = [torch.empty(nbytes, dtype=torch.uint8, device=like_field.device)
             for _ in range(seglen)]
    states = [torch.empty_like(like_state) for _ in range(seglen + 1)]
    return tapes, states


def mpdata_run(model: MPDATA, psi0, u, v, w, g, nsteps: int, ckpt: int = 5):
    """psi after nsteps steps, differentiable in psi0, U, V, W."""
    return MPDATAFunction.apply(psi0, u, v, w, g, model, nsteps, ckpt)
