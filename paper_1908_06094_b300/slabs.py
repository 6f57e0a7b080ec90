"""i-j slab decomposition of one MPDATA domain (Sec. 3.1.1, item 2: halo
exchange as a library component; Fig. 8: the grid split into partitions).

A domain of NX x NY x nz is cut into px x py slabs.  Each slab is a context
of the library in MPDATA_IJ_HALO mode: its step reads its i-j halo instead
of wrapping, so one exchange of psi's halo (depth 3, corners included)
before each step gives every slab the same values, point for point, as the
step of the undivided domain under the same kernel.  U, V, W and G are
exchanged once.  The exchange runs in two phases, x faces then y faces (the
y strips span the padded width, so they carry the corners); in each phase a
slab packs the strip next to face f and sends it to its neighbour across f,
which unpacks it beyond its face f ^ 1.  The strips are packed and unpacked
by the library's kernels; this module only orders the calls and moves the
buffers:

* ``SlabDecomposition``: every slab on one device; a neighbour's packed
  buffer is unpacked directly (device memory, no copy in between).
* ``SlabRank``: one slab per process of a torch.distributed group (NCCL on
  GPUs); buffers move by point-to-point send/recv, the global mass by one
  FP64 all-reduce.

The message order is fixed by ``exchange_plan`` so that backends that match
messages by order (not by tag) pair them correctly when both neighbours in a
direction are the same process (px or py = 2).
"""
from __future__ import annotations

from dataclasses import dataclass

FACES_X = (0, 1)   # -x, +x
FACES_Y = (2, 3)   # -y, +y


def split_sizes(n: int, parts: int) -> list[int]:
    """n cells over parts slabs, as even as possible (the first ones larger)."""
    if parts < 1 or n < parts:
        raise ValueError(f"cannot split {n} cells into {parts} slabs")
    q, r = divmod(n, parts)
    return [q + (1 if s < r else 0) for s in range(parts)]


def slab_coords(rank: int, px: int, py: int) -> tuple[int, int]:
    """(ix, iy) of a rank; ranks run along x first."""
    if not 0 <= rank < px * py:
        raise ValueError("rank outside the decomposition")
    return rank % px, rank // px


def neighbours(rank: int, px: int, py: int) -> dict[int, int]:
    """The rank across each face (the domain is periodic in i and j)."""
    ix, iy = slab_coords(rank, px, py)
    return {0: ((ix - 1) % px) + iy * px, 1: ((ix + 1) % px) + iy * px,
            2: ix + ((iy - 1) % py) * px, 3: ix + ((iy + 1) % py) * px}


@dataclass(frozen=True)
class Msg:
    face: int   # the face of this rank the message crosses
    peer: int   # the rank across it
    tag: int    # the sender's face (a send carries tag = face; a receive
                # expects tag = face ^ 1)


def exchange_plan(rank: int, px: int, py: int):
    """Per phase (x, then y): the sends (pack face f -> peer across f, in
    order of f), the receives (into face f from the peer across f, in order
    of the sender's face f ^ 1) and the faces served by the slab itself
    (a direction with one slab wraps onto itself: unpack(f) <- pack(f ^ 1))."""
    nb = neighbours(rank, px, py)
    plan = []
    for phase in (FACES_X, FACES_Y):
        sends, recvs, local = [], [], []
        for f in phase:
            if nb[f] == rank:
                local.append(f)
            else:
                sends.append(Msg(f, nb[f], f))
        for f in sorted(phase, key=lambda f: f ^ 1):
            if nb[f] != rank:
                recvs.append(Msg(f, nb[f], f ^ 1))
        plan.append((phase, sends, recvs, local))
    return plan


def slab_extent(NX: int, NY: int, px: int, py: int, rank: int):
    """(i0, nx, j0, ny): the slab's first interior column/row and its size."""
    xs, ys = split_sizes(NX, px), split_sizes(NY, py)
    ix, iy = slab_coords(rank, px, py)
    return sum(xs[:ix]), xs[ix], sum(ys[:iy]), ys[iy]


def halo_exchange(field, rank: int, px: int, py: int, pack, unpack, transfer):
    """Fill the i-j halo of one slab's field from its neighbours.

    pack(field, f) -> buffer of the strip next to face f; unpack(buf, f,
    field) writes a buffer into the halo beyond face f; transfer(sends,
    recvs, out) moves the buffers: sends = [(Msg, buf)], recvs = [Msg] and
    it returns {face: received buffer}."""
    for phase, sends, recvs, local in exchange_plan(rank, px, py):
        out = {f: pack(field, f) for f in phase}
        got = transfer([(m, out[m.face]) for m in sends], recvs, out) if (sends or recvs) else {}
        for f in local:
            got[f] = out[f ^ 1]
        for f in phase:
            unpack(got[f], f, field)


# ------------------------------------------------------------------ device --

class _SlabCtx:
    """One slab's library context plus the pack/unpack buffers."""

    def __init__(self, nx, ny, nz, halo, dtype, device, nonoscillatory, k_bc):
        import torch
        from . import _capi as C
        from .mpdata import MPDATA
        self.m = MPDATA(nx, ny, nz, halo=halo, iord=2, nonoscillatory=nonoscillatory,
                        dtype=dtype, device=device, k_bc=k_bc)
        C.mpdata_set_ij_boundary(self.m._ctx, C.MPDATA_IJ_HALO)
        self.C = C
        self.bufs = {f: torch.empty(C.mpdata_halo_strip_elems(self.m._ctx, f), dtype=dtype,
                                    device=self.m.device) for f in range(4)}

    def pack(self, field, f):
        self.m._sync_stream()
        self.C.mpdata_halo_pack(self.m._ctx, self.m._ptr(field, "field"), f,
                                self.bufs[f].data_ptr())
        return self.bufs[f]

    def unpack(self, buf, f, field):
        self.m._sync_stream()
        self.C.mpdata_halo_unpack(self.m._ctx, buf.data_ptr(), f, self.m._ptr(field, "field"))


class SlabDecomposition:
    """px x py slabs of one NX x NY x nz domain, all on one device.

    Fields are lists of padded slab tensors (one per slab, rank order).
    ``scatter`` cuts a global interior array into slab fields and exchanges
    their halos; ``step`` runs nsteps steps (an exchange of psi before each
    one); ``gather`` reassembles the interior; ``mass`` adds the slabs'
    FP64 masses in rank order."""

    def __init__(self, NX, NY, nz, px, py, halo=3, dtype=None, device=None,
                 nonoscillatory=True, k_bc=0):
        import torch
        self.NX, self.NY, self.nz, self.px, self.py, self.h = NX, NY, nz, px, py, halo
        self.dtype = torch.float64 if dtype is None else dtype
        self.ext = [slab_extent(NX, NY, px, py, r) for r in range(px * py)]
        self.slabs = [_SlabCtx(nx, ny, nz, halo, self.dtype, device, nonoscillatory, k_bc)
                      for (_, nx, _, ny) in self.ext]
        self.device = self.slabs[0].m.device
        self._tmp = None

    @property
    def nslabs(self):
        return len(self.slabs)

    def scatter(self, interior):
        """interior: (nz, NY, NX) array or tensor -> exchanged slab fields."""
        import torch
        t = torch.as_tensor(interior).to(self.device, self.dtype)
        h = self.h
        out = []
        for (i0, nx, j0, ny), s in zip(self.ext, self.slabs):
            f = torch.full(s.m.shape, float("nan"), dtype=self.dtype, device=self.device)
            f[h:h + self.nz, h:h + ny, h:h + nx] = t[:, j0:j0 + ny, i0:i0 + nx]
            out.append(f)
        self.exchange(out)
        return out

    def exchange(self, fields):
        """Fill every slab's i-j halo of one field (x phase, then y phase)."""
        for phase in (FACES_X, FACES_Y):
            # every slab packs into its own per-face buffers, so all packs of
            # a phase can run before the unpacks that read them
            packed = [{f: s.pack(fld, f) for f in phase} for s, fld in zip(self.slabs, fields)]
            for r, (s, fld) in enumerate(zip(self.slabs, fields)):
                nb = neighbours(r, self.px, self.py)
                for f in phase:
                    s.unpack(packed[nb[f]][f ^ 1], f, fld)

    def step(self, psi, u, v, w, g, nsteps=1):
        """Advance the slab fields psi in place by nsteps steps."""
        import torch
        if self._tmp is None:
            self._tmp = [torch.empty_like(p) for p in psi]
        for _ in range(nsteps):
            self.exchange(psi)
            for s, p, t, a, b, c, d in zip(self.slabs, psi, self._tmp, u, v, w, g):
                s.m.step_out(p, t, a, b, c, d)
            for p, t in zip(psi, self._tmp):
                p.copy_(t)
        return psi

    def gather(self, fields):
        """Slab fields -> the (nz, NY, NX) interior of the domain."""
        import torch
        h = self.h
        out = torch.empty((self.nz, self.NY, self.NX), dtype=self.dtype, device=self.device)
        for (i0, nx, j0, ny), f in zip(self.ext, fields):
            out[:, j0:j0 + ny, i0:i0 + nx] = f[h:h + self.nz, h:h + ny, h:h + nx]
        return out

    def mass(self, psi, g):
        """The domain's FP64 mass: the slabs' sums added in rank order."""
        tot = None
        for s, p, gg in zip(self.slabs, psi, g):
            m = s.m.mass(p, gg)
            tot = m if tot is None else tot + m
        return tot

    def close(self):
        for s in self.slabs:
            s.m.close()


# ------------------------------------------------------------- one per rank --

def dist_transfer(group=None):
    """A transfer function over torch.distributed point-to-point calls: the
    sends in plan order, then the receives in plan order, all posted before
    any wait."""
    import torch
    import torch.distributed as dist

    def transfer(sends, recvs, out):
        got = {m.face: torch.empty_like(out[m.face ^ 1]) for m in recvs}
        ops = [dist.P2POp(dist.isend, buf, m.peer, group, m.tag) for m, buf in sends]
        ops += [dist.P2POp(dist.irecv, got[m.face], m.peer, group, m.tag) for m in recvs]
        for req in dist.batch_isend_irecv(ops):
            req.wait()
        return got
    return transfer


def global_mass(local_mass, group=None):
    """Sum of the ranks' FP64 masses (one all-reduce; without a process
    group, the one rank's mass)."""
    import torch
    import torch.distributed as dist
    t = torch.as_tensor(local_mass, dtype=torch.float64).reshape(1).clone()
    if dist.is_available() and dist.is_initialized():
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t[0]


class SlabRank:
    """This process's slab of a px x py decomposition (rank = the group
    rank); the exchange goes over torch.distributed (NCCL on GPUs)."""

    def __init__(self, NX, NY, nz, px, py, rank, halo=3, dtype=None, device=None,
                 nonoscillatory=True, k_bc=0, group=None):
        import torch
        self.NX, self.NY, self.nz, self.px, self.py, self.rank = NX, NY, nz, px, py, rank
        self.h = halo
        self.dtype = torch.float64 if dtype is None else dtype
        self.i0, self.nx, self.j0, self.ny = slab_extent(NX, NY, px, py, rank)
        self.s = _SlabCtx(self.nx, self.ny, nz, halo, self.dtype, device, nonoscillatory, k_bc)
        self.transfer = dist_transfer(group)
        self.group = group
        self._tmp = None

    def exchange(self, field):
        halo_exchange(field, self.rank, self.px, self.py, self.s.pack, self.s.unpack,
                      self.transfer)

    def step(self, psi, u, v, w, g, nsteps=1):
        import torch
        if self._tmp is None:
            self._tmp = torch.empty_like(psi)
        for _ in range(nsteps):
            self.exchange(psi)
            self.s.m.step_out(psi, self._tmp, u, v, w, g)
            psi.copy_(self._tmp)
        return psi

    def mass(self, psi, g):
        return global_mass(self.s.m.mass(psi, g), self.group)

    def close(self):
        self.s.m.close()
