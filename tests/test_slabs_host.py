"""Host logic of the i-j slab decomposition (no GPU): the slab sizes, the
neighbour map, the order of the exchange's messages, and the exchange and
FP64 mass all-reduce run as gloo processes on CPU tensors.

In the gloo runs the strips are packed and unpacked by numpy slicing that
follows the strip geometry the library's header states (x faces: interior
rows, h columns; y faces: h rows of the padded width); the GPU tests check
the library's own pack/unpack kernels.  After the exchange every rank's halo
must equal the periodic padding of the undivided domain."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1908_06094_b300 import slabs  # noqa: E402


def test_split_sizes_cover_the_domain():
    for n, p in ((256, 2), (256, 3), (97, 4), (5, 5)):
        s = slabs.split_sizes(n, p)
        assert sum(s) == n and len(s) == p and max(s) - min(s) <= 1
    with pytest.raises(ValueError):
        slabs.split_sizes(3, 4)


def test_neighbours_are_mutual():
    for px, py in ((1, 1), (2, 1), (1, 3), (2, 2), (3, 2), (4, 3)):
        for r in range(px * py):
            nb = slabs.neighbours(r, px, py)
            for f in range(4):
                assert slabs.neighbours(nb[f], px, py)[f ^ 1] == r


def test_plan_pairs_messages_in_order():
    """Backends that match messages by order: for every pair of ranks, the
    k-th send from a to b must be the k-th receive b posts from a, and carry
    the face b expects."""
    for px, py in ((2, 1), (1, 2), (2, 2), (3, 2), (2, 3), (4, 4)):
        n = px * py
        plans = [slabs.exchange_plan(r, px, py) for r in range(n)]
        for ph in range(2):
            for a in range(n):
                for b in range(n):
                    sends = [m for m in plans[a][ph][1] if m.peer == b]
                    recvs = [m for m in plans[b][ph][2] if m.peer == a]
                    assert len(sends) == len(recvs)
                    for s, r in zip(sends, recvs):
                        assert s.tag == r.tag          # the sender's face
                        assert r.face == s.face ^ 1    # lands beyond the opposite face


def test_self_exchange_when_one_slab_spans_a_direction():
    plan = slabs.exchange_plan(0, 1, 1)
    for phase, sends, recvs, local in plan:
        assert not sends and not recvs and sorted(local) == sorted(phase)


# ---------------------------------------------------------------- gloo ranks --

def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


H = 3


def _np_strip(g_nx, g_ny, face, unpack):
    """(k, j, i) slices of the strip of face f in padded coordinates."""
    h = H
    if face < 2:
        js = slice(h, h + g_ny)
        if face == 0:
            i0 = 0 if unpack else h
        else:
            i0 = h + g_nx if unpack else g_nx
        return js, slice(i0, i0 + h)
    is_ = slice(0, g_nx + 2 * h)
    if face == 2:
        j0 = 0 if unpack else h
    else:
        j0 = h + g_ny if unpack else g_ny
    return slice(j0, j0 + h), is_


def _global(NX, NY, nz, seed):
    rng = np.random.default_rng(seed)
    return rng.random((nz, NY, NX)) + 0.5


def _rank_main(rank, ws, port, out_dir, NX, NY, nz, px, py):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=ws)
    try:
        psi = _global(NX, NY, nz, 1)
        G = _global(NX, NY, nz, 2)
        i0, nx, j0, ny = slabs.slab_extent(NX, NY, px, py, rank)
        f = torch.full((nz + 2 * H, ny + 2 * H, nx + 2 * H), float("nan"), dtype=torch.float64)
        f[H:H + nz, H:H + ny, H:H + nx] = torch.from_numpy(psi[:, j0:j0 + ny, i0:i0 + nx])

        def pack(fl, face):
            js, is_ = _np_strip(nx, ny, face, False)
            return fl[H:H + nz, js, is_].contiguous().reshape(-1)

        def unpack(buf, face, fl):
            js, is_ = _np_strip(nx, ny, face, True)
            fl[H:H + nz, js, is_] = buf.reshape(fl[H:H + nz, js, is_].shape)

        slabs.halo_exchange(f, rank, px, py, pack, unpack, slabs.dist_transfer())
        local = float(np.sum(psi[:, j0:j0 + ny, i0:i0 + nx] * G[:, j0:j0 + ny, i0:i0 + nx]))
        tot = float(slabs.global_mass(local))
        np.save(os.path.join(out_dir, f"f{rank}.npy"), f.numpy())
        with open(os.path.join(out_dir, f"m{rank}.txt"), "w") as fh:
            fh.write(repr(tot))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("px,py,NX,NY", [(2, 1, 11, 9), (2, 2, 12, 10)])
def test_gloo_exchange_and_mass(tmp_path, px, py, NX, NY):
    ws, nz = px * py, 3
    mp.start_processes(_rank_main, args=(ws, _free_port(), str(tmp_path), NX, NY, nz, px, py),
                       nprocs=ws, start_method="spawn")
    psi = _global(NX, NY, nz, 1)
    G = _global(NX, NY, nz, 2)
    wrapped = np.pad(psi, ((0, 0), (H, H), (H, H)), mode="wrap")   # the periodic domain
    for r in range(ws):
        f = np.load(tmp_path / f"f{r}.npy")
        i0, nx, j0, ny = slabs.slab_extent(NX, NY, px, py, r)
        want = wrapped[:, j0:j0 + ny + 2 * H, i0:i0 + nx + 2 * H]
        # every level's whole padded plane: interior, i-j halo and corners
        assert np.array_equal(f[H:H + nz], want), r
        tot = float((tmp_path / f"m{r}.txt").read_text())
        assert tot == pytest.approx(float(np.sum(psi * G)), rel=1e-14)
