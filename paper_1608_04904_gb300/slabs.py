"""x-slab decomposition of one MPCD system over several ranks: which rank
owns which cells of the collision grid, the migration of particles to the
owners of their cells, and the global storage slots that keep the stable
within-cell order of a single-rank run.

The module moves particles; it computes nothing of the method.  One step of
a decomposed system is: every rank streams its particles; the ranks agree on
the step's grid shift (it is a function of the seed and the step); every
particle goes to the rank owning the x-column of its cell on that grid
(`owners`, `migrate`); every rank puts what it received back into the
previous global storage order (sort by `slot`), bins, collides and reacts
its own cells, and numbers its particles in the new global order
(`global_slots`).  The collision's per-cell sums then run over the same
particles in the same order as on one rank, so the decomposed run equals the
single-rank run bit for bit.  Because the grid shift moves every step, the
columns a rank owns are those of the shifted grid, not fixed positions.

With colloids, one rank integrates them: before each interval every rank
sends it the particles that may come near a colloid (`within`, a
conservative superset of the near list: the integrating rank's MD decides
near or far exactly, and a far particle flies the same there as at home),
and after the interval the colloid state is broadcast (`broadcast_array`).
The colloid force sums are exact fixed-point sums, so their order does not
matter and the decomposed run still equals the single-rank run.

Transport is `torch.distributed` on host arrays (the gloo backend); a
device version moves the same packed buffers as CUDA tensors over NCCL."""
from __future__ import annotations

import numpy as np
import torch
import torch.distributed as dist


def slab_bounds(Lx: int, world: int) -> np.ndarray:
    """Column ranges [b[r], b[r + 1]) of the collision grid owned by rank r,
    as even as integer division allows."""
    if world < 1 or Lx < world:
        raise ValueError(f"cannot split {Lx} cell columns over {world} ranks")
    return np.array([(Lx * r) // world for r in range(world + 1)], dtype=np.int64)


def owners(cell_x, bounds) -> np.ndarray:
    """Rank owning each cell column index (0 <= cell_x < Lx)."""
    cell_x = np.asarray(cell_x, dtype=np.int64)
    return (np.searchsorted(bounds, cell_x, side="right") - 1).astype(np.int64)


def _exchange(arr: np.ndarray, order: np.ndarray, send: np.ndarray, recv: np.ndarray, group) -> np.ndarray:
    """All-to-all of the rows of arr, taken in `order` (grouped by destination).
    Rows travel as whole 8-byte words, so every dtype arrives bit for bit."""
    src = np.ascontiguousarray(arr[order])
    item = src.dtype.itemsize * (int(np.prod(arr.shape[1:])) if arr.ndim > 1 else 1)
    width = (item + 7) // 8
    buf = np.zeros((len(src), width * 8), dtype=np.uint8)
    if len(src):
        buf[:, :item] = src.reshape(len(src), -1).view(np.uint8)
    out = torch.empty(int(recv.sum()) * width, dtype=torch.int64)
    dist.all_to_all_single(out, torch.from_numpy(buf.view(np.int64).reshape(-1).copy()),
                           [int(c) * width for c in recv], [int(c) * width for c in send], group=group)
    got = np.ascontiguousarray(out.numpy().view(np.uint8).reshape(-1, width * 8)[:, :item])
    return got.view(arr.dtype).reshape((-1,) + arr.shape[1:])


def migrate(fields: dict, dest, group=None) -> dict:
    """Send particle i (row i of every array in `fields`) to rank dest[i].
    Returns the received particles: grouped by source rank in rank order,
    each source's particles in their order on that rank."""
    world = dist.get_world_size(group)
    dest = np.asarray(dest, dtype=np.int64)
    n = len(dest)
    for k, a in fields.items():
        if len(a) != n:
            raise ValueError(f"field {k} has {len(a)} rows, dest has {n}")
    order = np.argsort(dest, kind="stable")
    send = np.bincount(dest, minlength=world).astype(np.int64)
    recv_t = torch.empty(world, dtype=torch.int64)
    dist.all_to_all_single(recv_t, torch.from_numpy(send.copy()), group=group)
    recv = recv_t.numpy()
    return {k: _exchange(np.asarray(a), order, send, recv, group) for k, a in fields.items()}


def global_slots(key_sorted, n_cells: int, group=None) -> np.ndarray:
    """Slot of every local particle in the global storage order (all cells in
    key order, each cell's particles in their sorted order), given this
    rank's particles sorted by cell key; every cell belongs to one rank."""
    key = np.asarray(key_sorted, dtype=np.int64)
    local = np.bincount(key, minlength=n_cells).astype(np.int64)
    total = torch.from_numpy(local.copy())
    dist.all_reduce(total, op=dist.ReduceOp.SUM, group=group)
    gstart = np.concatenate([[0], np.cumsum(total.numpy())[:-1]])
    lstart = np.concatenate([[0], np.cumsum(local)[:-1]])
    i = np.arange(len(key), dtype=np.int64)
    return gstart[key] + (i - lstart[key])


def within(x, centers, radius, L, walls: bool = False) -> np.ndarray:
    """Particles closer than radius[j] to some centers[j] (a scalar radius
    applies to every centre; minimum image on the periodic axes): the routing
    test that picks the particles to send to the rank integrating the
    colloids."""
    x = np.asarray(x, dtype=np.float64).reshape(-1, 3)
    out = np.zeros(len(x), dtype=bool)
    L = np.asarray(L, dtype=np.float64)
    per = np.array([True, True, not walls])
    centers = np.asarray(centers, dtype=np.float64).reshape(-1, 3)
    radius = np.broadcast_to(np.asarray(radius, dtype=np.float64), (len(centers),))
    for c, r in zip(centers, radius):
        d = x - c
        d[:, per] -= L[per] * np.round(d[:, per] / L[per])
        out |= (d * d).sum(1) < float(r) * float(r)
    return out


def broadcast_array(a, src: int = 0, group=None) -> np.ndarray:
    """The array held by rank src, on every rank (same shape and dtype on
    all ranks), bit for bit."""
    a = np.ascontiguousarray(a)
    buf = torch.from_numpy(a.view(np.uint8).reshape(-1).copy())
    dist.broadcast(buf, src=src, group=group)
    return buf.numpy().view(a.dtype).reshape(a.shape)
