"""The x-slab decomposition of one system (paper_1608_04904_gb300.slabs) on
CPU ranks with gloo: a Poiseuille channel with walls, body force, virtual
wall particles and bulk reaction, stepped on two and three ranks with the
oracle as each rank's compute, equals the single-rank oracle run bit for bit
-- positions, velocities and species of every particle -- while particles
migrate between ranks as the random grid shift moves the owned columns."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STEPS = 4


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _case():
    from paper_1608_04904_gb300 import synth
    cfg = synth.base_config(L=(12, 6, 5), walls=1, rho_wall=10, g=(0.02, 0.0, 0.0), bulk_rate=0.2,
                            alpha=np.radians(130.0), tau=0.5, kT=1.0, seed=11, precision="fp64")
    x, v, fl = synth.solvent(cfg, seed=12, frac_b=0.3)
    return cfg, x, v, fl


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import oracle as orc
        from paper_1608_04904_gb300 import slabs
        cfg, x, v, fl = _case()
        L0 = cfg["L"][0]
        n = len(x)
        ids = np.arange(n, dtype=np.uint32)
        slot = np.arange(n, dtype=np.int64)          # the initial storage order
        if rank != 0:                                # everything starts on rank 0
            x, v, fl, ids, slot = x[:0], v[:0], fl[:0], ids[:0], slot[:0]
        bounds = slabs.slab_bounds(L0, world)
        moved = 0
        for step in range(STEPS):
            o = orc.OracleSystem(cfg, x, v, fl, ids=ids, step=step)
            o.interval()                             # streaming (no colloids)
            s = orc.grid_shift(cfg["seed"], step)
            key = orc.cell_keys(cfg, o.x, s)
            dest = slabs.owners(key % L0, bounds)
            moved += int((dest != rank).sum())
            got = slabs.migrate({"x": o.x, "v": o.v, "flags": o.flags, "id": o.id, "slot": slot}, dest)
            order = np.argsort(got["slot"], kind="stable")   # the previous global order
            o2 = orc.OracleSystem(cfg, got["x"][order], got["v"][order], got["flags"][order],
                                  ids=got["id"][order], step=step)
            o2.shift_and_sort()
            mine = slabs.owners(o2.key % L0, bounds)
            assert np.all(mine == rank)
            o2.collide()
            o2.react()
            slot = slabs.global_slots(o2.key, o2.ncells)
            x, v, fl, ids = o2.x, o2.v, o2.flags, o2.id
        parts = [None] * world
        dist.all_gather_object(parts, (ids, x, v, fl, slot, moved))
        if rank == 0:
            out[0] = parts
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_slab_decomposition_equals_single_rank_run(orc, world):
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    parts = out[0]
    ids = np.concatenate([p[0] for p in parts])
    x = np.concatenate([p[1] for p in parts])
    v = np.concatenate([p[2] for p in parts])
    fl = np.concatenate([p[3] for p in parts])
    slot = np.concatenate([p[4] for p in parts])
    assert all(p[5] > 0 for p in parts[:1])          # particles did change ranks
    assert sum(len(p[0]) for p in parts[1:]) > 0     # and every rank holds some

    cfg, x0, v0, fl0 = _case()
    ref = orc.OracleSystem(cfg, x0, v0, fl0, step=0)
    for _ in range(STEPS):
        ref.step(1)
    assert np.array_equal(np.sort(slot), np.arange(len(x0)))
    # the global slots are the single-rank storage order
    order = np.argsort(slot)
    assert np.array_equal(ids[order], ref.id)
    assert np.array_equal(x[order], ref.x)
    assert np.array_equal(v[order], ref.v)
    assert np.array_equal(fl[order], ref.flags)


def test_bounds_and_owners():
    from paper_1608_04904_gb300 import slabs
    b = slabs.slab_bounds(10, 3)
    assert b.tolist() == [0, 3, 6, 10]
    assert slabs.owners([0, 2, 3, 5, 6, 9], b).tolist() == [0, 0, 1, 1, 2, 2]
    with pytest.raises(ValueError):
        slabs.slab_bounds(2, 3)
