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


def _dimer_case():
    from paper_1608_04904_gb300 import synth
    cfg, col, bonds = synth.dimer32(precision="fp64", L=12)
    cfg = dict(cfg, L=(24, 12, 12), bulk_rate=0.05)
    col = [dict(c, x=(c["x"][0] + 6.0, c["x"][1], c["x"][2]), v=(0.03, -0.01, 0.0)) for c in col]
    x, v, fl = synth.solvent(cfg, col, seed=31, frac_b=0.2)
    return cfg, col, bonds, x, v, fl


def _dimer_worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import oracle as orc
        from paper_1608_04904_gb300 import slabs, synth
        cfg, col, bonds, x, v, fl = _dimer_case()
        ca = synth.colloid_arrays(col)
        X, V = np.array(ca["x"], float), np.array(ca["v"], float)
        L0 = cfg["L"][0]
        n = len(x)
        ids = np.arange(n, dtype=np.uint32)
        slot = np.arange(n, dtype=np.int64)
        if rank != 0:
            x, v, fl, ids, slot = x[:0], v[:0], fl[:0], ids[:0], slot[:0]
        bounds = slabs.slab_bounds(L0, world)
        sent = 0
        for step in range(STEPS):
            # particles that may come near a colloid go to rank 0 for the interval
            speed = np.sqrt((v * v).sum(1)) if len(v) else np.zeros(0)
            reach = 2.0 ** (1 / 6) * np.asarray(ca["sigma"]) + cfg["skin"] + 1.0
            near = slabs.within(x, X, reach.max() + speed.max(initial=0.0) * cfg["tau"], cfg["L"])
            dest = np.where(near, 0, rank)
            sent += int(near.sum()) if rank else 0
            got = slabs.migrate({"x": x, "v": v, "flags": fl, "id": ids, "slot": slot}, dest)
            cols = dict(ca, x=X, v=V)
            if rank == 0:
                o = orc.OracleSystem(cfg, got["x"], got["v"], got["flags"], ids=got["id"], colloids=cols,
                                     bonds=list(bonds), step=step)
            else:
                o = orc.OracleSystem(cfg, got["x"], got["v"], got["flags"], ids=got["id"], step=step)
            o.interval()
            X = slabs.broadcast_array(o.X if rank == 0 else X)
            V = slabs.broadcast_array(o.V if rank == 0 else V)
            s = orc.grid_shift(cfg["seed"], step)
            key = orc.cell_keys(cfg, o.x, s)
            dest = slabs.owners(key % L0, bounds)
            got = slabs.migrate({"x": o.x, "v": o.v, "flags": o.flags, "id": o.id, "slot": got["slot"]}, dest)
            order = np.argsort(got["slot"], kind="stable")
            o2 = orc.OracleSystem(cfg, got["x"][order], got["v"][order], got["flags"][order],
                                  ids=got["id"][order], step=step)
            o2.shift_and_sort()
            o2.collide()
            o2.react()
            slot = slabs.global_slots(o2.key, o2.ncells)
            x, v, fl, ids = o2.x, o2.v, o2.flags, o2.id
        parts = [None] * world
        dist.all_gather_object(parts, (ids, x, v, fl, slot, sent))
        if rank == 0:
            out[0] = (parts, X, V)
    finally:
        dist.destroy_process_group()


def test_slab_decomposition_with_a_dimer_equals_single_rank_run(orc):
    """The sphere dimer in a 24 x 12 x 12 box on two ranks: particles near the
    colloids are integrated on rank 0, the rest fly at home, then every
    particle goes to the owner of its cell; states and colloids equal the
    single-rank run bit for bit."""
    from paper_1608_04904_gb300 import synth
    out = mp.Manager().dict()
    mp.spawn(_dimer_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    parts, X, V = out[0]
    ids = np.concatenate([p[0] for p in parts])
    x = np.concatenate([p[1] for p in parts])
    v = np.concatenate([p[2] for p in parts])
    fl = np.concatenate([p[3] for p in parts])
    slot = np.concatenate([p[4] for p in parts])
    assert sum(p[5] for p in parts) > 0                # rank 1 sent near particles over
    cfg, col, bonds, x0, v0, fl0 = _dimer_case()
    ref = orc.OracleSystem(cfg, x0, v0, fl0, colloids=synth.colloid_arrays(col), bonds=list(bonds), step=0)
    for _ in range(STEPS):
        ref.step(1)
    order = np.argsort(slot)
    assert np.array_equal(ids[order], ref.id)
    assert np.array_equal(x[order], ref.x)
    assert np.array_equal(v[order], ref.v)
    assert np.array_equal(fl[order], ref.flags)
    assert np.array_equal(X, ref.X) and np.array_equal(V, ref.V)


def test_within_tests_every_centre():
    from paper_1608_04904_gb300 import slabs
    x = np.array([[1.0, 1.0, 1.0], [9.0, 1.0, 1.0], [5.0, 5.0, 5.0], [9.8, 9.9, 0.1]])
    c = np.array([[1.0, 1.0, 1.5], [9.0, 1.2, 1.0]])
    assert slabs.within(x, c, 1.0, (10, 10, 10)).tolist() == [True, True, False, False]
    assert slabs.within(x, c, [1.0, 0.1], (10, 10, 10)).tolist() == [True, False, False, False]
    # minimum image: (9.8, 9.9, 0.1) is 0.5 from (0.3, 9.9, 0.1) across x
    assert slabs.within(x, [[0.3, 9.9, 0.1]], 0.6, (10, 10, 10)).tolist() == [False, False, False, True]
    # walls in z: no wrap along z
    assert not slabs.within([[1.0, 1.0, 9.9]], [[1.0, 1.0, 0.1]], 0.5, (10, 10, 10), walls=True)[0]
