"""The multi-rank path of bench.py on CPU (gloo, world size 2): whole-job
throughput is every rank's particles over the slowest rank's time, and each
rank runs its own independent replicas (weak scaling, no collective on the
data path)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms = [10.0, 25.0][rank]           # the second rank is the slower one
        n = [1000, 3000][rank]
        value, ms_job = bench.job_throughput(ms, n, steps=7)
        reps, _ = bench.workload("dimer32", "mixed", seed_offset=rank)
        out[rank] = (value, ms_job, reps[0][0]["seed"], tuple(reps[0][0]["L"]))
    finally:
        dist.destroy_process_group()


def test_job_throughput_and_replica_seeds_over_two_ranks():
    port = _free_port()
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    for rank in (0, 1):
        value, ms_job, seed, L = out[rank]
        assert ms_job == 25.0                                  # max over ranks
        assert value == pytest.approx((1000 + 3000) * 7 / 0.025)  # all particles / slowest time
        assert L == (32, 32, 32)
    assert out[0][2] != out[1][2]                              # independent replicas per rank


def test_job_throughput_single_process():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    value, ms = bench.job_throughput(20.0, 500, steps=4)
    assert ms == 20.0 and value == pytest.approx(500 * 4 / 0.02)
