"""Multi-GPU runs are replicas only: each rank solves its own instances and
the job's time is the slowest rank's. The rank logic of bench.py is checked
here on CPU with two gloo ranks (no GPU involved)."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seeds = bench.rank_seeds(rank, 10)
        gathered = [None] * world
        dist.all_gather_object(gathered, seeds)
        flat = [s for g in gathered for s in g]
        elapsed = bench.max_over_ranks(1.0 + rank)       # rank 1 is slower
        out[rank] = (len(flat) == len(set(flat)), elapsed,
                     bench.replica_throughput(20, world, elapsed))
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        disjoint, elapsed, value = res[rank]
        assert disjoint                      # no instance is solved twice
        assert elapsed == 2.0                # every rank sees the slowest time
        assert value == 20 * 2 / 2.0         # all ranks' solves over that time


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.rank_seeds(0, 3) == [0, 1, 2]
