"""The multi-GPU form is independent replicas (no data-path collective): each
rank synthesises its own seeded volume, the timed region is bracketed by
barriers, and the whole-job value is the units all ranks processed over the
slowest rank's time. This checks that bookkeeping of bench.py with two gloo
ranks on the CPU (127.0.0.1 rendezvous)."""
import multiprocessing as mp
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        w, r, local = bench.dist_setup()
        dist.barrier()
        value, slowest = bench.replica_throughput(100.0 * (rank + 1), 0.5 + rank, "cpu")
        seeds = [None] * world
        dist.all_gather_object(seeds, bench.replica_seed(rank))
        q.put((rank, w, r, local, value, slowest, seeds))
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas_aggregate_max_time_and_total_units():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    try:
        out = sorted(q.get(timeout=120) for _ in range(world))
    finally:
        for p in procs:
            p.join(timeout=60)
    for p in procs:
        assert p.exitcode == 0
    for rank, w, r, local, value, slowest, seeds in out:
        assert (w, r, local) == (world, rank, rank)
        assert slowest == pytest.approx(1.5)            # max over ranks of 0.5, 1.5 s
        assert value == pytest.approx(300.0 / 1.5)     # (100 + 200) units / slowest
        assert len(set(seeds)) == world                 # every replica draws its own volume


def test_single_process_is_identity():
    import bench
    assert bench.replica_throughput(42.0, 2.0, "cpu") == (21.0, 2.0)
