"""The multi-GPU path is replicas only: no data-path collective, a barrier
around the timed region and the maximum step time over ranks.  This runs
bench.py's plumbing as two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.barrier(world)
        ms = 1.0 + rank                       # rank 1 is the slower replica
        worst = bench.max_over_ranks(ms, world)
        value = bench.replica_throughput(1_000_000, world, worst)
        bench.barrier(world)
        q.put((rank, worst, value))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_replica():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, worst, value in got:
        assert worst == 2.0                     # max over ranks
        assert abs(value - 1000.0) < 1e-9       # 2 ranks x 1e6 samples / 2 ms = 1000 MPix/s


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert abs(bench.replica_throughput(79_550_464, 1, 0.16) - 497190.4) < 1e-3
