"""Sharding one batch across ranks (host logic, on the CPU): the partition
into contiguous sample-balanced shares, and the per-image SSE gather run as
two and three gloo ranks whose worker codes its share with the CPU oracle.
The gathered list must equal the single-rank list item for item."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_1306_1373_gb300.shard import gather_sse, partition_by_samples


def test_partition_is_contiguous_complete_and_balanced():
    rng = np.random.default_rng(1)
    for trial in range(200):
        n = int(rng.integers(1, 60))
        world = int(rng.integers(1, 9))
        samples = [int(v) for v in rng.integers(64, 4_000_000, size=n)]
        shares = partition_by_samples(samples, world)
        assert len(shares) == world
        assert shares[0][0] == 0 and shares[-1][1] == n
        for (b0, e0), (b1, e1) in zip(shares, shares[1:]):
            assert e0 == b1 and b0 <= e0
        total = sum(samples)
        for b, e in shares:
            assert sum(samples[b:e]) <= total / world + max(samples)


def test_partition_edge_cases():
    assert partition_by_samples([5], 1) == [(0, 1)]
    assert partition_by_samples([10], 2) in ([(0, 0), (0, 1)], [(0, 1), (1, 1)])
    assert partition_by_samples([1, 1, 1, 1], 2) == [(0, 2), (2, 4)]
    assert partition_by_samples([100, 1, 1, 1], 2) == [(0, 1), (1, 4)]
    assert partition_by_samples([], 3) == [(0, 0)] * 3
    with pytest.raises(ValueError):
        partition_by_samples([1], 0)


def workload():
    from synth import powerlaw_image
    rng = np.random.default_rng(4)
    items = []
    for i in range(9):
        h, w = int(rng.integers(8, 70)), int(rng.integers(8, 90))
        items.append((powerlaw_image(h, w, seed=90 + i).numpy(), int(rng.integers(10, 96))))
    return items


def oracle_sse(img, quality):
    from oracle import codec, ijg, psnr
    Q = ijg.luma_table(quality)
    return psnr.sse(img, codec.reconstruct_plane(codec.compress_plane(img, Q), Q, *img.shape))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        items = workload()
        shares = partition_by_samples([img.size for img, _ in items], world)
        b, e = shares[rank]
        local = torch.tensor([oracle_sse(img, qq) for img, qq in items[b:e]], dtype=torch.int64)
        full = gather_sse(local, shares, rank, world)
        q.put((rank, (b, e), full.tolist()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_gather_the_single_rank_sse_list(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=180) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    expect = [oracle_sse(img, qq) for img, qq in workload()]
    spans = [span for _, span, _ in got]
    assert spans[0][0] == 0 and spans[-1][1] == len(expect)
    assert all(e > b for b, e in spans)            # every rank had work in this workload
    for rank, _, full in got:
        assert full == expect, rank


def test_single_rank_gather_is_identity():
    t = torch.tensor([3, 1, 4], dtype=torch.int64)
    assert gather_sse(t, [(0, 3)], 0, 1) is t
