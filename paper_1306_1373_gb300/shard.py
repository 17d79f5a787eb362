"""Sharding one batch of images across GPUs (one process per GPU).

Every 8x8 block, and so every image, is coded independently (Sec. 2.5.2's
transform works on single blocks), so a batch splits without any exchange
on the data path: rank r codes a contiguous share of the item list through
its own plan and graph, and the only message is the per-image SSE (one
uint64 word per image) gathered at the end, from which the PSNR of Eq. 23
follows on any rank.

The shares are balanced by sample count, not by image count: uneven image
sizes would otherwise leave the rank with the large images behind.
"""
import torch


def partition_by_samples(samples, world):
    """Contiguous shares of items with the given sample counts: a list of
    `world` (begin, end) index ranges covering 0..len(samples) in order,
    where share r ends at the first item whose running total reaches
    (r + 1) / world of the whole.  Shares may be empty (more ranks than
    items, or one item larger than a share)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    n = len(samples)
    total = sum(int(s) for s in samples)
    bounds = [0]
    acc = 0
    i = 0
    for r in range(1, world):
        goal = total * r / world
        while i < n and acc + int(samples[i]) <= goal:
            acc += int(samples[i])
            i += 1
        # take the item that straddles the goal when that ends nearer to it
        if i < n and (acc + int(samples[i]) - goal) < (goal - acc):
            acc += int(samples[i])
            i += 1
        bounds.append(max(i, bounds[-1]))
    bounds.append(n)
    return [(bounds[r], bounds[r + 1]) for r in range(world)]


def gather_sse(local_sse, shares, rank, world, device=None):
    """All ranks' per-image SSE words in item order.  local_sse is this
    rank's int64 tensor (its share's length); shares the partition.  One
    all_gather of max-share-length int64 words per rank (padded); with a
    single rank it returns local_sse unchanged."""
    if world == 1:
        return local_sse
    import torch.distributed as dist
    device = local_sse.device if device is None else device
    width = max(1, max(e - b for b, e in shares))
    buf = torch.zeros(width, dtype=torch.int64, device=device)
    b, e = shares[rank]
    if e > b:
        buf[:e - b] = local_sse.to(device=device, dtype=torch.int64)
    parts = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(parts, buf)
    return torch.cat([parts[r][:e - b] for r, (b, e) in enumerate(shares)])
