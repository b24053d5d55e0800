"""Beam sharding across processes (one process per GPU).

TDSC and FDSC are independent per beam (Sec. IV: statistics are taken per
channel row or per time column of one beam's batch), so a multi-GPU job
partitions whole beams across ranks with no exchange on the data path: each
rank cleans its share with its own context, and only host-side results
(counters, latencies, optionally the cleaned beams) are gathered.

`partition_beams` balances the ranks by bytes (largest beam first onto the
least-loaded rank; ties broken by index, so every rank computes the same
plan without communication).
"""
from __future__ import annotations

import heapq


def partition_beams(beam_bytes, world: int):
    """Indices of the beams each of `world` ranks cleans, balanced by bytes.

    Every beam goes to exactly one rank; each rank's list is in increasing
    beam order.  The most-loaded rank exceeds the least-loaded one by at most
    the largest beam."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(beam_bytes)), key=lambda i: (-int(beam_bytes[i]), i))
    heap = [(0, r) for r in range(world)]
    shares = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        shares[r].append(i)
        heapq.heappush(heap, (load + int(beam_bytes[i]), r))
    return [sorted(s) for s in shares]


def rank_share(beam_bytes, world: int, rank: int):
    return partition_beams(beam_bytes, world)[rank]


def clean_sharded(beams, clean_fn, group=None):
    """Clean a list of beams across the ranks of a torch.distributed group.

    beams: the full list (every rank holds the same list of arrays, or of any
    objects clean_fn accepts); clean_fn(beam) -> result.  Each rank cleans
    its share and the results are gathered on every rank, in beam order.
    Collectives are host-side (all_gather_object); no device data moves."""
    import torch.distributed as dist

    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    sizes = [getattr(b, "nbytes", 1) for b in beams]
    mine = rank_share(sizes, world, rank)
    local = {i: clean_fn(beams[i]) for i in mine}
    gathered = [None] * world
    dist.all_gather_object(gathered, local, group=group)
    out = [None] * len(beams)
    for part in gathered:
        for i, r in part.items():
            out[i] = r
    return out
