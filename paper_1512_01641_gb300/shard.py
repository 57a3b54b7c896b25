"""Sharding document pairs over ranks (one process per GPU).

Document pairs are independent (the paper parallelises mining over article
pairs, Section 5), so ranks exchange nothing while they mine: the pairs are
partitioned by greedy longest-processing-time on their cell count N*M (the
largest pairs first, each to the currently least-loaded rank), every rank
mines its shard, and the variable-length results are gathered once at the
end.
"""
from __future__ import annotations

import heapq

import numpy as np


def lpt_partition(cost, world: int) -> list[np.ndarray]:
    """Indices of the pairs of each rank (ascending).  Greedy LPT: within 4/3
    of the optimal makespan."""
    cost = np.asarray(cost, np.float64)
    if world < 1:
        raise ValueError("world must be >= 1")
    order = np.argsort(-cost, kind="stable")
    heap = [(0.0, r) for r in range(world)]
    owner = np.empty(len(cost), np.int64)
    for k in order:
        load, r = heapq.heappop(heap)
        owner[k] = r
        heapq.heappush(heap, (load + cost[k], r))
    return [np.nonzero(owner == r)[0] for r in range(world)]


def shard_of(batch, rank: int, world: int):
    """(pair indices, sub-batch) of this rank."""
    cost = batch.src.doc_sizes() * batch.tgt.doc_sizes()
    idx = lpt_partition(cost, world)[rank]
    return idx, batch.subset(idx)


def gather_results(idx, scores, links, group=None, dst: int = 0):
    """Gather per-rank (pair indices, pair scores, per-pair link lists) to dst;
    returns (scores, links) over all pairs in original order on dst, None
    elsewhere.  One collective at the end of mining (gather of Python objects;
    no tensor exchange while mining)."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    payload = (np.asarray(idx).tolist(), [float(s) for s in scores], links)
    out = [None] * world if rank == dst else None
    dist.gather_object(payload, out, dst=dst, group=group)
    if rank != dst:
        return None
    n = sum(len(p[0]) for p in out)
    all_scores = [None] * n
    all_links = [None] * n
    for ids, sc, lk in out:
        for x, k in enumerate(ids):
            all_scores[k] = sc[x]
            all_links[k] = lk[x]
    return all_scores, all_links
