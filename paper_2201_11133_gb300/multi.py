"""Host-side logic for running the detector on several GPUs (one process per GPU).

Windows are independent (the inference batch of the paper's TensorRT paragraph
is a stack of independent 1 s windows), and so are analysis segments: ranks
take whole segments and need no data exchange while they compute.  The only
communication is around the computation: the maximum of the per-rank times for
the throughput figure, and gathering the (small) trigger lists to one rank.
Nothing here touches the GPU; the functions work with any torch.distributed
backend (NCCL on GPUs, gloo on CPUs).
"""
from __future__ import annotations

import heapq

import numpy as np


def rank_segments(seg_lengths, world: int, rank: int, window: int = 4096, stride: int = 2048):
    """Indices of the segments assigned to `rank`: longest-first to the rank with the fewest
    windows so far (ties to the lower rank), so that every rank gets about the same work.
    Segments shorter than one window carry no work and go nowhere."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("bad world/rank")
    work = []
    for i, n in enumerate(seg_lengths):
        nw = (int(n) - window) // stride + 1 if int(n) >= window else 0
        if nw > 0:
            work.append((nw, i))
    work.sort(key=lambda t: (-t[0], t[1]))
    heap = [(0, r) for r in range(world)]
    owner = {}
    for nw, i in work:
        load, r = heapq.heappop(heap)
        owner[i] = r
        heapq.heappush(heap, (load + nw, r))
    return sorted(i for i, r in owner.items() if r == rank)


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """Maximum of a per-rank scalar over all ranks (the job time is the slowest rank's)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_triggers(records: np.ndarray, segment_ids: np.ndarray, dist=None, dst: int = 0):
    """Gather trigger records (structured arrays) with the id of the segment each one belongs to.

    Returns, on `dst`, one array with a leading `segment` field, sorted by (segment, slide,
    model, index) (ensemble records, model -1, after the per-model ones of their slide), and None
    on the other ranks.  With one process it just tags and sorts."""
    recs = np.asarray(records)
    seg = np.asarray(segment_ids, dtype=np.int64)
    if recs.shape[0] != seg.shape[0]:
        raise ValueError("one segment id per record")
    dt = np.dtype([("segment", np.int64)] + [(n, recs.dtype[n]) for n in recs.dtype.names])
    mine = np.zeros(recs.shape[0], dtype=dt)
    mine["segment"] = seg
    for n in recs.dtype.names:
        mine[n] = recs[n]
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        parts = [None] * dist.get_world_size() if dist.get_rank() == dst else None
        dist.gather_object(mine, parts, dst=dst)
        if dist.get_rank() != dst:
            return None
        allr = np.concatenate(parts) if parts else mine
    else:
        allr = mine
    model_key = np.where(allr["model"] < 0, np.iinfo(np.int32).max, allr["model"])
    order = np.lexsort((allr["index"], model_key, allr["slide"], allr["segment"]))
    return allr[order]
