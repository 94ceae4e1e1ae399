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


# ---------------------------------------------------------------------------------------------
# Time shards of one long stream (the paper fans a month of data out over 160 GPUs, section
# "Inference-optimized AI ensemble"): rank r takes a contiguous range of windows (its core) and
# computes them with `margin` windows of context on each side (its span).  Sample g of the stitched
# series (window 0 gives samples [0, W), window w >= 1 its last `stride` samples) is strain sample g,
# so a span's local indices are global indices minus the span's first sample.  Positions of the
# core are computed exactly as in one process; peaks and ensemble triggers are found on the span's
# stitched series and kept when their index lies in the core's part of the global series, so the
# cores partition the triggers (peaks whose prominence or width walks reach beyond the span can
# differ from whole-stream peak finding: walks_leave_span flags them, and an exact value for them needs
# the neighbouring shards' running maxima and minima, which is not exchanged here).  Time slides pair Hanford window
# w with Livingston window (w + k) mod n_windows: a shard also needs the Livingston windows its
# offsets reach, wrapping at the end of the stream.


def shard_windows(n_windows: int, world: int, rank: int):
    """Core [w0, w1) of `rank`: contiguous, sizes differing by at most one window."""
    if world < 1 or not (0 <= rank < world) or n_windows < 0:
        raise ValueError("bad world/rank/n_windows")
    q, r = divmod(n_windows, world)
    w0 = rank * q + min(rank, r)
    return w0, w0 + q + (1 if rank < r else 0)


def shard_span(n_windows: int, window: int, stride: int, w0: int, w1: int, margin: int):
    """(ws, we, s0, s1): windows [ws, we) computed by the shard (core plus margin, clipped) and the
    strain samples [s0, s1) they read."""
    ws = max(0, w0 - margin)
    we = min(n_windows, w1 + margin)
    if we <= ws:
        return ws, ws, ws * stride, ws * stride
    return ws, we, ws * stride, (we - 1) * stride + window


def core_series_range(n_windows: int, window: int, stride: int, w0: int, w1: int):
    """[g0, g1): the part of the global stitched series that the core windows [w0, w1) give."""
    def start(w):
        return 0 if w == 0 else window + (w - 1) * stride
    if w1 <= w0:
        return start(w0), start(w0)
    return start(w0), start(w1)


def livingston_windows(n_windows: int, w0: int, w1: int, offsets):
    """Sorted Livingston windows that Hanford windows [w0, w1) pair with under the slide offsets
    (offset k pairs w with (w + k) mod n_windows)."""
    need = set()
    for k in offsets:
        for w in range(w0, w1):
            need.add((w + int(k)) % n_windows)
    return np.array(sorted(need), dtype=np.int64)


def keep_core(records: np.ndarray, span_first_sample: int, g0: int, g1: int) -> np.ndarray:
    """Records of a shard's span (indices local to the span's first sample) whose global index lies
    in the core range [g0, g1), with their indices made global."""
    recs = np.array(records, copy=True)
    recs["index"] = recs["index"] + int(span_first_sample)
    return recs[(recs["index"] >= g0) & (recs["index"] < g1)]


def walks_leave_span(series: np.ndarray, index, exact_lo: int, at_start: bool, at_end: bool) -> np.ndarray:
    """Boolean per peak (indices into a span's stitched `series`): its prominence walk on some side
    reaches the end of the span's exact part without meeting a higher sample, so that its base (and
    the width derived from it) depends on samples of other shards.  exact_lo: first exact sample of
    the span (its first window also gives W - stride samples that the global series takes from the
    previous window); at_start / at_end: the span touches the start / end of the stream, where a walk
    ends anyway."""
    x = np.asarray(series)
    idx = np.asarray(index, dtype=np.int64)
    out = np.zeros(idx.shape[0], dtype=bool)
    n = x.shape[0]
    # running maxima from the exact start to the left of each sample, and from the right end
    left_max = np.maximum.accumulate(np.concatenate([[-np.inf], x[exact_lo:]]))[:-1]
    right_max = np.maximum.accumulate(np.concatenate([x[::-1], [-np.inf]]))[::-1][1:]
    for k, p in enumerate(idx):
        v = x[p]
        left_open = (not at_start) and (p <= exact_lo or left_max[p - exact_lo] <= v)
        right_open = (not at_end) and (p >= n - 1 or right_max[p] <= v)
        out[k] = left_open or right_open
    return out


def gather_shard_triggers(records: np.ndarray, dist=None, dst: int = 0):
    """Gather the shards' core records on `dst`, sorted by (slide, model with the ensemble last,
    index) as one process would list them; None on the other ranks."""
    recs = np.asarray(records)
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        parts = [None] * dist.get_world_size() if dist.get_rank() == dst else None
        dist.gather_object(recs, parts, dst=dst)
        if dist.get_rank() != dst:
            return None
        allr = np.concatenate(parts)
    else:
        allr = recs
    model_key = np.where(allr["model"] < 0, np.iinfo(np.int32).max, allr["model"])
    order = np.lexsort((allr["index"], model_key, allr["slide"]))
    return allr[order]
