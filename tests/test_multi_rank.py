"""The multi-process host logic on CPU with the gloo backend (world size 2):
segment assignment, the max-over-ranks time, and the trigger gather."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2201_11133_gb300 import multi, TRIGGER_DTYPE


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_rank_segments_partitions_and_balances():
    rng = np.random.default_rng(3)
    lengths = list(rng.integers(1000, 4096 * 300, size=57)) + [100, 4095]
    world = 4
    parts = [multi.rank_segments(lengths, world, r) for r in range(world)]
    flat = sorted(i for p in parts for i in p)
    nonempty = [i for i, n in enumerate(lengths) if n >= 4096]
    assert flat == nonempty                             # each segment with work goes to exactly one rank
    loads = [sum((lengths[i] - 4096) // 2048 + 1 for i in p) for p in parts]
    biggest = max((n - 4096) // 2048 + 1 for n in lengths if n >= 4096)
    assert max(loads) - min(loads) <= biggest          # greedy longest-first bound
    with pytest.raises(ValueError):
        multi.rank_segments(lengths, 2, 2)


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = multi.max_over_ranks(1.5 + rank, dist)
        recs = np.zeros(3, dtype=TRIGGER_DTYPE)
        recs["index"] = [30 + rank, 10, 20]
        recs["model"] = [0, -1, 1]
        recs["slide"] = [0, 0, 0]
        recs["height"] = rank
        seg = np.full(3, rank, dtype=np.int64)
        out = multi.gather_triggers(recs, seg, dist)
        if rank == 0:
            q.put((t, out.tolist()))
        else:
            q.put((t, out))
    finally:
        dist.destroy_process_group()


def test_gloo_world_size_two():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    times = sorted(r[0] for r in res)
    assert times == [2.5, 2.5]                           # max over ranks on both
    gathered = [r[1] for r in res if r[1] is not None]
    assert len(gathered) == 1                            # only rank 0 receives
    g = gathered[0]
    segs = [row[0] for row in g]
    assert segs == [0, 0, 0, 1, 1, 1]
    # within a segment: per-model peaks by model then index, the ensemble record last
    assert [row[3] for row in g[:3]] == [0, 1, -1]       # model field
    assert [row[1] for row in g[:3]] == [30, 20, 10]     # index field


def test_gather_single_process_sorts():
    recs = np.zeros(4, dtype=TRIGGER_DTYPE)
    recs["index"] = [5, 1, 9, 2]
    recs["model"] = [1, -1, 0, 0]
    recs["slide"] = [0, 0, 0, 1]
    out = multi.gather_triggers(recs, np.array([2, 2, 2, 1]))
    assert list(out["segment"]) == [1, 2, 2, 2]
    assert list(out["model"]) == [0, 0, 1, -1]
