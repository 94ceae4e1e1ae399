"""Time shards of one stream across ranks (gloo, world size 2 and 3 on CPU):
each rank computes its core windows plus a margin of context (zero lag and
time slides, whose Livingston windows wrap at the end of the stream), finds
peaks and ensemble triggers on its span, keeps those in its core and gathers
them to rank 0, which must hold exactly the records of one process working on
the whole stream, except the records that multi.walks_leave_span flags (a
prominence walk that leaves the span's exact part: its base lies in another
shard), whose indices and heights must still match.  Probabilities come from the oracle (no GPU here); the
library's forward computes the same windows on a GPU."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
import workload
from paper_2201_11133_gb300 import multi, TRIGGER_DTYPE

W, STRIDE, NW, COINC, MW = 1024, 512, 30, 512, 0.0
OFFSETS = [0, 3, -5, 17]
CFG = workload.config("small", n_models=2)


def _records(per_model, ens, slides_first=0):
    rows = []
    for s, pm in enumerate(per_model):
        for m, (idx, h, pr, wd) in enumerate(pm):
            for i, hh, pp, ww in zip(idx, h, pr, wd):
                rows.append((int(i), s, m, float(hh), float(pp), float(ww)))
        info = {int(i): (hh, pp, ww) for i, hh, pp, ww in zip(*pm[0])}
        for i in ens[s]:
            hh, pp, ww = info[int(i)]
            rows.append((int(i), s, -1, float(hh), float(pp), float(ww)))
    return np.array(rows, dtype=TRIGGER_DTYPE)


def _inputs():
    n = W + (NW - 1) * STRIDE
    sh, sl, _ = workload.stream(n, seed=71)
    wb = workload.init_weights(CFG, seed=3100, bias_std=0.1)
    return sh, sl, wb


def _probs(sh, sl, wb, hw, lw_of):
    """[slides, models, len(hw), W] for Hanford windows hw, Livingston window lw_of(si, w)."""
    out = np.zeros((len(OFFSETS), CFG["n_models"], len(hw), W), dtype=np.float32)
    xh = np.stack([sh[w * STRIDE:w * STRIDE + W] for w in hw]).astype(np.float64)
    for si in range(len(OFFSETS)):
        xl = np.stack([sl[lw_of(si, w) * STRIDE:lw_of(si, w) * STRIDE + W] for w in hw]).astype(np.float64)
        for m in range(CFG["n_models"]):
            out[si, m] = 1.0 / (1.0 + np.exp(-oracle.forward_windows(CFG, wb[m], xh, xl, nthreads=2)))
    return out


def _shard_records(rank, world, margin):
    sh, sl, wb = _inputs()
    w0, w1 = multi.shard_windows(NW, world, rank)
    ws, we, s0, _ = multi.shard_span(NW, W, STRIDE, w0, w1, margin)
    need = multi.livingston_windows(NW, ws, we, OFFSETS)
    assert all(((w + k) % NW) in set(need.tolist()) for w in range(ws, we) for k in OFFSETS)
    p = _probs(sh, sl, wb, list(range(ws, we)), lambda si, w: (w + OFFSETS[si]) % NW)
    per_model, ens = oracle.triggers(p, W, STRIDE, 0.0, MW, COINC)
    g0, g1 = multi.core_series_range(NW, W, STRIDE, w0, w1)
    recs = _records(per_model, ens)
    # flag the records whose prominence walks leave the span's exact part (model-0's walk for ensembles)
    risky = np.zeros(len(recs), dtype=bool)
    exact_lo = (W - STRIDE) if ws > 0 else 0
    for si in range(len(OFFSETS)):
        for m in range(CFG["n_models"]):
            x = oracle.stitch(p[si, m], W, STRIDE)
            sel = (recs["slide"] == si) & ((recs["model"] == m) | ((recs["model"] == -1) & (m == 0)))
            risky[sel] = multi.walks_leave_span(x, recs["index"][sel], exact_lo, ws == 0, we == NW)
    kept = multi.keep_core(recs, s0, g0, g1)
    kept_risky = risky[(recs["index"] + s0 >= g0) & (recs["index"] + s0 < g1)]
    return kept, kept_risky


def _whole_stream_records():
    sh, sl, wb = _inputs()
    p = _probs(sh, sl, wb, list(range(NW)), lambda si, w: (w + OFFSETS[si]) % NW)
    per_model, ens = oracle.triggers(p, W, STRIDE, 0.0, MW, COINC)
    return multi.gather_shard_triggers(_records(per_model, ens))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, margin, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        recs, risky = _shard_records(rank, world, margin)
        out = multi.gather_shard_triggers(recs, dist)
        flagged = multi.gather_shard_triggers(recs[risky], dist)
        q.put((rank, None if out is None else (out.tolist(), flagged.tolist())))
    finally:
        dist.destroy_process_group()


def test_shard_plan_partitions_the_series():
    for world in (1, 2, 3, 7):
        cores = [multi.shard_windows(NW, world, r) for r in range(world)]
        assert cores[0][0] == 0 and cores[-1][1] == NW
        assert all(a[1] == b[0] for a, b in zip(cores, cores[1:]))
        ranges = [multi.core_series_range(NW, W, STRIDE, *c) for c in cores]
        assert ranges[0][0] == 0 and ranges[-1][1] == W + (NW - 1) * STRIDE
        assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))
    ws, we, s0, s1 = multi.shard_span(NW, W, STRIDE, 10, 20, 4)
    assert (ws, we, s0, s1) == (6, 24, 6 * STRIDE, 23 * STRIDE + W)
    # wrap at the end of the stream
    assert list(multi.livingston_windows(NW, NW - 2, NW, [1, 2])) == [0, 1, NW - 1]
    x = np.array([0.0, 3.0, 1.0, 2.0, 0.5, 5.0, 1.0, 4.0, 0.0])
    # peaks 1 (3.0), 3 (2.0), 5 (5.0), 7 (4.0): 5 is the span maximum (both walks leave), 7's right
    # walk leaves (nothing higher to its right), 1's left walk leaves unless the span starts the stream
    got = multi.walks_leave_span(x, [1, 3, 5, 7], 0, False, False)
    assert list(got) == [True, False, True, True]
    assert list(multi.walks_leave_span(x, [1, 3, 5, 7], 0, True, True)) == [False, False, False, False]


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_time_shards_equal_one_process(world):
    ref = _whole_stream_records()
    assert len(ref) > 0 and np.any(ref["model"] == -1)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, 6, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert all(res[r] is None for r in range(1, world))
    got = np.array([tuple(r) for r in res[0][0]], dtype=TRIGGER_DTYPE)
    flagged = np.array([tuple(r) for r in res[0][1]], dtype=TRIGGER_DTYPE)
    assert len(got) == len(ref)
    for f in ("index", "slide", "model", "height"):
        np.testing.assert_array_equal(got[f], ref[f])
    key = lambda a: set(zip(a["index"].tolist(), a["slide"].tolist(), a["model"].tolist()))
    bad = key(flagged)
    ok = np.array([k not in bad for k in zip(got["index"].tolist(), got["slide"].tolist(), got["model"].tolist())])
    np.testing.assert_array_equal(got["prominence"][ok], ref["prominence"][ok])
    # widths are differences of interpolated absolute positions: a span's index origin changes their
    # FP64 rounding at the 1e-12 level
    np.testing.assert_allclose(got["width"][ok], ref["width"][ok], rtol=1e-9, atol=0)
    assert len(bad) <= 0.002 * len(got)                 # a handful of span-wide maxima
    print(f"world {world}: {len(got)} records equal to one process; {len(bad)} flagged (walks leave the span)")
