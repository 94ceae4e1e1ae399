"""Streaming search (gwe_search_run): a long raw stream cut into chunks, each
whitened on its own span, run through the ensemble and searched for triggers in
its core.  Every chunk equals, record for record, the library's single calls on
that span (gwe_whiten -> gwe_forward -> gwe_triggers, cut to the core), for FP16
and FP32 input, from device and from pinned host memory; the cores partition the
stream; and the ensemble triggers of a small stream agree with the FP64 oracle
run through the same chunking (every solid ensemble trigger recalled)."""
import numpy as np
import pytest

import oracle
import workload
from gpu_util import require_gpu

pytestmark = pytest.mark.gpu

FS = 4096


def _chunks(n, W, S, K, M, G):
    nw = (n - W) // S + 1
    out = []
    for i in range((nw + K - 1) // K):
        wa, wb = i * K, min(nw, i * K + K)
        wlo, whi = max(0, wa - M), min(nw, wb + M)
        xa, xb = max(0, wlo * S - G), min(n, (whi - 1) * S + W + G)
        out.append((wa, wb, wlo, whi, xa, xb))
    return nw, out


def _reference(gwe, m, xH, xL, n, W, S, K, M, G, seg, thr, minw, coinc, flags):
    import torch
    nw, chunks = _chunks(n, W, S, K, M, G)
    n_st = (nw - 1) * S + W
    recs = []
    for wa, wb, wlo, whi, xa, xb in chunks:
        span = xb - xa
        wh = torch.empty(span, dtype=torch.float32, device=xH.device)
        wl = torch.empty_like(wh)
        gwe.gwe_whiten(xH[xa:xb].contiguous(), span, float(FS), seg, wh)
        gwe.gwe_whiten(xL[xa:xb].contiguous(), span, float(FS), seg, wl)
        nws = whi - wlo
        off = wlo * S - xa
        ln = (nws - 1) * S + W
        p = m.forward(wh[off:off + ln], wl[off:off + ln], W, S)
        r = gwe.gwe_triggers(p, m.cfg["n_models"], 1, nws, W, S, thr, minw, coinc, flags=flags)
        r = r.copy()
        r["index"] += wlo * S
        ca = 0 if wa == 0 else wa * S + W - S
        cb = n_st if wb == nw else wb * S + W - S
        recs.append(r[(r["index"] >= ca) & (r["index"] < cb)])
    return np.concatenate(recs)


@pytest.mark.parametrize("dtype,host", [("f16", False), ("f32", True), ("f16", True)])
def test_search_equals_per_chunk_calls(dtype, host, tmp_path):
    import torch
    import paper_2201_11133_gb300 as gwe
    dev = require_gpu()
    cfg = workload.config("ensemble", n_models=2)
    W, S, K, M, G, seg = 4096, 2048, 23, 5, 8192, 16384
    n = 101 * S + W + 1234                        # 102 windows: five chunks, the last one short
    sh, sl, _ = workload.coloured_stream(n, seed=91, n_inj=6)
    wb = workload.init_weights(cfg, seed=3000, bias_std=0.05)
    m = gwe.Model(cfg, wb, gwe.GWE_BF16)
    tdt = torch.float16 if dtype == "f16" else torch.float32
    hH = torch.from_numpy(sh).to(tdt)
    hL = torch.from_numpy(sl).to(tdt)
    # the reference sees exactly the FP32 values the search converts to
    xH = hH.float().to(dev)
    xL = hL.float().to(dev)
    flags = gwe.GWE_TRIG_PER_MODEL
    # threshold from the data so that records exist
    wh = torch.empty(n, dtype=torch.float32, device=dev)
    wl = torch.empty_like(wh)
    gwe.gwe_whiten(xH, n, float(FS), seg, wh)
    gwe.gwe_whiten(xL, n, float(FS), seg, wl)
    p = m.forward(wh, wl, W, S)
    thr = float(torch.quantile(p[0, 0, :, ::31].reshape(-1), 0.7).item())
    ref = _reference(gwe, m, xH, xL, n, W, S, K, M, G, seg, thr, 0.0, 2048, flags)
    assert len(ref) > 10 and np.sum(ref["model"] == -1) > 0
    sr = gwe.gwe_search_create(m.handle, window=W, stride=S, chunk_windows=K, margin_windows=M, guard_samples=G,
                               fs=float(FS), welch_seg=seg,
                               input_dtype=gwe.GWE_INPUT_F16 if dtype == "f16" else gwe.GWE_INPUT_F32,
                               input_scale=1.0, height_thr=thr, min_width=0.0, coinc=2048, trigger_flags=flags)
    try:
        if host:
            iH, iL = hH.pin_memory(), hL.pin_memory()
        else:
            iH, iL = hH.to(dev), hL.to(dev)
        got = gwe.gwe_search_run(sr, iH, iL, n)
        assert len(got) == len(ref)
        for f in ("index", "slide", "model", "height", "prominence", "width"):
            np.testing.assert_array_equal(got[f], ref[f])
        # a second run on the same handle gives the same records
        got2 = gwe.gwe_search_run(sr, iH, iL, n)
        np.testing.assert_array_equal(got2, got)
        # chunk ranges concatenate to the whole run; a checkpointed run stopped after one range and
        # resumed from its checkpoint gives the same records
        assert gwe.gwe_search_chunks(sr, n) == 5
        parts = [gwe.gwe_search_run_range(sr, iH, iL, n, a, b) for a, b in ((0, 2), (2, 3), (3, 99))]
        np.testing.assert_array_equal(np.concatenate(parts), got)
        ck = str(tmp_path / "search_checkpoint.npz")
        first = gwe.gwe_search_resumable(sr, iH, iL, n, ck, chunks_per_step=2, max_steps=1)
        np.testing.assert_array_equal(first, np.concatenate(parts[:1]))
        rest = gwe.gwe_search_resumable(sr, iH, iL, n, ck, chunks_per_step=2)
        np.testing.assert_array_equal(rest, got)
        with pytest.raises(gwe.GweError) as e:
            gwe.gwe_search_run_range(sr, iH, iL, n, 3, 2)
        assert e.value.status == 1
        with pytest.raises(gwe.GweError) as e:
            gwe.gwe_search_run(sr, iH, iL, n, cap=1)
        assert e.value.status == 6
    finally:
        gwe.gwe_search_destroy(sr)


def test_search_cores_partition_and_arguments():
    import torch
    import paper_2201_11133_gb300 as gwe
    require_gpu()
    W, S = 4096, 2048
    for n, K, M in ((57 * S + W, 10, 3), (9 * S + W + 5, 4, 0), (W, 7, 2)):
        nw, chunks = _chunks(n, W, S, K, M, 4096)
        n_st = (nw - 1) * S + W
        cover = np.zeros(n_st, dtype=np.int32)
        for wa, wb, wlo, whi, xa, xb in chunks:
            ca = 0 if wa == 0 else wa * S + W - S
            cb = n_st if wb == nw else wb * S + W - S
            cover[ca:cb] += 1
            assert wlo <= wa < wb <= whi and xa <= wlo * S and (whi - 1) * S + W <= xb <= n
        assert np.all(cover == 1)
    cfg = workload.config("small")
    m = gwe.Model(cfg, workload.init_weights(cfg, seed=3000), gwe.GWE_BF16)
    with pytest.raises(gwe.GweError) as e:
        gwe.gwe_search_create(m.handle, chunk_windows=0)
    assert e.value.status == 1
    with pytest.raises(gwe.GweError) as e:
        gwe.gwe_search_create(m.handle, welch_seg=1000)
    assert e.value.status == 1
    sr = gwe.gwe_search_create(m.handle, window=1024, stride=512, chunk_windows=4, margin_windows=0, guard_samples=0,
                               welch_seg=4096)
    try:
        x = torch.zeros(1024 + 3 * 512, dtype=torch.float32, device="cuda")
        with pytest.raises(gwe.GweError) as e:          # span shorter than the Welch segment
            gwe.gwe_search_run(sr, x, x, x.numel())
        assert e.value.status == 1
        assert len(gwe.gwe_search_run(sr, x[:100], x[:100], 100)) == 0   # no window at all
    finally:
        gwe.gwe_search_destroy(sr)


def test_search_triggers_agree_with_oracle():
    """The small model on a short stream, two chunks: the oracle whitens each span (FP64), runs the
    network (FP64) and finds peaks and ensemble triggers on the span's stitched series; every solid
    oracle ensemble trigger is recalled by the device search within 256 samples."""
    import torch
    import paper_2201_11133_gb300 as gwe
    from oracle import whiten as ow
    dev = require_gpu()
    cfg = workload.config("small", n_models=2)
    W, S, K, M, G, seg = 1024, 512, 24, 4, 4096, 4096
    n = 47 * S + W
    sh, sl, _ = workload.coloured_stream(n, seed=97, n_inj=2)
    wb = workload.init_weights(cfg, seed=3000, bias_std=0.1)
    m = gwe.Model(cfg, wb, gwe.GWE_BF16)
    nw, chunks = _chunks(n, W, S, K, M, G)
    n_st = (nw - 1) * S + W
    # oracle: per chunk span
    probs = []
    for wa, wb_, wlo, whi, xa, xb in chunks:
        h = ow.whiten(sh[xa:xb].astype(np.float64), float(FS), seg)
        l_ = ow.whiten(sl[xa:xb].astype(np.float64), float(FS), seg)
        off = wlo * S - xa
        ln = (whi - wlo - 1) * S + W
        probs.append(oracle.forward_stream(cfg, wb, h[off:off + ln], l_[off:off + ln], W, S)[0])
    thr = float(np.quantile(np.concatenate([p.reshape(2, -1) for p in probs], axis=1)[0], 0.6))
    want = []
    for (wa, wb_, wlo, whi, xa, xb), p in zip(chunks, probs):
        per_model, ens = oracle.triggers(p[None].astype(np.float32), W, S, thr, 0.0, 2048)
        idx0, h0, pr0, _ = per_model[0][0]
        info = {int(i): (hh, pp) for i, hh, pp in zip(idx0, h0, pr0)}
        # solid triggers only: prominence >= 0.05 and height farther than the tolerance from thr
        idx = np.array([int(i) for i in ens[0] if info[int(i)][1] >= 0.05 and abs(info[int(i)][0] - thr) > 1e-2],
                       dtype=np.int64) + wlo * S
        ca = 0 if wa == 0 else wa * S + W - S
        cb = n_st if wb_ == nw else wb_ * S + W - S
        want.append(idx[(idx >= ca) & (idx < cb)])
    want = np.concatenate(want)
    sr = gwe.gwe_search_create(m.handle, window=W, stride=S, chunk_windows=K, margin_windows=M, guard_samples=G,
                               fs=float(FS), welch_seg=seg, height_thr=thr, min_width=0.0, coinc=2048)
    try:
        got = gwe.gwe_search_run(sr, torch.from_numpy(sh).to(dev), torch.from_numpy(sl).to(dev), n)
    finally:
        gwe.gwe_search_destroy(sr)
    gi = np.sort(got[got["model"] == -1]["index"])
    assert len(want) > 3
    hit = [np.min(np.abs(gi - i)) <= 256 if len(gi) else False for i in want]
    assert np.mean(hit) >= 0.999, (np.mean(hit), len(want), len(gi))
