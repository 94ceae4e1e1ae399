"""Batched science segments of uneven length (one launch over all segments):
equal, bit for bit, to one gwe_forward per segment; triggers per segment equal
gwe_triggers on each segment's output.  Segment lengths include one shorter than
a window and one of exactly one window."""
import numpy as np
import pytest

import oracle
import workload
from gpu_util import require_gpu

pytestmark = pytest.mark.gpu

W, STRIDE = 4096, 2048


def _segments():
    lens = [3000, W + 39 * STRIDE + 1000, W, W + 22 * STRIDE, W + 64 * STRIDE + 77]
    gaps = [500, 1234, 0, 4096, 17]
    starts, pos = [], 0
    for ln, gp in zip(lens, gaps):
        pos += gp
        starts.append(pos)
        pos += ln
    return np.array(starts, dtype=np.int64), np.array(lens, dtype=np.int64), pos + 100


def _per_segment(m, th, tl, starts, lens, slides):
    import torch
    outs = []
    for s0, ln in zip(starts, lens):
        if ln < W:
            continue
        outs.append(m.forward(th[s0:s0 + ln], tl[s0:s0 + ln], W, STRIDE, slides=slides))
    m.sync()
    return torch.cat(outs, dim=2)


@pytest.mark.parametrize("prec", ["bf16", "fp8", "fp32"])
@pytest.mark.parametrize("slides", [None, [1, -2, 5]])
def test_segments_equal_per_segment_calls(prec, slides):
    import torch
    import paper_2201_11133_gb300 as gwe
    dev = require_gpu()
    cfg = workload.config("ensemble")
    starts, lens, n = _segments()
    sh, sl, _ = workload.stream(n, seed=61, n_inj=4)
    wb = workload.init_weights(cfg, seed=3000, bias_std=0.05)
    code = {"bf16": gwe.GWE_BF16, "fp8": gwe.GWE_FP8, "fp32": gwe.GWE_FP32}[prec]
    m = gwe.Model(cfg, wb, code)
    th, tl = torch.from_numpy(sh).to(dev), torch.from_numpy(sl).to(dev)
    nws = gwe.segment_windows(lens, W, STRIDE)
    ns = 1 if slides is None else len(slides)
    out = torch.empty((ns, cfg["n_models"], int(nws.sum()), W), dtype=torch.float32, device=dev)
    gwe.gwe_forward_segments(m.handle, th, tl, starts, lens, W, STRIDE, slides, out)
    m.sync()
    ref = _per_segment(m, th, tl, starts, lens, slides)
    assert out.shape == ref.shape
    assert torch.equal(out, ref)
    if prec == "bf16" and slides is None:
        # one window of the last segment against the oracle
        g, w = 4, 50
        x0 = starts[g] + w * STRIDE
        lg = oracle.forward_windows(cfg, wb[1], sh[None, x0:x0 + W].astype(np.float64),
                                    sl[None, x0:x0 + W].astype(np.float64))
        got = out[0, 1, int(nws[:g].sum()) + w].cpu().numpy().astype(np.float64)
        assert np.max(np.abs(got - 1.0 / (1.0 + np.exp(-lg[0])))) <= 1e-2


def test_segment_triggers_equal_per_segment_triggers():
    import torch
    import paper_2201_11133_gb300 as gwe
    dev = require_gpu()
    cfg = workload.config("ensemble", n_models=2)
    starts, lens, n = _segments()
    sh, sl, _ = workload.stream(n, seed=67, n_inj=6)
    wb = workload.init_weights(cfg, seed=3000, bias_std=0.05)
    m = gwe.Model(cfg, wb, gwe.GWE_BF16)
    th, tl = torch.from_numpy(sh).to(dev), torch.from_numpy(sl).to(dev)
    nws = gwe.segment_windows(lens, W, STRIDE)
    slides = [0, 3]
    out = torch.empty((2, 2, int(nws.sum()), W), dtype=torch.float32, device=dev)
    gwe.gwe_forward_segments(m.handle, th, tl, starts, lens, W, STRIDE, slides, out)
    m.sync()
    thr = float(torch.quantile(out[0, 0, :, ::53].reshape(-1), 0.6).item())
    recs, segs = gwe.gwe_triggers_segments(out, 2, 2, lens, W, STRIDE, thr, 0.0, 2048)
    assert len(recs) > 0
    wo = 0
    got_any = 0
    for g, nw in enumerate(nws):
        if nw == 0:
            assert np.sum(segs == g) == 0
            continue
        sub = out[:, :, wo:wo + nw].contiguous()
        want = gwe.gwe_triggers(sub, 2, 2, int(nw), W, STRIDE, thr, 0.0, 2048)
        mine = recs[segs == g]
        assert len(mine) == len(want)
        for f in ("index", "slide", "model", "height", "prominence", "width"):
            np.testing.assert_array_equal(mine[f], want[f])
        got_any += len(mine)
        wo += int(nw)
    assert got_any == len(recs)
