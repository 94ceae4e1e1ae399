"""Forward plans: many uneven science segments x many time-slide offsets
recorded into one CUDA graph, with the slide heads' launch shape chosen by the
autotuner.  A plan's output equals, bit for bit, gwe_forward_segments on the
same arguments, for the tuned shape and for every candidate shape; a refilled
input buffer is picked up by the next execution; a sampled slid window matches
the FP64 oracle within the tensor-core tolerance."""
import numpy as np
import pytest

import oracle
import workload
from gpu_util import require_gpu, sigmoid

pytestmark = pytest.mark.gpu

W, STRIDE = 4096, 2048


def _segments(rng, n_seg=6):
    # uneven lengths (lognormal around ~40 windows), one shorter than a window, gaps between segments
    lens = np.maximum(1000, (W + STRIDE * rng.lognormal(np.log(40.0), 0.6, n_seg)).astype(np.int64))
    lens[2] = 3000
    starts, pos = [], 0
    for ln in lens:
        pos += int(rng.integers(0, 3000))
        starts.append(pos)
        pos += int(ln)
    return np.array(starts, dtype=np.int64), lens, pos + 64


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_plan_equals_segments_forward(prec):
    import torch
    import paper_2201_11133_gb300 as gwe
    dev = require_gpu()
    rng = np.random.default_rng(7)
    cfg = workload.config("ensemble", n_models=2)
    starts, lens, n = _segments(rng)
    sh, sl, _ = workload.stream(n, seed=71, n_inj=5)
    wb = workload.init_weights(cfg, seed=3000, bias_std=0.05)
    m = gwe.Model(cfg, wb, gwe.GWE_BF16 if prec == "bf16" else gwe.GWE_FP8)
    th, tl = torch.from_numpy(sh).to(dev), torch.from_numpy(sl).to(dev)
    nws = gwe.segment_windows(lens, W, STRIDE)
    slides = [2 * (k + 1) for k in range(9)]            # 1 .. 9 s offsets
    shape = (len(slides), cfg["n_models"], int(nws.sum()), W)
    ref = torch.empty(shape, dtype=torch.float32, device=dev)
    gwe.gwe_forward_segments(m.handle, th, tl, starts, lens, W, STRIDE, slides, ref)
    m.sync()
    out = torch.full(shape, -1.0, dtype=torch.float32, device=dev)
    plan = gwe.gwe_plan_create(m.handle, th, tl, starts, lens, W, STRIDE, slides, out, gwe.GWE_PLAN_AUTOTUNE)
    try:
        info = gwe.gwe_plan_shape(plan)
        assert info["window_tile"] in (2, 4) and info["offset_tile"] in (4, 8)
        assert 1 <= info["pieces_per_block"] <= len(slides)
        assert info["n_kernels"] == 2 * cfg["n_models"]       # per model: branch pass + slide heads
        assert info["tuned_ms"] > 0 and info["tuned_ms"] <= info["default_ms"] * 1.0001
        gwe.gwe_plan_execute(plan)
        m.sync()
        assert torch.equal(out, ref)
        # the bound input buffers are read at every execution: refill them in place
        sh2, sl2, _ = workload.stream(n, seed=73, n_inj=5)
        th.copy_(torch.from_numpy(sh2))
        tl.copy_(torch.from_numpy(sl2))
        gwe.gwe_forward_segments(m.handle, th, tl, starts, lens, W, STRIDE, slides, ref)
        m.sync()
        out.fill_(-1.0)
        gwe.gwe_plan_execute(plan)
        gwe.gwe_plan_execute(plan)
        m.sync()
        assert torch.equal(out, ref)
    finally:
        gwe.gwe_plan_destroy(plan)
    if prec == "bf16":
        # one slid window of the longest segment against the FP64 oracle
        g = int(np.argmax(nws))
        w, si = int(nws[g]) - 3, 4                          # near the end: the Livingston window wraps
        k = slides[si]
        wl = (w + k) % int(nws[g])
        xh = sh2[None, starts[g] + w * STRIDE:starts[g] + w * STRIDE + W].astype(np.float64)
        xl = sl2[None, starts[g] + wl * STRIDE:starts[g] + wl * STRIDE + W].astype(np.float64)
        lg = oracle.forward_windows(cfg, wb[1], xh, xl)
        got = out[si, 1, int(nws[:g].sum()) + w].cpu().numpy().astype(np.float64)
        assert np.max(np.abs(got - sigmoid(lg[0]))) <= 1e-2


def test_every_candidate_shape_gives_the_same_output():
    """Every slide-head launch shape the autotuner chooses from computes the same sums in the same
    order: plans forced to each shape equal gwe_forward_segments bit for bit, on segments whose window
    tiles straddle the segment boundaries, with offsets in runs of step 1 and 2, gaps, negative
    offsets and offsets longer than a segment; then the oracle on the first segment's slid windows."""
    import torch
    import paper_2201_11133_gb300 as gwe
    dev = require_gpu()
    cfg = workload.config("small")
    Ws, Ss = 1024, 512
    lens = np.array([Ws + 30 * Ss, Ws + 7 * Ss + 100, Ws, Ws + 2 * Ss], dtype=np.int64)
    starts = np.array([0, int(lens[0]) + 50, int(lens[0] + lens[1]) + 99, int(lens[:3].sum()) + 200],
                      dtype=np.int64)
    n = int(starts[-1] + lens[-1])
    sh, sl, _ = workload.stream(n, seed=79)
    wb = workload.init_weights(cfg, seed=3000, bias_std=0.1)
    m = gwe.Model(cfg, wb, gwe.GWE_BF16)
    th, tl = torch.from_numpy(sh).to(dev), torch.from_numpy(sl).to(dev)
    nws = gwe.segment_windows(lens, Ws, Ss)
    slide_sets = [list(range(1, 14)), [2, 4, 6, 8, 10, 12, 14, 16, 18, 3, -5, 0, 40, 41]]
    for slides in slide_sets:
        shape = (len(slides), 1, int(nws.sum()), Ws)
        ref = torch.empty(shape, dtype=torch.float32, device=dev)
        gwe.gwe_forward_segments(m.handle, th, tl, starts, lens, Ws, Ss, slides, ref)
        m.sync()
        try:
            for a in (2, 4):
                for b in (4, 8):
                    for ppb in (0, 1, 3):
                        gwe.gwe_set_slide_shape(a, b, ppb)
                        out = torch.full(shape, -1.0, dtype=torch.float32, device=dev)
                        plan = gwe.gwe_plan_create(m.handle, th, tl, starts, lens, Ws, Ss, slides, out, 0)
                        try:
                            info = gwe.gwe_plan_shape(plan)
                            assert (info["window_tile"], info["offset_tile"]) == (a, b)
                            gwe.gwe_plan_execute(plan)
                            m.sync()
                            assert torch.equal(out, ref), (slides, a, b, ppb)
                        finally:
                            gwe.gwe_plan_destroy(plan)
        finally:
            gwe.gwe_set_slide_shape(4, 8, 0)
        # and the oracle on the whole batch of slid windows of the first segment, model 0
        ref_o = oracle.forward_stream(cfg, wb, sh[:lens[0]], sl[:lens[0]], Ws, Ss, slides=slides)
        got = ref[:, :, :int(nws[0])].cpu().numpy().astype(np.float64)
        assert np.max(np.abs(got - ref_o)) <= 1e-2
    # the tuned plan picks one of the candidates and gives the same output
    slides = slide_sets[1]
    shape = (len(slides), 1, int(nws.sum()), Ws)
    ref = torch.empty(shape, dtype=torch.float32, device=dev)
    gwe.gwe_forward_segments(m.handle, th, tl, starts, lens, Ws, Ss, slides, ref)
    out = torch.empty(shape, dtype=torch.float32, device=dev)
    plan = gwe.gwe_plan_create(m.handle, th, tl, starts, lens, Ws, Ss, slides, out, gwe.GWE_PLAN_AUTOTUNE)
    try:
        gwe.gwe_plan_execute(plan)
        m.sync()
        assert torch.equal(out, ref)
    finally:
        gwe.gwe_plan_destroy(plan)
    with pytest.raises(gwe.GweError):
        gwe.gwe_set_slide_shape(3, 4, 0)
    with pytest.raises(gwe.GweError):
        gwe.gwe_set_slide_shape(4, 5, 0)


def test_every_candidate_shape_ensemble_width():
    """The same for the 256-channel head (four warps per block, shared-memory reduction)."""
    import torch
    import paper_2201_11133_gb300 as gwe
    dev = require_gpu()
    cfg = workload.config("ensemble", n_models=1)
    lens = np.array([W + 21 * STRIDE, W + 2 * STRIDE + 7, W + 9 * STRIDE], dtype=np.int64)
    starts = np.array([0, int(lens[0]) + 10, int(lens[:2].sum()) + 20], dtype=np.int64)
    n = int(starts[-1] + lens[-1])
    sh, sl, _ = workload.stream(n, seed=80)
    wb = workload.init_weights(cfg, seed=3000, bias_std=0.05)
    m = gwe.Model(cfg, wb, gwe.GWE_BF16)
    th, tl = torch.from_numpy(sh).to(dev), torch.from_numpy(sl).to(dev)
    nws = gwe.segment_windows(lens, W, STRIDE)
    slides = [2 * (k + 1) for k in range(11)] + [1, -3, 30]
    shape = (len(slides), 1, int(nws.sum()), W)
    ref = torch.empty(shape, dtype=torch.float32, device=dev)
    gwe.gwe_forward_segments(m.handle, th, tl, starts, lens, W, STRIDE, slides, ref)
    m.sync()
    try:
        for a in (2, 4):
            for b in (4, 8):
                for ppb in (0, 2):
                    gwe.gwe_set_slide_shape(a, b, ppb)
                    out = torch.full(shape, -1.0, dtype=torch.float32, device=dev)
                    plan = gwe.gwe_plan_create(m.handle, th, tl, starts, lens, W, STRIDE, slides, out, 0)
                    try:
                        gwe.gwe_plan_execute(plan)
                        m.sync()
                        assert torch.equal(out, ref), (a, b, ppb)
                    finally:
                        gwe.gwe_plan_destroy(plan)
    finally:
        gwe.gwe_set_slide_shape(4, 8, 0)
    # a sampled slid window of the last segment against the oracle
    g, si = 2, 3
    w = int(nws[g]) - 1
    k = slides[si]
    wl = (w + k) % int(nws[g])
    s0 = int(starts[g])
    xh = sh[None, s0 + w * STRIDE:s0 + w * STRIDE + W].astype(np.float64)
    xl = sl[None, s0 + wl * STRIDE:s0 + wl * STRIDE + W].astype(np.float64)
    lg = oracle.forward_windows(cfg, wb[0], xh, xl)
    got = ref[si, 0, int(nws[:g].sum()) + w].cpu().numpy().astype(np.float64)
    assert np.max(np.abs(got - sigmoid(lg[0]))) <= 1e-2


def test_zero_lag_plan_and_bad_arguments():
    import torch
    import paper_2201_11133_gb300 as gwe
    dev = require_gpu()
    cfg = workload.config("small")
    Ws, Ss = 1024, 512
    n = Ws + 20 * Ss
    sh, sl, _ = workload.stream(n, seed=83)
    wb = workload.init_weights(cfg, seed=3000, bias_std=0.1)
    m = gwe.Model(cfg, wb, gwe.GWE_BF16)
    th, tl = torch.from_numpy(sh).to(dev), torch.from_numpy(sl).to(dev)
    nw = gwe.gwe_n_windows(n, Ws, Ss)
    out = torch.empty((1, 1, nw, Ws), dtype=torch.float32, device=dev)
    ref = m.forward(th, tl, Ws, Ss)
    plan = gwe.gwe_plan_create(m.handle, th, tl, [0], [n], Ws, Ss, None, out, gwe.GWE_PLAN_AUTOTUNE)
    try:
        assert gwe.gwe_plan_shape(plan)["n_kernels"] == 1
        gwe.gwe_plan_execute(plan)
        m.sync()
        assert torch.equal(out, ref)
    finally:
        gwe.gwe_plan_destroy(plan)
    with pytest.raises(gwe.GweError) as e:
        gwe.gwe_plan_create(m.handle, th, tl, [0], [100], Ws, Ss, None, out)    # no window
    assert e.value.status == 1
    m32 = gwe.Model(cfg, wb, gwe.GWE_FP32)
    with pytest.raises(gwe.GweError) as e:
        gwe.gwe_plan_create(m32.handle, th, tl, [0], [n], Ws, Ss, None, out)
    assert e.value.status == 5
