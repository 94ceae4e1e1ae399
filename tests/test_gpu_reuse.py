"""Cross-window reuse of the tensor-core forward is exact: with it on, every
output bit equals the run that computes every window in full (and that run is
the one the oracle parity tests check).  Enough windows per model that each
persistent CTA takes several consecutive windows."""
import numpy as np
import pytest

import oracle
import workload
from gpu_util import require_gpu

pytestmark = pytest.mark.gpu


def _run(m, th, tl, W, stride, slides, reuse):
    import paper_2201_11133_gb300 as gwe
    gwe.gwe_set_cross_window_reuse(reuse)
    try:
        out = m.forward(th, tl, W, stride, slides=slides)
        m.sync()
    finally:
        gwe.gwe_set_cross_window_reuse(True)
    return out


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
@pytest.mark.parametrize("stride,slides", [(2048, None), (3072, None), (2048, [1, -3])])
def test_reuse_bit_exact_ensemble(prec, stride, slides):
    import torch
    import paper_2201_11133_gb300 as gwe
    dev = require_gpu()
    cfg = workload.config("ensemble")
    W = 4096
    n = W + 95 * stride + 77            # 96 windows x 4 models: more jobs than CTAs
    sh, sl, _ = workload.stream(n, seed=51, n_inj=3)
    wb = workload.init_weights(cfg, seed=3000, bias_std=0.05)
    m = gwe.Model(cfg, wb, gwe.GWE_BF16 if prec == "bf16" else gwe.GWE_FP8)
    th, tl = torch.from_numpy(sh).to(dev), torch.from_numpy(sl).to(dev)
    a = _run(m, th, tl, W, stride, slides, True)
    b = _run(m, th, tl, W, stride, slides, False)
    assert torch.equal(a, b)
    # and a sampled window against the oracle (the full-computation path's parity)
    if prec == "bf16" and slides is None:
        w = 57
        ref = oracle.forward_windows(cfg, wb[2], sh[None, w * stride:w * stride + W].astype(np.float64),
                                     sl[None, w * stride:w * stride + W].astype(np.float64))
        got = a[0, 2, w].cpu().numpy().astype(np.float64)
        assert np.max(np.abs(got - 1.0 / (1.0 + np.exp(-ref[0])))) <= 1e-2


def test_reuse_bit_exact_small_model_short_windows():
    import torch
    import paper_2201_11133_gb300 as gwe
    dev = require_gpu()
    cfg = workload.config("small", n_models=2)
    W, stride = 1024, 512
    n = W + 399 * stride                # 400 windows x 2 models
    sh, sl, _ = workload.stream(n, seed=53)
    wb = workload.init_weights(cfg, seed=3200, bias_std=0.1)
    m = gwe.Model(cfg, wb, gwe.GWE_BF16)
    th, tl = torch.from_numpy(sh).to(dev), torch.from_numpy(sl).to(dev)
    a = _run(m, th, tl, W, stride, None, True)
    b = _run(m, th, tl, W, stride, None, False)
    assert torch.equal(a, b)
