"""Parity of the tensor-core (BF16/FP16 operands, FP32 accumulation) forward
path with the FP64 oracle, through the C-ABI.  Tolerance: max |dprob| <= 1e-2."""
import numpy as np
import pytest

import oracle
import workload
from gpu_util import require_gpu, sigmoid

pytestmark = pytest.mark.gpu

TOL_BF16 = 1e-2


def _model(cfg, wb):
    import paper_2201_11133_gb300 as gwe
    return gwe.Model(cfg, wb, gwe.GWE_BF16)


def test_bf16_small_batch_of_8_windows():
    import torch
    dev = require_gpu()
    cfg = workload.config("small")
    xh, xl, _ = workload.small_batch(seed=1000)
    wb = workload.init_weights(cfg, seed=3000, bias_std=0.1)
    ref = oracle.forward_windows(cfg, wb[0], xh, xl)
    m = _model(cfg, wb)
    lg = m.logits(torch.from_numpy(xh).to(dev), torch.from_numpy(xl).to(dev))
    m.sync()
    got = lg.cpu().numpy()[0].astype(np.float64)
    err = np.max(np.abs(sigmoid(got) - sigmoid(ref)))
    print("bf16 small max|dprob|", err)
    assert err <= TOL_BF16


@pytest.mark.parametrize("slides", [None, [0, 3, -1]])
def test_bf16_stream_windows_slides_ragged_tail(slides):
    import torch
    dev = require_gpu()
    cfg = workload.config("small", n_models=2)
    W, stride = 1024, 512
    n = W + 6 * stride + 300
    sh, sl, _ = workload.stream(n, seed=23)
    wb = workload.init_weights(cfg, seed=3200, bias_std=0.1)
    ref = oracle.forward_stream(cfg, wb, sh, sl, W, stride, slides=slides)
    m = _model(cfg, wb)
    out = m.forward(torch.from_numpy(sh).to(dev), torch.from_numpy(sl).to(dev), W, stride, slides=slides)
    m.sync()
    err = np.max(np.abs(out.cpu().numpy() - ref))
    print("bf16 stream max|dprob|", err)
    assert err <= TOL_BF16


# n16: layers taking FP16 conv operands (None: the handle's default, the first third); with every
# layer in FP16 the error drops to the FP16 format's (~1.6e-3 on windows of this model), which checks
# the FP16 staging, lag-ring and descriptor path on its own
@pytest.mark.parametrize("n16,tol", [(None, TOL_BF16), (0, TOL_BF16), (30, 3e-3)])
def test_bf16_thirty_layer_ensemble(n16, tol):
    import torch
    import paper_2201_11133_gb300 as gwe
    dev = require_gpu()
    cfg = workload.config("ensemble")
    W, stride = 4096, 2048
    n = W + stride + 5
    sh, sl, _ = workload.stream(n, seed=31)
    wb = workload.init_weights(cfg, seed=3000, bias_std=0.05)
    ref = oracle.forward_stream(cfg, wb, sh, sl, W, stride)
    m = _model(cfg, wb)
    assert gwe.gwe_model_f16_layers(m.handle) == 10
    if n16 is not None:
        gwe.gwe_model_set_f16_layers(m.handle, n16)
        assert gwe.gwe_model_f16_layers(m.handle) == n16
    out = m.forward(torch.from_numpy(sh).to(dev), torch.from_numpy(sl).to(dev), W, stride)
    m.sync()
    err = np.max(np.abs(out.cpu().numpy() - ref))
    print(f"bf16 30-layer (n16={n16}) max|dprob| {err:.3e}")
    assert err <= tol


def test_bf16_ensemble_time_slides():
    """64-slide style background: branches once per window, slide heads on the projections."""
    import torch
    dev = require_gpu()
    cfg = workload.config("ensemble")
    W, stride = 1024, 512
    n = W + 5 * stride + 17
    sh, sl, _ = workload.stream(n, seed=37)
    wb = workload.init_weights(cfg, seed=3000, bias_std=0.05)
    slides = [1, 2, 5, -3, 0]
    ref = oracle.forward_stream(cfg, wb, sh, sl, W, stride, slides=slides)
    m = _model(cfg, wb)
    out = m.forward(torch.from_numpy(sh).to(dev), torch.from_numpy(sl).to(dev), W, stride, slides=slides)
    m.sync()
    err = np.max(np.abs(out.cpu().numpy() - ref))
    print("bf16 30-layer slides max|dprob|", err)
    assert err <= TOL_BF16
    # the zero-lag slide equals the plain forward
    z = m.forward(torch.from_numpy(sh).to(dev), torch.from_numpy(sl).to(dev), W, stride)
    m.sync()
    assert np.max(np.abs(out[4].cpu().numpy() - z[0].cpu().numpy())) <= 2e-3
