"""Parity of the FP32 CUDA forward path with the FP64 oracle (tolerance: max
|dprob| <= 1e-5), through the C-ABI."""
import numpy as np
import pytest

import oracle
import workload
from gpu_util import require_gpu, sigmoid

pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-5


def _model(cfg, wb, prec):
    import paper_2201_11133_gb300 as gwe
    return gwe.Model(cfg, wb, prec)


def test_fp32_small_batch_of_8_windows():
    """8 layers, R = S = Hc = 32, batch of 8 one-second windows, two with a chirp."""
    import torch
    import paper_2201_11133_gb300 as gwe
    dev = require_gpu()
    cfg = workload.config("small")
    xh, xl, meta = workload.small_batch(seed=1000)
    assert len(meta) == 2
    wb = workload.init_weights(cfg, seed=3000, bias_std=0.1)
    ref = oracle.forward_windows(cfg, wb[0], xh, xl)
    m = _model(cfg, wb, gwe.GWE_FP32)
    lg = m.logits(torch.from_numpy(xh).to(dev), torch.from_numpy(xl).to(dev))
    torch.cuda.synchronize()
    got = lg.cpu().numpy()[0].astype(np.float64)
    assert np.max(np.abs(sigmoid(got) - sigmoid(ref))) <= TOL_FP32
    assert np.max(np.abs(got - ref)) <= 1e-3 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("slides", [None, [0, 2, 5, -1]])
def test_fp32_stream_windows_slides_ragged_tail(slides):
    import torch
    import paper_2201_11133_gb300 as gwe
    dev = require_gpu()
    cfg = workload.config("small", n_models=2)
    W, stride = 4096, 2048
    n = W + 4 * stride + 777          # ragged tail is dropped
    sh, sl, _ = workload.stream(n, seed=21)
    wb = workload.init_weights(cfg, seed=3100, bias_std=0.1)
    ref = oracle.forward_stream(cfg, wb, sh, sl, W, stride, slides=slides)
    m = _model(cfg, wb, gwe.GWE_FP32)
    out = m.forward(torch.from_numpy(sh).to(dev), torch.from_numpy(sl).to(dev), W, stride, slides=slides)
    torch.cuda.synchronize()
    assert out.shape == ref.shape
    assert np.max(np.abs(out.cpu().numpy() - ref)) <= TOL_FP32


def test_fp32_thirty_layer_ensemble():
    """4 models x 3 stacks of dilations 1..512, R = 64, S = 128, Hc = 256, two windows."""
    import torch
    import paper_2201_11133_gb300 as gwe
    dev = require_gpu()
    cfg = workload.config("ensemble")
    W, stride = 4096, 2048
    n = W + stride + 5
    sh, sl, _ = workload.stream(n, seed=31)
    wb = workload.init_weights(cfg, seed=3000, bias_std=0.05)
    ref = oracle.forward_stream(cfg, wb, sh, sl, W, stride)
    m = _model(cfg, wb, gwe.GWE_FP32)
    out = m.forward(torch.from_numpy(sh).to(dev), torch.from_numpy(sl).to(dev), W, stride)
    torch.cuda.synchronize()
    assert np.max(np.abs(out.cpu().numpy() - ref)) <= TOL_FP32


def test_forward_argument_errors():
    import torch
    import paper_2201_11133_gb300 as gwe
    dev = require_gpu()
    cfg = workload.config("small")
    wb = workload.init_weights(cfg, seed=1)
    m = _model(cfg, wb, gwe.GWE_FP32)
    x = torch.zeros(100, device=dev)
    out = torch.zeros(4096, device=dev)
    with pytest.raises(gwe.GweError) as ei:
        gwe.gwe_forward(m.handle, x, x, 100, 4096, 2048, None, out)
    assert ei.value.status == 1
    with pytest.raises(gwe.GweError) as ei:
        gwe.gwe_forward(m.handle, x, x, 100, 64, 0, None, out)
    assert ei.value.status == 1
    with pytest.raises(gwe.GweError) as ei:
        c3 = dict(cfg, kernel=3)
        gwe.gwe_model_create(c3, np.zeros(gwe.gwe_param_count(c3), np.float32))
    assert ei.value.status in (1, 5)
