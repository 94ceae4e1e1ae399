"""Weights replaced from device memory (gwe_model_set_weights_device) and the
autograd wrapper that uses it.

The device packers must build exactly the images the host builders build:
a handle whose weights were replaced on the device gives bit-identical
forward outputs to one given the same weights from the host, for the FP32,
the 16-bit tensor-core and the FP8 paths, and the same gradients.  The
autograd wrapper must give each backward the weights of its own forward, also
when another forward with other weights ran on the handle in between."""
import numpy as np
import pytest

import workload
from gpu_util import require_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,prec", [("small", 0), ("small", 1), ("ensemble", 1), ("ensemble", 2), ("ensemble", 0)])
def test_device_weights_equal_host_weights(name, prec):
    import torch
    import paper_2201_11133_gb300 as gwe
    dev = require_gpu()
    cfg = workload.config(name, n_models=2)
    w1 = workload.init_weights(cfg, seed=5100, bias_std=0.05)
    w2 = workload.init_weights(cfg, seed=5200, bias_std=0.05)
    W, stride = 1024, 512
    n = W + 4 * stride + 9
    sh, sl, _ = workload.stream(n, seed=52)
    H, L = torch.from_numpy(sh).to(dev), torch.from_numpy(sl).to(dev)
    a = gwe.Model(cfg, w1, prec)
    b = gwe.Model(cfg, w1, prec)
    a.set_weights_device(torch.from_numpy(w2).to(dev))
    b.set_weights(w2)
    oa = a.forward(H, L, W, stride, slides=[0, 2])
    ob = b.forward(H, L, W, stride, slides=[0, 2])
    a.sync()
    b.sync()
    assert torch.equal(oa, ob)
    if prec == 1:
        # a fresh handle built from w2 on the host: the same images
        c = gwe.Model(cfg, w2, prec)
        oc = c.forward(H, L, W, stride, slides=[0, 2])
        c.sync()
        assert torch.equal(oa, oc)
        c.close()
    if prec != 2:
        # gradients: the backward's images come from the same device blob
        B = 2
        xh = torch.from_numpy(np.stack([sh[:W], sh[stride:stride + W]])).to(dev)
        xl = torch.from_numpy(np.stack([sl[:W], sl[stride:stride + W]])).to(dev)
        dl = torch.from_numpy(np.random.default_rng(3).standard_normal((B, W)).astype(np.float32)).to(dev)
        P = gwe.gwe_param_count(cfg)
        ga = torch.empty(P, device=dev)
        gb = torch.empty(P, device=dev)
        gwe.gwe_backward(a.handle, 1, xh, xl, B, W, dl, ga)
        gwe.gwe_backward(b.handle, 1, xh, xl, B, W, dl, gb)
        a.sync()
        b.sync()
        # weight gradients are summed with atomics (order not fixed)
        ref = gb.abs().max().item()
        assert (ga - gb).abs().max().item() <= 1e-5 * ref
    a.close()
    b.close()


def test_autograd_interleaved_forwards_keep_their_weights():
    import torch
    import paper_2201_11133_gb300 as gwe
    dev = require_gpu()
    cfg = workload.config("small", n_models=1)
    W = 512
    xh, xl, _ = workload.small_batch(seed=1001, B=2, W=W, chirp_windows=())
    x_H, x_L = torch.from_numpy(xh).to(dev), torch.from_numpy(xl).to(dev)
    wa = torch.from_numpy(workload.init_weights(cfg, seed=5300, bias_std=0.05)[0]).to(dev).requires_grad_(True)
    wb = torch.from_numpy(workload.init_weights(cfg, seed=5400, bias_std=0.05)[0]).to(dev).requires_grad_(True)
    m = gwe.Model(cfg, workload.init_weights(cfg, seed=1)[0:1], gwe.GWE_BF16)
    # reference: each forward immediately followed by its backward
    ref = []
    for w in (wa, wb):
        y = gwe.gwe_logits_autograd(m, w, x_H, x_L)
        (g,) = torch.autograd.grad((y * y).mean(), [w])
        ref.append(g.clone())
    # interleaved: both forwards, then both backwards
    ya = gwe.gwe_logits_autograd(m, wa, x_H, x_L)
    yb = gwe.gwe_logits_autograd(m, wb, x_H, x_L)
    (gb,) = torch.autograd.grad((yb * yb).mean(), [wb])
    (ga,) = torch.autograd.grad((ya * ya).mean(), [wa])
    torch.cuda.synchronize()
    for got, r in ((ga, ref[0]), (gb, ref[1])):
        assert (got - r).abs().max().item() <= 1e-5 * r.abs().max().item()
    assert (ga - gb).abs().max().item() > 1e-3 * ref[0].abs().max().item()   # the two weight sets differ
    m.close()
