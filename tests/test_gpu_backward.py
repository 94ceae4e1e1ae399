"""The FP32 backward pass (dgrad, wgrad, gate backward, per-stack recomputation)
against the FP64 oracle's reverse-mode gradient, and against central finite
differences of the library's own forward."""
import numpy as np
import pytest

import oracle
import workload
from gpu_util import require_gpu

pytestmark = pytest.mark.gpu


def _grads(cfg, wb, xh, xl, dlogit):
    import torch
    import paper_2201_11133_gb300 as gwe
    dev = require_gpu()
    m = gwe.Model(cfg, wb, gwe.GWE_FP32)
    B, W = xh.shape
    P = gwe.gwe_param_count(cfg)
    gw = torch.empty(P, dtype=torch.float32, device=dev)
    gh = torch.empty((B, W), dtype=torch.float32, device=dev)
    gl = torch.empty((B, W), dtype=torch.float32, device=dev)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(dev)
    gwe.gwe_backward(m.handle, 0, t(xh), t(xl), B, W, t(dlogit), gw, gh, gl)
    m.sync()
    out = gw.cpu().numpy().astype(np.float64), gh.cpu().numpy().astype(np.float64), gl.cpu().numpy().astype(np.float64)
    m.close()
    return out


def _check(got, ref, tol):
    scale = max(np.max(np.abs(ref)), 1e-30)
    err = np.max(np.abs(got - ref)) / scale
    assert err <= tol, (err, tol)
    return err


@pytest.mark.parametrize("name,W,B", [("small", 512, 3), ("ensemble", 384, 2)])
def test_backward_matches_oracle(name, W, B):
    cfg = workload.config(name, n_models=1)
    wb = workload.init_weights(cfg, seed=3400, bias_std=0.1)
    rng = np.random.default_rng(5)
    xh = rng.standard_normal((B, W)).astype(np.float32)
    xl = rng.standard_normal((B, W)).astype(np.float32)
    dlogit = (rng.standard_normal((B, W)) / (B * W)).astype(np.float32)
    gw, gh, gl = _grads(cfg, wb, xh, xl, dlogit)
    rw, rh, rl = oracle.backward(cfg, wb[0].astype(np.float64), xh, xl, dlogit.astype(np.float64))
    e1 = _check(gw, rw, 2e-4)
    e2 = _check(gh, rh, 2e-4)
    e3 = _check(gl, rl, 2e-4)
    # per parameter block: every group of the blob gets its gradient
    offs = workload.param_offsets(cfg)
    for pname, (o, shape) in offs.items():
        n = int(np.prod(shape))
        ref_blk = rw[o:o + n]
        if np.max(np.abs(ref_blk)) > 1e-3 * np.max(np.abs(rw)):
            rel = np.max(np.abs(gw[o:o + n] - ref_blk)) / np.max(np.abs(ref_blk))
            assert rel <= 2e-3, (pname, rel)
    print(f"{name}: rel err weights {e1:.2e} strain_H {e2:.2e} strain_L {e3:.2e}")


def test_backward_bce_training_batch_matches_oracle():
    """Gradient of the mean BCE over a labelled batch (labels 1 up to the merger)."""
    import torch
    import paper_2201_11133_gb300 as gwe
    dev = require_gpu()
    cfg = workload.config("small", n_models=1)
    wb = workload.init_weights(cfg, seed=3500, bias_std=0.1)
    xh, xl, y = workload.training_batch(B=4, W=1024, seed=77, merger_range=(256, 1023))
    m = gwe.Model(cfg, wb, gwe.GWE_FP32)
    lg = m.logits(torch.from_numpy(xh).to(dev), torch.from_numpy(xl).to(dev))[0]
    loss_t = torch.nn.functional.binary_cross_entropy_with_logits(lg, torch.from_numpy(y).to(dev))
    dl = torch.sigmoid(lg) - torch.from_numpy(y).to(dev)
    dl = (dl / dl.numel()).contiguous()
    m.close()
    gw, _, _ = _grads(cfg, wb, xh, xl, dl.cpu().numpy())
    ref_lg = oracle.forward_windows(cfg, wb[0], xh, xl)
    loss, dref = oracle.bce(ref_lg, y)
    assert abs(loss - float(loss_t.item())) <= 1e-5 * max(1.0, abs(loss))
    rw, _, _ = oracle.backward(cfg, wb[0].astype(np.float64), xh, xl, dref)
    _check(gw, rw, 2e-4)


def test_backward_central_differences_of_forward():
    """dL/dw from gwe_backward against (L(w + h e) - L(w - h e)) / 2h through gwe_forward_logits.

    The loss is evaluated by the FP32 forward, whose rounding adds ~1e-5 of noise to the loss, so the
    step must stay near 1e-2; the head's ReLUs would make such a step cross kinks (FP64 differences
    show it at h = 1e-3), so the skip and head biases are set to keep every ReLU input positive and
    the loss smooth.  The ReLU cases themselves are covered by the comparison with the oracle's
    gradient above (the oracle is pinned by FP64 central differences)."""
    import torch
    import paper_2201_11133_gb300 as gwe
    dev = require_gpu()
    cfg = workload.config("small", n_models=1)
    wb = workload.init_weights(cfg, seed=3600, bias_std=0.1).astype(np.float64)
    offs = workload.param_offsets(cfg)
    for tag in ("H", "L"):
        for l in range(workload.n_layers(cfg)):
            o, shape = offs[f"{tag}.{l}.b_skip"]
            wb[0, o:o + shape[0]] = 1.0
    o, shape = offs["b_h1"]
    wb[0, o:o + shape[0]] = 50.0
    rng = np.random.default_rng(9)
    B, W = 2, 256
    xh = rng.standard_normal((B, W)).astype(np.float32)
    xl = rng.standard_normal((B, W)).astype(np.float32)
    c = rng.standard_normal((B, W)) / (B * W)          # L = mean of c * logit
    gw, _, _ = _grads(cfg, wb.astype(np.float32), xh, xl, c.astype(np.float32))
    picks = []
    for pname in ("H.0.w_conv", "L.7.w_conv", "H.3.w_res", "L.5.w_skip", "w_h1", "w_h2", "b_h1", "H.w_in",
                  "L.2.b_conv", "H.6.b_res"):
        o, shape = offs[pname]
        picks += [o + int(i) for i in rng.choice(int(np.prod(shape)), size=2, replace=False)]
    m = gwe.Model(cfg, wb.astype(np.float32), gwe.GWE_FP32)
    H, Lt = torch.from_numpy(xh).to(dev), torch.from_numpy(xl).to(dev)

    def loss(wvec):
        gwe.gwe_model_set_weights(m.handle, wvec.astype(np.float32))
        lg = m.logits(H, Lt)[0].cpu().numpy().astype(np.float64)
        return float(np.sum(c * lg))

    h = 1e-2
    scale = float(np.max(np.abs(gw[picks])))
    for i in picks:
        wp = wb.copy(); wp[0, i] += h
        wn = wb.copy(); wn[0, i] -= h
        fd = (loss(wp) - loss(wn)) / (2 * h)
        assert abs(fd - gw[i]) <= 1e-2 * max(abs(fd), 0.05 * scale), (i, fd, gw[i])
    m.close()


def test_autograd_function_training_step():
    """torch autograd through the library: BCE on the logits, weight and input gradients equal to the
    oracle's, and a few SGD steps lower the loss."""
    import torch
    import paper_2201_11133_gb300 as gwe
    dev = require_gpu()
    cfg = workload.config("small", n_models=1)
    wb = workload.init_weights(cfg, seed=3700, bias_std=0.1)
    xh, xl, y = workload.training_batch(B=4, W=512, seed=78, merger_range=(128, 511))
    m = gwe.Model(cfg, wb, gwe.GWE_FP32)
    w = torch.from_numpy(wb[0].copy()).to(dev).requires_grad_(True)
    H = torch.from_numpy(xh).to(dev).requires_grad_(True)
    Lt = torch.from_numpy(xl).to(dev)
    Y = torch.from_numpy(y).to(dev)
    lg = gwe.gwe_logits_autograd(m, w, H, Lt)
    loss = torch.nn.functional.binary_cross_entropy_with_logits(lg, Y)
    loss.backward()
    ref_lg = oracle.forward_windows(cfg, wb[0], xh, xl)
    ref_loss, dref = oracle.bce(ref_lg, y)
    rw, rh, _ = oracle.backward(cfg, wb[0].astype(np.float64), xh, xl, dref)
    _check(w.grad.cpu().numpy().astype(np.float64), rw, 2e-4)
    _check(H.grad.cpu().numpy().astype(np.float64), rh, 2e-4)
    losses = [float(loss.item())]
    opt = torch.optim.SGD([w], lr=0.5)
    for _ in range(5):
        opt.zero_grad()
        lg = gwe.gwe_logits_autograd(m, w, H.detach(), Lt)
        loss = torch.nn.functional.binary_cross_entropy_with_logits(lg, Y)
        loss.backward()
        opt.step()
        losses.append(float(loss.item()))
    assert losses[-1] < losses[0], losses
    m.close()
