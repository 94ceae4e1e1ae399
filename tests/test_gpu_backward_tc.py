"""The tensor-core backward (BF16 operands, FP32 accumulation, per-stack
recomputation) against the oracle's BF16 reading of the backward
(oracle/bf16_backward.py: FP64 arithmetic with the operands of every
contraction rounded to BF16, the reading the kernels implement) and, for the
record, against the exact FP64 gradient and the FP32 backward.

Tolerances.  On these random-init networks the gradient is sensitive to any
perturbation of the forward at the 1e-7 level (ReLU masks of the head and
rounding boundaries flip), so the kernels' FP32 accumulation order moves them
about as far from the BF16 reading as the reading is from exact arithmetic
(~2e-2 relative on the 30-layer model).  The pins are therefore: the kernels'
distance from the exact gradient (relative L2, weights and strain) is at most
twice the BF16 reading's, plus 1e-3; the cosine with the exact gradient is at
least 0.99; and on a 1 s training batch with chirps and labels the gradient is
within 1e-2 (largest entry) and cosine 0.999 of the FP32 backward's."""
import numpy as np
import pytest

import oracle
import workload
from gpu_util import require_gpu

pytestmark = pytest.mark.gpu


def _grads(cfg, wb, xh, xl, dlogit, prec):
    import torch
    import paper_2201_11133_gb300 as gwe
    dev = require_gpu()
    m = gwe.Model(cfg, wb, prec)
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


def _rel(got, ref):
    return np.max(np.abs(got - ref)) / max(np.max(np.abs(ref)), 1e-30)


def _cos(a, b):
    a, b = np.ravel(a), np.ravel(b)
    return float(np.dot(a, b) / (np.linalg.norm(a) * np.linalg.norm(b)))


# BF16 handles with a window that is a multiple of 128 take the stack inputs and skip sums from the
# fused forward kernel; FP8 handles and other windows (tiles then span windows) from a forward pass
# of row GEMMs
@pytest.mark.parametrize("name,W,B,prec", [("small", 512, 3, "bf16"), ("ensemble", 384, 2, "bf16"),
                                           ("ensemble", 1024, 1, "bf16"), ("ensemble", 384, 2, "fp8"),
                                           ("small", 200, 2, "bf16")])
def test_tc_backward_as_accurate_as_bf16_arithmetic(name, W, B, prec):
    import paper_2201_11133_gb300 as gwe
    from oracle import bf16_backward as ob
    cfg = workload.config(name, n_models=1)
    wb = workload.init_weights(cfg, seed=3400, bias_std=0.1)
    rng = np.random.default_rng(5)
    xh = rng.standard_normal((B, W)).astype(np.float32)
    xl = rng.standard_normal((B, W)).astype(np.float32)
    dlogit = (rng.standard_normal((B, W)) / (B * W)).astype(np.float32)
    gw, gh, gl = _grads(cfg, wb, xh, xl, dlogit, gwe.GWE_BF16 if prec == "bf16" else gwe.GWE_FP8)
    qw, qh, ql = ob.backward(cfg, workload.param_offsets(cfg), wb[0], xh, xl, dlogit)
    rw, rh, rl = oracle.backward(cfg, wb[0].astype(np.float64), xh, xl, dlogit.astype(np.float64))
    l2 = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
    rows = []
    for got, q, ref, what in ((gw, qw, rw, "weights"), (gh, qh, rh, "strain_H"), (gl, ql, rl, "strain_L")):
        e_gpu, e_q = l2(got, ref), l2(q, ref)
        print(f"{name} W={W} B={B} {prec} {what}: rel L2 vs exact: kernels {e_gpu:.2e}, BF16 reading {e_q:.2e}; "
              f"kernels vs reading {l2(got, q):.2e}; cos vs exact {_cos(got, ref):.5f}")
        rows.append((what, e_gpu, e_q, _cos(got, ref)))
    for what, e_gpu, e_q, cos in rows:
        assert e_gpu <= 2.0 * e_q + 1e-3, (what, e_gpu, e_q)
        assert cos >= 0.99, (what, cos)


def test_tc_backward_close_to_fp32_backward_full_window():
    """A 1 s window batch of the 30-layer model with chirps and per-sample BCE labels: the tensor-core
    gradient against the FP32 SIMT gradient of the same weights."""
    import torch
    import paper_2201_11133_gb300 as gwe
    cfg = workload.config("ensemble", n_models=1)
    wb = workload.init_weights(cfg, seed=3000)
    xh, xl, y = workload.training_batch(B=6, W=4096, seed=2024)
    dev = require_gpu()
    m = gwe.Model(cfg, wb, gwe.GWE_FP32)
    lg = m.logits(torch.from_numpy(xh).to(dev), torch.from_numpy(xl).to(dev))[0]
    dl = ((torch.sigmoid(lg) - torch.from_numpy(y).to(dev)) / float(y.size)).cpu().numpy()
    m.close()
    g32, h32, l32 = _grads(cfg, wb, xh, xl, dl, gwe.GWE_FP32)
    g16, h16, l16 = _grads(cfg, wb, xh, xl, dl, gwe.GWE_BF16)
    e_w, e_h = _rel(g16, g32), _rel(h16, h32)
    print(f"full window: rel err vs FP32 weights {e_w:.2e} strain {e_h:.2e} cos {_cos(g16, g32):.6f}")
    assert e_w <= 1e-2 and _cos(g16, g32) >= 0.999


def test_tc_backward_training_steps_lower_the_loss():
    """torch autograd through a BF16 handle (tensor-core forward logits, tensor-core backward): a few
    SGD steps on a batch with chirps lower the BCE loss."""
    import torch
    import paper_2201_11133_gb300 as gwe
    dev = require_gpu()
    cfg = workload.config("small", n_models=1)
    wb = workload.init_weights(cfg, seed=3700, bias_std=0.1)
    xh, xl, y = workload.training_batch(B=8, W=1024, seed=79, merger_range=(256, 1023))
    m = gwe.Model(cfg, wb, gwe.GWE_BF16)
    w = torch.from_numpy(wb[0].copy()).to(dev).requires_grad_(True)
    H = torch.from_numpy(xh).to(dev)
    Lt = torch.from_numpy(xl).to(dev)
    Y = torch.from_numpy(y).to(dev)
    opt = torch.optim.SGD([w], lr=0.5)
    losses = []
    for _ in range(6):
        opt.zero_grad()
        lg = gwe.gwe_logits_autograd(m, w, H, Lt)
        loss = torch.nn.functional.binary_cross_entropy_with_logits(lg, Y)
        loss.backward()
        opt.step()
        losses.append(float(loss.item()))
    assert losses[-1] < losses[0], losses
    m.close()


def _smooth_net(cfg, seed):
    """Weights on which no ReLU of the network can change state: the skip and head weights are
    scaled by 0.1 (a valid network with small skip terms), every skip term W_skip z + b_skip is
    positive (|z| < 1 and b_skip[o] = 0.1 + sum_i |W_skip[o, i]|), so the skip sums h are positive
    and bounded by h_max, and the head's u = W_h1 h + b_h1 is positive
    (b_h1[j] = 0.1 + h_max sum_k |W_h1[j, k]|).  The network is then smooth in its weights and
    inputs, and gradients are comparable entry by entry."""
    wb = workload.init_weights(cfg, seed=seed, bias_std=0.1)[0].astype(np.float64)
    off = workload.param_offsets(cfg)
    L = int(cfg["stacks"]) * int(cfg["layers_per_stack"])
    h_max = 0.0
    for br in ("H", "L"):
        tot = 0.0
        for l in range(L):
            o, sh = off[f"{br}.{l}.w_skip"]
            n = int(np.prod(sh))
            wb[o:o + n] *= 0.1
            ws = wb[o:o + n].reshape(sh)
            ob_, _ = off[f"{br}.{l}.b_skip"]
            b = 0.1 + np.abs(ws).sum(1)
            wb[ob_:ob_ + b.size] = b
            tot += float((np.abs(ws).sum(1) + b).max())
        h_max = max(h_max, tot)
    o, sh = off["w_h1"]
    n = int(np.prod(sh))
    wb[o:o + n] *= 0.1
    w1 = wb[o:o + n].reshape(sh)
    ob_, _ = off["b_h1"]
    wb[ob_:ob_ + sh[0]] = 0.1 + h_max * np.abs(w1).sum(1)
    return wb.astype(np.float32)[None, :]


def _smooth_setup(seed_w, seed_x):
    cfg = dict(workload.config("small", n_models=1), stacks=1, layers_per_stack=3)
    wb = _smooth_net(cfg, seed_w)
    B, W = 2, 256
    rng = np.random.default_rng(seed_x)
    xh = rng.standard_normal((B, W)).astype(np.float32)
    xl = rng.standard_normal((B, W)).astype(np.float32)
    c = (rng.standard_normal((B, W)) / (B * W)).astype(np.float32)
    return cfg, wb, xh, xl, c, rng


def _handle_grad(cfg, wb, xh, xl, c, n16):
    import torch
    import paper_2201_11133_gb300 as gwe
    dev = require_gpu()
    m = gwe.Model(cfg, wb, gwe.GWE_BF16)
    gwe.gwe_model_set_f16_layers(m.handle, n16)
    B, W = xh.shape
    P = gwe.gwe_param_count(cfg)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(dev)
    gw = torch.empty(P, device=dev)
    gh = torch.empty((B, W), device=dev)
    gl = torch.empty((B, W), device=dev)
    gwe.gwe_backward(m.handle, 0, t(xh), t(xl), B, W, t(c), gw, gh, gl)
    m.sync()
    return m, tuple(a.cpu().numpy().astype(np.float64) for a in (gw, gh, gl))


def test_tc_backward_elementwise_on_smooth_net():
    """Entry by entry against the BF16 reading of the backward (R19), on a 3-layer network with no
    ReLU state changes; tolerance 1e-2 of the largest entry of each parameter tensor (and of each
    strain gradient), which covers BF16 operands that the kernels and the FP64 reading round to
    neighbouring values from inputs that differ at the 1e-7 level (FP32 vs FP64 accumulation)."""
    from oracle import bf16_backward as ob
    cfg, wb, xh, xl, c, _ = _smooth_setup(3500, 6)
    m, (gw, gh, gl) = _handle_grad(cfg, wb, xh, xl, c, 0)   # the reading rounds every conv operand to BF16
    m.close()
    qw, qh, ql = ob.backward(cfg, workload.param_offsets(cfg), wb[0], xh, xl, c)
    worst = 0.0
    for name, (o, sh) in workload.param_offsets(cfg).items():
        n = int(np.prod(sh))
        ref = qw[o:o + n]
        scale = max(float(np.max(np.abs(ref))), 1e-30)
        e = float(np.max(np.abs(gw[o:o + n] - ref))) / scale
        worst = max(worst, e)
        assert e <= 1e-2, (name, e)
    for got, ref, what in ((gh, qh, "strain_H"), (gl, ql, "strain_L")):
        e = float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
        print(f"smooth net {what}: max |kernels - reading| / max |reading| {e:.2e}")
        assert e <= 1e-2, (what, e)
    print(f"smooth net weights: worst per-tensor max |kernels - reading| / max |reading| {worst:.2e}")


def test_tc_backward_against_central_differences_of_exact_forward():
    """The tensor-core gradient against central differences of the FP64 forward (the oracle) along
    random directions over every parameter: within 1e-2 relative (the BF16 rounding of the
    backward's operands)."""
    cfg, wb, xh, xl, c, rng = _smooth_setup(3600, 7)
    m, (g, _, _) = _handle_grad(cfg, wb, xh, xl, c, 0)
    m.close()
    w = wb[0].astype(np.float64)
    L = lambda wv: float(np.sum(oracle.forward_windows(cfg, wv, xh, xl) * c))
    for trial in range(3):
        v = rng.standard_normal(w.size)
        v *= np.abs(w).max() / np.abs(v).max()
        h = 1e-5
        fd = (L(w + h * v) - L(w - h * v)) / (2 * h)
        an = float(np.dot(g, v))
        rel = abs(fd - an) / abs(fd)
        print(f"central differences of the FP64 forward, trial {trial}: fd {fd:.6e} tensor-core {an:.6e} rel {rel:.2e}")
        assert rel <= 1e-2


def test_tc_backward_central_differences_of_handle_forward():
    """The handle's gradient against central differences of its own tensor-core forward: along the
    head's FP32 parameters (b_h1, w_h2, b_h2: everything after the last 16-bit rounding, so the
    differences are exact up to FP32) within 1e-3, and along every parameter with a step large
    against the forward's FP16 rounding (n16 = L: all conv operands FP16) within 3e-2."""
    import torch
    cfg, wb, xh, xl, c, rng = _smooth_setup(3700, 8)
    dev = require_gpu()
    off = workload.param_offsets(cfg)
    L_ = int(cfg["stacks"]) * int(cfg["layers_per_stack"])
    m, (g, _, _) = _handle_grad(cfg, wb, xh, xl, c, L_)
    xt, lt = torch.from_numpy(xh).to(dev), torch.from_numpy(xl).to(dev)
    ct = torch.from_numpy(c).to(dev).double()
    w0 = torch.from_numpy(wb[0]).to(dev)

    def loss(wv):
        m.set_weights_device(wv)
        lg = m.logits(xt, lt)[0]
        m.sync()
        return float((lg.double() * ct).sum().item())

    P = w0.numel()
    for tag, names, h, tol in (("head", ["b_h1", "w_h2", "b_h2"], 1e-2, 1e-3),
                               ("all", list(off), 2e-2, 3e-2)):
        v = np.zeros(P)
        for n in names:
            o, sh = off[n]
            k = int(np.prod(sh))
            v[o:o + k] = rng.standard_normal(k) * max(float(np.abs(wb[0][o:o + k]).max()), 1e-3)
        v /= np.abs(v).max()
        vt = torch.from_numpy(v.astype(np.float32)).to(dev)
        fd = (loss(w0 + h * vt) - loss(w0 - h * vt)) / (2 * h)
        an = float(np.dot(g, v))
        rel = abs(fd - an) / max(abs(an), 1e-30)
        print(f"central differences of the handle forward ({tag}): fd {fd:.6e} analytic {an:.6e} rel {rel:.2e}")
        assert rel <= tol, (tag, fd, an)
    m.close()


def test_tensor_map_and_per_thread_staging_agree():
    """The backward with its GEMM operands brought in by tensor-map copies (128-byte swizzled tiles, the
    default) against the same backward with per-thread copies, on the 30-layer model with 1024-sample
    windows, where every GEMM takes the tensor-map form: dL/dstrain bit for bit (the row GEMMs multiply
    the same operands in the same K order), and the weight gradients within 1e-3 of each parameter
    tensor's largest entry (their atomic partial sums come in another order; a misplaced tile would
    move them by O(1))."""
    import paper_2201_11133_gb300 as gwe
    cfg = workload.config("ensemble", n_models=1)
    wb = workload.init_weights(cfg, seed=3800, bias_std=0.1)
    rng = np.random.default_rng(9)
    B, W = 2, 1024
    xh = rng.standard_normal((B, W)).astype(np.float32)
    xl = rng.standard_normal((B, W)).astype(np.float32)
    dlogit = (rng.standard_normal((B, W)) / (B * W)).astype(np.float32)
    try:
        gwe.gwe_set_tensor_map_copies(False)
        pw, ph, pl = _grads(cfg, wb, xh, xl, dlogit, gwe.GWE_BF16)
    finally:
        gwe.gwe_set_tensor_map_copies(True)
    tw, th, tl = _grads(cfg, wb, xh, xl, dlogit, gwe.GWE_BF16)
    assert np.array_equal(th, ph) and np.array_equal(tl, pl)
    worst = 0.0
    for name, (o, sh) in workload.param_offsets(cfg).items():
        n = int(np.prod(sh))
        ref = pw[o:o + n]
        e = float(np.max(np.abs(tw[o:o + n] - ref))) / max(float(np.max(np.abs(ref))), 1e-30)
        worst = max(worst, e)
        assert e <= 1e-3, (name, e)
    print(f"tensor-map vs per-thread staging: dL/dstrain identical; weights worst per-tensor {worst:.2e}")
