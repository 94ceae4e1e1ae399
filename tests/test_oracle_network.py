"""Pins of the FP64 oracle's network forward against things other than itself.

* the dilated causal convolution against torch's FP64 conv1d (a library routine)
  with left padding (k-1)*d, on every layer of a random network;
* the impulse response: a unit impulse at t0 yields the two taps at t0 and
  t0 + d (tap order and dilation per layer);
* closed forms of the gate, residual, skip and head on hand-built weights;
* the receptive field is exactly 1 + sum(d): a perturbation at t0 changes the
  output on [t0, t0 + RF - 1] and nowhere else;
* shift equivariance / window-vs-stream: overlapping windows agree at
  positions >= RF - 1.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import workload


def _blob(cfg, seed=7, bias_std=0.3):
    return workload.init_weights(cfg, seed=seed, bias_std=bias_std)[0].astype(np.float64)


def _set(blob, cfg, name, value):
    off, shape = workload.param_offsets(cfg)[name]
    n = int(np.prod(shape))
    blob[off:off + n] = np.broadcast_to(np.asarray(value, dtype=np.float64), shape).reshape(-1)


def test_param_count_matches_layout():
    for name in ("small", "ensemble", "tiny"):
        cfg = workload.config(name)
        assert oracle.param_count(cfg) == workload.param_count(cfg)
    # 30-layer model: per branch 2R + 30 * (4R^2 + 2R + R^2 + R + S R + S), head 2S Hc + 2Hc + 1
    assert oracle.param_count(workload.config("ensemble")) == 1805825


@pytest.mark.parametrize("name", ["small", "tiny"])
def test_conv_matches_torch_conv1d(name):
    cfg = workload.config(name)
    blob = _blob(cfg)
    rng = np.random.default_rng(1)
    W = 300
    s = rng.standard_normal(W)
    R = cfg["r_ch"]
    K = cfg["kernel"]
    offs = workload.param_offsets(cfg)
    for branch, tag in ((0, "H"), (1, "L")):
        xs, as_, zs, _ = oracle.branch_trace(cfg, blob, branch, s)
        for l, d in enumerate(workload.dilations(cfg)):
            o, shape = offs[f"{tag}.{l}.w_conv"]
            wc = blob[o:o + int(np.prod(shape))].reshape(shape)          # [2R, K, R] (out, tap, in)
            ob, _ = offs[f"{tag}.{l}.b_conv"]
            bc = blob[ob:ob + 2 * R]
            x = torch.from_numpy(xs[l].T.copy())[None]                    # [1, R, W]
            wt = torch.from_numpy(np.transpose(wc, (0, 2, 1)).copy())     # [2R, R, K]
            xp = torch.nn.functional.pad(x, ((K - 1) * d, 0))
            ref = torch.nn.functional.conv1d(xp, wt, torch.from_numpy(bc), dilation=d)[0].T.numpy()
            np.testing.assert_allclose(as_[l], ref, rtol=1e-12, atol=1e-12)


def test_impulse_response_gives_taps_at_0_and_d():
    cfg = workload.config("small")
    blob = _blob(cfg, bias_std=0.0)
    R = cfg["r_ch"]
    # residual path frozen so every layer sees the same impulse input x = delta(t - t0) * 1
    _set(blob, cfg, "H.w_in", 1.0)
    _set(blob, cfg, "H.b_in", 0.0)
    for l in range(workload.n_layers(cfg)):
        _set(blob, cfg, f"H.{l}.w_res", 0.0)
        _set(blob, cfg, f"H.{l}.b_res", 0.0)
    W, t0 = 600, 100
    s = np.zeros(W); s[t0] = 1.0
    xs, as_, _, _ = oracle.branch_trace(cfg, blob, 0, s)
    offs = workload.param_offsets(cfg)
    for l, d in enumerate(workload.dilations(cfg)):
        o, shape = offs[f"H.{l}.w_conv"]
        wc = blob[o:o + int(np.prod(shape))].reshape(shape)
        expect = np.zeros((W, 2 * R))
        expect[t0] += wc[:, 1, :].sum(axis=1)          # tap on x[t]
        expect[t0 + d] += wc[:, 0, :].sum(axis=1)      # tap on x[t - d]
        np.testing.assert_allclose(as_[l], expect, atol=1e-14)


def test_gate_residual_skip_head_closed_form():
    """All conv weights zero; the conv biases fix a = (atanh 0.5, 0) so z = 0.5 * 0.5 = 0.25."""
    cfg = workload.config("tiny")       # R = S = Hc = 2, 6 layers
    P = workload.param_count(cfg)
    blob = np.zeros(P)
    R, S, L = 2, 2, workload.n_layers(cfg)
    for tag in ("H", "L"):
        _set(blob, cfg, f"{tag}.w_in", [1.0, -1.0])
        _set(blob, cfg, f"{tag}.b_in", [0.5, 0.25])
        for l in range(L):
            _set(blob, cfg, f"{tag}.{l}.b_conv", [math.atanh(0.5), math.atanh(0.5), 0.0, 0.0])
            _set(blob, cfg, f"{tag}.{l}.w_res", np.eye(R) * 2.0)    # r = 2 z = 0.5
            _set(blob, cfg, f"{tag}.{l}.b_res", [0.1, -0.1])
            _set(blob, cfg, f"{tag}.{l}.w_skip", [[1.0, 1.0], [-1.0, 0.0]])  # q = (0.5, -0.25)
            _set(blob, cfg, f"{tag}.{l}.b_skip", [0.0, 0.05])
    s = np.linspace(-1, 1, 16)
    xs, as_, zs, sk = oracle.branch_trace(cfg, blob, 0, s)
    np.testing.assert_allclose(zs, 0.25, atol=1e-15)
    # residual: x_L = x_0 + L * (0.5 + b_res)
    x0 = np.stack([s * 1.0 + 0.5, -s + 0.25], axis=1)
    np.testing.assert_allclose(xs[L], x0 + L * np.array([0.6, 0.4]), atol=1e-13)
    # skip = L * (0.5, -0.25 + 0.05)
    np.testing.assert_allclose(sk, np.broadcast_to([L * 0.5, L * -0.2], sk.shape), atol=1e-13)
    # head: h = ReLU([3, -1.2, 3, -1.2]) = [3, 0, 3, 0]; u = ReLU(W1 h + b1); logit = w2 . u + b2
    _set(blob, cfg, "w_h1", [[1.0, 5.0, 1.0, 5.0], [-1.0, 0.0, 0.0, 0.0]])
    _set(blob, cfg, "b_h1", [0.5, 1.0])          # u = (6.5, ReLU(-2) = 0)
    _set(blob, cfg, "w_h2", [0.25, 3.0])
    _set(blob, cfg, "b_h2", [-1.0])              # logit = 1.625 - 1 = 0.625
    lg = oracle.forward_windows(cfg, blob, s[None], s[None])
    np.testing.assert_allclose(lg, 0.625, atol=1e-13)
    prob = oracle.forward_stream(cfg, blob[None], s.astype(np.float32), s.astype(np.float32), 16, 16)
    np.testing.assert_allclose(prob[0, 0, 0], 1.0 / (1.0 + math.exp(-0.625)), atol=1e-13)


def test_receptive_field_exact():
    cfg = workload.config("small")
    rf = workload.receptive_field(cfg)
    assert rf == 256
    blob = _blob(cfg)
    rng = np.random.default_rng(3)
    W, t0 = 1024, 300
    xh = rng.standard_normal((1, W)); xl = rng.standard_normal((1, W))
    base = oracle.forward_windows(cfg, blob, xh, xl)
    for which in (0, 1):
        xh2, xl2 = xh.copy(), xl.copy()
        (xh2 if which == 0 else xl2)[0, t0] += 0.5
        pert = oracle.forward_windows(cfg, blob, xh2, xl2)
        diff = np.abs(pert - base)[0]
        assert np.all(diff[:t0] == 0.0)
        assert np.all(diff[t0 + rf:] == 0.0)
        assert diff[t0 + rf - 1] > 0.0
        assert diff[t0] > 0.0


def test_windows_agree_with_stream_beyond_receptive_field():
    cfg = workload.config("small")
    rf = workload.receptive_field(cfg)
    blob = _blob(cfg)[None]
    rng = np.random.default_rng(4)
    W, stride = 1024, 384
    n = W + 3 * stride + 17
    sh = rng.standard_normal(n).astype(np.float32); sl = rng.standard_normal(n).astype(np.float32)
    prob = oracle.forward_stream(cfg, blob, sh, sl, W, stride)[0, 0]      # [nw, W]
    nw = prob.shape[0]
    assert nw == (n - W) // stride + 1 == oracle.n_windows(n, W, stride)
    for w in range(1, nw):
        # window w position p equals window w-1 position p + stride when p >= rf - 1
        np.testing.assert_allclose(prob[w, rf - 1:W - stride], prob[w - 1, rf - 1 + stride:], rtol=0, atol=1e-13)
        # and generally differs inside the receptive field (zero padding at the window start)
        assert np.max(np.abs(prob[w, :rf - 1] - prob[w - 1, stride:stride + rf - 1])) > 1e-6


def test_time_slides_pair_h_window_with_shifted_l_window():
    cfg = workload.config("small")
    blob = _blob(cfg)[None]
    rng = np.random.default_rng(5)
    W, stride = 512, 256
    n = W + 5 * stride
    sh = rng.standard_normal(n).astype(np.float32); sl = rng.standard_normal(n).astype(np.float32)
    nw = oracle.n_windows(n, W, stride)
    slides = [0, 1, 3, nw + 2]
    prob = oracle.forward_stream(cfg, blob, sh, sl, W, stride, slides=slides)
    for si, k in enumerate(slides):
        for w in range(nw):
            wl = (w + k) % nw
            lg = oracle.forward_windows(cfg, blob[0], sh[None, w * stride:w * stride + W].astype(np.float64),
                                        sl[None, wl * stride:wl * stride + W].astype(np.float64))
            np.testing.assert_allclose(prob[si, 0, w], 1 / (1 + np.exp(-lg[0])), atol=1e-14)


def test_branches_are_not_shared():
    """Swapping the detectors changes the output when the branch weights differ."""
    cfg = workload.config("tiny")
    blob = _blob(cfg)
    rng = np.random.default_rng(6)
    xh = rng.standard_normal((1, 64)); xl = rng.standard_normal((1, 64))
    a = oracle.forward_windows(cfg, blob, xh, xl)
    b = oracle.forward_windows(cfg, blob, xl, xh)
    assert np.max(np.abs(a - b)) > 1e-6
