"""Pins of the oracle's backward pass and loss.

* every weight gradient and both strain gradients against FP64 central finite
  differences on a tiny network (R = S = Hc = 2, 2 stacks x 3 layers, W = 64),
  for the scalar functional J = sum(g * logit) with random g (so dJ/dlogit = g);
* the BCE loss and its derivative against closed-form values;
* the per-sample label convention: the end-to-end training loss gradient is the
  backward of dL/dlogit = (sigmoid(z) - y) / n.
"""
import math

import numpy as np
import pytest

import oracle
import workload


def _setup(seed=11):
    cfg = workload.config("tiny")
    blob = workload.init_weights(cfg, seed=seed, bias_std=0.3)[0].astype(np.float64)
    rng = np.random.default_rng(seed)
    B, W = 2, 64
    xh = rng.standard_normal((B, W)); xl = rng.standard_normal((B, W))
    g = rng.standard_normal((B, W))
    return cfg, blob, xh, xl, g


def _J(cfg, blob, xh, xl, g):
    return float(np.sum(g * oracle.forward_windows(cfg, blob, xh, xl, nthreads=1)))


def test_weight_gradients_match_central_differences():
    cfg, blob, xh, xl, g = _setup()
    gw, _, _ = oracle.backward(cfg, blob, xh, xl, g, nthreads=1)
    h = 1e-6
    P = blob.shape[0]
    fd = np.zeros(P)
    for i in range(P):
        bp = blob.copy(); bp[i] += h
        bm = blob.copy(); bm[i] -= h
        fd[i] = (_J(cfg, bp, xh, xl, g) - _J(cfg, bm, xh, xl, g)) / (2 * h)
    scale = np.maximum(np.abs(fd), 1e-3)
    rel = np.abs(gw - fd) / scale
    assert rel.max() < 1e-6, (rel.argmax(), gw[rel.argmax()], fd[rel.argmax()])
    # every parameter group is exercised (no silently-zero gradient), except the
    # last layer's residual projection, whose output feeds nothing
    offs = workload.param_offsets(cfg)
    last = workload.n_layers(cfg) - 1
    for name, (o, shape) in offs.items():
        n = int(np.prod(shape))
        if name.endswith(f".{last}.w_res") or name.endswith(f".{last}.b_res"):
            assert np.all(gw[o:o + n] == 0.0) and np.all(np.abs(fd[o:o + n]) < 1e-9), name
        else:
            assert np.any(np.abs(fd[o:o + n]) > 1e-9), name


def test_strain_gradients_match_central_differences():
    cfg, blob, xh, xl, g = _setup(seed=12)
    _, gh, gl = oracle.backward(cfg, blob, xh, xl, g, nthreads=1)
    h = 1e-6
    for arr, grad in ((xh, gh), (xl, gl)):
        for (b, t) in [(0, 0), (0, 5), (1, 31), (1, 63), (0, 40)]:
            ap = arr.copy(); ap[b, t] += h
            am = arr.copy(); am[b, t] -= h
            if arr is xh:
                fd = (_J(cfg, blob, ap, xl, g) - _J(cfg, blob, am, xl, g)) / (2 * h)
            else:
                fd = (_J(cfg, blob, xh, ap, g) - _J(cfg, blob, xh, am, g)) / (2 * h)
            assert abs(grad[b, t] - fd) <= 1e-6 * max(abs(fd), 1e-3), (b, t, grad[b, t], fd)


def test_bce_closed_form():
    z = np.array([0.0, 0.0, 3.0, -3.0, 40.0, -40.0])
    y = np.array([1.0, 0.0, 0.0, 1.0, 1.0, 0.0])
    loss, dz = oracle.bce(z, y)
    per = np.array([math.log(2.0), math.log(2.0), 3.048587351573742, 3.048587351573742,
                    4.248354255291589e-18, 4.248354255291589e-18])
    assert loss == pytest.approx(per.mean(), rel=1e-14)
    sig = np.array([0.5, 0.5, 0.9525741268224334, 0.04742587317756678, 1.0, 0.0])
    np.testing.assert_allclose(dz, (sig - y) / 6.0, rtol=1e-12, atol=1e-18)
    # derivative of the mean loss by central differences
    rng = np.random.default_rng(0)
    z = rng.standard_normal(7) * 3; y = (rng.random(7) > 0.5).astype(float)
    _, dz = oracle.bce(z, y)
    for i in range(7):
        zp = z.copy(); zp[i] += 1e-6
        zm = z.copy(); zm[i] -= 1e-6
        fd = (oracle.bce(zp, y)[0] - oracle.bce(zm, y)[0]) / 2e-6
        assert dz[i] == pytest.approx(fd, rel=1e-6, abs=1e-10)


def test_training_gradient_through_bce_matches_finite_difference():
    cfg, blob, xh, xl, _ = _setup(seed=13)
    y = np.zeros_like(xh); y[0, :40] = 1.0      # merger at t = 39 in window 0: labels 1 up to it
    lg = oracle.forward_windows(cfg, blob, xh, xl)
    _, dz = oracle.bce(lg, y)
    gw, _, _ = oracle.backward(cfg, blob, xh, xl, dz)
    idx = [0, 7, 100, 250, blob.shape[0] - 1, blob.shape[0] - 5]
    for i in idx:
        h = 1e-6
        bp = blob.copy(); bp[i] += h
        bm = blob.copy(); bm[i] -= h
        fd = (oracle.bce(oracle.forward_windows(cfg, bp, xh, xl), y)[0]
              - oracle.bce(oracle.forward_windows(cfg, bm, xh, xl), y)[0]) / (2 * h)
        assert gw[i] == pytest.approx(fd, rel=1e-5, abs=1e-9)
