"""Pins of the BF16 reading of the backward pass (oracle/bf16_backward.py):
with rounding off it is the exact reverse-mode gradient (equal to the C
oracle's backward, itself pinned by finite differences); the rounding is BF16
round-to-nearest-even (equal to torch's bfloat16 casts, a library routine, on
random values and on constructed ties); and a network whose contraction
operands are rounded keeps the exact gradient's direction."""
import numpy as np
import pytest

import oracle
import workload
from oracle import bf16_backward as ob


@pytest.mark.parametrize("name,W,B,bias", [("small", 96, 2, 0.1), ("ensemble", 64, 1, 0.05)])
def test_unrounded_reading_is_the_exact_gradient(name, W, B, bias):
    cfg = workload.config(name, n_models=1)
    if name == "ensemble":
        cfg = dict(cfg, stacks=1, layers_per_stack=4)
    wb = workload.init_weights(cfg, seed=3401, bias_std=bias)
    rng = np.random.default_rng(11)
    xh = rng.standard_normal((B, W))
    xl = rng.standard_normal((B, W))
    dl = rng.standard_normal((B, W)) / (B * W)
    g, gh, gl = ob.backward(cfg, workload.param_offsets(cfg), wb[0].astype(np.float64), xh, xl, dl, rounding=False)
    rw, rh, rl = oracle.backward(cfg, wb[0].astype(np.float64), xh, xl, dl)
    for a, b in ((g, rw), (gh, rh), (gl, rl)):
        assert np.max(np.abs(a - b)) <= 1e-10 * max(1.0, np.max(np.abs(b)))


def test_bf16_round_matches_torch_casts_and_ties():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    v = np.concatenate([rng.standard_normal(100000) * 10.0 ** rng.integers(-20, 20, 100000),
                        [0.0, -0.0, 1.0, -1.5, 3.0e38, 1e-40]])
    want = torch.from_numpy(v.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(ob.bf16_round(v), want)
    # ties: 1 + 2^-8 lies halfway between 1 and 1 + 2^-7 -> even (1); 1 + 3 * 2^-8 -> 1 + 2^-6
    assert ob.bf16_round(np.array([1.0 + 2.0 ** -8]))[0] == 1.0
    assert ob.bf16_round(np.array([1.0 + 3 * 2.0 ** -8]))[0] == 1.0 + 2.0 ** -6


def test_f16_round_matches_torch_casts_and_ties():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4)
    v = np.concatenate([rng.standard_normal(100000) * 10.0 ** rng.integers(-9, 5, 100000),
                        [0.0, -0.0, 1.0, -1.5, 65504.0, 1e-8,
                         1.0 + 2.0 ** -11, 1.0 + 3 * 2.0 ** -11]])   # ties to even at 1
    want = torch.from_numpy(v.astype(np.float32)).to(torch.float16).to(torch.float64).numpy()
    np.testing.assert_array_equal(ob.f16_round(v.astype(np.float32).astype(np.float64)), want)
    assert ob.f16_round(1.0 + 2.0 ** -11) == 1.0 and ob.f16_round(1.0 + 3 * 2.0 ** -11) == 1.0 + 2.0 ** -9


def test_rounding_reaches_every_contraction():
    """Rounding changes the gradient (every contraction's operands are rounded, including the first
    layer's), but keeps its direction: the cosine with the exact gradient stays above 0.99.  The
    largest entry-wise changes sit in the head's gradients, whose ReLU masks follow the rounded
    forward (about 0.14 of the largest entry on this random-init network)."""
    cfg = workload.config("small", n_models=1)
    wb = workload.init_weights(cfg, seed=3402, bias_std=0.1)
    rng = np.random.default_rng(12)
    xh, xl = rng.standard_normal((2, 128)), rng.standard_normal((2, 128))
    dl = rng.standard_normal((2, 128)) / 256
    off = workload.param_offsets(cfg)
    g0, _, _ = ob.backward(cfg, off, wb[0], xh, xl, dl, rounding=False)
    g1, _, _ = ob.backward(cfg, off, wb[0], xh, xl, dl, rounding=True)
    rel = np.max(np.abs(g1 - g0)) / np.max(np.abs(g0))
    cos = float(g1 @ g0 / (np.linalg.norm(g1) * np.linalg.norm(g0)))
    assert rel > 1e-4 and cos > 0.99, (rel, cos)
    o, shape = off["H.0.w_conv"]
    n = int(np.prod(shape))
    assert np.max(np.abs(g1[o:o + n] - g0[o:o + n])) > 0.0
