"""Pins of the oracle's FP8 reading (E4M3 convolution operands with
per-channel scales), used for the error statements of the FP8 path.

* the E4M3 rounding against torch.float8_e4m3fn casts run as a library
  routine: every representable value, every midpoint between neighbours
  (ties to even), subnormals, and random values over the whole range;
  saturation at +-448 from the format's definition;
* a one-layer network evaluated in numpy with torch's casts for the
  quantisation and the scale conventions written out, against the oracle;
* the calibration maxima against the oracle's own per-layer trace.
"""
import numpy as np
import pytest

import oracle
import workload

torch = pytest.importorskip("torch")
if not hasattr(torch, "float8_e4m3fn"):
    pytest.skip("torch without float8_e4m3fn", allow_module_level=True)


def _torch_e4m3(v):
    t = torch.from_numpy(np.asarray(v, dtype=np.float32))
    return t.to(torch.float8_e4m3fn).to(torch.float64).numpy()


def _all_finite_e4m3():
    codes = torch.arange(0, 256, dtype=torch.int32).to(torch.uint8)
    vals = codes.view(torch.float8_e4m3fn).to(torch.float64).numpy()
    return np.unique(vals[np.isfinite(vals)])


def test_e4m3_representable_values_and_midpoints():
    vals = _all_finite_e4m3()
    assert vals.max() == 448.0 and vals.min() == -448.0
    assert np.min(vals[vals > 0]) == 2.0 ** -9          # smallest subnormal
    np.testing.assert_array_equal(oracle.e4m3(vals), vals)
    pos = vals[vals >= 0]
    mids = 0.5 * (pos[:-1] + pos[1:])                   # ties: to the even mantissa
    np.testing.assert_array_equal(oracle.e4m3(mids), _torch_e4m3(mids))
    np.testing.assert_array_equal(oracle.e4m3(-mids), _torch_e4m3(-mids))
    # a tie picks the neighbour whose last mantissa bit is 0
    codes = {float(v): int(c) for c, v in enumerate(torch.arange(0, 128, dtype=torch.int32).to(torch.uint8)
                                                   .view(torch.float8_e4m3fn).to(torch.float64).numpy())}
    for m in mids[:40]:
        r = float(oracle.e4m3(np.array([m]))[0])
        assert codes[r] % 2 == 0, (m, r)


def test_e4m3_random_values_and_saturation():
    rng = np.random.default_rng(7)
    v = (np.exp(rng.uniform(np.log(2.0 ** -12), np.log(440.0), 200000)) *
         rng.choice([-1.0, 1.0], 200000)).astype(np.float32)
    np.testing.assert_array_equal(oracle.e4m3(v.astype(np.float64)), _torch_e4m3(v))
    big = np.array([448.0, 449.0, 463.9, 464.0, 500.0, 1e6, -1e6, -470.0])
    np.testing.assert_array_equal(oracle.e4m3(big), np.sign(big) * 448.0)
    # relative error of a normal value is at most half a spacing: 2^-4
    w = rng.uniform(2.0 ** -6, 440.0, 10000)
    assert np.max(np.abs(oracle.e4m3(w) - w) / w) <= 2.0 ** -4 + 1e-15


def _one_layer_numpy(cfg, wb, amax, xh, xl, margin):
    """Logits of a one-layer (dilation 1) network under the FP8 reading, with torch's E4M3 casts."""
    R, S = int(cfg["r_ch"]), int(cfg["s_ch"])
    off = workload.param_offsets(cfg)
    P = {k: wb[o:o + int(np.prod(s))].astype(np.float64).reshape(s) for k, (o, s) in off.items()}
    skips = []
    for bi, (b, x_in) in enumerate((("H", xh), ("L", xl))):
        x = x_in[..., None] * P[f"{b}.w_in"] + P[f"{b}.b_in"]                   # [B, W, R]
        sc = np.where(amax[bi, 0] > 0, margin * amax[bi, 0] / 448.0, 1.0)
        qx = _q64(x / sc)
        Wc = P[f"{b}.0.w_conv"]                                                  # [2R, 2, R]
        Wp = Wc * sc[None, None, :]
        wo = np.abs(Wp).reshape(2 * R, -1).max(axis=1) / 448.0
        wo[wo == 0] = 1.0
        qw = _q64(Wp / wo[:, None, None])
        ql = np.zeros_like(qx)
        ql[:, 1:] = qx[:, :-1]
        a = wo * (ql @ qw[:, 0, :].T + qx @ qw[:, 1, :].T) + P[f"{b}.0.b_conv"]
        z = np.tanh(a[..., :R]) / (1.0 + np.exp(-a[..., R:]))
        skips.append(z @ P[f"{b}.0.w_skip"].T + P[f"{b}.0.b_skip"])
    h = np.maximum(np.concatenate(skips, -1), 0.0)
    u = np.maximum(h @ P["w_h1"].T + P["b_h1"], 0.0)
    return u @ P["w_h2"] + P["b_h2"][0]


def _q64(v):
    """torch E4M3 cast of FP64 values that sit on FP32 exactly; others are rounded to FP32 first,
    which changes the result only within 2^-24 of a rounding midpoint."""
    v = np.asarray(v, dtype=np.float64)
    return _torch_e4m3(np.clip(v, -448.0, 448.0).astype(np.float32)).reshape(v.shape)


def test_fp8_reading_one_layer_against_numpy():
    cfg = dict(n_models=1, stacks=1, layers_per_stack=1, kernel=2, r_ch=8, s_ch=8, head_ch=4)
    wb = workload.init_weights(cfg, seed=11, bias_std=0.2)[0]
    rng = np.random.default_rng(3)
    B, W = 3, 64
    # inputs on the FP32 grid so that the FP32 detour of the torch cast is exact at the first step
    xh = rng.standard_normal((B, W)).astype(np.float32).astype(np.float64)
    xl = rng.standard_normal((B, W)).astype(np.float32).astype(np.float64)
    amax = np.stack([oracle.act_amax(cfg, wb, 0, xh), oracle.act_amax(cfg, wb, 1, xl)])
    got = oracle.forward_windows_q8(cfg, wb, amax, xh, xl, margin=16.0)
    want = _one_layer_numpy(cfg, wb.astype(np.float64), amax, xh, xl, 16.0)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-9)
    # and it differs from exact arithmetic by a quantisation-sized amount, not more
    exact = oracle.forward_windows(cfg, wb, xh, xl)
    d = np.max(np.abs(got - exact))
    assert 1e-6 < d < 0.2 * np.max(np.abs(exact)), d


def test_fp8_reading_with_exact_operands_is_exact():
    """Weights and inputs on the E4M3 grid with unit activation scales and power-of-two weight
    scales: the reading changes nothing."""
    cfg = dict(n_models=1, stacks=1, layers_per_stack=1, kernel=2, r_ch=4, s_ch=4, head_ch=4)
    off = workload.param_offsets(cfg)
    rng = np.random.default_rng(5)
    grid = _all_finite_e4m3()
    grid = grid[(np.abs(grid) >= 0.125) & (np.abs(grid) <= 1.75)]
    wb = rng.choice(grid, workload.param_count(cfg)).astype(np.float64)
    for b in ("H", "L"):
        o, shp = off[f"{b}.0.w_conv"]
        blk = wb[o:o + int(np.prod(shp))].reshape(shp[0], -1)
        blk[:, 0] = 1.75                     # row max |W| = 1.75: w_o = 1.75 / 448 = 2^-8
        wb[o:o + int(np.prod(shp))] = blk.ravel()
        o, _ = off[f"{b}.w_in"]
        wb[o:o + 4] = 1.0
        o, _ = off[f"{b}.b_in"]
        wb[o:o + 4] = 0.0
    xh = rng.choice(grid, (2, 32))
    xl = rng.choice(grid, (2, 32))
    amax = np.full((2, 1, 4), 448.0 / 16.0)  # s = 16 * 28 / 448 = 1
    got = oracle.forward_windows_q8(cfg, wb, amax, xh, xl, margin=16.0)
    exact = oracle.forward_windows(cfg, wb, xh, xl)
    np.testing.assert_allclose(got, exact, rtol=0, atol=1e-12)


def test_act_amax_matches_trace():
    cfg = workload.config("small", n_models=1)
    wb = workload.init_weights(cfg, seed=21, bias_std=0.1)[0]
    rng = np.random.default_rng(2)
    s = rng.standard_normal((2, 512))
    am = oracle.act_amax(cfg, wb, 1, s)
    want = np.zeros_like(am)
    for k in range(2):
        xs, _, _, _ = oracle.branch_trace(cfg, wb, 1, s[k])
        want = np.maximum(want, np.max(np.abs(xs[:-1]), axis=1))
    np.testing.assert_array_equal(am, want)
