"""Threshold sweep of the trigger statistics (gwe_trigger_sweep) against the
oracle's peak finding and coincidence run once per threshold (section
"Statistical Analysis": ROC and false-alarm curves from sweeping the height
threshold over [0, 0.9998]).  Counts must be equal exactly: per slide, the
number of ensemble triggers and of each model's kept peaks at every
threshold."""
import numpy as np
import pytest

import oracle
from gpu_util import require_gpu, smooth_prob

pytestmark = pytest.mark.gpu


def _oracle_counts(prob, W, stride, thrs, mw, coinc):
    ns, nm = prob.shape[0], prob.shape[1]
    ens = np.zeros((ns, len(thrs)), dtype=np.int64)
    mod = np.zeros((ns, nm, len(thrs)), dtype=np.int64)
    for k, t in enumerate(thrs):
        per_model, e = oracle.triggers(prob, W, stride, float(t), mw, coinc)
        for s in range(ns):
            ens[s, k] = len(e[s])
            for m in range(nm):
                mod[s, m, k] = len(per_model[s][m][0])
    return ens, mod


def _check(prob, W, stride, thrs, mw, coinc):
    import torch
    import paper_2201_11133_gb300 as gwe
    dev = require_gpu()
    ns, nm, nw, _ = prob.shape
    thrs = np.asarray(thrs, dtype=np.float32)
    ens, mod = gwe.gwe_trigger_sweep(torch.from_numpy(prob).to(dev), nm, ns, nw, W, stride, thrs, mw, coinc)
    ens_ref, mod_ref = _oracle_counts(prob, W, stride, thrs, mw, coinc)
    np.testing.assert_array_equal(mod, mod_ref)
    np.testing.assert_array_equal(ens, ens_ref)
    # counts never grow with the threshold
    assert np.all(np.diff(ens, axis=-1) <= 0) and np.all(np.diff(mod, axis=-1) <= 0)
    return ens, mod


@pytest.mark.parametrize("mw", [0.0, 64.0, 300.0])
def test_sweep_matches_per_threshold_oracle(mw):
    rng = np.random.default_rng(17)
    W, stride = 4096, 2048
    prob = smooth_prob(rng, (3, 4, 7, W))
    thrs = np.quantile(prob, [0.0, 0.2, 0.5, 0.6, 0.7, 0.8, 0.9, 0.95, 0.99, 0.999])
    ens, _ = _check(prob, W, stride, thrs, mw, 2048)
    assert ens[:, 0].sum() > 0


def test_sweep_paper_grid_and_duplicates():
    """The paper's grid [0, 0.9998] (uniform steps plus the top end), repeated thresholds, one model
    (the ensemble triggers are then model 0's peaks) and a zero coincidence span."""
    rng = np.random.default_rng(18)
    W, stride = 1024, 512
    prob = smooth_prob(rng, (2, 3, 9, W), width=15)
    thrs = np.concatenate([np.linspace(0.0, 0.99, 34), [0.99, 0.995, 0.9998]])
    _check(prob, W, stride, thrs, 16.0, 256)
    _check(prob[:, :1], W, stride, thrs, 0.0, 256)
    _check(prob, W, stride, thrs, 0.0, 0)


def test_sweep_plateaus_long_walks_and_edges():
    rng = np.random.default_rng(19)
    W, stride = 4096, 1024
    nw = 10
    walk = np.cumsum(rng.standard_normal((2, 3, nw * W)), axis=-1)
    walk = np.round(walk * 0.05) / 50.0
    prob = (1 / (1 + np.exp(-walk))).astype(np.float32).reshape(2, 3, nw, W)
    _check(prob, W, stride, np.quantile(prob, np.linspace(0.05, 0.95, 12)), 10.0, 512)
    flat = np.full((1, 2, 3, 256), 0.25, dtype=np.float32)
    ens, mod = _check(flat, 256, 128, [0.0, 0.5], 0.0, 64)
    assert ens.sum() == 0 and mod.sum() == 0


def test_sweep_segments_sum_over_segments():
    import torch
    import paper_2201_11133_gb300 as gwe
    dev = require_gpu()
    rng = np.random.default_rng(20)
    W, stride = 1024, 512
    seg_len = [W + 3 * stride, W, 5 * W + 7]
    nws = [gwe.gwe_n_windows(n, W, stride) for n in seg_len]
    prob = smooth_prob(rng, (2, 3, sum(nws), W), width=15)
    thrs = np.asarray(np.quantile(prob, [0.1, 0.5, 0.9]), dtype=np.float32)
    ens, mod = gwe.gwe_trigger_sweep_segments(torch.from_numpy(prob).to(dev), 3, 2, seg_len, W, stride, thrs, 8.0, 128)
    e_ref = np.zeros_like(ens)
    m_ref = np.zeros_like(mod)
    o = 0
    for g, nw in enumerate(nws):
        e, m = _oracle_counts(np.ascontiguousarray(prob[:, :, o:o + nw]), W, stride, thrs, 8.0, 128)
        e_ref += e
        m_ref += m
        o += nw
    np.testing.assert_array_equal(ens, e_ref)
    np.testing.assert_array_equal(mod, m_ref)


def test_sweep_argument_errors():
    import torch
    import paper_2201_11133_gb300 as gwe
    dev = require_gpu()
    prob = torch.zeros((1, 1, 2, 256), device=dev)
    for thrs in ([0.5, 0.2], [float("nan")], []):
        with pytest.raises(gwe.GweError) as ei:
            gwe.gwe_trigger_sweep(prob, 1, 1, 2, 256, 128, thrs, 0.0, 10)
        assert ei.value.status == 1
