"""Trigger extraction on the device against the oracle, bit-exact given
identical probabilities: per-model peaks (index, height, prominence, width)
and ensemble coincidences, over several slides and models."""
import numpy as np
import pytest

import oracle
from gpu_util import require_gpu, smooth_prob

pytestmark = pytest.mark.gpu


def _compare(prob, W, stride, thr, mw, coinc):
    import torch
    import paper_2201_11133_gb300 as gwe
    dev = require_gpu()
    ns, nm, nw, _ = prob.shape
    recs = gwe.gwe_triggers(torch.from_numpy(prob).to(dev), nm, ns, nw, W, stride, thr, mw, coinc,
                            flags=gwe.GWE_TRIG_PER_MODEL)
    per_model, ens = oracle.triggers(prob, W, stride, thr, mw, coinc)
    n_ref = 0
    for s in range(ns):
        for m in range(nm):
            sel = recs[(recs["slide"] == s) & (recs["model"] == m)]
            idx, h, pr, wd = per_model[s][m]
            n_ref += len(idx)
            np.testing.assert_array_equal(sel["index"], idx)
            np.testing.assert_array_equal(sel["height"], h)
            np.testing.assert_array_equal(sel["prominence"], pr)
            np.testing.assert_array_equal(sel["width"], wd)
        e = recs[(recs["slide"] == s) & (recs["model"] == -1)]["index"]
        np.testing.assert_array_equal(e, ens[s])
        n_ref += len(ens[s])
    assert len(recs) == n_ref
    # records come sorted by (slide, model with ensemble last, index)
    return recs


@pytest.mark.parametrize("mw", [0.0, 64.0, 300.0])
def test_triggers_match_oracle_bit_exact(mw):
    rng = np.random.default_rng(7)
    W, stride = 4096, 2048
    prob = smooth_prob(rng, (3, 4, 9, W))
    thr = float(np.quantile(prob, 0.6))
    recs = _compare(prob, W, stride, thr, mw, 2048)
    assert len(recs) > 0


def test_triggers_plateaus_and_long_walks():
    """Quantised series: long plateaus and bases far from their peaks (block-skipping paths)."""
    rng = np.random.default_rng(8)
    W, stride = 4096, 1024
    nw = 12
    walk = np.cumsum(rng.standard_normal((2, 2, nw * W)), axis=-1)
    walk = np.round(walk * 0.05) / 50.0
    prob = (1 / (1 + np.exp(-walk))).astype(np.float32).reshape(2, 2, nw, W)
    _compare(prob, W, stride, float(np.quantile(prob, 0.3)), 10.0, 512)


def test_triggers_edge_cases():
    W, stride = 256, 128
    flat = np.full((1, 2, 3, W), 0.25, dtype=np.float32)      # no local maxima
    assert len(_compare(flat, W, stride, 0.0, 0.0, 64)) == 0
    one = np.random.default_rng(9).random((1, 1, 1, W)).astype(np.float32)   # single window
    _compare(one, W, stride, 0.5, 0.0, 0)
    rng = np.random.default_rng(10)
    p = smooth_prob(rng, (2, 3, 5, W), width=31)
    _compare(p, W, stride, 0.0, 1e9, 64)                     # width filter removes everything


def test_triggers_capacity_error():
    import torch
    import paper_2201_11133_gb300 as gwe
    dev = require_gpu()
    rng = np.random.default_rng(11)
    prob = rng.random((1, 1, 4, 512)).astype(np.float32)
    with pytest.raises(gwe.GweError) as ei:
        gwe.gwe_triggers(torch.from_numpy(prob).to(dev), 1, 1, 4, 512, 256, 0.0, 0.0, 10, cap=3)
    assert ei.value.status == 6


def test_triggers_superblock_walks():
    """A long quantised random walk (160 windows, 41 superblocks of 8192 samples): prominence and
    width walks that cross many blocks and superblocks, with equal minima in different blocks and
    superblocks (first / last argmin rules)."""
    rng = np.random.default_rng(12)
    W, stride = 4096, 2048
    nw = 160
    walk = np.cumsum(rng.standard_normal((1, 2, nw * W)), axis=-1)
    walk = np.round(walk * 0.02) / 20.0
    prob = (1 / (1 + np.exp(-walk / 8.0))).astype(np.float32).reshape(1, 2, nw, W)
    recs = _compare(prob, W, stride, float(np.quantile(prob, 0.2)), 0.0, 4096)
    assert len(recs) > 0
