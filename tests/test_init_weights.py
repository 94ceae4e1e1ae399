"""Seeded random initialisation of the library (gwe_init_weights, host only).

The generator is Philox4x64-10 (Salmon et al., SC 2011), pinned against
numpy's own Philox bit generator (a library implementation of the same
published function); the weights are pinned against a statement of the
documented transform on numpy's stream, and their statistics against the
N(0, 1/fan_in) law of the paper's random initialisation ("AI ensemble
construction": members differ in their random initialisation)."""
import math

import numpy as np

import paper_2201_11133_gb300 as gwe
import workload

MASK = (1 << 64) - 1


def _numpy_blocks(key, n_blocks):
    # numpy's Philox advances the counter before each block: start one below zero
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=np.array([MASK] * 4, dtype=np.uint64))
    return bg.random_raw(4 * n_blocks).reshape(n_blocks, 4)


def test_philox_matches_numpy_philox():
    gwe.build()
    for key in ([0, 0], [5, 7], [2 ** 63 + 11, 12345678901234567]):
        ref = _numpy_blocks(key, 64)
        for c in (0, 1, 2, 17, 63):
            got = gwe.gwe_philox4x64_10([c, 0, 0, 0], key)
            np.testing.assert_array_equal(got, ref[c])
    # a counter with high words set (carry propagation is numpy's, the function is the same)
    bg = np.random.Philox(key=np.array([3, 4], dtype=np.uint64),
                          counter=np.array([MASK, 6, 7, 8], dtype=np.uint64))
    np.testing.assert_array_equal(gwe.gwe_philox4x64_10([0, 7, 7, 8], [3, 4]), bg.random_raw(4))


def test_init_weights_is_the_documented_transform():
    cfg = workload.config("small", n_models=2)
    seed = 4242
    w = gwe.gwe_init_weights(cfg, seed)
    P = gwe.gwe_param_count(cfg)
    assert w.shape == (2, P)
    for m in range(2):
        blocks = _numpy_blocks([seed, m], (P + 1) // 2)
        e = np.arange(P)
        r = blocks[e // 2]
        j = e % 2
        u1 = ((r[e, 2 * j] >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0 ** -53
        u2 = (r[e, 2 * j + 1] >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
        z = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
        o = 0
        for _, shape, fan_in in workload.param_layout(cfg):
            n = int(np.prod(shape))
            if fan_in > 0:
                exp = (z[o:o + n] / math.sqrt(fan_in)).astype(np.float32)
                np.testing.assert_allclose(w[m, o:o + n], exp, rtol=2e-7, atol=1e-9)
            else:
                assert not np.any(w[m, o:o + n])
            o += n


def test_init_weights_statistics_and_seeds():
    cfg = workload.config("ensemble")
    w = gwe.gwe_init_weights(cfg, 7)
    assert w.dtype == np.float32 and np.all(np.isfinite(w))
    # members and seeds differ, the same seed repeats
    assert not np.array_equal(w[0], w[1])
    assert not np.array_equal(w[0], gwe.gwe_init_weights(cfg, 8)[0])
    np.testing.assert_array_equal(w, gwe.gwe_init_weights(cfg, 7))
    # every weight tensor of member 0 ~ N(0, 1/fan_in): mean and variance within 6 standard errors
    o = 0
    for name, shape, fan_in in workload.param_layout(cfg):
        n = int(np.prod(shape))
        x = w[0, o:o + n].astype(np.float64)
        if fan_in > 0 and n >= 64:
            v = x * math.sqrt(fan_in)
            assert abs(v.mean()) <= 6.0 / math.sqrt(n), name
            assert abs(v.var() - 1.0) <= 6.0 * math.sqrt(2.0 / n), name
        o += n
    # the whole blob: a standardised sample passes a Kolmogorov-Smirnov test against N(0, 1)
    from scipy import stats
    z = []
    o = 0
    for name, shape, fan_in in workload.param_layout(cfg):
        n = int(np.prod(shape))
        if fan_in > 0:
            z.append(w[0, o:o + n].astype(np.float64) * math.sqrt(fan_in))
        o += n
    z = np.concatenate(z)
    assert stats.kstest(z[:200000], "norm").pvalue > 1e-4
