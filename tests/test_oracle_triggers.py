"""Pins of the oracle's post-processing: stitching, peak finding, coincidence.

* find_peaks against SciPy's find_peaks (run as a library) on random and
  structured series, including plateaus, for several heights and widths;
* closed forms: a rectangle pulse of length n has width exactly n and
  prominence equal to its height; a symmetric triangle of height A and slope s
  has width A / s;
* coincidence against brute force over all tuples of peaks;
* stitching against an explicit index map on a ramp.
"""
import itertools

import numpy as np
import pytest

import oracle

scipy_signal = pytest.importorskip("scipy.signal")


def _series(rng, kind, n):
    if kind == "noise":
        return rng.random(n).astype(np.float32)
    if kind == "walk":
        return np.cumsum(rng.standard_normal(n)).astype(np.float32)
    if kind == "smooth":
        x = np.convolve(rng.standard_normal(n + 200), np.hanning(201), mode="valid")[:n]
        return (1 / (1 + np.exp(-x))).astype(np.float32)
    if kind == "plateau":     # heavy quantisation -> many flat runs
        return np.round(np.cumsum(rng.standard_normal(n)) * 0.7).astype(np.float32)
    raise ValueError(kind)


@pytest.mark.parametrize("kind", ["noise", "walk", "smooth", "plateau"])
def test_find_peaks_matches_scipy(kind):
    rng = np.random.default_rng(hash(kind) % 2**32)
    for trial in range(25):
        n = int(rng.integers(3, 3000))
        x = _series(rng, kind, n)
        thr = float(np.quantile(x, rng.choice([0.0, 0.5, 0.9])))
        mw = float(rng.choice([0.0, 1.5, 4.0, 20.0]))
        pk, h, pr, wd = oracle.find_peaks(x, thr, mw)
        ref, props = scipy_signal.find_peaks(x.astype(np.float64), height=thr, width=mw)
        np.testing.assert_array_equal(pk, ref)
        np.testing.assert_array_equal(h, props["peak_heights"])
        np.testing.assert_array_equal(pr, props["prominences"])
        np.testing.assert_array_equal(wd, props["widths"])


def test_rectangle_pulse_width_and_prominence():
    for a, n in [(10, 1), (10, 2), (37, 2048), (5, 4095)]:
        x = np.zeros(a + n + 10, dtype=np.float32)
        x[a:a + n] = 0.75
        pk, h, pr, wd = oracle.find_peaks(x, 0.5, 0.0)
        assert list(pk) == [a + (n - 1) // 2]
        assert pr[0] == 0.75 and h[0] == np.float32(0.75)
        assert wd[0] == float(n)
        # the minimum-width filter is inclusive
        assert len(oracle.find_peaks(x, 0.5, float(n))[0]) == 1
        assert len(oracle.find_peaks(x, 0.5, float(n) + 1e-9)[0]) == 0
        # the height filter is inclusive
        assert len(oracle.find_peaks(x, 0.75, 0.0)[0]) == 1
        assert len(oracle.find_peaks(x, 0.7500001, 0.0)[0]) == 0


def test_triangle_width_closed_form():
    slope = 1.0 / 64.0
    c = 500
    i = np.arange(1001)
    x = np.maximum(0.0, 1.0 - np.abs(i - c) * slope).astype(np.float32)
    pk, h, pr, wd = oracle.find_peaks(x, 0.0, 0.0)
    assert list(pk) == [c] and pr[0] == 1.0
    assert wd[0] == pytest.approx(1.0 / slope, abs=1e-12)


def test_edges_are_never_peaks():
    x = np.array([5, 1, 2, 1, 7], dtype=np.float32)
    pk, *_ = oracle.find_peaks(x, -1.0, 0.0)
    assert list(pk) == [2]
    assert len(oracle.find_peaks(np.array([1, 1, 1], dtype=np.float32), -1, 0)[0]) == 0
    assert len(oracle.find_peaks(np.array([1.0], dtype=np.float32), -1, 0)[0]) == 0


def _brute_coinc(lists, coinc):
    out = []
    for i0, p0 in enumerate(lists[0]):
        ok = False
        for combo in itertools.product(*lists[1:]):
            vals = (p0,) + combo
            if max(vals) - min(vals) <= coinc:
                ok = True
                break
        if ok:
            out.append(i0)
    return out


def test_coincidence_matches_brute_force():
    rng = np.random.default_rng(21)
    for trial in range(300):
        m = int(rng.integers(1, 5))
        lists = [np.sort(rng.choice(200, size=int(rng.integers(0, 7)), replace=False)) for _ in range(m)]
        coinc = int(rng.integers(0, 40))
        got = oracle.coincidence(lists, coinc)
        assert list(got) == _brute_coinc([list(l) for l in lists], coinc), (lists, coinc)


def test_coincidence_span_is_inclusive():
    assert list(oracle.coincidence([[100], [2148], [1000]], 2048)) == [0]
    assert list(oracle.coincidence([[100], [2149], [1000]], 2048)) == []
    # both sides of p0: span counts, not distance to p0
    assert list(oracle.coincidence([[3000], [1500], [4500]], 2048)) == []
    assert list(oracle.coincidence([[3000], [1500, 3100], [4500]], 2048)) == [0]


def test_stitch_index_map():
    W, stride, nw = 16, 6, 5
    prob = (np.arange(nw)[:, None] * 1000 + np.arange(W)[None, :]).astype(np.float32)
    s = oracle.stitch(prob, W, stride)
    assert s.shape[0] == (nw - 1) * stride + W
    for g in range(s.shape[0]):
        if g < W:
            w, p = 0, g
        else:
            w = (g - W) // stride + 1
            p = g - w * stride
        assert s[g] == prob[w, p]
        assert p >= W - stride or w == 0
