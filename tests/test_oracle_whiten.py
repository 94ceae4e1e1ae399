"""Pins of the oracle's whitening front end.

* Welch PSD against scipy.signal.welch run as a library (periodic Hann window,
  50 % overlap, constant detrend, one-sided density);
* a sinusoid on a frequency bin: the PSD integrates to A^2/2 exactly and the
  Hann leakage into the neighbouring bins is exactly a quarter;
* coloured Gaussian noise drawn from the analytic spectrum: the Welch estimate
  matches that spectrum, and the whitened output is flat at the unit-variance
  level 2/fs with unit standard deviation;
* whitened white noise of any variance is flat at 2/fs.
"""
import numpy as np
import pytest

import workload
from oracle import whiten as ow

scipy_signal = pytest.importorskip("scipy.signal")

FS = 4096.0
SEG = 4096


def _band_means(f, p, lo, hi, nb):
    edges = np.linspace(lo, hi, nb + 1)
    return np.array([np.mean(p[(f >= a) & (f < b)]) for a, b in zip(edges[:-1], edges[1:])])


@pytest.mark.parametrize("n", [SEG, 3 * SEG // 2 + 7, 10 * SEG + 123])
def test_welch_matches_scipy(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) * 3.0 + 0.7
    f, p = ow.welch_psd(x, FS, SEG)
    fr, pr = scipy_signal.welch(x, fs=FS, window="hann", nperseg=SEG, noverlap=SEG // 2, detrend="constant",
                                scaling="density", return_onesided=True, average="mean")
    np.testing.assert_allclose(f, fr, rtol=0, atol=1e-12)
    np.testing.assert_allclose(p, pr, rtol=1e-10, atol=0)


def test_sinusoid_power_and_hann_leakage():
    A, k0 = 2.5, 300
    n = 8 * SEG
    t = np.arange(n) / FS
    x = A * np.sin(2 * np.pi * (k0 * FS / SEG) * t)
    f, p = ow.welch_psd(x, FS, SEG)
    assert int(np.argmax(p)) == k0
    np.testing.assert_allclose(np.sum(p) * FS / SEG, A * A / 2, rtol=1e-10)
    np.testing.assert_allclose(p[k0 - 1] / p[k0], 0.25, rtol=1e-9)
    np.testing.assert_allclose(p[k0 + 1] / p[k0], 0.25, rtol=1e-9)


def test_coloured_noise_psd_and_whitening():
    n = 256 * int(FS)
    x = workload.coloured_noise(n, seed=1234)
    f, p = ow.welch_psd(x, FS, 4 * SEG)
    ref = workload.aligo_like_psd(f) * 1e42
    ratio = _band_means(f, p / ref, 20.0, 1800.0, 40)
    assert np.all(np.abs(ratio - 1.0) < 0.05), ratio
    y = ow.whiten(x, FS, 4 * SEG)
    assert abs(np.std(y) - 1.0) < 1e-12
    assert abs(np.mean(y)) < 1e-10
    fy, py = ow.welch_psd(y, FS, SEG)
    flat = _band_means(fy, py, 20.0, 2000.0, 40) / (2.0 / FS)
    assert np.all(np.abs(flat - 1.0) < 0.06), flat


@pytest.mark.parametrize("sigma", [0.01, 7.0])
def test_whitened_white_noise_is_flat(sigma):
    n = 128 * int(FS)
    x = np.random.default_rng(5).standard_normal(n) * sigma
    y = ow.whiten(x, FS, SEG)
    fy, py = ow.welch_psd(y, FS, SEG)
    flat = _band_means(fy, py, 20.0, 2000.0, 20) / (2.0 / FS)
    assert np.all(np.abs(flat - 1.0) < 0.06), flat
    low = np.mean(py[(fy > 2.0) & (fy < 12.0)]) / (2.0 / FS)
    assert low < 0.05                      # removed below 15 Hz
