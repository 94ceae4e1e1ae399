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


@pytest.mark.parametrize("n", [5 * SEG, 5 * SEG + SEG // 2, 12 * SEG + 77])
def test_median_welch_matches_scipy(n):
    """Odd and even numbers of segments (the even median averages the two middle values)."""
    rng = np.random.default_rng(n + 1)
    x = rng.standard_normal(n) * 2.0 - 0.3
    f, p = ow.welch_psd(x, FS, SEG, average="median")
    fr, pr = scipy_signal.welch(x, fs=FS, window="hann", nperseg=SEG, noverlap=SEG // 2, detrend="constant",
                                scaling="density", return_onesided=True, average="median")
    np.testing.assert_allclose(p, pr, rtol=1e-10, atol=0)


@pytest.mark.parametrize("n,alpha", [(100, 0.5), (101, 0.25), (16, 1.0), (7, 0.1), (4096, 0.1), (50, 0.0)])
def test_tukey_matches_scipy(n, alpha):
    np.testing.assert_allclose(ow.tukey(n, alpha), scipy_signal.windows.tukey(n, alpha), rtol=0, atol=1e-14)


def test_median_bias_closed_form():
    # the median of n (odd) exponential(1) values has mean H_n - H_{(n-1)/2} = 1 - 1/2 + ... + 1/n: check the
    # bias against a Monte-Carlo mean of medians (within 5 standard errors)
    rng = np.random.default_rng(3)
    for n in (3, 9, 33):
        med = np.median(rng.exponential(1.0, size=(200000, n)), axis=1)
        assert abs(med.mean() - ow.median_bias(n)) < 5.0 * med.std() / np.sqrt(med.size)
        h = lambda m: sum(1.0 / k for k in range(1, m + 1))
        assert abs(ow.median_bias(n) - (h(n) - h((n - 1) // 2))) < 1e-14
    assert ow.median_bias(1) == 1.0 and ow.median_bias(2) == 1.0 and abs(ow.median_bias(4) - (1 - 0.5 + 1 / 3)) < 1e-15


def test_median_psd_robust_to_glitches():
    """White noise with a few loud sine-Gaussian glitches at 200 Hz: the mean-averaged Welch PSD is
    inflated in the glitch band, the median-averaged one stays at the noise level 2 sigma^2 / fs."""
    n = 256 * int(FS)
    rng = np.random.default_rng(11)
    x = rng.standard_normal(n)
    for c in (40, 120, 200):
        g = workload.sine_gaussian(200.0, 20.0, fs=int(FS))
        h = g.shape[0] // 2
        x[c * int(FS) - h:c * int(FS) + h + 1] += 40.0 * g
    f, pm = ow.welch_psd(x, FS, SEG, average="mean")
    _, pd = ow.welch_psd(x, FS, SEG, average="median")
    band = (f > 190.0) & (f < 210.0)
    level = 2.0 / FS
    assert pm[band].mean() > 1.5 * level
    assert abs(pd[band].mean() / level - 1.0) < 0.15
    quiet = (f > 600.0) & (f < 1600.0)
    assert abs(pd[quiet].mean() / level - 1.0) < 0.05


@pytest.mark.parametrize("average,alpha", [("median", 0.0), ("mean", 0.1), ("median", 0.1)])
def test_whitening_variants_flat_on_coloured_noise(average, alpha):
    n = 128 * int(FS)
    x = workload.coloured_noise(n, seed=77)
    y = ow.whiten(x, FS, 4 * SEG, average=average, tukey_alpha=alpha)
    assert abs(np.std(y) - 1.0) < 1e-12
    core = y[n // 8:-n // 8]                 # away from the tapered ends
    fy, py = ow.welch_psd(core / np.std(core), FS, SEG)
    flat = _band_means(fy, py, 20.0, 2000.0, 20) / (2.0 / FS)
    assert np.all(np.abs(flat - 1.0) < 0.08), flat
