"""FP64 whitening front end (TEST INFRASTRUCTURE ONLY, part of the oracle).

The paper (section "Materials and Methods", paragraph "Data preparation")
whitens strain with power spectral densities estimated from the data and then
normalises the standard deviation to one; it does not state the estimator.
The reading taken here, written out plainly in numpy FP64 (numpy's FFT is the
library primitive; nothing else is shared with the CUDA library):

  Welch PSD: segments of `seg` samples at 50 % overlap (segment s starts at
  s * seg/2; floor((n - seg/2) / (seg/2)) segments), each minus its own mean,
  times the periodic Hann window w[i] = 0.5 - 0.5 cos(2 pi i / seg); one-sided
  density S_k = c_k * mean_s |X_s[k]|^2 / (fs * sum(w^2)), c_k = 2 except at
  DC and Nyquist (1).
  Median variant (robust against loud short glitches, which the paper's data
  contain, section "Event Detection"): the median over segments of |X_s[k]|^2
  instead of the mean (the average of the two middle values for an even count),
  divided by the bias of the median of exponentially distributed values,
  1 - 1/2 + 1/3 - ... up to the largest odd number of terms <= n_seg.
  Whitening of a segment of n samples: X = rfft(x w_T) with w_T the Tukey
  window of taper fraction alpha (w_T = 1 for alpha = 0): a cosine taper over the
  first and last alpha (n - 1) / 2 samples, w_T[i] = 0.5 (1 + cos(pi (2 i /
  (alpha (n - 1)) - 1))) on the first; S interpolated linearly at f_k = k fs / n
  on the Welch grid j fs / seg; Y_k = X_k / sqrt(fs S(f_k) / 2), Y_k = 0 below
  f_low (15 Hz); y = irfft(Y); y / std(y).

Pinned (tests/test_oracle_whiten.py) against scipy.signal.welch (mean and
median averages) and scipy.signal.windows.tukey as libraries, the Parseval
closed form of a sinusoid, the statistics of whitened white and coloured
Gaussian noise, and the robustness of the median to injected glitches.
"""
from __future__ import annotations

import numpy as np


def hann_periodic(n: int) -> np.ndarray:
    i = np.arange(n, dtype=np.float64)
    return 0.5 - 0.5 * np.cos(2.0 * np.pi * i / n)


def median_bias(n: int) -> float:
    """Bias of the median of n exponentially distributed values: 1 - 1/2 + 1/3 - ..., over the largest
    odd number of terms not above n."""
    terms = n if n % 2 == 1 else n - 1
    return float(sum((-1.0) ** (i + 1) / i for i in range(1, terms + 1))) if terms > 0 else 1.0


def tukey(n: int, alpha: float) -> np.ndarray:
    """Tukey (tapered cosine) window of n samples with taper fraction alpha in [0, 1]."""
    w = np.ones(n, dtype=np.float64)
    if alpha <= 0.0 or n < 2:
        return w
    width = alpha * (n - 1) / 2.0
    i = np.arange(n, dtype=np.float64)
    lo = i < width
    w[lo] = 0.5 * (1.0 + np.cos(np.pi * (i[lo] / width - 1.0)))
    hi = i > (n - 1) - width
    w[hi] = 0.5 * (1.0 + np.cos(np.pi * ((n - 1 - i[hi]) / width - 1.0)))
    return w


def welch_psd(x: np.ndarray, fs: float, seg: int, average: str = "mean"):
    """(frequencies [seg/2 + 1], one-sided PSD [seg/2 + 1]) of x, FP64; average 'mean' or 'median'."""
    x = np.asarray(x, dtype=np.float64)
    n = x.shape[0]
    step = seg // 2
    n_seg = (n - step) // step
    if n_seg < 1:
        raise ValueError("signal shorter than one Welch segment")
    w = hann_periodic(seg)
    p = np.zeros((n_seg, seg // 2 + 1), dtype=np.float64)
    for s in range(n_seg):
        x_s = x[s * step:s * step + seg]
        X = np.fft.rfft((x_s - x_s.mean()) * w)
        p[s] = X.real ** 2 + X.imag ** 2
    c = np.full(seg // 2 + 1, 2.0)
    c[0] = 1.0
    c[-1] = 1.0
    if average == "mean":
        avg = p.sum(axis=0) / n_seg
    elif average == "median":
        avg = np.median(p, axis=0) / median_bias(n_seg)
    else:
        raise ValueError("average must be 'mean' or 'median'")
    psd = c * avg / (fs * np.sum(w * w))
    f = np.arange(seg // 2 + 1, dtype=np.float64) * fs / seg
    return f, psd


def whiten(x: np.ndarray, fs: float, seg: int, f_low: float = 15.0, average: str = "mean",
           tukey_alpha: float = 0.0) -> np.ndarray:
    """Whitened, unit-standard-deviation copy of x (FP64)."""
    x = np.asarray(x, dtype=np.float64)
    n = x.shape[0]
    fw, psd = welch_psd(x, fs, seg, average)
    X = np.fft.rfft(x * tukey(n, tukey_alpha))
    f = np.arange(X.shape[0], dtype=np.float64) * fs / n
    s = np.interp(f, fw, psd)
    Y = X / np.sqrt(fs * s / 2.0)
    Y[f < f_low] = 0.0
    y = np.fft.irfft(Y, n)
    return y / np.std(y)
