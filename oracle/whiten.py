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
  Whitening of a segment of n samples: X = rfft(x); S interpolated linearly
  at f_k = k fs / n on the Welch grid j fs / seg; Y_k = X_k / sqrt(fs S(f_k) / 2),
  Y_k = 0 below f_low (15 Hz); y = irfft(Y); y / std(y).

Pinned (tests/test_oracle_whiten.py) against scipy.signal.welch as a library,
the Parseval closed form of a sinusoid, and the statistics of whitened white
and coloured Gaussian noise.
"""
from __future__ import annotations

import numpy as np


def hann_periodic(n: int) -> np.ndarray:
    i = np.arange(n, dtype=np.float64)
    return 0.5 - 0.5 * np.cos(2.0 * np.pi * i / n)


def welch_psd(x: np.ndarray, fs: float, seg: int):
    """(frequencies [seg/2 + 1], one-sided PSD [seg/2 + 1]) of x, FP64."""
    x = np.asarray(x, dtype=np.float64)
    n = x.shape[0]
    step = seg // 2
    n_seg = (n - step) // step
    if n_seg < 1:
        raise ValueError("signal shorter than one Welch segment")
    w = hann_periodic(seg)
    acc = np.zeros(seg // 2 + 1, dtype=np.float64)
    for s in range(n_seg):
        x_s = x[s * step:s * step + seg]
        X = np.fft.rfft((x_s - x_s.mean()) * w)
        acc += X.real ** 2 + X.imag ** 2
    c = np.full(seg // 2 + 1, 2.0)
    c[0] = 1.0
    c[-1] = 1.0
    psd = c * acc / (n_seg * fs * np.sum(w * w))
    f = np.arange(seg // 2 + 1, dtype=np.float64) * fs / seg
    return f, psd


def whiten(x: np.ndarray, fs: float, seg: int, f_low: float = 15.0) -> np.ndarray:
    """Whitened, unit-standard-deviation copy of x (FP64)."""
    x = np.asarray(x, dtype=np.float64)
    n = x.shape[0]
    fw, psd = welch_psd(x, fs, seg)
    X = np.fft.rfft(x)
    f = np.arange(X.shape[0], dtype=np.float64) * fs / n
    s = np.interp(f, fw, psd)
    Y = X / np.sqrt(fs * s / 2.0)
    Y[f < f_low] = 0.0
    y = np.fft.irfft(Y, n)
    return y / np.std(y)
