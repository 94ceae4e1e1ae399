"""The sine-Gaussian glitch generator of the synthetic inputs: each glitch lands
in exactly one detector, away from the chirp mergers, with the closed-form
shape exp(-t^2/tau^2) sin(2 pi f0 t + phi), tau = Q / (sqrt(2) pi f0), and a
whitened norm equal to the requested SNR (whitening with the analytic noise
spectrum the streams are drawn from)."""
import math

import numpy as np

import workload


def test_sine_gaussian_closed_form():
    f0, q = 120.0, 9.0
    g = workload.sine_gaussian(f0, q, fs=4096, phase0=0.3)
    tau = q / (math.sqrt(2.0) * math.pi * f0)
    half = len(g) // 2
    t = (np.arange(len(g)) - half) / 4096.0
    np.testing.assert_allclose(g, np.exp(-(t / tau) ** 2) * np.sin(2 * math.pi * f0 * t + 0.3), atol=1e-15)
    assert abs(t[-1] - 4 * tau) < 1.0 / 4096 + 1e-12      # spans +-4 tau


def test_glitches_one_detector_away_from_chirps_and_scaled():
    n = 120 * 4096
    xh = np.zeros(n)
    xl = np.zeros(n)
    mergers = [30 * 4096, 70 * 4096]
    gl = workload.add_glitches(xh, xl, 6, seed=3, snr_range=(20.0, 40.0), avoid=mergers, guard=4 * 4096)
    assert len(gl) == 6
    for c, det, snr, f0, q, ph in gl:
        assert all(abs(c - m) >= 4 * 4096 for m in mergers)
        other = xl if det == 0 else xh
        mine = xh if det == 0 else xl
        h = workload.sine_gaussian(f0, q, fs=4096, phase0=ph)
        half = len(h) // 2
        assert not np.any(other[c - half:c + half + 1])       # the other detector untouched
        seg = mine[c - half:c + half + 1]
        # the stored glitch is the closed form times one scale; its whitened norm is the SNR
        scale = float(np.dot(seg, h) / np.dot(h, h))
        np.testing.assert_allclose(seg, scale * h, rtol=0, atol=1e-12 * abs(scale) * 10 + 1e-300)
        pad = 8192
        m = len(h) + pad
        hf = np.fft.rfft(np.concatenate([seg, np.zeros(pad)]))
        f = np.fft.rfftfreq(m, 1.0 / 4096)
        wf = hf / np.sqrt(4096 * workload.aligo_like_psd(f) * 1e42 / 2.0)
        wf[f < 15.0] = 0.0
        assert abs(math.sqrt(float(np.sum(np.fft.irfft(wf, m) ** 2))) - snr) < 1e-6 * snr
