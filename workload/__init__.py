"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module draws random numbers and synthesises signals; it holds none of the
detector's arithmetic (no network, no whitening estimate, no peak finding).

* Model configurations (layer counts, widths, dilations) for the workloads the
  library is measured on.  The paper states none of these sizes ("AI
  architecture" section); they are the workload's own choices.
* Weight blobs: every weight ~ N(0, 1/fan_in) with fan_in = C_in * kernel;
  biases 0 unless ``bias_std`` is given (tests use non-zero biases so that bias
  handling is exercised).  numpy PCG64, model m seeded with seed + m.
* Strain: whitened-domain inputs, i.e. i.i.d. N(0, 1) noise plus leading-order
  (Newtonian) chirps that were coloured by an analytic advanced-LIGO-like noise
  spectrum and then divided by it again (the whitened template), scaled to a
  target signal-to-noise ratio.  This stands in for the paper's whitened GWOSC
  strain with SEOBNRv3 injections, which are not available.
* Coloured (unwhitened) noise from the same analytic spectrum for the
  whitening front end.
"""
from __future__ import annotations

import math

import numpy as np

FS = 4096            # sample rate (Hz) of the paper's strain
WINDOW = 4096        # 1 s windows
STRIDE = 2048        # 0.5 s stride between windows
MSUN_S = 4.925490947e-6   # G * M_sun / c^3 in seconds

CONFIGS = {
    # 1 model, 8 layers (dilations 1..128), R = S = Hc = 32, batch of 8 windows
    "small": dict(n_models=1, stacks=1, layers_per_stack=8, kernel=2, r_ch=32, s_ch=32, head_ch=32),
    # 4-model ensemble, 3 stacks x dilations 1..512 (30 layers), R=64, S=128, Hc=256
    "ensemble": dict(n_models=4, stacks=3, layers_per_stack=10, kernel=2, r_ch=64, s_ch=128, head_ch=256),
    # tiny network for finite-difference gradient checks
    "tiny": dict(n_models=1, stacks=2, layers_per_stack=3, kernel=2, r_ch=2, s_ch=2, head_ch=2),
}


def config(name: str, **over) -> dict:
    c = dict(CONFIGS[name])
    c.update(over)
    return c


def n_layers(cfg) -> int:
    return int(cfg["stacks"]) * int(cfg["layers_per_stack"])


def dilations(cfg):
    return [1 << (l % int(cfg["layers_per_stack"])) for l in range(n_layers(cfg))]


def receptive_field(cfg) -> int:
    k = int(cfg["kernel"])
    return 1 + (k - 1) * sum(dilations(cfg))


def param_layout(cfg):
    """Ordered (name, shape, fan_in) entries of one model's blob (layout documented in include/gwe.h)."""
    R, S, Hc, K = int(cfg["r_ch"]), int(cfg["s_ch"]), int(cfg["head_ch"]), int(cfg["kernel"])
    ent = []
    for b in ("H", "L"):
        ent.append((f"{b}.w_in", (R,), 1))
        ent.append((f"{b}.b_in", (R,), 0))
        for l in range(n_layers(cfg)):
            ent.append((f"{b}.{l}.w_conv", (2 * R, K, R), R * K))
            ent.append((f"{b}.{l}.b_conv", (2 * R,), 0))
            ent.append((f"{b}.{l}.w_res", (R, R), R))
            ent.append((f"{b}.{l}.b_res", (R,), 0))
            ent.append((f"{b}.{l}.w_skip", (S, R), R))
            ent.append((f"{b}.{l}.b_skip", (S,), 0))
    ent.append(("w_h1", (Hc, 2 * S), 2 * S))
    ent.append(("b_h1", (Hc,), 0))
    ent.append(("w_h2", (Hc,), Hc))
    ent.append(("b_h2", (1,), 0))
    return ent


def param_count(cfg) -> int:
    return int(sum(int(np.prod(s)) for _, s, _ in param_layout(cfg)))


def param_offsets(cfg) -> dict:
    off, o = {}, 0
    for name, shape, _ in param_layout(cfg):
        n = int(np.prod(shape))
        off[name] = (o, shape)
        o += n
    return off


def init_weights(cfg, seed: int = 3000, bias_std: float = 0.0) -> np.ndarray:
    """float32 [n_models, P]: weights N(0, 1/fan_in), biases N(0, bias_std^2) (0 by default)."""
    nm = int(cfg["n_models"])
    P = param_count(cfg)
    out = np.zeros((nm, P), dtype=np.float32)
    for m in range(nm):
        rng = np.random.Generator(np.random.PCG64(seed + m))
        o = 0
        for _, shape, fan_in in param_layout(cfg):
            n = int(np.prod(shape))
            if fan_in > 0:
                out[m, o:o + n] = rng.standard_normal(n) / math.sqrt(fan_in)
            elif bias_std > 0:
                out[m, o:o + n] = rng.standard_normal(n) * bias_std
            o += n
    return out


# ---------------------------------------------------------------------------
# Noise spectrum and chirps
# ---------------------------------------------------------------------------

def aligo_like_psd(f: np.ndarray) -> np.ndarray:
    """One-sided analytic advanced-LIGO-like noise PSD (1/Hz); held flat below 10 Hz.

    Zero-detuned high-power style analytic fit with x = f / 215 Hz and
    S0 = 1e-49 / Hz.  Only its shape matters here (a seismic wall, a bucket near
    200 Hz and a rise from shot noise)."""
    f = np.maximum(np.asarray(f, dtype=np.float64), 10.0)
    x = f / 215.0
    return 1e-49 * (x ** -4.14 - 5.0 * x ** -2 + 111.0 * (1.0 - x ** 2 + 0.5 * x ** 4) / (1.0 + 0.5 * x ** 2))


def newtonian_chirp(mchirp_msun: float, n_before: int, fs: int = FS, f_low: float = 20.0,
                    phase0: float = 0.0) -> np.ndarray:
    """Leading-order inspiral ending at the innermost stable circular orbit.

    Returns n_before + 1 samples; the last one is the merger sample.  With
    tau the time to merger: f(tau) = (5 / (256 tau))^(3/8) (G Mc / c^3)^(-5/8) / pi,
    phase = -2 (tau / (5 G Mc / c^3))^(5/8), amplitude ~ f^(2/3); the equal-mass
    total mass M = 2^(6/5) Mc sets f_isco = 1 / (6^(3/2) pi G M / c^3)."""
    mc = mchirp_msun * MSUN_S
    mtot = 2.0 ** 1.2 * mc
    f_isco = 1.0 / (6.0 ** 1.5 * math.pi * mtot)
    tau_of_f = lambda f: (5.0 / 256.0) * mc ** (-5.0 / 3.0) * (math.pi * f) ** (-8.0 / 3.0)
    tau_isco = tau_of_f(f_isco)
    tau_low = tau_of_f(f_low)
    t = np.arange(n_before, -1, -1, dtype=np.float64) / fs + tau_isco   # time to coalescence
    f = (5.0 / (256.0 * t)) ** 0.375 * mc ** (-0.625) / math.pi
    phi = -2.0 * (t / (5.0 * mc)) ** 0.625 + phase0
    h = f ** (2.0 / 3.0) * np.cos(phi)
    h[t > tau_low] = 0.0
    # smooth turn-on over the first 0.1 s of the band to avoid a step
    ramp = np.clip((tau_low - t) / 0.1, 0.0, 1.0)
    return h * (0.5 - 0.5 * np.cos(math.pi * ramp))


def whitened_template(mchirp_msun: float, n_before: int, fs: int = FS, phase0: float = 0.0,
                      pad: int = 8192) -> np.ndarray:
    """Chirp as seen in whitened data (unit-variance noise): divide its spectrum by sqrt(PSD).

    Returns n_before + 1 samples ending at the merger, unnormalised."""
    h = newtonian_chirp(mchirp_msun, n_before + pad, fs=fs, phase0=phase0)
    n = h.shape[0] + pad
    hf = np.fft.rfft(np.concatenate([h, np.zeros(pad)]))
    f = np.fft.rfftfreq(n, 1.0 / fs)
    w = hf / np.sqrt(aligo_like_psd(f))
    w[f < 15.0] = 0.0
    hw = np.fft.irfft(w, n)[:h.shape[0]]
    return hw[-(n_before + 1):]


def inject(x: np.ndarray, merger: int, mchirp: float, snr: float, phase0: float = 0.0) -> None:
    """Add a whitened chirp with merger at sample `merger`, scaled so sqrt(sum h_w^2) = snr."""
    n_before = min(merger, 6 * FS)
    hw = whitened_template(mchirp, n_before, phase0=phase0)
    norm = math.sqrt(float(np.sum(hw * hw)))
    if norm > 0:
        hw = hw * (snr / norm)
    x[merger - n_before:merger + 1] += hw.astype(x.dtype)


def small_batch(seed: int = 1000, B: int = 8, W: int = WINDOW, chirp_windows=(2, 5)):
    """Batch of B independent whitened windows per detector (float32 [B, W] each).

    Windows in `chirp_windows` carry a chirp: chirp mass U[5, 30] Msun, network
    SNR 10 (SNR / sqrt(2) per detector), merger at a uniform position in
    [W/2, W-1], Livingston delayed by U[-10, 10] ms with an independent phase."""
    rng = np.random.Generator(np.random.PCG64(seed))
    xh = rng.standard_normal((B, W)).astype(np.float32)
    xl = rng.standard_normal((B, W)).astype(np.float32)
    meta = []
    for b in chirp_windows:
        if b >= B:
            continue
        mc = rng.uniform(5.0, 30.0)
        tm = int(rng.integers(W // 2, W))
        dt = int(round(rng.uniform(-0.010, 0.010) * FS))
        ph = rng.uniform(0, 2 * math.pi)
        inject(xh[b], tm, mc, 10.0 / math.sqrt(2.0))
        tl = min(max(tm + dt, 0), W - 1)
        inject(xl[b], tl, mc, 10.0 / math.sqrt(2.0), phase0=ph)
        meta.append((b, tm, mc))
    return xh, xl, meta


def stream(n: int, seed: int = 1000, n_inj: int = 0, snr_range=(6.0, 20.0), mc_range=(5.0, 30.0),
           min_gap: int = 2 * FS):
    """Two whitened detector streams of n samples (float32) with n_inj chirps.

    Mergers are uniform over the stream and at least `min_gap` samples apart;
    network SNR U[snr_range], chirp mass U[mc_range]."""
    rng_h = np.random.Generator(np.random.PCG64(seed))
    rng_l = np.random.Generator(np.random.PCG64(seed + 1))
    xh = rng_h.standard_normal(n, dtype=np.float32)
    xl = rng_l.standard_normal(n, dtype=np.float32)
    rng = np.random.Generator(np.random.PCG64(seed + 1000))
    mergers = []
    lo = 6 * FS
    if n_inj > 0 and n > lo + 2 * FS:
        slots = np.sort(rng.choice(np.arange(lo, n - FS, min_gap), size=n_inj, replace=False))
        for tm in slots:
            mc = rng.uniform(*mc_range)
            snr = rng.uniform(*snr_range)
            dt = int(round(rng.uniform(-0.010, 0.010) * FS))
            ph = rng.uniform(0, 2 * math.pi)
            inject(xh, int(tm), mc, snr / math.sqrt(2.0))
            inject(xl, int(tm) + dt, mc, snr / math.sqrt(2.0), phase0=ph)
            mergers.append(int(tm))
    return xh, xl, mergers


def training_batch(B: int = 256, W: int = WINDOW, seed: int = 2000, frac_signal: float = 0.5,
                   mc_range=(5.0, 50.0), snr_range=(5.0, 25.0), merger_range=(1024, WINDOW - 1)):
    """(xh, xl, y): B windows per detector and per-sample labels.

    Labels: every sample up to and including the merger is 1 ("waveform"),
    later samples 0 ("noise"); noise-only windows are 0 everywhere."""
    rng = np.random.Generator(np.random.PCG64(seed))
    xh = rng.standard_normal((B, W)).astype(np.float32)
    xl = rng.standard_normal((B, W)).astype(np.float32)
    y = np.zeros((B, W), dtype=np.float32)
    n_sig = int(round(B * frac_signal))
    for b in range(n_sig):
        mc = rng.uniform(*mc_range)
        snr = rng.uniform(*snr_range)
        tm = int(rng.integers(merger_range[0], merger_range[1] + 1))
        dt = int(round(rng.uniform(-0.010, 0.010) * FS))
        ph = rng.uniform(0, 2 * math.pi)
        inject(xh[b], tm, mc, snr / math.sqrt(2.0))
        inject(xl[b], min(max(tm + dt, 0), W - 1), mc, snr / math.sqrt(2.0), phase0=ph)
        y[b, :tm + 1] = 1.0
    return xh, xl, y


def coloured_noise(n: int, seed: int = 1000, fs: int = FS) -> np.ndarray:
    """Gaussian noise of n samples with one-sided PSD aligo_like_psd (float64), scaled by 1e21."""
    rng = np.random.Generator(np.random.PCG64(seed))
    f = np.fft.rfftfreq(n, 1.0 / fs)
    amp = np.sqrt(aligo_like_psd(f) * fs / 2.0 * n)
    spec = (rng.standard_normal(f.shape[0]) + 1j * rng.standard_normal(f.shape[0])) * amp / math.sqrt(2.0)
    spec[0] = 0.0
    return np.fft.irfft(spec, n) * 1e21


def sine_gaussian(f0: float, q: float, fs: int = FS, phase0: float = 0.0) -> np.ndarray:
    """Sine-Gaussian burst exp(-t^2 / tau^2) sin(2 pi f0 t + phase0), tau = q / (sqrt(2) pi f0), over
    |t| <= 4 tau (the usual model of short instrumental glitches); centred sample at index len // 2."""
    tau = q / (math.sqrt(2.0) * math.pi * f0)
    half = max(1, int(math.ceil(4.0 * tau * fs)))
    t = np.arange(-half, half + 1, dtype=np.float64) / fs
    return np.exp(-(t / tau) ** 2) * np.sin(2.0 * math.pi * f0 * t + phase0)


def _whitened_norm(h: np.ndarray, fs: int, psd_scale: float) -> float:
    pad = 8192
    m = h.shape[0] + pad
    hf = np.fft.rfft(np.concatenate([h, np.zeros(pad)]))
    f = np.fft.rfftfreq(m, 1.0 / fs)
    wf = hf / np.sqrt(fs * aligo_like_psd(f) * psd_scale / 2.0)
    wf[f < 15.0] = 0.0
    return math.sqrt(float(np.sum(np.fft.irfft(wf, m) ** 2)))


def add_glitches(xh: np.ndarray, xl: np.ndarray, n_glitch: int, seed: int, snr_range=(10.0, 100.0),
                 f0_range=(30.0, 500.0), q_range=(3.0, 30.0), fs: int = FS, psd_scale: float = 1e42,
                 avoid=(), guard: int = 4 * FS):
    """Add n_glitch sine-Gaussian glitches, each in one detector only (chosen at random), to the
    coloured streams xh, xl (in place), scaled so that the whitened glitch has norm `snr`; centres
    uniform, at least `guard` samples from every index in `avoid` (the chirp mergers).
    Returns [(centre, detector (0 = H, 1 = L), snr, f0, q, phase)]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = xh.shape[0]
    av = np.sort(np.asarray(list(avoid), dtype=np.int64))
    out = []
    tries = 0
    while len(out) < n_glitch and tries < 100 * max(1, n_glitch):
        tries += 1
        c = int(rng.integers(fs, n - fs))
        if av.size:
            j = np.searchsorted(av, c)
            near = [av[k] for k in (j - 1, j) if 0 <= k < av.size]
            if any(abs(int(a) - c) < guard for a in near):
                continue
        det = int(rng.integers(0, 2))
        snr = rng.uniform(*snr_range)
        f0 = rng.uniform(*f0_range)
        q = rng.uniform(*q_range)
        phase = rng.uniform(0, 2 * math.pi)
        h = sine_gaussian(f0, q, fs=fs, phase0=phase)
        half = h.shape[0] // 2
        if c - half < 0 or c + half >= n:
            continue
        nrm = _whitened_norm(h, fs, psd_scale)
        x = xh if det == 0 else xl
        x[c - half:c + half + 1] += (h * (snr / nrm)).astype(x.dtype)
        out.append((c, det, float(snr), float(f0), float(q), float(phase)))
    return out


def coloured_stream(n: int, seed: int = 1000, n_inj: int = 0, snr_range=(6.0, 20.0), mc_range=(5.0, 30.0),
                    min_gap: int = 2 * FS, fs: int = FS, with_params: bool = False):
    """Two detector streams of n samples (float32) of coloured Gaussian noise with the analytic
    spectrum (scaled by 1e21) and n_inj unwhitened leading-order chirps.

    Each chirp is scaled so that, whitened with the true spectrum (division of its transform by
    sqrt(fs S / 2), S the spectrum of the scaled noise), its norm is the detector SNR
    (network SNR / sqrt(2)); mergers uniform, >= min_gap apart; Livingston delayed by U[-10, 10] ms
    with an independent phase.  Stands in for unwhitened GWOSC strain with injections.
    with_params: also return a list of (merger, network SNR, chirp mass) per injection."""
    xh = coloured_noise(n, seed=seed)
    xl = coloured_noise(n, seed=seed + 1)
    rng = np.random.Generator(np.random.PCG64(seed + 1000))
    mergers = []
    params = []
    lo = 6 * fs
    if n_inj > 0 and n > lo + 2 * fs:
        slots = np.sort(rng.choice(np.arange(lo, n - fs, min_gap), size=n_inj, replace=False))
        for tm in slots:
            mc = rng.uniform(*mc_range)
            snr_net = rng.uniform(*snr_range)
            snr = snr_net / math.sqrt(2.0)
            params.append((int(tm), float(snr_net), float(mc)))
            dt = int(round(rng.uniform(-0.010, 0.010) * fs))
            ph = rng.uniform(0, 2 * math.pi)
            for x, t_m, p0 in ((xh, int(tm), 0.0), (xl, int(tm) + dt, ph)):
                n_before = min(t_m, 6 * fs)
                h = newtonian_chirp(mc, n_before, fs=fs, phase0=p0)
                pad = 8192
                m = h.shape[0] + pad
                hf = np.fft.rfft(np.concatenate([h, np.zeros(pad)]))
                f = np.fft.rfftfreq(m, 1.0 / fs)
                wf = hf / np.sqrt(fs * aligo_like_psd(f) * 1e42 / 2.0)
                wf[f < 15.0] = 0.0
                norm = math.sqrt(float(np.sum(np.fft.irfft(wf, m) ** 2)))
                if norm > 0:
                    x[t_m - n_before:t_m + 1] += h * (snr / norm)
            mergers.append(int(tm))
    if with_params:
        return xh.astype(np.float32), xl.astype(np.float32), mergers, params
    return xh.astype(np.float32), xl.astype(np.float32), mergers
