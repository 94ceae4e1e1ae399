"""Sensitivity of a trained ensemble (paper, section "Statistical Analysis":
injections recovered as a function of signal strength, and false alarms
counted on time-slid data, at a probability threshold).

An injection with merger at sample tm counts as recovered when an ensemble
trigger (gwe_triggers record with model == -1) lies in [tm - before, tm + after]
(the trigger is the midpoint of the probability plateau that precedes the
merger; 4 s before and 0.5 s after by default).  The false-alarm rate is the
number of ensemble triggers of the time-slid copies per slid hour."""
from __future__ import annotations

import numpy as np

FS = 4096


def recovered(ens_idx, mergers, before: int = 4 * FS, after: int = FS // 2) -> np.ndarray:
    """Boolean per injection: an ensemble trigger lies in [tm - before, tm + after]."""
    e = np.sort(np.asarray(ens_idx, dtype=np.int64))
    out = np.zeros(len(mergers), dtype=bool)
    for k, tm in enumerate(mergers):
        j = np.searchsorted(e, tm - before)
        out[k] = j < len(e) and e[j] <= tm + after
    return out


def recovery_by_snr(ens_idx, params, edges=(6.0, 8.0, 10.0, 12.0, 15.0, 20.0)):
    """[(snr_lo, snr_hi, injections, recovered)] for injections (merger, network SNR, chirp mass)."""
    tm = [p[0] for p in params]
    snr = np.array([p[1] for p in params])
    hit = recovered(ens_idx, tm)
    rows = []
    for lo, hi in zip(edges[:-1], edges[1:]):
        sel = (snr >= lo) & (snr < hi) if hi < edges[-1] else (snr >= lo) & (snr <= hi)
        rows.append((float(lo), float(hi), int(sel.sum()), int(hit[sel].sum())))
    return rows


def far_per_hour(n_background_triggers: int, n_slides: int, seconds: float) -> float:
    """Ensemble triggers per hour of slid background."""
    return float(n_background_triggers) / (n_slides * seconds / 3600.0)
