"""Training of the ensemble members (paper, section "Materials and Methods",
paragraph "AI ensemble construction": models of one architecture trained from
different random initialisations on whitened two-detector windows with
injected waveforms, labelled per time step: 1 up to the merger, 0 after it and
in noise-only windows; BCE on the logits).

Every forward and backward runs in the library's kernels through
gwe_logits_autograd (tensor-core forward logits, tensor-core backward with
per-stack recomputation); torch supplies the synthetic batches on the device
and the Adam update of the FP32 master weights.

Synthetic batches (the paper's SEOBNRv3 injections into O2 noise are not
available): unit-variance white Gaussian noise per detector (whitened strain),
half of the windows with a leading-order chirp from a bank of whitened
templates (chirp mass on a grid over [mc_lo, mc_hi], two quadratures each, so
that any phase is a combination of the two), network SNR uniform in
[snr_lo, snr_hi] (SNR / sqrt(2) per detector against the template's full
norm), merger uniform in [W/4, W - 1], Livingston shifted by up to +-10 ms
with an independent phase.

Command line (writes the trained FP32 blobs and the loss history):
    python -m paper_2201_11133_gb300.train --steps 1000 --out trained.npz
"""
from __future__ import annotations

import argparse
import math
import time

import numpy as np

from . import GWE_BF16, Model, gwe_init_weights, gwe_logits_autograd, gwe_param_count

FS = 4096


def template_bank(n_mass: int = 96, mc_lo: float = 5.0, mc_hi: float = 50.0, W: int = 4096):
    """(templates [n_mass, 2, W] float32, norms [n_mass]): the last W samples up to the merger of the
    whitened chirp at two quadrature phases (0, pi/2) for chirp masses spaced evenly in mc^(-5/3)
    (duration), and the full-template norm of the phase-0 quadrature."""
    import workload
    inv = np.linspace(mc_lo ** (-5.0 / 3.0), mc_hi ** (-5.0 / 3.0), n_mass)
    masses = inv ** (-3.0 / 5.0)
    n_before = 6 * FS
    T = np.zeros((n_mass, 2, W), dtype=np.float32)
    norms = np.zeros(n_mass, dtype=np.float64)
    for i, mc in enumerate(masses):
        h0 = workload.whitened_template(float(mc), n_before, phase0=0.0)
        h1 = workload.whitened_template(float(mc), n_before, phase0=0.5 * math.pi)
        norms[i] = math.sqrt(float(np.sum(h0 * h0)))
        T[i, 0] = h0[-W:]
        T[i, 1] = h1[-W:]
    return T, norms, masses


class Batches:
    """Synthetic training batches on the device (see the module docstring)."""

    def __init__(self, device, W: int = 4096, seed: int = 0, snr=(5.0, 25.0), mc=(5.0, 50.0), n_mass: int = 96):
        import torch
        self.torch = torch
        self.dev = device
        self.W = W
        T, norms, _ = template_bank(n_mass, mc[0], mc[1], W)
        self.T = torch.from_numpy(T).to(device)
        self.norm = torch.from_numpy(norms.astype(np.float32)).to(device)
        self.snr = snr
        self.gen = torch.Generator(device=device)
        self.gen.manual_seed(int(seed))

    def __call__(self, B: int = 256):
        torch = self.torch
        W = self.W
        g = self.gen
        xh = torch.randn((B, W), device=self.dev, generator=g)
        xl = torch.randn((B, W), device=self.dev, generator=g)
        y = torch.zeros((B, W), device=self.dev)
        ns = B // 2
        tm = torch.randint(W // 4, W, (ns,), device=self.dev, generator=g)
        snr = self.snr[0] + (self.snr[1] - self.snr[0]) * torch.rand(ns, device=self.dev, generator=g)
        per_det = snr / math.sqrt(2.0)
        ph_h = 2 * math.pi * torch.rand(ns, device=self.dev, generator=g)
        ph_l = 2 * math.pi * torch.rand(ns, device=self.dev, generator=g)
        dt = torch.randint(-41, 42, (ns,), device=self.dev, generator=g)
        # the same chirp (mass) in both detectors: draw the mass once
        i = torch.randint(0, self.T.shape[0], (ns,), device=self.dev, generator=g)
        t = torch.arange(W, device=self.dev)[None, :]
        for x, ph, sh in ((xh, ph_h, torch.zeros_like(dt)), (xl, ph_l, dt)):
            m = (tm + sh).clamp(0, W - 1)[:, None]
            k = (t + (W - 1) - m).clamp(0, W - 1)
            valid = t <= m
            h = (torch.cos(ph)[:, None] * torch.gather(self.T[i, 0], 1, k)
                 - torch.sin(ph)[:, None] * torch.gather(self.T[i, 1], 1, k)) * valid
            x[:ns] += h * (per_det / self.norm[i])[:, None]
        y[:ns] = (t <= tm[:, None]).float()
        return xh, xl, y


def train_member(cfg, init_seed: int, data_seed: int, steps: int, batch: int = 256, W: int = 4096,
                 lr: float = 5e-4, clip: float = 1.0, device=None, log_every: int = 50, verbose: bool = True):
    """Train one member (cfg with n_models = 1) from gwe_init_weights(cfg, init_seed); returns
    (FP32 blob [P], loss history)."""
    import torch
    dev = device or torch.device("cuda:0")
    one = dict(cfg, n_models=1)
    w0 = gwe_init_weights(one, init_seed)
    m = Model(one, w0, GWE_BF16)
    w = torch.from_numpy(w0[0].copy()).to(dev).requires_grad_(True)
    opt = torch.optim.Adam([w], lr=lr)
    data = Batches(dev, W=W, seed=data_seed)
    hist = []
    t0 = time.time()
    for it in range(steps):
        xh, xl, y = data(batch)
        lg = gwe_logits_autograd(m, w, xh, xl)
        loss = torch.nn.functional.binary_cross_entropy_with_logits(lg, y)
        opt.zero_grad(set_to_none=True)
        loss.backward()
        torch.nn.utils.clip_grad_norm_([w], clip)
        opt.step()
        if it % log_every == 0 or it == steps - 1:
            lv = float(loss.item())
            if not math.isfinite(lv):
                raise FloatingPointError(f"loss is {lv} at step {it}")
            hist.append((it, lv))
            if verbose:
                print(f"step {it}: loss {lv:.4f} ({time.time() - t0:.1f} s)", flush=True)
    out = w.detach().cpu().numpy().astype(np.float32)
    m.close()
    return out, hist


def main(argv=None):
    ap = argparse.ArgumentParser(description="train the ensemble members on synthetic chirps")
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--members", type=int, default=4)
    ap.add_argument("--lr", type=float, default=5e-4)
    ap.add_argument("--init-seed", type=int, default=3000)
    ap.add_argument("--data-seed", type=int, default=7000)
    ap.add_argument("--out", default="trained.npz")
    a = ap.parse_args(argv)
    import workload
    cfg = workload.config("ensemble")
    P = gwe_param_count(dict(cfg, n_models=1))
    blobs = np.zeros((a.members, P), dtype=np.float32)
    hists = []
    for k in range(a.members):
        print(f"member {k}", flush=True)
        blobs[k], h = train_member(cfg, a.init_seed + k, a.data_seed + 101 * k, a.steps, a.batch, lr=a.lr)
        hists.append(h)
        # saved after every member (members 0 .. k trained)
        np.savez(a.out, weights=blobs[:k + 1], loss=np.array(hists, dtype=np.float64),
                 meta=np.array([a.steps, a.batch, a.lr, a.init_seed, a.data_seed], dtype=np.float64))
        print("saved", a.out, flush=True)


if __name__ == "__main__":
    main()
