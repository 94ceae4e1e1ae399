#!/usr/bin/env python
"""Throughput of the two-detector AI-ensemble detector (arXiv:2201.11133) on
one hour of 4096 Hz Hanford + Livingston strain.

One step = the whole inference hot path over the hour: whitening of both
detectors' coloured strain (Welch PSD, spectral division, unit std), ensemble
forward of 4 models (3 stacks x dilations 1..512 = 30 layers, R = 64, S = 128,
Hc = 256) on every 1 s window at 0.5 s stride (7199 windows), then peak finding
and ensemble coincidence on the device.  Metric: strain-seconds (two detectors,
whole ensemble) processed per wall-second.

Prints ONE JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
instead on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workload  # noqa: E402

FS = workload.FS
WINDOW, STRIDE = workload.WINDOW, workload.STRIDE
HOUR = 3600
METRIC = "strain-sec/s (2-det, ensemble)"
UNIT = "strain-s/s"
PREC_NAMES = {"fp32": 0, "bf16": 1, "fp8": 2}
L2_BYTES = 129 * 1024 * 1024


def flops_per_sample(cfg) -> int:
    """Algorithmic FLOPs per output sample of one model (both branches and the head)."""
    R, S, Hc, L = cfg["r_ch"], cfg["s_ch"], cfg["head_ch"], workload.n_layers(cfg)
    per_layer = 2 * (2 * R) * (2 * R) + 2 * (R + S) * R
    return 2 * (2 * R + L * per_layer) + 2 * (2 * S) * Hc + 2 * Hc


def reuse_plan(cfg, W: int, stride: int, tile: int = 128):
    """First computed layer per tile of a window that follows its predecessor in the same CTA
    (cross-window reuse of the tensor-core path): tile t starts at layer lstar[t] + 1, where lstar[t]
    is the last layer whose receptive field r_l satisfies r_l - 1 <= 128 t (at most L - 2); only
    tiles t < NT - stride/128, and only for W/2 <= stride < W with stride a multiple of 128."""
    L = workload.n_layers(cfg)
    NT = W // tile
    first = [0] * NT
    if stride % tile or stride >= W or 2 * stride < W or NT > 64 or L < 2:
        return first
    shift = stride // tile
    r, rl = 1, []
    for d in workload.dilations(cfg):
        r += (int(cfg["kernel"]) - 1) * d
        rl.append(r)
    for t in range(NT - shift):
        ls = -1
        for l in range(min(L - 1, 127)):
            if rl[l] - 1 <= tile * t:
                ls = l
            else:
                break
        first[t] = ls + 1
    return first


def executed_flops(cfg, nw: int, W: int, stride: int, grid: int, reuse: bool = True) -> int:
    """FLOPs the tensor-core forward executes for all models over nw windows: per window and
    model the input projections, the computed (tile, layer) pairs of both branches and the head.
    A job (model, window) reuses layers when it is not the first job of its CTA's contiguous
    range and not window 0."""
    R, S, Hc = cfg["r_ch"], cfg["s_ch"], cfg["head_ch"]
    L, T = workload.n_layers(cfg), 128
    per_layer_row = 2 * (2 * R) * (2 * R) + 2 * (R + S) * R
    fixed = W * (2 * 2 * R + 2 * (2 * S) * Hc + 2 * Hc)
    full = fixed + 2 * W * L * per_layer_row
    first = reuse_plan(cfg, W, stride) if reuse else [0] * (W // T)
    reduced = fixed + 2 * T * per_layer_row * sum(L - f for f in first)
    n_jobs = cfg["n_models"] * nw
    q, rm = divmod(n_jobs, grid)
    n_reuse = 0
    for c in range(grid):
        j0 = c * q + min(c, rm)
        j1 = j0 + q + (1 if c < rm else 0)
        n_reuse += sum(1 for j in range(j0 + 1, j1) if j % nw > 0)
    return n_reuse * reduced + (n_jobs - n_reuse) * full


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
        "fallback"


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.gpu)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() in ("active", "1"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def traffic_for(kernel: str, src_files):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, or None when
    the kernel sources changed since the counters were taken."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get(kernel)
    if not e:
        return None
    h = hashlib.sha256()
    for f in src_files:
        h.update(open(f, "rb").read())
    sha = h.hexdigest()[:16]
    if e.get("src_sha") != sha:
        return None
    return e.get("bytes_per_launch")


WELCH_SEG = 16384      # 4 s Welch segments


def make_inputs(seed: int, minutes: float = 60.0):
    """Coloured (unwhitened) two-detector strain with leading-order chirps, float32; with the injections'
    (merger, network SNR, chirp mass)."""
    n = int(round(minutes * 60)) * FS
    n_inj = max(1, int(round(200 * minutes / 60.0)))
    sh, sl, mergers, params = workload.coloured_stream(n, seed=seed, n_inj=n_inj, snr_range=(6.0, 20.0),
                                                       mc_range=(5.0, 30.0), with_params=True)
    return sh, sl, mergers, params


TRAINED = os.path.join(ROOT, "paper_2201_11133_gb300", "weights", "ensemble_trained_lite.npz")


def ensemble_weights(cfg):
    """(FP32 blobs [n_models, P], description): the trained-lite members when their file is present
    (paper_2201_11133_gb300.train), else seeded random initialisation."""
    if os.path.exists(TRAINED):
        z = np.load(TRAINED)
        w = z["weights"].astype(np.float32)
        if w.shape == (cfg["n_models"], workload.param_count(cfg)):
            steps = int(z["meta"][0]) if "meta" in z else -1
            return w, f"trained-lite ({steps} steps per member, synthetic chirps)"
    return workload.init_weights(cfg, seed=3000), "seeded random init"


# ---------------------------------------------------------------------------
# Reference arm / CPU baseline: the FP64 oracle on a bounded sample
# ---------------------------------------------------------------------------

def oracle_whiten_pair(sh, sl):
    """FP64 oracle whitening of both detectors; returns (whitened pair float32, seconds)."""
    from oracle import whiten as ow
    t0 = time.perf_counter()
    wh = ow.whiten(sh.astype(np.float64), float(FS), WELCH_SEG).astype(np.float32)
    wl = ow.whiten(sl.astype(np.float64), float(FS), WELCH_SEG).astype(np.float32)
    return (wh, wl), time.perf_counter() - t0


def oracle_network(whitened, cfg, wb, n_win: int):
    """FP64 oracle forward + triggers on the first n_win windows; returns (seconds, threads)."""
    import oracle
    threads = os.cpu_count() or 1
    n_s = (n_win - 1) * STRIDE + WINDOW
    t0 = time.perf_counter()
    prob = oracle.forward_stream(cfg, wb, whitened[0][:n_s], whitened[1][:n_s], WINDOW, STRIDE, nthreads=threads)
    oracle.triggers(prob.astype(np.float32), WINDOW, STRIDE, 0.5, 2048.0, 2048)
    return time.perf_counter() - t0, threads


def cpu_seconds_per_strain_second(t_white, n, t_net, n_win):
    """Whitening is charged per strain-second of the whole stream, the network per window (0.5 s)."""
    return t_white / (n / FS) + t_net / (n_win * STRIDE / FS)


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cfg = workload.config("ensemble")
    wb, _ = ensemble_weights(cfg)
    sh, sl, _, _ = make_inputs(1000)
    import oracle
    oracle.build()
    n_win = args.ref_windows
    whitened, t_white = oracle_whiten_pair(sh, sl)
    for _ in range(args.warmup):
        oracle_network(whitened, cfg, wb, 1)
    per_s_tot = 0.0
    threads = 1
    for _ in range(args.steps):
        t_net, threads = oracle_network(whitened, cfg, wb, n_win)
        per_s_tot += cpu_seconds_per_strain_second(t_white, sh.shape[0], t_net, n_win)
    v = args.steps / per_s_tot
    tot = per_s_tot * HOUR
    sample = (f"FP64 whitening of the whole hour (both detectors, {t_white:.1f} s, charged per strain-second) + "
              f"{n_win} windows x 4 models per step (FP64 forward + triggers, charged 0.5 s each)")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * tot / args.steps,
        "ms_per_step_note": "extrapolated to the one-hour step from the sampled CPU time per strain-second",
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "1h-2det-4model-30layer", "window": WINDOW, "stride": STRIDE,
                   "sample_windows": n_win},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def lognormal_segments(total: int, seed: int = 2024, median_s: float = 1200.0, sigma: float = 1.0,
                       lo_s: float = 60.0, hi_s: float = 14400.0, gap_max_s: float = 60.0):
    """Science segments with lognormal lengths (median 20 min, clipped to 60 s .. 4 h) and gaps of up
    to a minute, laid out from sample 0 until `total` samples are used (the last one cut)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    starts, lens, pos = [], [], 0
    while pos < total:
        ln = int(np.clip(rng.lognormal(np.log(median_s), sigma), lo_s, hi_s) * FS)
        ln = min(ln, total - pos)
        if ln >= WINDOW:
            starts.append(pos)
            lens.append(ln)
        pos += ln + int(rng.uniform(0, gap_max_s) * FS)
    return np.array(starts, dtype=np.int64), np.array(lens, dtype=np.int64)


def batched_slides(gwe, cfg, wb, Hw, Lw, n, thr, minutes, dist, dev, stream, world):
    """Segments cut from the whitened hour (lognormal lengths, gaps between them) x 64 offsets of
    1..64 s, FP8 ensemble, one autotuned CUDA-graph plan per step, then triggers per segment."""
    import torch
    from paper_2201_11133_gb300 import multi
    starts, lens = lognormal_segments(min(n, int(minutes * 60) * FS))
    nws = gwe.segment_windows(lens, WINDOW, STRIDE)
    k_sl = 64
    offs = [2 * (i + 1) for i in range(k_sl)]
    m8 = gwe.Model(cfg, wb, PREC_NAMES["fp8"])
    out = torch.empty((k_sl, cfg["n_models"], int(nws.sum()), WINDOW), dtype=torch.float32, device=dev)
    t0 = time.perf_counter()
    plan = gwe.gwe_plan_create(m8.handle, Hw, Lw, starts, lens, WINDOW, STRIDE, offs, out, gwe.GWE_PLAN_AUTOTUNE,
                               stream=stream)
    t_create = time.perf_counter() - t0
    shape = gwe.gwe_plan_shape(plan)

    def step():
        gwe.gwe_plan_execute(plan, stream=stream)
        return gwe.gwe_triggers_segments(out, cfg["n_models"], k_sl, lens, WINDOW, STRIDE, thr, 2048.0, 2048,
                                         flags=0, stream=stream)[0]

    step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ts, tf = [], []
    for _ in range(2):
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        gwe.gwe_plan_execute(plan, stream=stream)
        e1.record(stream)
        recs = gwe.gwe_triggers_segments(out, cfg["n_models"], k_sl, lens, WINDOW, STRIDE, thr, 2048.0, 2048,
                                         flags=0, stream=stream)[0]
        e2.record(stream)
        e2.synchronize()
        ts.append(e0.elapsed_time(e2))
        tf.append(e0.elapsed_time(e1))
    gwe.gwe_sync(m8.handle)
    t_step = multi.max_over_ranks(sum(ts) / len(ts), dist, dev)
    t_fwd = multi.max_over_ranks(sum(tf) / len(tf), dist, dev)
    strain_s = float(lens.sum()) / FS
    res = {"segments": int(len(lens)), "strain_s": strain_s, "windows": int(nws.sum()), "offsets": k_sl,
           "precision": "fp8", "ms_per_step": t_step, "forward_graph_ms": t_fwd,
           "physical_strain_s_per_s": world * strain_s / (t_step / 1000.0),
           "effective_strain_s_per_s": world * strain_s * k_sl / (t_step / 1000.0),
           "ensemble_triggers": int(np.sum(recs["model"] == -1)) if len(recs) else 0,
           "plan": {"graph_kernels": shape["n_kernels"], "slide_window_tile": shape["window_tile"],
                    "slide_offset_tile": shape["offset_tile"], "slide_pieces_per_block": shape["pieces_per_block"],
                    "slide_heads_ms_tuned": shape["tuned_ms"],
                    "slide_heads_ms_default": shape["default_ms"], "create_s": t_create},
           "segment_lengths_s": {"min": float(lens.min()) / FS, "median": float(np.median(lens)) / FS,
                                 "max": float(lens.max()) / FS},
           "note": "lognormal segment lengths (median 20 min, clipped 60 s..4 h) cut from the whitened hour; "
                   "one graph launch per step (all models, branch passes + slide heads), then triggers per "
                   "segment on every (offset, model) series"}
    gwe.gwe_plan_destroy(plan)
    del out
    m8.close()
    return res


def stream_search(gwe, cfg, wb, sh, sl, thr, hours, dist, dev, stream, world):
    """FP16 raw strain (x 1e21) in pinned host memory, `hours` long (the hour repeated), searched in
    chunks of 7151 windows (+16 windows of context and 4 s of whitening guard per side: 1 h spans):
    H2D copies, conversion, whitening, ensemble forward and triggers, for BF16 and FP8."""
    import torch
    from paper_2201_11133_gb300 import multi
    reps = max(1, int(round(hours)))
    hH = torch.from_numpy(np.tile(sh, reps).astype(np.float16)).pin_memory()
    hL = torch.from_numpy(np.tile(sl, reps).astype(np.float16)).pin_memory()
    n_all = int(hH.numel())
    res = {"hours": n_all / FS / 3600.0, "input": "fp16 x 1e21, pinned host memory", "chunk_windows": 7151,
           "margin_windows": 16, "guard_samples": 16384, "h2d_bytes": int(hH.nbytes + hL.nbytes)}
    for pname in ("bf16", "fp8"):
        m = gwe.Model(cfg, wb, PREC_NAMES[pname])
        sr = gwe.gwe_search_create(m.handle, window=WINDOW, stride=STRIDE, chunk_windows=7151, margin_windows=16,
                                   guard_samples=16384, fs=float(FS), welch_seg=WELCH_SEG,
                                   input_dtype=gwe.GWE_INPUT_F16, input_scale=1.0, height_thr=thr,
                                   min_width=2048.0, coinc=2048, trigger_flags=0)
        gwe.gwe_search_run(sr, hH[:WINDOW * 8], hL[:WINDOW * 8], WINDOW * 8, stream=stream)   # warm the plans
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        recs = gwe.gwe_search_run(sr, hH, hL, n_all, stream=stream)
        torch.cuda.synchronize()
        t = multi.max_over_ranks(time.perf_counter() - t0, dist, dev)
        rate = world * n_all / FS / t
        res[pname] = {"seconds": t, "strain_s_per_s": rate, "ensemble_triggers": int(np.sum(recs["model"] == -1)),
                      "month_seconds_extrapolated": 30 * 86400 / (rate / world)}
        gwe.gwe_search_destroy(sr)
        m.close()
    return res


def training_roofline(cfg1, B, W, kernels, peaks, peak_kind):
    """Roofline of the backward's row GEMMs (k_tc_rows, bound by HBM) from their measured time per
    step.  Algorithmic bytes per row (one sample of one branch) and layer, with the stack inputs
    and skip sums taken from the fused forward (BF16 handles, W a multiple of 128): recomputed
    conv 8R (x in, gate cache and z out), residual 12R (z, x in; x FP32 and BF16 out), dz 10R + 2S
    (dL/dx, dL/dskip, gate cache in; da out), dgrad 14R (da, dL/dx in; dL/dx FP32 and BF16 out).
    The head's two row GEMMs (timed as k_tc_rows:head_u and k_tc_rows:head_dh) are not counted."""
    kr = kernels.get("k_tc_rows")
    if not kr or kr["ms_per_step"] <= 0:
        return None
    ms = kr["ms_per_step"] - sum(kernels.get(k, {}).get("ms_per_step", 0.0)
                                 for k in ("k_tc_rows:head_u", "k_tc_rows:head_dh"))
    if ms <= 0:
        return None
    R, S, L = cfg1["r_ch"], cfg1["s_ch"], workload.n_layers(cfg1)
    bytes_step = 2 * B * W * L * (44 * R + 2 * S)
    ach = bytes_step / (ms / 1000.0) / 1e9
    return {"kernel": "k_tc_rows", "bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": ach / peaks["hbm_gbs"], "peak_source": f"of {peak_kind}", "bytes_per_step": bytes_step}


def training_step(gwe, cfg, B, dist, dev, stream, world):
    """Forward logits, dL/dlogit of the mean BCE, and the backward pass (weight and input gradients,
    per-stack recomputation) of one member on B windows of 2 x 4096 samples, half with chirps: with
    a BF16 handle (tensor-core forward and backward, FP32 accumulation) and with an FP32 handle
    (the FP32 SIMT kernels)."""
    import torch
    from paper_2201_11133_gb300 import multi
    cfg1 = dict(cfg, n_models=1)
    wb = workload.init_weights(cfg1, seed=3000)
    xh, xl, y = workload.training_batch(B=B, W=WINDOW, seed=2000)
    XH, XL, Y = (torch.from_numpy(a).to(dev) for a in (xh, xl, y))
    fwd = B * WINDOW * flops_per_sample(cfg1)
    res = {"batch": B, "window": WINDOW, "layers": workload.n_layers(cfg1),
           "tflop_per_step_algorithmic": 3 * fwd / 1e12,
           "note": "algorithmic FLOPs = forward + 2x forward for the backward; the per-stack recomputation "
                   "of the forward is executed on top"}
    for pname in ("bf16", "fp32"):
        m = gwe.Model(cfg1, wb, PREC_NAMES[pname])
        lg = torch.empty((1, B, WINDOW), dtype=torch.float32, device=dev)
        gw = torch.empty(gwe.gwe_param_count(cfg1), dtype=torch.float32, device=dev)
        gH = torch.empty((B, WINDOW), dtype=torch.float32, device=dev)
        gL = torch.empty_like(gH)

        def step():
            gwe.gwe_forward_logits(m.handle, XH, XL, B, WINDOW, lg, stream)
            dlg = (torch.sigmoid(lg[0]) - Y) / float(B * WINDOW)      # mean-BCE gradient on the logits
            gwe.gwe_backward(m.handle, 0, XH, XL, B, WINDOW, dlg, gw, gH, gL, stream)

        step()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        gwe.gwe_profile_enable(True)
        ts = []
        for _ in range(2):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        prof = gwe.gwe_profile_read()
        gwe.gwe_profile_enable(False)
        t = multi.max_over_ranks(sum(ts) / len(ts), dist, dev)
        res[pname] = {"path": "tensor cores (BF16 operands, FP32 accumulation)" if pname == "bf16" else "FP32 SIMT",
                      "ms_per_step": t, "windows_per_s": world * B / (t / 1000.0),
                      "achieved_tflops": 3 * fwd / (t / 1000.0) / 1e12,
                      "kernels": {k: {"ms_per_step": v[0] / 2, "launches_per_step": v[1] / 2}
                                  for k, v in prof.items()}}
        m.close()
    res["speedup_bf16_vs_fp32"] = res["fp32"]["ms_per_step"] / res["bf16"]["ms_per_step"]
    peaks, peak_kind = load_peaks()
    res["bf16"]["roofline"] = training_roofline(cfg1, B, WINDOW, res["bf16"]["kernels"], peaks, peak_kind)
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gwe", choices=["gwe", "reference"])
    ap.add_argument("--precision", default=os.environ.get("GWE_BENCH_PRECISION", "bf16"), choices=list(PREC_NAMES))
    ap.add_argument("--minutes", type=float, default=60.0,
                    help="strain duration per detector (60 = the one-hour workload; smaller only for profiler captures)")
    ncpu = max(1, min(32, os.cpu_count() or 1))
    ap.add_argument("--ref-windows", type=int, default=ncpu,
                    help="windows per reference-arm step (the oracle runs one window per host core)")
    ap.add_argument("--cpu-windows", type=int, default=ncpu,
                    help="windows of the CPU-baseline sample (one per host core)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--slides", type=int, default=64,
                    help="also time the time-slide background pass with this many Livingston offsets (0: skip)")
    ap.add_argument("--batched-minutes", type=float, default=60.0,
                    help="science segments (lognormal lengths) totalling this many minutes x 64 offsets through a "
                         "graph plan in FP8 (0: skip)")
    ap.add_argument("--stream-hours", type=float, default=3.0,
                    help="stream this many hours of FP16 strain from pinned host memory through the chunked "
                         "search (0: skip)")
    ap.add_argument("--train-batch", type=int, default=256,
                    help="time one training step (forward logits, BCE gradient, hand-written backward) of one "
                         "30-layer model on this many windows (0: skip)")
    ap.add_argument("--thr", type=float, default=0.9,
                    help="probability threshold of the triggers with trained members")
    ap.add_argument("--min-width", type=float, default=None,
                    help="peak width cut in samples (default: the paper's 0.5 s = 2048 with random-init members; "
                         "256 with the trained-lite members, whose detection plateaus last 0.06-0.36 s)")
    ap.add_argument("--sweep-thresholds", type=int, default=64,
                    help="thresholds of the on-device ROC / false-alarm sweep over [0, 0.9998] (0: skip)")
    ap.add_argument("--glitches", type=int, default=100,
                    help="trained members: sine-Gaussian glitches (one detector each) injected into a copy of the "
                         "hour, triggers near them counted per model and for the ensemble (0: skip)")
    ap.add_argument("--compare-minutes", type=float, default=6.0,
                    help="time the other precisions' forward steps too (FP8 on the whole workload, FP32 on "
                         "this many minutes of it); 0: skip")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import paper_2201_11133_gb300 as gwe
    from paper_2201_11133_gb300 import evaluate as ev
    from paper_2201_11133_gb300 import multi

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    gwe.build()
    cfg = workload.config("ensemble")
    wb, weights_desc = ensemble_weights(cfg)
    trained = weights_desc.startswith("trained")
    prec = PREC_NAMES[args.precision]
    model = gwe.Model(cfg, wb, prec)
    sh, sl, mergers, inj_params = make_inputs(1000 + 7 * rank, args.minutes)   # each rank its own hour (weak scaling)
    n = sh.shape[0]
    nw = gwe.gwe_n_windows(n, WINDOW, STRIDE)
    H = torch.from_numpy(sh).to(dev)          # coloured (unwhitened) strain
    L = torch.from_numpy(sl).to(dev)
    Hw = torch.empty_like(H)
    Lw = torch.empty_like(L)
    out = torch.empty((1, cfg["n_models"], nw, WINDOW), dtype=torch.float32, device=dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    # trigger threshold: args.thr for trained members; for random-init members the 99.9th percentile of
    # one forward's probabilities (fixed before timing)
    gwe.gwe_whiten(H, n, float(FS), WELCH_SEG, Hw)
    gwe.gwe_whiten(L, n, float(FS), WELCH_SEG, Lw)
    model.forward(Hw, Lw, WINDOW, STRIDE, out=out)
    torch.cuda.synchronize()
    if trained:
        thr = float(args.thr)
    else:
        thr = float(torch.quantile(out[0, 0, :, ::97].reshape(-1).float(), 0.999).item())
    min_width = float(args.min_width) if args.min_width is not None else (256.0 if trained else 2048.0)
    coinc = 2048

    def step(h, l_):
        gwe.gwe_whiten(h, n, float(FS), WELCH_SEG, Hw, stream=stream)
        gwe.gwe_whiten(l_, n, float(FS), WELCH_SEG, Lw, stream=stream)
        gwe.gwe_forward(model.handle, Hw, Lw, n, WINDOW, STRIDE, None, out, stream)
        return gwe.gwe_triggers(out, cfg["n_models"], 1, nw, WINDOW, STRIDE, thr, min_width, coinc, flags=0,
                                stream=stream)

    for _ in range(args.warmup):
        step(H, L)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()

    clocks = Clocks(local)
    clocks.start()
    gwe.gwe_profile_enable(True)
    launches0 = gwe.load().gwe_launch_count()
    times = []
    n_trig = 0
    for _ in range(args.steps):
        flush.fill_(1.0)                                  # evict L2 between timed steps
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        recs = step(H, L)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        n_trig = len(recs)
    launches = gwe.load().gwe_launch_count() - launches0
    prof = gwe.gwe_profile_read()
    gwe.gwe_profile_enable(False)
    clk = clocks.stop()
    torch.cuda.synchronize()
    total_ms = multi.max_over_ranks(sum(times), dist, dev)
    if dist:
        dist.barrier()
    ms_per_step = total_ms / args.steps
    strain_s = n / FS
    value = world * strain_s * args.steps / (total_ms / 1000.0)

    # end to end through the public API with host buffers (pinned), copies inside the timed region
    e2e = None
    if not args.no_e2e:
        hH = torch.from_numpy(sh).pin_memory()
        hL = torch.from_numpy(sl).pin_memory()
        dH = torch.empty_like(H)
        dL = torch.empty_like(L)
        e2e_steps = max(1, min(args.steps, 3))
        t_tot = 0.0
        d2h = 0
        for _ in range(e2e_steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            if dist:
                dist.barrier()
            t0 = time.perf_counter()
            dH.copy_(hH, non_blocking=True)
            dL.copy_(hL, non_blocking=True)
            recs = step(dH, dL)            # trigger records come back to host memory
            torch.cuda.synchronize()
            t_tot += time.perf_counter() - t0
            d2h = recs.nbytes + 8
        t_tot = multi.max_over_ranks(t_tot, dist, dev)
        e2e = {"value": world * strain_s * e2e_steps / t_tot, "unit": UNIT,
               "h2d_bytes_per_step": int(hH.nbytes + hL.nbytes), "d2h_bytes_per_step": int(d2h)}

    # time slides (the background estimate): offsets of 1..K seconds on the same hour, whitening +
    # branch pass once + slide heads + triggers on all K x 4 series
    slides_res = None
    if args.slides > 0 and prec == 1:
        k_sl = args.slides
        offs = [2 * (i + 1) for i in range(k_sl)]          # 1 s = 2 windows at 0.5 s stride
        out_sl = torch.empty((k_sl, cfg["n_models"], nw, WINDOW), dtype=torch.float32, device=dev)

        def slide_step():
            gwe.gwe_whiten(H, n, float(FS), WELCH_SEG, Hw, stream=stream)
            gwe.gwe_whiten(L, n, float(FS), WELCH_SEG, Lw, stream=stream)
            gwe.gwe_forward(model.handle, Hw, Lw, n, WINDOW, STRIDE, offs, out_sl, stream)
            return gwe.gwe_triggers(out_sl, cfg["n_models"], k_sl, nw, WINDOW, STRIDE, thr, min_width, coinc,
                                    flags=0, stream=stream)

        slide_step()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        gwe.gwe_profile_enable(True)
        st_ms = []
        for _ in range(2):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            recs = slide_step()
            e1.record(stream)
            e1.synchronize()
            st_ms.append(e0.elapsed_time(e1))
        prof_sl = gwe.gwe_profile_read()
        gwe.gwe_profile_enable(False)
        t_sl = multi.max_over_ranks(sum(st_ms) / len(st_ms), dist, dev)
        # on-device threshold sweep over the zero-lag and the 64 slid outputs (ROC / false-alarm curve)
        if args.sweep_thresholds > 0:
            thr_grid = np.linspace(0.0, 0.9998, args.sweep_thresholds).astype(np.float32)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            bg, _ = gwe.gwe_trigger_sweep(out_sl, cfg["n_models"], k_sl, nw, WINDOW, STRIDE, thr_grid, min_width,
                                          coinc, per_model=False, stream=stream)
            t_sweep_bg = time.perf_counter() - t0
            fg, fg_model = gwe.gwe_trigger_sweep(out, cfg["n_models"], 1, nw, WINDOW, STRIDE, thr_grid, min_width,
                                                 coinc, stream=stream)
            hours_bg = k_sl * strain_s / 3600.0
            sweep_res = {"thresholds": [float(t) for t in thr_grid], "min_width": min_width, "coinc": coinc,
                         "zero_lag_ensemble": [int(v) for v in fg[0]],
                         "zero_lag_per_model": [[int(v) for v in row] for row in fg_model[0]],
                         "background_ensemble": [int(v) for v in bg.sum(0)],
                         "background_hours": hours_bg,
                         "far_per_hour": [float(v) / hours_bg for v in bg.sum(0)],
                         "seconds_64_slides": t_sweep_bg,
                         "note": "one pass over the 64 slid series per threshold vector (peaks found once at the "
                                 "lowest threshold, each model-0 peak's largest threshold as an ensemble trigger)"}
            if trained:
                # recovered injections at a few thresholds of the sweep grid (zero lag)
                rec_at = {}
                for tq in (0.5, 0.9, 0.99):
                    r_t = gwe.gwe_triggers(out, cfg["n_models"], 1, nw, WINDOW, STRIDE, tq, min_width, coinc,
                                           flags=0, stream=stream)
                    hit = ev.recovered(r_t["index"][r_t["model"] == -1], [p[0] for p in inj_params])
                    bg_t = gwe.gwe_trigger_sweep(out_sl, cfg["n_models"], k_sl, nw, WINDOW, STRIDE,
                                                 np.array([tq], dtype=np.float32), min_width, coinc,
                                                 per_model=False, stream=stream)[0].sum()
                    rec_at[f"{tq:g}"] = {"recovered_fraction": float(hit.mean()),
                                         "far_per_hour": float(bg_t) / hours_bg}
                sweep_res["recovery_at"] = rec_at
        # roofline of the slide heads (one launch = one model, all offsets): FP16x2 instructions against the
        # FP16x2 FMA rate of the SMs (152 SMs x 128 lanes per clock at the 2.07 GHz maximum clock), and the
        # Livingston-tile bytes the register blocking streams from L2 (default shape: 4 windows x pieces
        # of 8 offsets in step 2, so 11 tiles per 32 pairs), for context
        sl_roof = None
        if "k_slide_head" in prof_sl and prof_sl["k_slide_head"][1] > 0:
            hc = int(cfg["head_ch"])
            ms_l = prof_sl["k_slide_head"][0] / prof_sl["k_slide_head"][1]
            off_samples = k_sl * nw * WINDOW
            inst = off_samples * hc                                    # Hc/2 ReLU-adds + Hc/2 FMAs, FP16x2
            peak = 152 * 128 * 2.07e9
            l2_bytes = off_samples * (2 * hc) * 11 / 32 + nw * WINDOW * 2 * hc
            sl_roof = {"kernel": "k_slide_head", "bound": "alu", "achieved": inst / (ms_l / 1e3) / 1e12,
                       "peak": peak / 1e12, "unit": "T FP16x2 inst/s", "frac": inst / (ms_l / 1e3) / peak,
                       "peak_source": "derived: 152 SMs x 128 FP16x2 FMA lanes/clk x 2.07 GHz",
                       "ms_per_launch": ms_l, "offset_samples_per_launch": off_samples,
                       "l2_bytes_per_launch": l2_bytes, "l2_gbs": l2_bytes / (ms_l / 1e3) / 1e9,
                       "traffic": None}
        slides_res = {"offsets": k_sl, "ms_per_step": t_sl, "roofline": sl_roof,
                      "threshold_sweep": sweep_res if args.sweep_thresholds > 0 else None,
                      "physical_strain_s_per_s": world * strain_s / (t_sl / 1000.0),
                      "effective_strain_s_per_s": world * strain_s * k_sl / (t_sl / 1000.0),
                      "ensemble_triggers": int(np.sum(recs["model"] == -1)) if len(recs) else 0,
                      "kernels": {k: {"ms_per_step": v[0] / 2, "launches_per_step": v[1] / 2}
                                  for k, v in prof_sl.items()},
                      "note": "branch pass once per window (projections of the head's first conv kept in FP16), "
                              "slide heads per offset, triggers on every (offset, model) series"}
        out_sl_keep = out_sl if trained else None
        del out_sl

    # sensitivity of the trained ensemble (the last timed step's zero-lag triggers at thr): injections
    # recovered per network-SNR bin, and the false-alarm rate from the slid background
    sensitivity = None
    if trained:
        sensitivity = {"threshold": thr, "coinc": coinc, "recovery_window_s": [-4.0, 0.5],
                       "injections": len(inj_params), "by_min_width": []}
        for mw_s in sorted({min_width, 2048.0}):
            r0 = gwe.gwe_triggers(out, cfg["n_models"], 1, nw, WINDOW, STRIDE, thr, mw_s, coinc, flags=0,
                                  stream=stream)
            ens0 = r0["index"][r0["model"] == -1]
            rows = ev.recovery_by_snr(ens0, inj_params)
            bg = None
            if slides_res:
                bgc = gwe.gwe_trigger_sweep(out_sl_keep, cfg["n_models"], args.slides, nw, WINDOW, STRIDE,
                                            np.array([thr], dtype=np.float32), mw_s, coinc, per_model=False,
                                            stream=stream)[0].sum()
                bg = ev.far_per_hour(int(bgc), args.slides, strain_s)
            sensitivity["by_min_width"].append({
                "min_width": mw_s, "ensemble_triggers": int(len(ens0)),
                "recovered_by_snr": [{"snr": [lo, hi], "injections": k, "recovered": h} for lo, hi, k, h in rows],
                "recovered_total": int(sum(r[3] for r in rows)), "false_alarms_per_hour": bg})

    # glitches: sine-Gaussians in one detector each, whitened with the mean and the median PSD; triggers
    # within 1 s of a glitch counted per model and for the ensemble (coincidence of the members)
    glitches = None
    if trained and args.glitches > 0:
        gh, gl = sh.copy(), sl.copy()
        glist = workload.add_glitches(gh, gl, args.glitches, seed=4242 + rank, snr_range=(10.0, 60.0),
                                      avoid=mergers, guard=8 * FS)
        cent = np.array(sorted(g[0] for g in glist), dtype=np.int64)
        Hg, Lg = torch.from_numpy(gh).to(dev), torch.from_numpy(gl).to(dev)
        glitches = {"n": len(glist), "snr": [10.0, 60.0], "f0_hz": [30.0, 500.0], "q": [3.0, 30.0]}
        for avg_name, avg in (("mean_psd", gwe.GWE_PSD_MEAN), ("median_psd", gwe.GWE_PSD_MEDIAN)):
            gwe.gwe_whiten_ex(Hg, n, float(FS), WELCH_SEG, Hw, psd_average=avg, stream=stream)
            gwe.gwe_whiten_ex(Lg, n, float(FS), WELCH_SEG, Lw, psd_average=avg, stream=stream)
            gwe.gwe_forward(model.handle, Hw, Lw, n, WINDOW, STRIDE, None, out, stream)
            rg = gwe.gwe_triggers(out, cfg["n_models"], 1, nw, WINDOW, STRIDE, thr, min_width, coinc,
                                  flags=gwe.GWE_TRIG_PER_MODEL, stream=stream)
            near = lambda idx: int(ev.recovered(idx, cent, before=FS, after=FS).sum())
            glitches[avg_name] = {
                "glitches_with_model_peak": [near(rg["index"][rg["model"] == mi]) for mi in range(cfg["n_models"])],
                "glitches_with_ensemble_trigger": near(rg["index"][rg["model"] == -1]),
                "injections_recovered": int(ev.recovered(rg["index"][rg["model"] == -1],
                                                         [p[0] for p in inj_params]).sum())}
        del Hg, Lg
        # the later legs read the clean whitened hour
        gwe.gwe_whiten(H, n, float(FS), WELCH_SEG, Hw, stream=stream)
        gwe.gwe_whiten(L, n, float(FS), WELCH_SEG, Lw, stream=stream)
        torch.cuda.synchronize()

    out_sl_keep = None
    torch.cuda.empty_cache()

    # many uneven science segments x 64 offsets, FP8, through one autotuned CUDA-graph plan
    batched = None
    if args.batched_minutes > 0:
        batched = batched_slides(gwe, cfg, wb, Hw, Lw, n, thr, args.batched_minutes, dist, dev, stream, world)
    # month-scale streaming: FP16 strain in pinned host memory, chunked whitening + forward + triggers
    streaming = None
    if args.stream_hours > 0:
        streaming = stream_search(gwe, cfg, wb, sh, sl, thr, args.stream_hours, dist, dev, stream, world)

    # one training step of one 30-layer member (forward logits + BCE gradient + backward)
    train = None
    if args.train_batch > 0:
        train = training_step(gwe, cfg, args.train_batch, dist, dev, stream, world)

    # the same step in the other precisions (FP32: the plain SIMT path the speed-ups are quoted against)
    precisions = None
    if args.compare_minutes > 0:
        precisions = {args.precision: {"value": value, "ms_per_step": ms_per_step, "strain_s": strain_s}}
        for pname, pcode in PREC_NAMES.items():
            if pname == args.precision:
                continue
            n_p = n if pname != "fp32" else min(n, int(args.compare_minutes * 60 * FS))
            nw_p = gwe.gwe_n_windows(n_p, WINDOW, STRIDE)
            m_p = gwe.Model(cfg, wb, pcode)
            out_p = out if nw_p == nw else torch.empty((1, cfg["n_models"], nw_p, WINDOW), dtype=torch.float32,
                                                       device=dev)
            Hp, Lp = H[:n_p], L[:n_p]

            def step_p():
                gwe.gwe_whiten(Hp, n_p, float(FS), WELCH_SEG, Hw[:n_p], stream=stream)
                gwe.gwe_whiten(Lp, n_p, float(FS), WELCH_SEG, Lw[:n_p], stream=stream)
                gwe.gwe_forward(m_p.handle, Hw[:n_p], Lw[:n_p], n_p, WINDOW, STRIDE, None, out_p, stream)
                return gwe.gwe_triggers(out_p, cfg["n_models"], 1, nw_p, WINDOW, STRIDE, thr, min_width, coinc,
                                        flags=0, stream=stream)

            step_p()
            torch.cuda.synchronize()
            if dist:
                dist.barrier()
            ts = []
            for _ in range(2):
                flush.fill_(1.0)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                step_p()
                e1.record(stream)
                e1.synchronize()
                ts.append(e0.elapsed_time(e1))
            t_p = multi.max_over_ranks(sum(ts) / len(ts), dist, dev)
            precisions[pname] = {"value": world * (n_p / FS) / (t_p / 1000.0), "ms_per_step": t_p,
                                 "strain_s": n_p / FS}
            m_p.close()
        if "fp32" in precisions:
            for pname in precisions:
                precisions[pname]["speedup_vs_fp32"] = precisions[pname]["value"] / precisions["fp32"]["value"]

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    # roofline of the dominant kernel
    peaks, peak_kind = load_peaks()
    dom = max(prof.items(), key=lambda kv: kv[1][0]) if prof else None
    roof = None
    if dom:
        kname, (kms, kn) = dom
        fps = flops_per_sample(cfg)
        per_layer = 2 * (2 * cfg["r_ch"]) ** 2 + 2 * (cfg["r_ch"] + cfg["s_ch"]) * cfg["r_ch"]
        if kname == "k_fp32_layer":
            # one launch = one layer over 2 branches x all windows of a chunk: all windows of the step
            flops_step = cfg["n_models"] * nw * WINDOW * 2 * workload.n_layers(cfg) * per_layer
            sms = torch.cuda.get_device_properties(dev).multi_processor_count
            peak = sms * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
            bound, unit, src = "alu", "TFLOP/s", ["fp32_path.cu"]
        else:
            # FLOPs the launch executes (cross-window reuse skips the layers that the previous
            # window already computed; the algorithmic count without reuse is reported beside it)
            sms = torch.cuda.get_device_properties(dev).multi_processor_count
            flops_step = executed_flops(cfg, nw, WINDOW, STRIDE, min(sms, cfg["n_models"] * nw))
            flops_norecompute = cfg["n_models"] * nw * WINDOW * fps
            peak = peaks["bf16_tflops_sustained"] * (2.0 if prec == 2 else 1.0)
            bound, unit, src = "tensor", "TFLOP/s", ["branch_tc.cu", "tc_ptx.cuh"]
        flops_launch = flops_step * args.steps / kn
        achieved = flops_launch / (kms / kn / 1000.0) / 1e12
        src_paths = [os.path.join(ROOT, "paper_2201_11133_gb300", "csrc", f) for f in src]
        traffic = traffic_for(kname, src_paths) if all(os.path.exists(f) for f in src_paths) else None
        roof = {"kernel": kname, "bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
                "frac": achieved / peak, "peak_source": f"of {peak_kind}",
                "traffic": traffic, "launches": kn, "kernel_ms_per_step": kms / args.steps,
                "flops_per_launch": flops_launch}
        if kname != "k_fp32_layer":
            roof["flops_per_launch_without_reuse"] = flops_norecompute * args.steps / kn
            roof["flops_note"] = ("achieved counts the FLOPs executed; without cross-window reuse the same "
                                  "outputs take flops_per_launch_without_reuse")

    cpu = None
    if not args.no_cpu_baseline and world == 1:
        whitened, t_white = oracle_whiten_pair(sh, sl)
        t_net, threads = oracle_network(whitened, cfg, wb, args.cpu_windows)
        per_s = cpu_seconds_per_strain_second(t_white, n, t_net, args.cpu_windows)
        cpu = {"value": 1.0 / per_s, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"FP64 whitening of the whole hour (both detectors, charged per strain-second) + the first "
                         f"{args.cpu_windows} windows x 4 models (FP64 forward + triggers, charged 0.5 s each), "
                         f"{threads} host threads"}

    res = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {0: "f32", 1: "bf16", 2: "fp8e4m3"}[prec], "data": "synthetic",
        "config": {"workload": "1h-2det-4model-30layer" if args.minutes == 60 else f"{args.minutes:g}min-2det-4model-30layer", "n_samples_per_detector": n, "window": WINDOW,
                   "input": "coloured Gaussian noise (analytic aLIGO-like PSD) + leading-order chirps, whitened on the device",
                   "stride": STRIDE, "n_windows": nw, "models": cfg["n_models"], "layers": workload.n_layers(cfg),
                   "r_ch": cfg["r_ch"], "s_ch": cfg["s_ch"], "head_ch": cfg["head_ch"],
                   "precision": args.precision, "injections": len(mergers), "trigger_thr": thr,
                   "l2": "flushed before every timed step (256 MiB write)", "triggers_last_step": n_trig,
                   "weights": weights_desc},
        "gpu_launches": int(launches),
        "clocks": clk,
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "time_slides": slides_res,
        "sensitivity": sensitivity,
        "glitches": glitches,
        "batched_slides": batched,
        "streaming": streaming,
        "training": train,
        "precisions": precisions,
        "kernels": {k: {"ms_per_step": v[0] / args.steps, "launches_per_step": v[1] / args.steps}
                    for k, v in prof.items()},
    }
    print(json.dumps(res), flush=True)
    model.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
