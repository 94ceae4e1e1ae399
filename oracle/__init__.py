"""FP64 CPU oracle for the two-detector WaveNet-ensemble detector (arXiv:2201.11133).

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
baseline leg of the benchmark may import this package.  It shares no code with
the CUDA library: the network, backward pass, stitching, peak finding and
coincidence are written out plainly in ``gwe_oracle.c`` (FP64, libm) and the
whitening front end in ``whiten.py`` (numpy FP64).

Parity status of each function (what pins it is in tests/test_oracle_*.py):
  forward_windows / forward_stream / branch_trace  pinned (torch conv1d, closed
      forms, impulse response, receptive field, shift equivariance)
  backward   pinned (central finite differences in FP64)
  bce        pinned (closed form)
  find_peaks pinned (SciPy find_peaks as a library, rectangle/triangle closed forms)
  coincidence pinned (brute force over all tuples)
  stitch     pinned (explicit index map on a ramp)
  whiten.welch_psd / whiten.whiten  pinned (scipy.signal.welch as a library, sinusoid
      closed forms, statistics of whitened white and coloured noise)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gwe_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libgwe_oracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (OpenMP over independent windows, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        i64 = ctypes.c_int64
        lib.orc_param_count.argtypes = [P]
        lib.orc_param_count.restype = i64
        lib.orc_forward_windows.argtypes = [P, P, P, P, ctypes.c_int, ctypes.c_int, P, ctypes.c_int]
        lib.orc_forward_windows.restype = None
        lib.orc_branch_trace.argtypes = [P, P, ctypes.c_int, P, ctypes.c_int, P, P, P, P]
        lib.orc_branch_trace.restype = None
        lib.orc_n_windows.argtypes = [i64, ctypes.c_int, ctypes.c_int]
        lib.orc_n_windows.restype = i64
        lib.orc_forward_stream.argtypes = [P, P, P, P, i64, ctypes.c_int, ctypes.c_int, P, ctypes.c_int,
                                           P, ctypes.c_int]
        lib.orc_forward_stream.restype = None
        lib.orc_backward.argtypes = [P, P, P, P, ctypes.c_int, ctypes.c_int, P, P, P, P, ctypes.c_int]
        lib.orc_backward.restype = None
        lib.orc_bce.argtypes = [P, P, i64, P]
        lib.orc_bce.restype = ctypes.c_double
        lib.orc_stitch.argtypes = [P, i64, ctypes.c_int, ctypes.c_int, P]
        lib.orc_stitch.restype = i64
        lib.orc_find_peaks.argtypes = [P, i64, ctypes.c_double, ctypes.c_double, P, P, P, P, i64]
        lib.orc_find_peaks.restype = i64
        lib.orc_coincidence.argtypes = [P, P, ctypes.c_int, i64, P]
        lib.orc_coincidence.restype = i64
        lib.orc_e4m3.argtypes = [ctypes.c_double]
        lib.orc_e4m3.restype = ctypes.c_double
        lib.orc_forward_windows_q8.argtypes = [P, P, P, ctypes.c_double, P, P, ctypes.c_int, ctypes.c_int, P,
                                               ctypes.c_int]
        lib.orc_forward_windows_q8.restype = None
        lib.orc_act_amax.argtypes = [P, P, ctypes.c_int, P, ctypes.c_int, ctypes.c_int, P, ctypes.c_int]
        lib.orc_act_amax.restype = None
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _cfg_arr(cfg) -> np.ndarray:
    keys = ("n_models", "stacks", "layers_per_stack", "kernel", "r_ch", "s_ch", "head_ch")
    return np.array([int(cfg[k]) for k in keys], dtype=np.int32)


def param_count(cfg) -> int:
    return int(_load().orc_param_count(_ptr(_cfg_arr(cfg))))


def _threads(nthreads):
    return int(nthreads) if nthreads else (os.cpu_count() or 1)


def forward_windows(cfg, wblob: np.ndarray, xh: np.ndarray, xl: np.ndarray, nthreads=None) -> np.ndarray:
    """Logits [B, W] of one model (blob [P], converted to FP64) on explicit windows xh, xl [B, W]."""
    lib = _load()
    c = _cfg_arr(cfg)
    w = np.ascontiguousarray(wblob, dtype=np.float64)
    xh = np.ascontiguousarray(xh, dtype=np.float64)
    xl = np.ascontiguousarray(xl, dtype=np.float64)
    B, W = xh.shape
    out = np.zeros((B, W), dtype=np.float64)
    lib.orc_forward_windows(_ptr(c), _ptr(w), _ptr(xh), _ptr(xl), B, W, _ptr(out), _threads(nthreads))
    return out


def branch_trace(cfg, wblob: np.ndarray, branch: int, s: np.ndarray):
    """Per-layer traces of one branch on one window: xs [L+1,W,R], as [L,W,2R], zs [L,W,R], skip [W,S]."""
    lib = _load()
    c = _cfg_arr(cfg)
    L = int(cfg["stacks"]) * int(cfg["layers_per_stack"])
    R, S = int(cfg["r_ch"]), int(cfg["s_ch"])
    s = np.ascontiguousarray(s, dtype=np.float64)
    W = s.shape[0]
    xs = np.zeros((L + 1, W, R)); as_ = np.zeros((L, W, 2 * R)); zs = np.zeros((L, W, R))
    sk = np.zeros((W, S))
    w = np.ascontiguousarray(wblob, dtype=np.float64)
    lib.orc_branch_trace(_ptr(c), _ptr(w), int(branch), _ptr(s), W, _ptr(xs), _ptr(as_), _ptr(zs), _ptr(sk))
    return xs, as_, zs, sk


def e4m3(v) -> np.ndarray:
    """E4M3 rounding (nearest, ties to even, saturating at +-448) of every element, as FP64."""
    lib = _load()
    a = np.asarray(v, dtype=np.float64)
    return np.vectorize(lambda x: lib.orc_e4m3(float(x)), otypes=[np.float64])(a) if a.size else a.copy()


def act_amax(cfg, wblob: np.ndarray, branch: int, s: np.ndarray, nthreads=None) -> np.ndarray:
    """Calibration of the FP8 reading: max |x_l[i]| [L, R] of one branch over windows s [B, W]."""
    lib = _load()
    c = _cfg_arr(cfg)
    L = int(cfg["stacks"]) * int(cfg["layers_per_stack"])
    R = int(cfg["r_ch"])
    s = np.ascontiguousarray(np.atleast_2d(s), dtype=np.float64)
    B, W = s.shape
    out = np.zeros((L, R), dtype=np.float64)
    w = np.ascontiguousarray(wblob, dtype=np.float64)
    lib.orc_act_amax(_ptr(c), _ptr(w), int(branch), _ptr(s), B, W, _ptr(out), _threads(nthreads))
    return out


def forward_windows_q8(cfg, wblob: np.ndarray, amax: np.ndarray, xh: np.ndarray, xl: np.ndarray,
                       margin: float = 16.0, nthreads=None) -> np.ndarray:
    """Logits [B, W] of one model under the FP8 reading (E4M3 convolution operands, scales from
    amax [2, L, R]); everything else exact."""
    lib = _load()
    c = _cfg_arr(cfg)
    w = np.ascontiguousarray(wblob, dtype=np.float64)
    a = np.ascontiguousarray(amax, dtype=np.float64)
    L = int(cfg["stacks"]) * int(cfg["layers_per_stack"])
    assert a.shape == (2, L, int(cfg["r_ch"]))
    xh = np.ascontiguousarray(xh, dtype=np.float64)
    xl = np.ascontiguousarray(xl, dtype=np.float64)
    B, W = xh.shape
    out = np.zeros((B, W), dtype=np.float64)
    lib.orc_forward_windows_q8(_ptr(c), _ptr(w), _ptr(a), float(margin), _ptr(xh), _ptr(xl), B, W, _ptr(out),
                               _threads(nthreads))
    return out


def n_windows(n: int, window: int, stride: int) -> int:
    return int(_load().orc_n_windows(int(n), int(window), int(stride)))


def forward_stream(cfg, wblobs: np.ndarray, sh: np.ndarray, sl: np.ndarray, window: int, stride: int,
                   slides=None, nthreads=None) -> np.ndarray:
    """Probabilities [n_slides|1, n_models, n_windows, window] (FP64) over one segment."""
    lib = _load()
    c = _cfg_arr(cfg)
    wb = np.ascontiguousarray(wblobs, dtype=np.float64)
    sh = np.ascontiguousarray(sh, dtype=np.float32)
    sl = np.ascontiguousarray(sl, dtype=np.float32)
    n = sh.shape[0]
    nw = n_windows(n, window, stride)
    if slides is None or len(slides) == 0:
        sarr = np.zeros(1, dtype=np.int32); ns = 0; nout = 1
    else:
        sarr = np.ascontiguousarray(slides, dtype=np.int32); ns = len(sarr); nout = ns
    out = np.zeros((nout, int(cfg["n_models"]), nw, window), dtype=np.float64)
    if nw > 0:
        lib.orc_forward_stream(_ptr(c), _ptr(wb), _ptr(sh), _ptr(sl), n, window, stride, _ptr(sarr), ns,
                               _ptr(out), _threads(nthreads))
    return out


def backward(cfg, wblob: np.ndarray, xh: np.ndarray, xl: np.ndarray, dlogit: np.ndarray, nthreads=None):
    """(grad_w [P], grad_h [B,W], grad_l [B,W]) for one model given dL/dlogit [B,W]."""
    lib = _load()
    c = _cfg_arr(cfg)
    w = np.ascontiguousarray(wblob, dtype=np.float64)
    xh = np.ascontiguousarray(xh, dtype=np.float64)
    xl = np.ascontiguousarray(xl, dtype=np.float64)
    dl = np.ascontiguousarray(dlogit, dtype=np.float64)
    B, W = xh.shape
    gw = np.zeros(param_count(cfg), dtype=np.float64)
    gh = np.zeros((B, W)); gl = np.zeros((B, W))
    lib.orc_backward(_ptr(c), _ptr(w), _ptr(xh), _ptr(xl), B, W, _ptr(dl), _ptr(gw), _ptr(gh), _ptr(gl),
                     _threads(nthreads))
    return gw, gh, gl


def bce(logit: np.ndarray, y: np.ndarray):
    """(mean BCE loss, dL/dlogit) on logits."""
    lib = _load()
    z = np.ascontiguousarray(logit, dtype=np.float64)
    yy = np.ascontiguousarray(y, dtype=np.float64)
    dz = np.zeros_like(z)
    loss = lib.orc_bce(_ptr(z), _ptr(yy), z.size, _ptr(dz))
    return float(loss), dz


def stitch(prob: np.ndarray, window: int, stride: int) -> np.ndarray:
    """Stitched FP32 series from window outputs prob [n_w, window]."""
    lib = _load()
    p = np.ascontiguousarray(prob, dtype=np.float32)
    nw = p.shape[0]
    if nw == 0:
        return np.zeros(0, dtype=np.float32)
    out = np.zeros((nw - 1) * stride + window, dtype=np.float32)
    lib.orc_stitch(_ptr(p), nw, window, stride, _ptr(out))
    return out


def find_peaks(x: np.ndarray, thr: float, min_width: float):
    """(index int64, height, prominence, width) of the kept peaks of an FP32 series."""
    lib = _load()
    xf = np.ascontiguousarray(x, dtype=np.float32)
    n = xf.shape[0]
    cap = max(1, n // 2 + 1)
    pk = np.zeros(cap, dtype=np.int64); h = np.zeros(cap); pr = np.zeros(cap); wd = np.zeros(cap)
    cnt = lib.orc_find_peaks(_ptr(xf), n, float(thr), float(min_width), _ptr(pk), _ptr(h), _ptr(pr),
                             _ptr(wd), cap)
    cnt = int(cnt)
    return pk[:cnt].copy(), h[:cnt].copy(), pr[:cnt].copy(), wd[:cnt].copy()


def coincidence(peak_lists, coinc: int) -> np.ndarray:
    """Indices into peak_lists[0] of the model-0 peaks that are ensemble triggers."""
    lib = _load()
    arrs = [np.ascontiguousarray(p, dtype=np.int64) for p in peak_lists]
    m = len(arrs)
    ptrs = (ctypes.c_void_p * m)(*[a.ctypes.data for a in arrs])
    npk = np.array([a.shape[0] for a in arrs], dtype=np.int64)
    out = np.zeros(max(1, npk[0]), dtype=np.int64)
    cnt = lib.orc_coincidence(ctypes.cast(ptrs, ctypes.c_void_p), _ptr(npk), m, int(coinc), _ptr(out))
    return out[:int(cnt)].copy()


def triggers(prob: np.ndarray, window: int, stride: int, thr: float, min_width: float, coinc: int):
    """Full post-processing of prob [n_slides, n_models, n_w, window]:
    per (slide, model) stitched series -> peaks; per slide -> ensemble triggers.
    Returns (per_model, ensemble): per_model[s][m] = (idx, height, prom, width),
    ensemble[s] = int64 array of trigger sample indices (model-0 peak index)."""
    prob = np.asarray(prob, dtype=np.float32)
    ns, nm = prob.shape[0], prob.shape[1]
    per_model, ens = [], []
    for s in range(ns):
        pm = []
        for m in range(nm):
            x = stitch(prob[s, m], window, stride)
            pm.append(find_peaks(x, thr, min_width))
        per_model.append(pm)
        sel = coincidence([pm[m][0] for m in range(nm)], coinc)
        ens.append(pm[0][0][sel])
    return per_model, ens
