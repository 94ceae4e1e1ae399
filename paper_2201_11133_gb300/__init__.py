"""Python binding of libgwe, the GB300 (sm_103a) two-detector gravitational-wave
ensemble detector of arXiv:2201.11133.

Argument marshalling only: every step of the hot path runs in the CUDA
library's kernels.  The functions carry the C-ABI names declared in
``include/gwe.h``; device buffers are passed as torch CUDA tensors (their
``data_ptr()``), host buffers as numpy arrays.  There is no CPU fallback: if
the library is missing or no GB300 is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

__all__ = [
    "GWE_FP32", "GWE_BF16", "GWE_FP8", "GweError", "load", "build",
    "gwe_param_count", "gwe_n_windows", "gwe_model_create", "gwe_model_set_weights", "gwe_model_set_weights_device", "gwe_init_weights",
    "gwe_model_init_random", "gwe_philox4x64_10", "gwe_model_set_f16_layers", "gwe_model_f16_layers", "gwe_model_calibrate", "gwe_model_set_fp8_amax", "gwe_model_get_fp8_amax",
    "gwe_model_destroy",
    "gwe_trigger_sweep", "gwe_trigger_sweep_segments", "gwe_forward", "gwe_forward_segments", "gwe_triggers_segments", "gwe_forward_logits", "gwe_backward", "gwe_triggers", "gwe_whiten", "gwe_whiten_ex", "GWE_PSD_MEAN", "GWE_PSD_MEDIAN", "gwe_last_error",
    "gwe_version", "gwe_sync", "gwe_set_cross_window_reuse", "gwe_forward_static",
    "gwe_plan_create", "gwe_plan_execute", "gwe_plan_shape", "gwe_set_slide_shape", "gwe_plan_destroy", "GWE_PLAN_AUTOTUNE",
    "gwe_set_tensor_map_copies",
    "gwe_search_create", "gwe_search_run", "gwe_search_run_range", "gwe_search_chunks", "gwe_search_resumable",
    "gwe_search_destroy", "GWE_INPUT_F32", "GWE_INPUT_F16", "gwe_logits_autograd", "gwe_profile_enable", "gwe_profile_read", "Model", "TRIGGER_DTYPE",
]

GWE_FP32, GWE_BF16, GWE_FP8 = 0, 1, 2
GWE_TRIG_PER_MODEL = 1
GWE_PLAN_AUTOTUNE = 1
GWE_INPUT_F32, GWE_INPUT_F16 = 0, 1
GWE_PSD_MEAN, GWE_PSD_MEDIAN = 0, 1
_STATUS = {0: "GWE_OK", 1: "GWE_ERR_ARG", 2: "GWE_ERR_CUDA", 3: "GWE_ERR_OOM", 4: "GWE_ERR_TIMEOUT",
           5: "GWE_ERR_UNSUPPORTED", 6: "GWE_ERR_CAPACITY"}

_lib = None
_lock = threading.Lock()


class GweError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {_STATUS.get(status, status)}: {msg}")
        self.status = status


class _Config(ctypes.Structure):
    _fields_ = [("n_models", ctypes.c_int), ("stacks", ctypes.c_int), ("layers_per_stack", ctypes.c_int),
                ("kernel", ctypes.c_int), ("r_ch", ctypes.c_int), ("s_ch", ctypes.c_int),
                ("head_ch", ctypes.c_int)]


class _Trigger(ctypes.Structure):
    _fields_ = [("index", ctypes.c_int64), ("slide", ctypes.c_int32), ("model", ctypes.c_int32),
                ("height", ctypes.c_double), ("prominence", ctypes.c_double), ("width", ctypes.c_double)]


class _SearchConfig(ctypes.Structure):
    _fields_ = [("window", ctypes.c_int), ("stride", ctypes.c_int), ("chunk_windows", ctypes.c_int),
                ("margin_windows", ctypes.c_int), ("guard_samples", ctypes.c_int64), ("fs", ctypes.c_double),
                ("welch_seg", ctypes.c_int), ("input_dtype", ctypes.c_int), ("input_scale", ctypes.c_float),
                ("height_thr", ctypes.c_float), ("min_width", ctypes.c_double), ("coinc", ctypes.c_int64),
                ("trigger_flags", ctypes.c_int)]


TRIGGER_DTYPE = np.dtype([("index", np.int64), ("slide", np.int32), ("model", np.int32),
                          ("height", np.float64), ("prominence", np.float64), ("width", np.float64)])
assert TRIGGER_DTYPE.itemsize == ctypes.sizeof(_Trigger)


def build(force: bool = False) -> str:
    """Compile libgwe.so in-tree for sm_103a (nvcc); returns its path."""
    return _build.build(force=force)


def load():
    """Load libgwe.so (built in-tree); raises if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"libgwe.so not built ({path}); call paper_2201_11133_gb300.build() first")
        lib = ctypes.CDLL(path)
        P, I, I64, F, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_float, ctypes.c_double
        sig = {
            "gwe_param_count": (I64, [P]),
            "gwe_n_windows": (I64, [I64, I, I]),
            "gwe_model_create": (I, [P, P, I, P]),
            "gwe_model_set_weights": (I, [P, P]),
            "gwe_model_set_weights_device": (I, [P, P, P]),
            "gwe_init_weights": (I, [P, ctypes.c_uint64, P]),
            "gwe_model_init_random": (I, [P, ctypes.c_uint64, I, P]),
            "gwe_philox4x64_10": (None, [P, P, P]),
            "gwe_model_set_f16_layers": (I, [P, I]),
            "gwe_model_f16_layers": (I, [P]),
            "gwe_model_calibrate": (I, [P, P, P, I64, I, I, P]),
            "gwe_model_set_fp8_amax": (I, [P, P]),
            "gwe_model_get_fp8_amax": (I, [P, P]),
            "gwe_model_destroy": (None, [P]),
            "gwe_forward": (I, [P, P, P, I64, I, I, P, I, P, P]),
            "gwe_forward_segments": (I, [P, P, P, P, P, I, I, I, P, I, P, P]),
            "gwe_triggers_segments": (I, [P, I, I, P, I, I, I, F, D, I64, I, P, P, I64, P, P]),
            "gwe_forward_logits": (I, [P, P, P, I, I, P, P]),
            "gwe_backward": (I, [P, I, P, P, I, I, P, P, P, P, P]),
            "gwe_triggers": (I, [P, I, I, I64, I, I, F, D, I64, I, P, I64, P, P]),
            "gwe_whiten": (I, [P, I64, D, I, I, P, P]),
            "gwe_whiten_ex": (I, [P, I64, D, I, P, P, P]),
            "gwe_trigger_sweep": (I, [P, I, I, I64, I, I, P, I, D, I64, P, P, P]),
            "gwe_trigger_sweep_segments": (I, [P, I, I, P, I, I, I, P, I, D, I64, P, P, P]),
            "gwe_sync": (I, [P, P]),
            "gwe_set_cross_window_reuse": (I, [I]),
            "gwe_debug_config": (I, [I, D]),
            "gwe_debug_ring_margin": (I, [I64]),
            "gwe_forward_static": (I, [P, P, P, I64, I, I, P, P, P]),
            "gwe_plan_create": (I, [P, P, P, P, P, I, I, I, P, I, P, I, P, P]),
            "gwe_plan_execute": (I, [P, P]),
            "gwe_plan_shape": (I, [P, P, P, P, P, P, P]),
            "gwe_set_slide_shape": (I, [I, I, I]),
            "gwe_set_tensor_map_copies": (I, [I]),
            "gwe_plan_destroy": (None, [P]),
            "gwe_search_create": (I, [P, P, P]),
            "gwe_search_run": (I, [P, P, P, I64, I, P, I64, P, P]),
            "gwe_search_destroy": (None, [P]),
            "gwe_search_chunks": (I64, [P, I64]),
            "gwe_search_run_range": (I, [P, P, P, I64, I, I64, I64, P, I64, P, P]),
            "gwe_profile_enable": (I, [I]),
            "gwe_profile_read": (I, [I, P, I, P, P]),
            "gwe_last_error": (ctypes.c_char_p, []),
            "gwe_version": (ctypes.c_char_p, []),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _check(status: int, where: str):
    if status != 0:
        raise GweError(status, where, load().gwe_last_error().decode())


def _cfg(cfg) -> _Config:
    return _Config(int(cfg["n_models"]), int(cfg["stacks"]), int(cfg["layers_per_stack"]), int(cfg["kernel"]),
                   int(cfg["r_ch"]), int(cfg["s_ch"]), int(cfg["head_ch"]))


def _dptr(t) -> int:
    """Device pointer of a CUDA tensor (or 0 for None)."""
    if t is None:
        return 0
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def _stream(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def gwe_version() -> str:
    return load().gwe_version().decode()


def gwe_last_error() -> str:
    return load().gwe_last_error().decode()


def gwe_param_count(cfg) -> int:
    c = _cfg(cfg)
    return int(load().gwe_param_count(ctypes.byref(c)))


def gwe_n_windows(n_samples: int, window: int, stride: int) -> int:
    return int(load().gwe_n_windows(int(n_samples), int(window), int(stride)))


def gwe_model_create(cfg, host_weights: np.ndarray, precision: int = GWE_FP32) -> int:
    """Create a model handle on the current device from an FP32 host blob [n_models, P]."""
    lib = load()
    c = _cfg(cfg)
    w = np.ascontiguousarray(host_weights, dtype=np.float32)
    expect = int(cfg["n_models"]) * gwe_param_count(cfg)
    if w.size != expect:
        raise ValueError(f"weights have {w.size} floats, expected {expect}")
    h = ctypes.c_void_p()
    _check(lib.gwe_model_create(ctypes.byref(c), w.ctypes.data, int(precision), ctypes.byref(h)),
           "gwe_model_create")
    return h.value


def gwe_init_weights(cfg, seed: int) -> np.ndarray:
    """Seeded FP32 weight blobs [n_models, P] (Philox4x64-10, N(0, 1/fan_in) weights, zero biases)."""
    c = _cfg(cfg)
    out = np.zeros((int(cfg["n_models"]), gwe_param_count(cfg)), dtype=np.float32)
    _check(load().gwe_init_weights(ctypes.byref(c), int(seed), out.ctypes.data), "gwe_init_weights")
    return out


def gwe_model_init_random(cfg, seed: int, precision: int = GWE_FP32) -> int:
    """Model handle with seeded random weights (gwe_init_weights + gwe_model_create)."""
    c = _cfg(cfg)
    h = ctypes.c_void_p()
    _check(load().gwe_model_init_random(ctypes.byref(c), int(seed), int(precision), ctypes.byref(h)),
           "gwe_model_init_random")
    return h.value


def gwe_philox4x64_10(counter, key) -> np.ndarray:
    """Philox4x64-10 block (4 uint64) of the library's generator."""
    ctr = np.ascontiguousarray(counter, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    load().gwe_philox4x64_10(ctr.ctypes.data, k.ctypes.data, out.ctypes.data)
    return out


def gwe_model_set_f16_layers(model: int, n: int) -> None:
    """GWE_BF16 handle: layers l < n take FP16 conv operands, the rest BF16 (default L // 3)."""
    _check(load().gwe_model_set_f16_layers(model, int(n)), "gwe_model_set_f16_layers")


def gwe_model_f16_layers(model: int) -> int:
    return int(load().gwe_model_f16_layers(model))


def gwe_model_set_weights(model: int, host_weights: np.ndarray) -> None:
    w = np.ascontiguousarray(host_weights, dtype=np.float32)
    _check(load().gwe_model_set_weights(model, w.ctypes.data), "gwe_model_set_weights")


def gwe_model_set_weights_device(model: int, weights, stream=None) -> None:
    """Replace the weights from a CUDA FP32 tensor (blob layout); rebuilt on the device, asynchronous."""
    _check(load().gwe_model_set_weights_device(model, _dptr(weights), _stream(stream)),
           "gwe_model_set_weights_device")


def gwe_model_calibrate(model: int, strain_H, strain_L, n_samples: int, window: int, stride: int,
                        stream=None) -> None:
    """FP8 activation scales from the FP32 forward over one segment of (device) whitened strain."""
    _check(load().gwe_model_calibrate(model, _dptr(strain_H), _dptr(strain_L), int(n_samples), int(window),
                                      int(stride), _stream(stream)), "gwe_model_calibrate")


def gwe_model_set_fp8_amax(model: int, amax: np.ndarray) -> None:
    """Set the FP8 calibration maxima, host [n_models, 2, L, R]; rebuilds the E4M3 weights."""
    a = np.ascontiguousarray(amax, dtype=np.float32)
    _check(load().gwe_model_set_fp8_amax(model, a.ctypes.data), "gwe_model_set_fp8_amax")


def gwe_model_get_fp8_amax(model: int, shape) -> np.ndarray:
    """The FP8 calibration maxima as float32 [n_models, 2, L, R] (`shape`)."""
    out = np.zeros(shape, dtype=np.float32)
    _check(load().gwe_model_get_fp8_amax(model, out.ctypes.data), "gwe_model_get_fp8_amax")
    return out


def gwe_model_destroy(model: int) -> None:
    if model:
        load().gwe_model_destroy(model)


def gwe_forward(model: int, strain_H, strain_L, n_samples: int, window: int, stride: int, slides,
                out_prob, stream=None) -> None:
    """Ensemble forward over one segment; out_prob [max(n_slides,1), n_models, n_windows, window] (device)."""
    if slides is None or len(slides) == 0:
        sl = None
        ns = 0
    else:
        sl = np.ascontiguousarray(slides, dtype=np.int32)
        ns = int(sl.shape[0])
    _check(load().gwe_forward(model, _dptr(strain_H), _dptr(strain_L), int(n_samples), int(window), int(stride),
                              sl.ctypes.data if sl is not None else None, ns, _dptr(out_prob), _stream(stream)),
           "gwe_forward")


def segment_windows(seg_len, window: int, stride: int) -> np.ndarray:
    """Windows per segment (int64), as gwe_forward_segments lays them out."""
    return np.array([gwe_n_windows(int(n), window, stride) for n in seg_len], dtype=np.int64)


def gwe_forward_segments(model: int, strain_H, strain_L, seg_start, seg_len, window: int, stride: int, slides,
                         out_prob, stream=None) -> None:
    """Ensemble forward over segments [seg_start[g], seg_start[g] + seg_len[g]) of the (device) strain;
    out_prob [max(n_slides,1), n_models, sum of windows, window] (device)."""
    s0 = np.ascontiguousarray(seg_start, dtype=np.int64)
    ln = np.ascontiguousarray(seg_len, dtype=np.int64)
    if s0.shape != ln.shape or s0.ndim != 1:
        raise ValueError("seg_start and seg_len must be 1-D of equal length")
    if slides is None or len(slides) == 0:
        sl, ns = None, 0
    else:
        sl = np.ascontiguousarray(slides, dtype=np.int32)
        ns = int(sl.shape[0])
    _check(load().gwe_forward_segments(model, _dptr(strain_H), _dptr(strain_L), s0.ctypes.data, ln.ctypes.data,
                                       int(s0.shape[0]), int(window), int(stride),
                                       sl.ctypes.data if sl is not None else None, ns, _dptr(out_prob),
                                       _stream(stream)), "gwe_forward_segments")


def gwe_triggers_segments(prob, n_models: int, n_slides: int, seg_len, window: int, stride: int, height_thr: float,
                          min_width: float, coinc: int, flags: int = GWE_TRIG_PER_MODEL, cap: int = 1 << 20,
                          stream=None):
    """(records of TRIGGER_DTYPE, their segment ids) over the segments of a gwe_forward_segments output."""
    lib = load()
    ln = np.ascontiguousarray(seg_len, dtype=np.int64)
    out = np.zeros(max(1, int(cap)), dtype=TRIGGER_DTYPE)
    seg = np.zeros(max(1, int(cap)), dtype=np.int32)
    n_out = ctypes.c_int64(0)
    st = lib.gwe_triggers_segments(_dptr(prob), int(n_models), int(n_slides), ln.ctypes.data, int(ln.shape[0]),
                                   int(window), int(stride), float(height_thr), float(min_width), int(coinc),
                                   int(flags), out.ctypes.data, seg.ctypes.data, int(cap), ctypes.byref(n_out),
                                   _stream(stream))
    _check(st, "gwe_triggers_segments")
    return out[:n_out.value].copy(), seg[:n_out.value].copy()


def gwe_forward_logits(model: int, x_H, x_L, batch: int, window: int, out_logit, stream=None) -> None:
    """Logits [n_models, batch, window] for explicit windows x_H, x_L [batch, window] (device)."""
    _check(load().gwe_forward_logits(model, _dptr(x_H), _dptr(x_L), int(batch), int(window), _dptr(out_logit),
                                     _stream(stream)), "gwe_forward_logits")


def gwe_backward(model: int, model_index: int, x_H, x_L, batch: int, window: int, dlogit, grad_weights,
                 grad_H=None, grad_L=None, stream=None) -> None:
    _check(load().gwe_backward(model, int(model_index), _dptr(x_H), _dptr(x_L), int(batch), int(window),
                               _dptr(dlogit), _dptr(grad_weights), _dptr(grad_H), _dptr(grad_L), _stream(stream)),
           "gwe_backward")


def gwe_triggers(prob, n_models: int, n_slides: int, n_windows: int, window: int, stride: int, height_thr: float,
                 min_width: float, coinc: int, flags: int = GWE_TRIG_PER_MODEL, cap: int = 1 << 20,
                 stream=None) -> np.ndarray:
    """Peaks and ensemble triggers (structured array of TRIGGER_DTYPE records)."""
    lib = load()
    out = np.zeros(max(1, int(cap)), dtype=TRIGGER_DTYPE)
    n_out = ctypes.c_int64(0)
    st = lib.gwe_triggers(_dptr(prob), int(n_models), int(n_slides), int(n_windows), int(window), int(stride),
                          float(height_thr), float(min_width), int(coinc), int(flags), out.ctypes.data, int(cap),
                          ctypes.byref(n_out), _stream(stream))
    _check(st, "gwe_triggers")
    return out[:n_out.value].copy()


def gwe_trigger_sweep(prob, n_models: int, n_slides: int, n_windows: int, window: int, stride: int, thresholds,
                      min_width: float, coinc: int, per_model: bool = True, stream=None):
    """(ensemble counts [slides, K], per-model peak counts [slides, models, K] or None) of a threshold sweep."""
    thr = np.ascontiguousarray(thresholds, dtype=np.float32)
    ns = max(1, int(n_slides))
    ens = np.zeros((ns, thr.shape[0]), dtype=np.int64)
    mod = np.zeros((ns, int(n_models), thr.shape[0]), dtype=np.int64) if per_model else None
    _check(load().gwe_trigger_sweep(_dptr(prob), int(n_models), int(n_slides), int(n_windows), int(window),
                                    int(stride), thr.ctypes.data, int(thr.shape[0]), float(min_width), int(coinc),
                                    ens.ctypes.data, mod.ctypes.data if mod is not None else None, _stream(stream)),
           "gwe_trigger_sweep")
    return ens, mod


def gwe_trigger_sweep_segments(prob, n_models: int, n_slides: int, seg_len, window: int, stride: int, thresholds,
                               min_width: float, coinc: int, per_model: bool = True, stream=None):
    """As gwe_trigger_sweep over the segments of a gwe_forward_segments output (counts summed)."""
    thr = np.ascontiguousarray(thresholds, dtype=np.float32)
    ln = np.ascontiguousarray(seg_len, dtype=np.int64)
    ns = max(1, int(n_slides))
    ens = np.zeros((ns, thr.shape[0]), dtype=np.int64)
    mod = np.zeros((ns, int(n_models), thr.shape[0]), dtype=np.int64) if per_model else None
    _check(load().gwe_trigger_sweep_segments(_dptr(prob), int(n_models), int(n_slides), ln.ctypes.data,
                                             int(ln.shape[0]), int(window), int(stride), thr.ctypes.data,
                                             int(thr.shape[0]), float(min_width), int(coinc), ens.ctypes.data,
                                             mod.ctypes.data if mod is not None else None, _stream(stream)),
           "gwe_trigger_sweep_segments")
    return ens, mod


def gwe_forward_static(model: int, strain_H, strain_L, n_samples: int, window: int, stride: int, out_prob,
                       status=None, stream=None) -> None:
    """Zero-lag forward that allocates no device memory (scratch in a fixed array of the library)."""
    _check(load().gwe_forward_static(model, _dptr(strain_H), _dptr(strain_L), int(n_samples), int(window),
                                     int(stride), _dptr(out_prob), _dptr(status), _stream(stream)),
           "gwe_forward_static")


def gwe_plan_create(model: int, strain_H, strain_L, seg_start, seg_len, window: int, stride: int, slides, out_prob,
                    flags: int = GWE_PLAN_AUTOTUNE, stream=None) -> int:
    """Forward plan over segments x slides recorded into one CUDA graph (see include/gwe.h); returns the handle."""
    s0 = np.ascontiguousarray(seg_start, dtype=np.int64)
    ln = np.ascontiguousarray(seg_len, dtype=np.int64)
    if s0.shape != ln.shape or s0.ndim != 1:
        raise ValueError("seg_start and seg_len must be 1-D of equal length")
    if slides is None or len(slides) == 0:
        sl, ns = None, 0
    else:
        sl = np.ascontiguousarray(slides, dtype=np.int32)
        ns = int(sl.shape[0])
    h = ctypes.c_void_p()
    _check(load().gwe_plan_create(model, _dptr(strain_H), _dptr(strain_L), s0.ctypes.data, ln.ctypes.data,
                                  int(s0.shape[0]), int(window), int(stride),
                                  sl.ctypes.data if sl is not None else None, ns, _dptr(out_prob), int(flags),
                                  _stream(stream), ctypes.byref(h)), "gwe_plan_create")
    return h.value


def gwe_plan_execute(plan: int, stream=None) -> None:
    """One launch of the plan's CUDA graph (asynchronous)."""
    _check(load().gwe_plan_execute(plan, _stream(stream)), "gwe_plan_execute")


def gwe_plan_shape(plan: int) -> dict:
    """Launch shape of a plan's slide heads (Hanford windows per block, offsets per piece, pieces per
    block), kernels in the graph, tuning times (ms)."""
    wt, ot, ppb, nk = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    t_ms, d_ms = ctypes.c_double(), ctypes.c_double()
    _check(load().gwe_plan_shape(plan, ctypes.byref(wt), ctypes.byref(ot), ctypes.byref(ppb), ctypes.byref(nk),
                                 ctypes.byref(t_ms), ctypes.byref(d_ms)), "gwe_plan_shape")
    return {"window_tile": wt.value, "offset_tile": ot.value, "pieces_per_block": ppb.value, "n_kernels": nk.value,
            "tuned_ms": t_ms.value, "default_ms": d_ms.value}


def gwe_set_slide_shape(window_tile: int = 4, offset_tile: int = 8, pieces_per_block: int = 0) -> None:
    """Slide-head shape of launches that are not autotuned (forward calls with slides and plans created
    without GWE_PLAN_AUTOTUNE), process-wide, from now on."""
    _check(load().gwe_set_slide_shape(int(window_tile), int(offset_tile), int(pieces_per_block)),
           "gwe_set_slide_shape")


def gwe_set_tensor_map_copies(on: bool) -> None:
    """Operand staging of the tensor-core backward's GEMMs, process-wide, from now on: tensor-map copies
    where the shapes allow (True, the default) or per-thread copies everywhere (False)."""
    _check(load().gwe_set_tensor_map_copies(1 if on else 0), "gwe_set_tensor_map_copies")


def gwe_plan_destroy(plan: int) -> None:
    if plan:
        load().gwe_plan_destroy(plan)


def gwe_search_create(model: int, window: int = 4096, stride: int = 2048, chunk_windows: int = 7151,
                      margin_windows: int = 16, guard_samples: int = 16384, fs: float = 4096.0, welch_seg: int = 16384,
                      input_dtype: int = GWE_INPUT_F32, input_scale: float = 1.0, height_thr: float = 0.5,
                      min_width: float = 2048.0, coinc: int = 2048, trigger_flags: int = 0) -> int:
    """Streaming search over a long raw two-detector stream (see include/gwe.h); returns the handle."""
    c = _SearchConfig(int(window), int(stride), int(chunk_windows), int(margin_windows), int(guard_samples),
                      float(fs), int(welch_seg), int(input_dtype), float(input_scale), float(height_thr),
                      float(min_width), int(coinc), int(trigger_flags))
    h = ctypes.c_void_p()
    _check(load().gwe_search_create(model, ctypes.byref(c), ctypes.byref(h)), "gwe_search_create")
    return h.value


def gwe_search_run(search: int, strain_H, strain_L, n_samples: int, cap: int = 1 << 20, stream=None) -> np.ndarray:
    """Records (TRIGGER_DTYPE) of the whole stream.  strain_H/L: CUDA tensors (device input) or host
    tensors / numpy arrays (host input; pin them for overlapped copies)."""
    def ptr(x):
        if hasattr(x, "is_cuda"):
            if not x.is_contiguous():
                raise ValueError("expected a contiguous tensor")
            return x.data_ptr(), bool(x.is_cuda)
        a = np.ascontiguousarray(x)
        return a.ctypes.data, False
    (ph, dh), (pl, dl) = ptr(strain_H), ptr(strain_L)
    if dh != dl:
        raise ValueError("strain_H and strain_L must both be on the device or both on the host")
    out = np.zeros(max(1, int(cap)), dtype=TRIGGER_DTYPE)
    n_out = ctypes.c_int64(0)
    _check(load().gwe_search_run(search, ph, pl, int(n_samples), 0 if dh else 1, out.ctypes.data, int(cap),
                                 ctypes.byref(n_out), _stream(stream)), "gwe_search_run")
    return out[:n_out.value].copy()


def gwe_search_chunks(search: int, n_samples: int) -> int:
    return int(load().gwe_search_chunks(search, int(n_samples)))


def _strain_ptrs(strain_H, strain_L):
    def ptr(x):
        if hasattr(x, "is_cuda"):
            if not x.is_contiguous():
                raise ValueError("expected a contiguous tensor")
            return x.data_ptr(), bool(x.is_cuda)
        a = np.ascontiguousarray(x)
        return a.ctypes.data, False
    (ph, dh), (pl, dl) = ptr(strain_H), ptr(strain_L)
    if dh != dl:
        raise ValueError("strain_H and strain_L must both be on the device or both on the host")
    return ph, pl, dh


def gwe_search_run_range(search: int, strain_H, strain_L, n_samples: int, chunk_begin: int, chunk_end: int,
                         cap: int = 1 << 20, stream=None) -> np.ndarray:
    """Records (TRIGGER_DTYPE) of chunks [chunk_begin, chunk_end) of the stream."""
    ph, pl, dev = _strain_ptrs(strain_H, strain_L)
    out = np.zeros(max(1, int(cap)), dtype=TRIGGER_DTYPE)
    n_out = ctypes.c_int64(0)
    _check(load().gwe_search_run_range(search, ph, pl, int(n_samples), 0 if dev else 1, int(chunk_begin),
                                       int(chunk_end), out.ctypes.data, int(cap), ctypes.byref(n_out),
                                       _stream(stream)), "gwe_search_run_range")
    return out[:n_out.value].copy()


def gwe_search_resumable(search: int, strain_H, strain_L, n_samples: int, checkpoint: str, chunks_per_step: int = 1,
                         max_steps=None, stream=None) -> np.ndarray:
    """Run a search in ranges of `chunks_per_step` chunks, saving the next chunk index and the records
    found so far to `checkpoint` (an .npz file) after every range, and continuing from it when it
    exists.  Returns the records so far (all of them once the last chunk is done); stops early after
    `max_steps` ranges if given."""
    import os
    n_chunks = gwe_search_chunks(search, n_samples)
    nxt, recs = 0, np.zeros(0, dtype=TRIGGER_DTYPE)
    if os.path.exists(checkpoint):
        z = np.load(checkpoint)
        if int(z["n_samples"]) != int(n_samples) or int(z["n_chunks"]) != n_chunks:
            raise ValueError("checkpoint belongs to another stream")
        nxt, recs = int(z["next_chunk"]), z["records"].astype(TRIGGER_DTYPE)
    steps = 0
    while nxt < n_chunks and (max_steps is None or steps < max_steps):
        end = min(n_chunks, nxt + int(chunks_per_step))
        part = gwe_search_run_range(search, strain_H, strain_L, n_samples, nxt, end, stream=stream)
        recs = np.concatenate([recs, part])
        nxt = end
        steps += 1
        tmp = checkpoint + ".tmp.npz"
        np.savez(tmp, next_chunk=nxt, n_chunks=n_chunks, n_samples=int(n_samples), records=recs)
        os.replace(tmp, checkpoint)
    return recs


def gwe_search_destroy(search: int) -> None:
    if search:
        load().gwe_search_destroy(search)


def gwe_set_cross_window_reuse(enable: bool) -> None:
    """Process-wide switch of the tensor-core path's cross-window reuse (results are bit-identical)."""
    _check(load().gwe_set_cross_window_reuse(1 if enable else 0), "gwe_set_cross_window_reuse")


def gwe_debug_config(drop: int, wait_seconds: float) -> None:
    """Failure-detection test hook: bound of device waits and a dropped producer (see include/gwe.h)."""
    _check(load().gwe_debug_config(int(drop), float(wait_seconds)), "gwe_debug_config")


def gwe_debug_ring_margin(nbytes: int) -> None:
    """Test hook of the kernel's address checks (see include/gwe.h)."""
    _check(load().gwe_debug_ring_margin(int(nbytes)), "gwe_debug_ring_margin")


def gwe_sync(model: int, stream=None) -> None:
    """Wait for the stream and raise if a device-side wait of the handle's kernels timed out."""
    _check(load().gwe_sync(model, _stream(stream)), "gwe_sync")


def gwe_whiten(strain, n: int, fs: float, seg_len: int, out, flags: int = 0, stream=None) -> None:
    _check(load().gwe_whiten(_dptr(strain), int(n), float(fs), int(seg_len), int(flags), _dptr(out),
                             _stream(stream)), "gwe_whiten")


class _WhitenOptions(ctypes.Structure):
    _fields_ = [("psd_average", ctypes.c_int), ("tukey_alpha", ctypes.c_double), ("f_low", ctypes.c_double)]


def gwe_whiten_ex(strain, n: int, fs: float, seg_len: int, out, psd_average: int = GWE_PSD_MEAN,
                  tukey_alpha: float = 0.0, f_low: float = 15.0, stream=None) -> None:
    """Whitening with options: mean or median Welch PSD, Tukey taper, low-frequency cut."""
    o = _WhitenOptions(int(psd_average), float(tukey_alpha), float(f_low))
    _check(load().gwe_whiten_ex(_dptr(strain), int(n), float(fs), int(seg_len), ctypes.byref(o), _dptr(out),
                                _stream(stream)), "gwe_whiten_ex")


def gwe_profile_enable(on: bool = True) -> None:
    _check(load().gwe_profile_enable(1 if on else 0), "gwe_profile_enable")


def gwe_profile_read() -> dict:
    """{kernel name: (total device ms, launches)} of the launches recorded since gwe_profile_enable."""
    lib = load()
    out = {}
    i = 0
    buf = ctypes.create_string_buffer(128)
    while True:
        ms = ctypes.c_double(0.0)
        n = ctypes.c_int64(0)
        if lib.gwe_profile_read(i, buf, 128, ctypes.byref(ms), ctypes.byref(n)) != 0:
            break
        out[buf.value.decode()] = (ms.value, n.value)
        i += 1
    return out


class Model:
    """Owning wrapper of a gwe_model handle."""

    def __init__(self, cfg, host_weights: np.ndarray, precision: int = GWE_FP32):
        self.cfg = dict(cfg)
        self.precision = int(precision)
        self.handle = gwe_model_create(cfg, host_weights, precision)
        self.weights_token = 0      # changes whenever the handle's weights are replaced through set_weights*

    def set_weights(self, host_weights: np.ndarray) -> None:
        gwe_model_set_weights(self.handle, host_weights)
        self.weights_token += 1

    def set_weights_device(self, weights, stream=None) -> int:
        """Replace the weights from a CUDA FP32 tensor; returns the new weights token."""
        gwe_model_set_weights_device(self.handle, weights.detach().float().contiguous(), stream)
        self.weights_token += 1
        return self.weights_token

    def close(self):
        if getattr(self, "handle", None):
            gwe_model_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def forward(self, strain_H, strain_L, window: int, stride: int, slides=None, out=None, stream=None):
        import torch
        n = int(strain_H.shape[0])
        nw = gwe_n_windows(n, window, stride)
        ns = 1 if slides is None or len(slides) == 0 else len(slides)
        if out is None:
            out = torch.empty((ns, int(self.cfg["n_models"]), nw, window), dtype=torch.float32,
                              device=strain_H.device)
        gwe_forward(self.handle, strain_H, strain_L, n, window, stride, slides, out, stream)
        return out

    def sync(self, stream=None):
        gwe_sync(self.handle, stream)

    def calibrate(self, strain_H, strain_L, window: int, stride: int, stream=None):
        gwe_model_calibrate(self.handle, strain_H, strain_L, int(strain_H.shape[0]), window, stride, stream)

    def _amax_shape(self):
        c = self.cfg
        return (int(c["n_models"]), 2, int(c["stacks"]) * int(c["layers_per_stack"]), int(c["r_ch"]))

    @property
    def fp8_amax(self) -> np.ndarray:
        return gwe_model_get_fp8_amax(self.handle, self._amax_shape())

    @fp8_amax.setter
    def fp8_amax(self, amax) -> None:
        a = np.asarray(amax, dtype=np.float32)
        if a.shape != self._amax_shape():
            raise ValueError(f"amax must have shape {self._amax_shape()}")
        gwe_model_set_fp8_amax(self.handle, a)

    def logits(self, x_H, x_L, out=None, stream=None):
        import torch
        B, W = int(x_H.shape[0]), int(x_H.shape[1])
        if out is None:
            out = torch.empty((int(self.cfg["n_models"]), B, W), dtype=torch.float32, device=x_H.device)
        gwe_forward_logits(self.handle, x_H, x_L, B, W, out, stream)
        return out


def _autograd_function():
    import torch

    class GweLogits(torch.autograd.Function):
        """Logits of a one-member handle as a differentiable function of its FP32 weight blob
        and of the two detector windows; the backward pass runs gwe_backward."""

        @staticmethod
        def forward(ctx, weights, x_H, x_L, model):
            if int(model.cfg["n_models"]) != 1:
                raise ValueError("GweLogits needs a one-member handle")
            if not weights.is_cuda:
                raise ValueError("GweLogits: the weight blob must be a CUDA tensor")
            # weights go to the handle on the device (no host round trip); the token identifies them
            ctx.wtoken = model.set_weights_device(weights)
            out = model.logits(x_H.contiguous(), x_L.contiguous())[0]
            ctx.save_for_backward(weights, x_H, x_L)
            ctx.model = model
            ctx.wdevice = weights.device
            return out

        @staticmethod
        def backward(ctx, grad_out):
            weights, x_H, x_L = ctx.saved_tensors
            model = ctx.model
            if model.weights_token != ctx.wtoken:
                # another forward replaced the handle's weights since this one: restore this
                # forward's weights (saved_tensors raises if they were modified in place)
                ctx.wtoken = model.set_weights_device(weights)
            B, W = int(x_H.shape[0]), int(x_H.shape[1])
            dev = x_H.device
            gw = torch.empty(gwe_param_count(model.cfg), dtype=torch.float32, device=dev)
            gH = torch.empty((B, W), dtype=torch.float32, device=dev) if ctx.needs_input_grad[1] else None
            gL = torch.empty((B, W), dtype=torch.float32, device=dev) if ctx.needs_input_grad[2] else None
            gwe_backward(model.handle, 0, x_H.contiguous(), x_L.contiguous(), B, W,
                         grad_out.contiguous().float(), gw, gH, gL)
            return gw.to(ctx.wdevice), gH, gL, None

    return GweLogits


_GWE_LOGITS = None


def gwe_logits_autograd(model, weights, x_H, x_L):
    """Differentiable logits [batch, window] of a one-member handle (weights: FP32 blob [P])."""
    global _GWE_LOGITS
    if _GWE_LOGITS is None:
        _GWE_LOGITS = _autograd_function()
    return _GWE_LOGITS.apply(weights, x_H, x_L, model)
