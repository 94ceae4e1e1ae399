"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/gwe.h declares (no compute call: this runs without a GPU)."""
import ctypes
import os
import re

import paper_2201_11133_gb300 as gwe

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(gwe_[a-z0-9_]+)\s*\(", txt))
    return names


def test_library_exports_every_declared_symbol():
    path = gwe.build()
    assert os.path.exists(path)
    lib = ctypes.CDLL(path)
    names = _declared()
    assert {"gwe_model_create", "gwe_forward", "gwe_backward", "gwe_triggers"} <= names
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_host_only_calls():
    assert gwe.gwe_version().startswith("gwe")
    cfg = dict(n_models=4, stacks=3, layers_per_stack=10, kernel=2, r_ch=64, s_ch=128, head_ch=256)
    assert gwe.gwe_param_count(cfg) == 1805825
    assert gwe.gwe_n_windows(14745600, 4096, 2048) == 7199
    assert gwe.gwe_n_windows(4095, 4096, 2048) == 0
    assert gwe.gwe_n_windows(4096 + 2047, 4096, 2048) == 1
    bad = dict(cfg, r_ch=0)
    assert gwe.gwe_param_count(bad) == -1


def test_model_create_without_gpu_fails_loudly():
    import torch
    if torch.cuda.is_available():
        return
    cfg = dict(n_models=1, stacks=1, layers_per_stack=8, kernel=2, r_ch=32, s_ch=32, head_ch=32)
    import numpy as np
    w = np.zeros(gwe.gwe_param_count(cfg), dtype=np.float32)
    try:
        gwe.gwe_model_create(cfg, w, gwe.GWE_FP32)
    except gwe.GweError as e:
        assert e.status == 2
    else:
        raise AssertionError("model creation succeeded without a GPU")


def test_reuse_switch_host_only():
    gwe.gwe_set_cross_window_reuse(False)
    gwe.gwe_set_cross_window_reuse(True)
    try:
        gwe._check(gwe.load().gwe_set_cross_window_reuse(2), "gwe_set_cross_window_reuse")
    except gwe.GweError as e:
        assert e.status == 1
    else:
        raise AssertionError("enable = 2 accepted")
