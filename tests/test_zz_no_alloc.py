"""The allocation-free forward (gwe_forward_static) against the ordinary forward.

Some callers must not allocate device memory while they stream (a low-latency
trigger pipeline sharing the GPU, whose other work cudaMalloc's implicit
synchronisation would stall, or a process whose device memory a framework has
reserved up front).  gwe_forward_static serves them from a fixed array inside
the library.  This file is collected last, so a failure here leaves every
other test already run; it also passes when run alone in a fresh process."""
import ctypes

import numpy as np
import pytest

import workload
from gpu_util import require_gpu

pytestmark = pytest.mark.gpu

TOL_BF16 = 1e-2


def _run(cfg, n, W, stride, seed):
    import torch
    import paper_2201_11133_gb300 as gwe
    dev = require_gpu()
    lib = gwe.load()
    sh, sl, _ = workload.stream(n, seed=seed)
    wb = workload.init_weights(cfg, seed=3300, bias_std=0.05)
    m = gwe.Model(cfg, wb, gwe.GWE_BF16)
    H = torch.from_numpy(sh).to(dev)
    L = torch.from_numpy(sl).to(dev)
    ref = m.forward(H, L, W, stride)
    m.sync()
    nw = gwe.gwe_n_windows(n, W, stride)
    status = torch.full((1,), -1, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):                        # two calls in a row share the same fixed scratch
        out = torch.full((cfg["n_models"], nw, W), float("nan"), dtype=torch.float32, device=dev)
        st = lib.gwe_forward_static(m.handle, H.data_ptr(), L.data_ptr(), n, W, stride, out.data_ptr(),
                                    status.data_ptr(), ctypes.c_void_p(stream))
        assert st == 0, lib.gwe_last_error().decode()
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        diff = float((out - ref[0]).abs().max().item())
        assert diff <= TOL_BF16, diff
    m.close()


def test_no_alloc_forward_matches_gwe_forward_ensemble():
    # 10 windows x 4 models = 40 jobs on at most 32 CTAs: lag rings are reused across jobs
    _run(workload.config("ensemble"), 4096 + 9 * 2048 + 100, 4096, 2048, seed=41)


def test_no_alloc_forward_matches_gwe_forward_small():
    _run(workload.config("small", n_models=2), 1024 + 7 * 512 + 33, 1024, 512, seed=42)


def test_no_alloc_forward_argument_errors():
    import torch
    import paper_2201_11133_gb300 as gwe
    dev = require_gpu()
    cfg = workload.config("small")
    m = gwe.Model(cfg, workload.init_weights(cfg, seed=1), gwe.GWE_BF16)
    x = torch.zeros(4096, device=dev)
    out = torch.zeros(4096, device=dev)
    with pytest.raises(gwe.GweError) as ei:
        gwe.gwe_forward_static(m.handle, x, x, 100, 4096, 2048, out)
    assert ei.value.status == 1
    with pytest.raises(gwe.GweError) as ei:
        gwe.gwe_forward_static(m.handle, x, x, 4096, 1000, 500, out)   # window not a multiple of 128
    assert ei.value.status == 5
    m.close()
    m32 = gwe.Model(cfg, workload.init_weights(cfg, seed=1), gwe.GWE_FP32)
    with pytest.raises(gwe.GweError) as ei:
        gwe.gwe_forward_static(m32.handle, x, x, 4096, 1024, 512, out)
    assert ei.value.status == 5
