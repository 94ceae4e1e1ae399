"""The allocation-free forward (gwe_forward_static) against the ordinary forward.

Some callers must not allocate device memory while they stream: a low-latency
trigger pipeline that shares the GPU with other work (cudaMalloc synchronises
the device and would stall that work), or a process whose device memory a
framework's pool has reserved up front.  gwe_forward_static serves them from a
fixed array inside the library.  Checked here: its output equals gwe_forward's
within the tensor-core tolerance on two calls in a row; a first call on a fresh
handle; a NULL status word (a timeout then surfaces through gwe_sync); and
repeated calls leave the device's free memory unchanged.  This file is
collected last, so a failure here leaves every other test already run; it also
passes when run alone in a fresh process."""
import ctypes

import numpy as np
import pytest

import workload
from gpu_util import require_gpu

pytestmark = pytest.mark.gpu

TOL_BF16 = 1e-2


def _static(lib, m, H, L, n, W, stride, out, status):
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    st = lib.gwe_forward_static(m.handle, H.data_ptr(), L.data_ptr(), n, W, stride, out.data_ptr(),
                                status.data_ptr() if status is not None else None, ctypes.c_void_p(stream))
    assert st == 0, lib.gwe_last_error().decode()


def _run(cfg, n, W, stride, seed, static_first=False):
    import torch
    import paper_2201_11133_gb300 as gwe
    dev = require_gpu()
    lib = gwe.load()
    sh, sl, _ = workload.stream(n, seed=seed)
    wb = workload.init_weights(cfg, seed=3300, bias_std=0.05)
    m = gwe.Model(cfg, wb, gwe.GWE_BF16)
    H = torch.from_numpy(sh).to(dev)
    L = torch.from_numpy(sl).to(dev)
    nw = gwe.gwe_n_windows(n, W, stride)
    status = torch.full((1,), -1, dtype=torch.int32, device=dev)
    first = None
    if static_first:                          # the handle's first forward is the static one
        first = torch.full((cfg["n_models"], nw, W), float("nan"), dtype=torch.float32, device=dev)
        _static(lib, m, H, L, n, W, stride, first, None)
        m.sync()
    ref = m.forward(H, L, W, stride)
    m.sync()
    if first is not None:
        assert float((first - ref[0]).abs().max().item()) <= TOL_BF16
    for _ in range(2):                        # two calls in a row share the same fixed scratch
        out = torch.full((cfg["n_models"], nw, W), float("nan"), dtype=torch.float32, device=dev)
        _static(lib, m, H, L, n, W, stride, out, status)
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


def test_no_alloc_forward_first_call_on_fresh_handle():
    _run(workload.config("small", n_models=2), 1024 + 5 * 512, 1024, 512, seed=43, static_first=True)


def test_no_alloc_forward_allocates_nothing_and_null_status():
    import torch
    import paper_2201_11133_gb300 as gwe
    dev = require_gpu()
    lib = gwe.load()
    cfg = workload.config("ensemble")
    W, stride = 4096, 2048
    n = W + 5 * stride
    sh, sl, _ = workload.stream(n, seed=44)
    m = gwe.Model(cfg, workload.init_weights(cfg, seed=3301, bias_std=0.05), gwe.GWE_BF16)
    H = torch.from_numpy(sh).to(dev)
    L = torch.from_numpy(sl).to(dev)
    nw = gwe.gwe_n_windows(n, W, stride)
    outs = [torch.empty((cfg["n_models"], nw, W), dtype=torch.float32, device=dev) for _ in range(3)]
    _static(lib, m, H, L, n, W, stride, outs[0], None)    # warm-up: symbol lookup, module loaded
    m.sync()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info(dev)[0]
    for k in (1, 2):
        _static(lib, m, H, L, n, W, stride, outs[k], None)
    m.sync()                                               # status NULL: gwe_sync reports failures
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info(dev)[0] == free0
    assert torch.equal(outs[1], outs[2])
    ref = m.forward(H, L, W, stride)
    m.sync()
    assert float((outs[2] - ref[0]).abs().max().item()) <= TOL_BF16
    m.close()


def test_no_alloc_forward_timeout_with_null_status_reaches_gwe_sync():
    import torch
    import paper_2201_11133_gb300 as gwe
    dev = require_gpu()
    lib = gwe.load()
    cfg = workload.config("small")
    W, stride = 1024, 512
    n = W + 3 * stride
    sh, sl, _ = workload.stream(n, seed=45)
    m = gwe.Model(cfg, workload.init_weights(cfg, seed=3302, bias_std=0.1), gwe.GWE_BF16)
    H = torch.from_numpy(sh).to(dev)
    L = torch.from_numpy(sl).to(dev)
    nw = gwe.gwe_n_windows(n, W, stride)
    out = torch.empty((1, nw, W), dtype=torch.float32, device=dev)
    try:
        gwe.gwe_debug_config(1, 0.2)          # a producer that issues nothing: a bounded wait runs out
        _static(lib, m, H, L, n, W, stride, out, None)
        with pytest.raises(gwe.GweError) as ei:
            m.sync()
        assert ei.value.status == 4
    finally:
        gwe.gwe_debug_config(0, 4.0)
    _static(lib, m, H, L, n, W, stride, out, None)
    m.sync()
    ref = m.forward(H, L, W, stride)
    m.sync()
    assert float((out - ref[0]).abs().max().item()) <= TOL_BF16
    m.close()


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
