"""Failure detection without a GPU fault: a producer that issues nothing makes a
bounded device-side wait run out (limit 0.2 s); the kernel records the wait
site and returns, gwe_sync reports GWE_ERR_TIMEOUT, and the same context then
runs a normal forward that matches the oracle."""
import numpy as np
import pytest

import oracle
import workload
from gpu_util import require_gpu

pytestmark = pytest.mark.gpu


def test_dropped_producer_times_out_and_context_survives():
    import torch
    import paper_2201_11133_gb300 as gwe
    dev = require_gpu()
    cfg = workload.config("small")
    W, stride = 1024, 512
    n = W + 3 * stride
    sh, sl, _ = workload.stream(n, seed=51)
    wb = workload.init_weights(cfg, seed=3900, bias_std=0.1)
    m = gwe.Model(cfg, wb, gwe.GWE_BF16)
    H, L = torch.from_numpy(sh).to(dev), torch.from_numpy(sl).to(dev)
    try:
        gwe.gwe_debug_config(1, 0.2)
        m.forward(H, L, W, stride)
        with pytest.raises(gwe.GweError) as ei:
            m.sync()
        assert ei.value.status == 4
        assert "timed out" in str(ei.value)
    finally:
        gwe.gwe_debug_config(0, 4.0)
    out = m.forward(H, L, W, stride)
    m.sync()
    ref = oracle.forward_stream(cfg, wb, sh, sl, W, stride)
    assert np.max(np.abs(out.cpu().numpy() - ref)) <= 1e-2
    m.close()


def test_debug_config_rejects_bad_arguments():
    import paper_2201_11133_gb300 as gwe
    require_gpu()
    for drop, wait in [(2, 1.0), (-1, 1.0), (0, 0.0), (0, 100.0)]:
        with pytest.raises(gwe.GweError) as ei:
            gwe.gwe_debug_config(drop, wait)
        assert ei.value.status == 1


def test_address_check_stops_the_copies_and_is_reported():
    """The ring is reported 4 KiB smaller to the kernel's address checks: the lag copies that would
    reach into the missing part are not made, the site is recorded, gwe_sync reports it, and a normal
    forward on the same context matches the oracle afterwards.  No access outside the real ring is
    made at any point (the real ring is larger than the checked size)."""
    import torch
    import paper_2201_11133_gb300 as gwe
    dev = require_gpu()
    cfg = workload.config("small")
    W, stride = 1024, 512
    n = W + 3 * stride
    sh, sl, _ = workload.stream(n, seed=52)
    wb = workload.init_weights(cfg, seed=3901, bias_std=0.1)
    m = gwe.Model(cfg, wb, gwe.GWE_BF16)
    H, L = torch.from_numpy(sh).to(dev), torch.from_numpy(sl).to(dev)
    try:
        gwe.gwe_debug_config(0, 0.2)
        gwe.gwe_debug_ring_margin(1 << 40)        # every lag source fails the check
        m.forward(H, L, W, stride)
        with pytest.raises(gwe.GweError) as ei:
            m.sync()
        assert ei.value.status == 2
        assert "address check" in str(ei.value)
    finally:
        gwe.gwe_debug_ring_margin(0)
        gwe.gwe_debug_config(0, 4.0)
    out = m.forward(H, L, W, stride)
    m.sync()
    ref = oracle.forward_stream(cfg, wb, sh, sl, W, stride)
    assert np.max(np.abs(out.cpu().numpy() - ref)) <= 1e-2
    m.close()
