"""The device whitening front end against the FP64 oracle (numpy) on coloured
Gaussian noise drawn from the analytic detector spectrum."""
import numpy as np
import pytest

import workload
from gpu_util import require_gpu
from oracle import whiten as ow

pytestmark = pytest.mark.gpu

FS = 4096.0


def _gpu_whiten(x, seg):
    import torch
    import paper_2201_11133_gb300 as gwe
    dev = require_gpu()
    xt = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).to(dev)
    out = torch.empty_like(xt)
    gwe.gwe_whiten(xt, xt.numel(), FS, seg, out)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("n,seg", [(64 * 4096, 16384), (100000 + 7, 4096), (3600 * 4096, 16384)])
def test_whiten_matches_oracle(n, seg):
    x = workload.coloured_noise(n, seed=2024).astype(np.float32)
    ref = ow.whiten(x.astype(np.float64), FS, seg)
    got = _gpu_whiten(x, seg)
    err = np.abs(got - ref)
    print(f"n={n}: max |dy| {err.max():.2e}, rms {np.sqrt(np.mean(err ** 2)):.2e}")
    # FP32 transforms of up to 2^24 points: a few 1e-6 of relative error per bin
    assert err.max() <= 2e-4
    assert np.sqrt(np.mean(err ** 2)) <= 1e-5
    assert abs(np.std(got) - 1.0) < 1e-5


def test_whiten_argument_errors():
    import torch
    import paper_2201_11133_gb300 as gwe
    dev = require_gpu()
    x = torch.zeros(5000, device=dev)
    out = torch.zeros(5000, device=dev)
    for args in [(x, 5000, FS, 1000, out), (x, 5000, FS, 8192, out), (x, 5000, -1.0, 1024, out), (x, 5000, FS, 1024, x)]:
        with pytest.raises(gwe.GweError) as ei:
            gwe.gwe_whiten(*args)
        assert ei.value.status == 1
