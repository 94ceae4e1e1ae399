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


@pytest.mark.parametrize("average,alpha,n", [("median", 0.0, 64 * 4096), ("median", 0.1, 100000 + 7),
                                             ("mean", 0.1, 64 * 4096), ("median", 0.0, 3600 * 4096)])
def test_whiten_variants_match_oracle(average, alpha, n):
    """Median-averaged Welch PSD and Tukey-tapered whitening, on coloured noise with loud sine-Gaussian
    glitches in it (what the median average is for)."""
    import torch
    import paper_2201_11133_gb300 as gwe
    dev = require_gpu()
    x = workload.coloured_noise(n, seed=2025)
    xl = np.zeros_like(x)
    workload.add_glitches(x, xl, max(1, n // (30 * 4096)), seed=5, snr_range=(50.0, 200.0))
    x = x.astype(np.float32)
    seg = 16384 if n >= 64 * 4096 else 4096
    ref = ow.whiten(x.astype(np.float64), FS, seg, average=average, tukey_alpha=alpha)
    xt = torch.from_numpy(x).to(dev)
    out = torch.empty_like(xt)
    gwe.gwe_whiten_ex(xt, n, FS, seg, out, psd_average=gwe.GWE_PSD_MEDIAN if average == "median" else gwe.GWE_PSD_MEAN,
                      tukey_alpha=alpha)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    err = np.abs(got - ref)
    print(f"{average} alpha={alpha} n={n}: max |dy| {err.max():.2e}, rms {np.sqrt(np.mean(err ** 2)):.2e}")
    assert err.max() <= 2e-4
    assert np.sqrt(np.mean(err ** 2)) <= 1e-5
    assert abs(np.std(got) - 1.0) < 1e-5


def test_whiten_ex_argument_errors():
    import torch
    import paper_2201_11133_gb300 as gwe
    dev = require_gpu()
    x = torch.zeros(5000, device=dev)
    out = torch.zeros(5000, device=dev)
    for kw in [dict(psd_average=2), dict(tukey_alpha=1.5), dict(tukey_alpha=-0.1), dict(f_low=3000.0)]:
        with pytest.raises(gwe.GweError) as ei:
            gwe.gwe_whiten_ex(x, 5000, FS, 1024, out, **kw)
        assert ei.value.status == 1
