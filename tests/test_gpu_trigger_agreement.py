"""Trigger-set agreement between the tensor-core path and the FP64 oracle on the
same strain: ensemble triggers found on the device from the device's
probabilities against those the oracle finds from its own probabilities.
Reading of "trigger agreement": triggers match when their indices differ by at
most 256 samples; triggers whose oracle height lies within the probability
tolerance of the threshold, or whose width lies within 1 % of the minimum
width, are marginal and counted separately (they may flip either way)."""
import numpy as np
import pytest

import oracle
import workload
from gpu_util import require_gpu

pytestmark = pytest.mark.gpu

TOL = 1e-2


def _match(a, b, radius=256):
    a, b = np.sort(np.asarray(a)), np.sort(np.asarray(b))
    used = np.zeros(len(b), dtype=bool)
    hits = 0
    for x in a:
        j = np.searchsorted(b, x - radius)
        while j < len(b) and b[j] <= x + radius:
            if not used[j]:
                used[j] = True
                hits += 1
                break
            j += 1
    return hits


@pytest.mark.parametrize("q", [0.5, 0.8])
def test_trigger_agreement(q):
    """Random-init models give jagged probability series (median prominence ~0.15), so the
    threshold sweep uses quantiles of the oracle's probabilities and no width cut."""
    import torch
    import paper_2201_11133_gb300 as gwe
    dev = require_gpu()
    cfg = workload.config("small", n_models=4)
    W, stride = 1024, 512
    n = W + 40 * stride
    sh, sl, _ = workload.stream(n, seed=61, n_inj=2)
    wb = workload.init_weights(cfg, seed=3000, bias_std=0.1)
    ref = oracle.forward_stream(cfg, wb, sh, sl, W, stride).astype(np.float32)
    thr = float(np.quantile(ref, q))
    coinc = 2048
    per_model, ens = oracle.triggers(ref, W, stride, thr, 0.0, coinc)
    m = gwe.Model(cfg, wb, gwe.GWE_BF16)
    prob = m.forward(torch.from_numpy(sh).to(dev), torch.from_numpy(sl).to(dev), W, stride)
    m.sync()
    recs = gwe.gwe_triggers(prob, 4, 1, prob.shape[2], W, stride, thr, 0.0, coinc)
    for mi in range(4):
        idx, h, pr, _ = per_model[0][mi]
        solid = idx[(pr >= 0.05) & (np.abs(h - thr) > TOL)]
        got_m = recs[recs["model"] == mi]["index"]
        if len(solid):
            recall = _match(solid, got_m) / len(solid)
            print(f"q {q} model {mi}: {len(idx)} oracle peaks, {len(solid)} solid, recall {recall:.5f}")
            assert recall >= 0.999
    got = recs[recs["model"] == -1]["index"]
    idx0, h0, pr0, _ = per_model[0][0]
    info = {int(i): (hh, pp) for i, hh, pp in zip(idx0, h0, pr0)}
    marginal = {int(i) for i in ens[0] if abs(info[int(i)][0] - thr) <= TOL or info[int(i)][1] < 0.05}
    solid_e = [int(i) for i in ens[0] if int(i) not in marginal]
    hits = _match(solid_e, got)
    union = len(solid_e) + len(got) - _match(got, ens[0])
    jacc = hits / max(1, len(solid_e))
    print(f"q {q}: {len(ens[0])} oracle ensemble triggers ({len(marginal)} marginal), device {len(got)}, "
          f"solid recall {jacc:.5f}")
    assert len(solid_e) > 0
    assert jacc >= 0.999
    m.close()
