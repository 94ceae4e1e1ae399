"""Host-side arithmetic of bench.py (no GPU): the algorithmic byte count behind the training
roofline."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402
import workload  # noqa: E402


def test_training_roofline_bytes():
    cfg = dict(workload.config("ensemble"), n_models=1)
    R, S, L = cfg["r_ch"], cfg["s_ch"], workload.n_layers(cfg)
    # per row and layer: conv x in (2R), gate cache (4R) and z (2R) out; residual z (2R) and x
    # (4R) in, x out in FP32 (4R) and BF16 (2R); dz dL/dx (2R), dL/dskip (2S) and the gate cache
    # (4R) in, da (4R) out; dgrad da (4R) and dL/dx (4R) in, dL/dx out in FP32 (4R) and BF16 (2R)
    per_row_layer = (2 * R + 4 * R + 2 * R) + (2 * R + 4 * R + 4 * R + 2 * R) + (2 * R + 2 * S + 4 * R + 4 * R) \
        + (4 * R + 4 * R + 4 * R + 2 * R)
    r = bench.training_roofline(cfg, 256, 4096, {"k_tc_rows": {"ms_per_step": 100.0}}, {"hbm_gbs": 5000.0},
                                "measured")
    assert r["bytes_per_step"] == 2 * 256 * 4096 * L * per_row_layer
    assert abs(r["achieved"] - r["bytes_per_step"] / 0.1 / 1e9) < 1e-6
    assert abs(r["frac"] - r["achieved"] / 5000.0) < 1e-12
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert bench.training_roofline(cfg, 256, 4096, {}, {"hbm_gbs": 5000.0}, "measured") is None
