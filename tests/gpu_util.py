"""Helpers shared by the GPU tests (no method arithmetic here)."""
import numpy as np
import pytest


def require_gpu():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device (GB300)"
    import paper_2201_11133_gb300 as gwe
    gwe.build()
    gwe.load()
    return torch.device("cuda:0")


def sigmoid(x):
    return 1.0 / (1.0 + np.exp(-np.asarray(x, dtype=np.float64)))


def smooth_prob(rng, shape, width=301):
    """Smooth random series in (0, 1) with peaks of a few hundred samples."""
    n = int(np.prod(shape[:-1]))
    L = shape[-1]
    out = np.empty((n, L), dtype=np.float32)
    k = np.hanning(width)
    k /= k.sum()
    for i in range(n):
        x = np.convolve(rng.standard_normal(L + width - 1) * 8.0, k, mode="valid")
        out[i] = (1.0 / (1.0 + np.exp(-x))).astype(np.float32)
    return out.reshape(shape)
