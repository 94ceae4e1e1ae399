"""BF16 reading of the backward pass (test infrastructure: only tests/ and
bench.py's CPU legs use it).

The paper trains its models in mixed precision without stating the scheme
(section "Materials and Methods", paragraph "AI ensemble construction"); this
module states the reading the tensor-core backward implements: FP64 arithmetic
everywhere, except that the two operands of every contraction of the branches
(the dilated convolution, the residual and skip projections, and in the
backward the dz, dgrad and weight-gradient contractions) are rounded to BF16
(round to nearest even) first.  The head's contractions take their operands
rounded as the kernels do: u = h . W_h1^T from FP16 h and W_h1 (the forward
kernel's head operands), dh = du . W_h1 from BF16 du and W_h1, and
dW_h1 = du^T h from the BF16 splits x = hi + lo (hi = BF16(x), lo = BF16(x - hi))
of du and h as hi.hi + hi.lo + lo.hi.  The biases, the input projection and every elementwise step are
exact.  With rounding switched off it is the plain
reverse-mode gradient of the network (pinned against the C oracle's
`backward`, which is pinned by finite differences).

Layout of the gradient: the model's blob (workload.param_layout).
"""
from __future__ import annotations

import numpy as np


def bf16_round(x) -> np.ndarray:
    """Round to the nearest BF16 value, ties to even (float64 in, float64 out)."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64).astype(np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    nan = np.isnan(a)
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    out[nan] = np.nan
    return out


def f16_round(x) -> np.ndarray:
    """Round to the nearest FP16 value, ties to even (float64 in, float64 out)."""
    return np.asarray(x, dtype=np.float64).astype(np.float16).astype(np.float64)


def _lag(x, s, W):
    """Row t of the result is row t + s of x within each window (zero outside [0, W)); x [B, W, C]."""
    out = np.zeros_like(x)
    if abs(s) >= W:
        return out
    if s >= 0:
        out[:, :W - s] = x[:, s:]
    else:
        out[:, -s:] = x[:, :W + s]
    return out


def backward(cfg, offsets, blob, xh, xl, dlogit, rounding: bool = True):
    """(dL/dblob, dL/dx_H, dL/dx_L) for windows xh, xl [B, W] and dL/dlogit [B, W].

    offsets: {name: (offset, shape)} of the blob (workload.param_offsets)."""
    q = bf16_round if rounding else (lambda v: np.asarray(v, dtype=np.float64))
    q16 = f16_round if rounding else (lambda v: np.asarray(v, dtype=np.float64))
    R, S = int(cfg["r_ch"]), int(cfg["s_ch"])
    lps = int(cfg["layers_per_stack"])
    L = int(cfg["stacks"]) * lps
    xh = np.asarray(xh, dtype=np.float64)
    xl = np.asarray(xl, dtype=np.float64)
    dlogit = np.asarray(dlogit, dtype=np.float64)
    B, W = xh.shape
    blob = np.asarray(blob, dtype=np.float64)

    def par(name):
        o, shape = offsets[name]
        return blob[o:o + int(np.prod(shape))].reshape(shape)

    sig = lambda v: 1.0 / (1.0 + np.exp(-v))
    grad = {name: np.zeros(shape) for name, (_, shape) in offsets.items()}
    saved, skips = {}, {}
    # forward of both branches, keeping every layer's input, pre-activation and gate output
    for br, s in (("H", xh), ("L", xl)):
        x = par(f"{br}.w_in")[None, None, :] * s[:, :, None] + par(f"{br}.b_in")
        skip = np.zeros((B, W, S))
        keep = []
        for l in range(L):
            d = 2 ** (l % lps)
            w = par(f"{br}.{l}.w_conv").reshape(2 * R, 2 * R)          # [out][tap * R + in]
            a = np.concatenate([q(_lag(x, -d, W)), q(x)], -1) @ q(w).T + par(f"{br}.{l}.b_conv")
            z = np.tanh(a[..., :R]) * sig(a[..., R:])
            zq = q(z)
            keep.append((x, a, zq))
            x = x + zq @ q(par(f"{br}.{l}.w_res")).T + par(f"{br}.{l}.b_res")
            skip = skip + zq @ q(par(f"{br}.{l}.w_skip")).T + par(f"{br}.{l}.b_skip")
        saved[br], skips[br] = keep, skip
    # head: u from FP16 operands, dh from BF16 operands, dW_h1 from BF16 hi/lo splits
    h = np.concatenate([np.maximum(skips["H"], 0.0), np.maximum(skips["L"], 0.0)], -1)
    u = q16(h) @ q16(par("w_h1")).T + par("b_h1")
    du = dlogit[..., None] * par("w_h2") * (u > 0)
    grad["w_h2"] = np.einsum("bt,btj->j", dlogit, np.maximum(u, 0.0))
    grad["b_h2"] = np.array([dlogit.sum()])
    lo = lambda v: q(v - q(v))
    grad["w_h1"] = (np.einsum("btj,btk->jk", q(du), q(h)) + np.einsum("btj,btk->jk", q(du), lo(h)) +
                    np.einsum("btj,btk->jk", lo(du), q(h)))
    grad["b_h1"] = du.sum((0, 1))
    dh = q(du) @ q(par("w_h1"))
    dstrain = []
    for bi, (br, s) in enumerate((("H", xh), ("L", xl))):
        dskip = dh[..., bi * S:(bi + 1) * S] * (skips[br] > 0)
        dsq = q(dskip)
        dx = np.zeros((B, W, R))
        for l in reversed(range(L)):
            d = 2 ** (l % lps)
            x, a, zq = saved[br][l]
            wres, wskip = q(par(f"{br}.{l}.w_res")), q(par(f"{br}.{l}.w_skip"))
            dz = q(dx) @ wres + dsq @ wskip
            th, sg = np.tanh(a[..., :R]), sig(a[..., R:])
            da = np.concatenate([dz * sg * (1.0 - th * th), dz * th * sg * (1.0 - sg)], -1)
            daq = q(da)
            xin = np.concatenate([q(_lag(x, -d, W)), q(x)], -1)
            grad[f"{br}.{l}.w_conv"] = np.einsum("bto,btk->ok", daq, xin).reshape(2 * R, 2, R)
            grad[f"{br}.{l}.b_conv"] = da.sum((0, 1))
            grad[f"{br}.{l}.w_res"] = np.einsum("bto,bti->oi", q(dx), zq)
            grad[f"{br}.{l}.b_res"] = dx.sum((0, 1))
            grad[f"{br}.{l}.w_skip"] = np.einsum("bto,bti->oi", dsq, zq)
            grad[f"{br}.{l}.b_skip"] = dskip.sum((0, 1))
            wc = q(par(f"{br}.{l}.w_conv"))                              # [out][tap][in]
            dx = dx + daq @ wc[:, 1, :] + _lag(daq, d, W) @ wc[:, 0, :]
        grad[f"{br}.w_in"] = np.einsum("btc,bt->c", dx, s)
        grad[f"{br}.b_in"] = dx.sum((0, 1))
        dstrain.append(dx @ par(f"{br}.w_in"))
    flat = np.concatenate([grad[name].reshape(-1) for name in offsets])
    return flat, dstrain[0], dstrain[1]
