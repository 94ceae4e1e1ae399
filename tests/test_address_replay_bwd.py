"""Host-side replay of the tensor-map operand copies of the tensor-core backward
(bwd_tc.cu: the row GEMMs' A tiles and both operands of the weight-gradient
GEMMs), for every GEMM of one backward chunk of the 30-layer ensemble at the
windows the GPU tests and the bench use (384, 1024, 4096 samples; chunks of up
to 128 windows) and of the 8-layer model (whose dgrad alone takes the tensor-map
form: its 2R = 64-channel da segments).

For each GEMM it recomputes, as the host and the kernels do: whether the shapes
take the tensor-map form; the box coordinates (innermost coordinate 16-byte
aligned); the shared-memory destination of every box (inside its A tile or
stage, never on a stage's constant blocks); the bytes each mbarrier expects
(exactly those of the boxes issued on it); the shared-memory span of every MMA
descriptor (inside the operand it describes); the dynamic shared memory
against the SM's capacity at the CTAs per SM the launch assumes; the TMEM
columns; the tile ranges of the CTAs; and the largest element each tensor map
can address against the device buffer the host allocates for it.  No GPU is
needed: this pins the index arithmetic against the buffer sizes, not the values
the kernels compute."""
import pytest

import workload

KROWS = 128                 # row GEMM tile (the MMA's M)
TMA_ROWS = 64               # weight-gradient tile
TMA_BLK = TMA_ROWS * 128    # one 64-channel block of a weight-gradient stage
TMA_SMEM = 226 * 1024       # dynamic shared memory of the weight-gradient kernels
SM_SMEM = 228 * 1024        # shared memory per SM
CTA_RESERVED = 1024         # per CTA, reserved by the system
WARP_STAGE, WARP_STAGE_NARROW = 32 * 80, 32 * 48
SMS = 152


def seg(buf_elems, boff, ld, C, shift):
    return dict(buf=buf_elems, boff=boff, ld=ld, C=C, shift=shift)


def chunk_gemms(cfg, W, Cc):
    """The row GEMMs and weight-gradient GEMMs of one chunk, with the buffers their operands lie in
    (element counts of the slice the base pointer starts), as tc_backward sets them up."""
    R, S, Hc, lps = cfg["r_ch"], cfg["s_ch"], cfg["head_ch"], cfg["layers_per_stack"]
    rb = Cc * W                       # rows per branch
    rows2 = 2 * rb
    xo = rb * R
    off = workload.param_offsets(cfg)
    Pb = off["L.w_in"][0] - off["H.w_in"][0]
    rows, wgs = [], []
    for l in range(int(cfg["stacks"]) * lps):
        dl = 1 << (l % lps)
        x = rows2 * R                 # one layer's slice of x16 / z16 / dx16 (both branches)
        rows.append(dict(name=f"conv {l}", epi=0, segs=[seg(x, xo, R, R, -dl), seg(x, xo, R, R, 0)], K=2 * R,
                         N=2 * R, bn=2 * R, nbranch=2))
        rows.append(dict(name=f"res {l}", epi=1, segs=[seg(x, xo, R, R, 0)], K=R, N=R, bn=R + S, nbranch=2))
        rows.append(dict(name=f"dz {l}", epi=2, segs=[seg(x, xo, R, R, 0), seg(rows2 * S, rb * S, S, S, 0)],
                         K=R + S, N=R, bn=R, nbranch=2))
        da = rows2 * 2 * R
        rows.append(dict(name=f"dgrad {l}", epi=3, segs=[seg(da, rb * 2 * R, 2 * R, 2 * R, 0),
                                                         seg(da, rb * 2 * R, 2 * R, 2 * R, dl)],
                         K=4 * R, N=R, bn=R, nbranch=2))
        wconv = off[f"H.{l}.w_conv"][0]
        assert off[f"L.{l}.w_conv"][0] == wconv + Pb
        wgs.append(dict(name=f"wconv {l}", G=da, g_boff=rb * 2 * R, ldg=2 * R, M=2 * R,
                        xs=[seg(x, xo, R, R, -dl), seg(x, xo, R, R, 0)], nx=2 * R, N=2 * R + 16,
                        dW=wconv, ldw=2 * R, w_boff=Pb, rows=rb))
        wgs.append(dict(name=f"wres {l}", G=x, g_boff=xo, ldg=R, M=R, xs=[seg(x, xo, R, R, 0)], nx=R, N=R + 16,
                        dW=off[f"H.{l}.w_res"][0], ldw=R, w_boff=Pb, rows=rb))
        wgs.append(dict(name=f"wskip {l}", G=rows2 * S, g_boff=rb * S, ldg=S, M=S, xs=[seg(x, xo, R, R, 0)],
                        nx=R, N=R + 16, dW=off[f"H.{l}.w_skip"][0], ldw=R, w_boff=Pb, rows=rb))
    if Hc <= 256 and 2 * S <= 256 and Hc % 32 == 0:
        # h in FP16 [branch][row][S] (the L half from + rb S, boff 0), du [row][Hc]
        rows.append(dict(name="head u", epi=4, segs=[seg(rows2 * S, 0, S, S, 0), seg(rb * S, 0, S, S, 0)],
                         K=2 * S, N=Hc, bn=Hc, nbranch=1))
        rows.append(dict(name="head dh", epi=5, segs=[seg(rb * Hc, 0, Hc, Hc, 0)], K=Hc, N=2 * S, bn=2 * S,
                         nbranch=1))
        for m0 in range(0, Hc, 128):
            wgs.append(dict(name=f"wh1 {m0}", G=rb * Hc - m0, g_boff=0, ldg=Hc, M=min(128, Hc - m0),
                            xs=[seg(rows2 * S, rb * S, S, S, 0)], nx=S, N=S + 16,
                            dW=off["w_h1"][0] + m0 * 2 * S, ldw=2 * S, w_boff=S, rows=rb))
    return rows, wgs


def map_extent(s, rows, W, nb_dims):
    """Largest element index + 1 a 4-D segment map {C, W, windows, branches} can address."""
    nwin = rows // W
    nb = 2 if s["boff"] else 1
    assert nb_dims == nb
    return (nb - 1) * s["boff"] + (nwin - 1) * W * s["ld"] + (W - 1) * s["ld"] + s["C"]


def check_rows(g, W, rows):
    segs = g["segs"]
    tma = W % KROWS == 0 and rows % W == 0 and all(s["C"] % 64 == 0 and s["C"] <= s["ld"] for s in segs)
    assert sum(s["C"] for s in segs) == g["K"]
    a_bytes = KROWS * g["K"] * 2
    staging = 8 * WARP_STAGE if g["epi"] <= 2 else (8 * WARP_STAGE_NARROW if g["epi"] == 3 else 0)
    bn = max(g["bn"], g["N"])
    smem = max(a_bytes + bn * g["K"] * 2 + staging + 1024, 80 * 1024)
    per_sm = 2 if smem <= 112 * 1024 else 1
    assert per_sm * (smem + 32 + CTA_RESERVED) <= SM_SMEM, (g["name"], smem)
    assert smem <= 200 * 1024
    ncols = 32
    while ncols < g["N"]:
        ncols *= 2
    assert per_sm * ncols <= 512
    if not tma:
        return False
    # boxes of one tile (the same for every tile; t0 + shift may leave the window: zero fill)
    blk = 0
    for s in segs:
        for j in range(s["C"] // 64):
            assert (64 * j * 2) % 16 == 0
            dst = blk * KROWS * 128
            assert 0 <= dst and dst + KROWS * 128 <= a_bytes
            blk += 1
        assert map_extent(s, rows, W, 2 if s["boff"] else 1) <= s["buf"], g["name"]
    assert blk * KROWS * 128 == a_bytes            # expect_tx = 128 K 2 = the boxes' bytes
    # the A descriptors: K step ks at byte 32 (ks % 4) of 64-channel block ks / 4; 16 groups of 8 rows
    for ks in range(g["K"] // 16):
        start = (ks >> 2) * KROWS * 128 + (ks & 3) * 32
        assert start % 1024 < 128                    # the atom's row 0: base offset 0
        last = start - start % 128 + (KROWS // 8 - 1) * 1024 + 7 * 128 + 128
        assert last <= ((ks >> 2) + 1) * KROWS * 128 <= a_bytes
    for t0 in range(0, W, KROWS):
        assert t0 + KROWS <= W                       # a tile lies in one window
        for s in segs:
            assert -2 ** 31 <= t0 + s["shift"] < 2 ** 31
    return True


def check_wgrad(g, W):
    rows = g["rows"]
    tma = (W % TMA_ROWS == 0 and rows % W == 0 and g["M"] in (64, 128) and g["nx"] in (64, 128)
           and g["N"] == g["nx"] + 16 and all(s["C"] in (64, 128) for s in g["xs"])
           and sum(s["C"] for s in g["xs"]) == g["nx"] and g["dW"] % 4 == 0 and g["ldw"] % 4 == 0
           and g["w_boff"] % 4 == 0)
    if not tma:
        return False
    NB = g["nx"] // 64 + 1
    stage = (2 + NB) * TMA_BLK
    stages = min(6, (TMA_SMEM - 1024) // stage)
    assert stages >= 2
    smem = stages * stage + 1024
    assert smem <= TMA_SMEM and smem + 112 + CTA_RESERVED <= SM_SMEM
    assert g["N"] <= (128 if g["N"] <= 128 else 256) <= 512
    a_end, b0 = 2 * TMA_BLK, 2 * TMA_BLK
    # boxes: G blocks j < M / 64 in A, X blocks blk < nx / 64 in B, never the ones block (NB - 1)
    gb = g["M"] // 64
    for j in range(gb):
        assert (j + 1) * TMA_BLK <= a_end
    xb = 0
    for s in g["xs"]:
        for j in range(s["C"] // 64):
            assert (64 * j * 2) % 16 == 0
            assert b0 + (xb + 1) * TMA_BLK <= b0 + (NB - 1) * TMA_BLK
            xb += 1
        assert map_extent(s, rows, W, 2 if s["boff"] else 1) <= s["buf"], g["name"]
    assert xb == NB - 1
    # G map {M, rows, branches}
    nbg = 2 if g["g_boff"] else 1
    assert (nbg - 1) * g["g_boff"] + (rows - 1) * g["ldg"] + g["M"] <= g["G"], g["name"]
    # descriptors: K step ks at 2048 ks; MN blocks 8 KB apart (two for A, NB for B), two 8-row groups
    for ks in range(TMA_ROWS // 16):
        assert (ks * 2048) % 1024 == 0
        assert ks * 2048 + TMA_BLK + 1024 + 8 * 128 <= a_end
        assert b0 + ks * 2048 + (NB - 1) * TMA_BLK + 1024 + 8 * 128 <= stage
    # tile ranges of the CTAs cover each branch's tiles once
    tiles = rows // TMA_ROWS
    per_branch = SMS // 2
    tpc = max(1, -(-tiles // per_branch))
    grid_x = -(-tiles // tpc)
    covered = sum(max(0, min(tiles, (x + 1) * tpc) - x * tpc) for x in range(grid_x))
    assert covered == tiles
    return True


@pytest.mark.parametrize("W,batch", [(384, 2), (1024, 2), (1024, 1), (4096, 6), (4096, 256)])
def test_ensemble_backward_tensor_map_copies_stay_in_bounds(W, batch):
    cfg = workload.config("ensemble", n_models=1)
    Cc = min(batch, 128)
    rows, wgs = chunk_gemms(cfg, W, Cc)
    n_rows = sum(check_rows(g, W, Cc * W) for g in rows)
    n_wg = sum(check_wgrad(g, W) for g in wgs)
    # every GEMM of the 30-layer model takes the tensor-map form at these windows
    assert n_rows == len(rows) and n_wg == len(wgs), (n_rows, len(rows), n_wg, len(wgs))


@pytest.mark.parametrize("W,batch", [(512, 3), (200, 2)])
def test_small_model_mixes_both_stagings(W, batch):
    """R = S = Hc = 32: only dgrad's segments (da, 2R = 64 channels) take the tensor-map form, and only
    where the window is a multiple of 128; every other GEMM stages with per-thread copies (no weight
    gradient has 64-channel X segments).  The shared memory and TMEM checks hold for all."""
    cfg = workload.config("small", n_models=1)
    Cc = min(batch, 128)
    rows, wgs = chunk_gemms(cfg, W, Cc)
    tma = [g["name"] for g in rows if check_rows(g, W, Cc * W)]
    expect = [g["name"] for g in rows if g["epi"] == 3] if W % KROWS == 0 else []
    assert tma == expect
    assert not any(check_wgrad(g, W) for g in wgs)
