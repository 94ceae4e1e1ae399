"""Host-side replay of the global-memory and staging-buffer address arithmetic of
the fused tensor-core forward (branch_tc.cu) in its time-slide projection mode
and zero-lag mode, and of the slide heads, for every geometry the GPU tests run
(including the 30-layer ensemble at W = 1024, stride 512, slides [1, 2, 5, -3, 0]).

For each CTA, job, tile and layer it walks the same job ranges, cross-window
reuse plan (lstar), lag-ring offsets, carry slots and projection indices as the
kernel and checks that every bulk-copy source and destination, ring row store,
carry access, projection store and slide-head load or store lies inside the
allocation the host sets up for it (sizes computed as the host does, from the
configuration).  No GPU is needed; this pins the index arithmetic against the
allocation sizes, not the numbers the kernel computes."""
import numpy as np
import pytest

KT = 128          # time tile


def shape(R, S, HC, f8):
    XB = 1 if f8 else 2
    N1 = 2 * R
    RC = R * XB // 16
    NH = 1 if HC <= 128 else 2
    HP = HC // NH
    HQ = S // 2
    STAGE_LBO = 256 * 16
    STAGE_BYTES = max(STAGE_LBO * RC, 256 * S)
    CONV_BYTES = N1 * 2 * R * XB
    RS_BYTES = R * R * 2 + S * R * 2
    HEADP_BYTES = HP * HQ * 2
    CB = 16 * R if f8 else 8 * R
    RB = 8 * R if f8 else 4 * R
    HDR = 8 * R + 4 * S + (4 * R if f8 else 0)
    return dict(XB=XB, XROW=R * XB, RC=RC, NH=NH, HP=HP, HQ=HQ, STAGE_LBO=STAGE_LBO, STAGE_BYTES=STAGE_BYTES,
                CONV_BYTES=CONV_BYTES, RS_BYTES=RS_BYTES, HEADP_BYTES=HEADP_BYTES, NHP=4 * NH,
                LAYER_IMG=2 * CONV_BYTES + 2 * RS_BYTES, PL=CB + RB, CB=CB, RB=RB, HDR=HDR)


def plan_reuse(L, lps, W, stride):
    NT = W // KT
    lstar = [-1] * 64
    if stride % KT != 0 or stride >= W or 2 * stride < W or NT > 64 or L < 2:
        return 0, lstar
    shift = stride // KT
    rl, rf = [], 1
    for l in range(L):
        rf += 1 << (l % lps)
        rl.append(rf)
    anyr = False
    for t in range(NT - shift):
        ls = -1
        for l in range(min(L - 1, 127)):
            if rl[l] - 1 <= KT * t:
                ls = l
            else:
                break
        lstar[t] = ls
        anyr = anyr or ls >= 0
    return (shift if anyr else 0), lstar


def job_range(n_jobs, grid, c):
    q, rm = divmod(n_jobs, grid)
    j0 = c * q + min(c, rm)
    return j0, j0 + q + (1 if c < rm else 0)


def replay(R, S, HC, f8, stacks, lps, W, stride, n, n_models, slides, sms=152, reuse=True, ring_short=0,
           proj_short=0):
    """Walk every access of one gwe_forward call; returns the number of checked accesses."""
    sh = shape(R, S, HC, f8)
    L = stacks * lps
    nw = (n - W) // stride + 1
    NT = W // KT
    ring_rows = sum(1 << (l % lps) for l in range(L))
    ring_cta = (2 * ring_rows * sh["XROW"] + 255) & ~255
    shift, lstar = plan_reuse(L, lps, W, stride) if reuse else (0, [-1] * 64)
    n_rings = 2 if shift > 0 else 1
    grid_max = min(sms, n_models * nw)
    ring_alloc = n_rings * ring_cta * grid_max - ring_short
    ring_cta_bytes = n_rings * ring_cta
    ring_pp = ring_cta if n_rings > 1 else 0
    ntr = NT - shift
    carry_cta_floats = 2 * ntr * (R // 2 + S // 2) * 256 if shift > 0 else 0
    carry_alloc = carry_cta_floats * grid_max
    img_stride = (L * sh["LAYER_IMG"] + sh["NHP"] * sh["HEADP_BYTES"] + 255) & ~255
    pb_bytes = sh["HDR"] + L * sh["PL"]
    pb_stride = (2 * pb_bytes + ((8 * HC + 4 + 15) & ~15) + 255) & ~255
    proj_alloc = 2 * nw * HC * W - proj_short         # FP16 elements
    n_sl = len(slides) if slides else 0
    out_alloc = max(n_sl, 1) * n_models * nw * W     # FP32 elements
    RH, SH = R // 2, S // 2
    checks = 0

    def inside(lo, size, alloc, what):
        nonlocal checks
        checks += 1
        assert 0 <= lo and lo + size <= alloc, (what, lo, size, alloc)

    launches = []
    if n_sl == 0:
        launches.append(dict(models=n_models, model0=0, grid=grid_max, proj=False))
    else:
        for mi in range(n_models):
            launches.append(dict(models=1, model0=mi, grid=min(sms, nw), proj=True))
    for la in launches:
        n_jobs = la["models"] * nw
        for c in range(la["grid"]):
            j0, j1 = job_range(n_jobs, la["grid"], c)
            for j in range(j0, j1):
                w = j % nw
                m = la["model0"] + j // nw
                inside(m * img_stride, img_stride, img_stride * n_models, "weight image")
                inside(m * pb_stride + 2 * pb_bytes, 8 * HC + 4, pb_stride * n_models, "head parameters")
                ru = shift > 0 and j > j0 and w > 0
                cw = shift > 0 and j + 1 < j1 and w + 1 < nw
                par = (j - j0) & 1
                for b in range(2):
                    ring_c = c * ring_cta_bytes + b * ring_rows * sh["XROW"]
                    ring_b = ring_c + par * ring_pp
                    for tt in range(NT):
                        t0 = tt * KT
                        l0 = lstar[tt] + 1 if ru else 0
                        lgive = lstar[tt - shift] if (cw and tt >= shift) else -1
                        inside(w * stride + t0, KT, n, "strain rows")
                        if l0 > 0 or lgive >= 0:
                            slot = tt if l0 > 0 else tt - shift
                            base = c * carry_cta_floats + (b * ntr * ((RH + SH) // 4) * 256 + slot * ((RH + SH) // 4) * 256) * 4
                            inside(base, ((RH + SH) // 4) * 256 * 4, carry_alloc, "carry slot")
                        for l in range(l0, L):
                            d = 1 << (l % lps)
                            nn = min(d, KT)
                            roff = (l // lps) * ((1 << lps) - 1) + (d - 1)
                            inside(l * sh["LAYER_IMG"] + b * sh["CONV_BYTES"], sh["CONV_BYTES"], img_stride, "conv piece")
                            inside(l * sh["LAYER_IMG"] + 2 * sh["CONV_BYTES"] + b * sh["RS_BYTES"], sh["RS_BYTES"],
                                   img_stride, "res/skip piece")
                            inside(b * pb_bytes + sh["HDR"] + l * sh["PL"], sh["PL"], pb_stride, "bias slots")
                            # producer: lagged rows into the staging buffer (rows 128 - n .. 127 of every chunk column)
                            for cc in range(sh["RC"]):
                                inside(cc * sh["STAGE_LBO"] + (KT - nn) * 16, nn * 16, sh["STAGE_BYTES"], "lag destination")
                            if t0 >= d:
                                ts = tt - (1 if d < KT else d // KT)
                                prev = ru and 0 <= ts < NT - shift and l <= lstar[ts]
                                src0 = ring_c + (par ^ (1 if prev else 0)) * ring_pp + roff * sh["XROW"] + (t0 & (d - 1)) * 16
                                for cc in range(sh["RC"]):
                                    inside(src0 + cc * d * 16, nn * 16, ring_alloc, "lag source")
                                    # the rows stay inside this layer's region of this CTA's ring
                                    lay = ring_c + (par ^ (1 if prev else 0)) * ring_pp + roff * sh["XROW"]
                                    assert lay <= src0 + cc * d * 16 and src0 + cc * d * 16 + nn * 16 <= lay + d * sh["XROW"]
                            else:
                                assert nn * 16 <= 4096, "zero rows"
                            # epilogue: history rows of layer l (rows r >= 128 - n)
                            if tt + 1 < NT or cw:
                                for r in (KT - nn, KT - 1):
                                    dst = ring_b + roff * sh["XROW"] + ((t0 + r) & (d - 1)) * 16
                                    for hf in range(2):
                                        for ck in range(sh["RC"] // 2):
                                            o = dst + (hf * (sh["RC"] // 2) + ck) * d * 16
                                            inside(o, 16, ring_alloc, "history store")
                                            lay = ring_b + roff * sh["XROW"]
                                            assert lay <= o and o + 16 <= lay + d * sh["XROW"]
                        # head operand in the staging buffer, then the projections or the probabilities
                        for ch in (0, S - 16):
                            inside((ch // 8 + 1) * (KT * 16) + (KT - 1) * 16, 16, sh["STAGE_BYTES"], "head operand")
                        if la["proj"]:
                            pw = (b * nw + w) * HC * W
                            for ch in (0, HC - 16):
                                for r in (0, KT - 1):
                                    inside(pw + ((ch // 8) * W + t0 + r) * 8, 8, proj_alloc, "projection store")
                                    inside(pw + ((ch // 8 + 1) * W + t0 + r) * 8, 8, proj_alloc, "projection store")
                        elif b == 0:
                            inside(((m - la["model0"]) * nw + w) * W + t0, KT, out_alloc, "probability store")
    # slide heads: every launch shape the autotuner can choose
    if n_sl:
        for A, B, ppb in SLIDE_SHAPES:
            checks += replay_slide_heads(HC, W, [nw], n_models, slides, A, B, ppb, proj_alloc, out_alloc)
    return checks


# (Hanford windows per block, offsets per piece, pieces per block; 0 = all, -1 = a quarter)
SLIDE_SHAPES = [(a, b, ppb) for a in (2, 4) for b in (4, 8) for ppb in (0, -1)]


def slide_step(slides, nw):
    """The offsets' most common positive step (smaller on a tie), 1 when none is below nw."""
    cnt = {}
    for a, b in zip(slides[:-1], slides[1:]):
        d = b - a
        if 0 < d < nw and d <= 1 << 20:
            cnt[d] = cnt.get(d, 0) + 1
    best, nb = 1, 0
    for d in sorted(cnt):
        if cnt[d] > nb:
            best, nb = d, cnt[d]
    return best


def slide_pieces(slides, bmax, step=1):
    """Pieces of offsets in arithmetic progression with `step` (first index, count), at most bmax long,
    as the host builds them."""
    out, i, n = [], 0, len(slides)
    while i < n:
        j = i + 1
        while j < n and j - i < bmax and slides[j] == slides[j - 1] + step:
            j += 1
        out.append((i, j - i))
        i = j
    return out


def replay_slide_heads(HC, W, seg_nw, n_models, slides, A, B, ppb, proj_alloc, out_alloc):
    """Walk the slide heads' loads and stores for one launch shape (all models); returns the count.

    Block (x, y, z): windows [x A dw, (x + 1) A dw) taken per residue mod dw in passes of windows
    wa + a dw that stay within one segment, samples [y SPW, y SPW + SPW), pieces [z ppb, z ppb + ppb).
    Each thread reads chunks 2q and 2q + 1 of the Hanford windows and of the Livingston windows
    (r0 + s dw) mod n_seg_w, s < na + nb - 1, and the block stores (slide first + b, window
    wa + a dw) for a < na, b < nb.  Every window of every slide is stored exactly once."""
    NP = HC // 16
    SPW = 32 // min(NP, 4)                  # samples per block (pairs per warp x samples = 32 lanes)
    nw = int(sum(seg_nw))
    seg_w0 = np.concatenate([[0], np.cumsum(seg_nw)]).astype(np.int64)
    dw = slide_step(slides, nw)
    pieces = slide_pieces(slides, B, dw)
    np_ = len(pieces)
    if ppb == -1:
        ppb = max(1, (np_ + 3) // 4)
    ppb = min(ppb, np_) if ppb > 0 else np_
    wst = HC * W // 8                      # 16-byte chunks per window
    alloc16 = proj_alloc // 8               # the projections in 16-byte chunks
    slide_stride = n_models * nw * W
    checks = 0
    ys = sorted({0, W // SPW - 1})
    zs = range((np_ + ppb - 1) // ppb)

    def load(chunk_index):
        nonlocal checks
        checks += 1
        assert 0 <= chunk_index < alloc16, ("slide-head load", chunk_index, alloc16)

    stored = np.zeros((len(slides), nw), dtype=np.int64)
    for mi in range(n_models):
        for x in range((nw + A * dw - 1) // (A * dw)):
            wrun, wend = x * A * dw, min(nw, (x + 1) * A * dw)
            for rho in range(dw):
                wa = wrun + rho
                while wa < wend:
                    g = int(np.searchsorted(seg_w0, wa, side="right") - 1)
                    sw0, snw = int(seg_w0[g]), int(seg_w0[g + 1] - seg_w0[g])
                    na = (min(wend, sw0 + snw) - wa + dw - 1) // dw
                    assert 1 <= na <= A
                    assert wa + (na - 1) * dw < sw0 + snw          # the pass stays in its segment
                    for y in ys:
                        for q in (0, NP - 1):
                            base = 2 * q * W + y * SPW
                            for ts in (0, SPW - 1):
                                for a in range(na):
                                    load((wa + a * dw) * wst + base + ts)
                                    load((wa + a * dw) * wst + base + W + ts)
                        for z in zs:
                            for pc in range(z * ppb, min(np_, z * ppb + ppb)):
                                i0, nb = pieces[pc]
                                r0 = (wa - sw0 + slides[i0]) % snw
                                for s in range(na + nb - 1):
                                    wl = sw0 + (r0 + s * dw) % snw
                                    # the Livingston window of pair (a, s - a) is the plain definition's
                                    for a in range(max(0, s - nb + 1), min(na, s + 1)):
                                        b = s - a
                                        assert wl == sw0 + (wa + a * dw - sw0 + slides[i0 + b]) % snw
                                    for q in (0, NP - 1):
                                        base = nw * wst + wl * wst + 2 * q * W + y * SPW
                                        load(base)
                                        load(base + W + SPW - 1)
                                for a in range(na):
                                    for b in range(nb):
                                        o = mi * nw * W + (i0 + b) * slide_stride + (wa + a * dw) * W + y * SPW
                                        checks += 1
                                        assert 0 <= o and o + SPW <= out_alloc, ("slide-head store", o, out_alloc)
                                        if mi == 0 and y == 0:
                                            stored[i0 + b, wa + a * dw] += 1
                    wa += na * dw
    assert np.all(stored == 1), "every (slide, window) stored exactly once"
    return checks


GEOMETRIES = [
    # (R, S, HC, stacks, lps, W, stride, n, n_models, slides)
    (64, 128, 256, 3, 10, 1024, 512, 1024 + 5 * 512 + 17, 4, [1, 2, 5, -3, 0]),
    (64, 128, 256, 3, 10, 1024, 512, 1024 + 5 * 512 + 17, 2, [1, 2, 5, -3, 0]),
    (64, 128, 256, 3, 10, 4096, 2048, 4096 + 2048 + 5, 4, None),
    (64, 128, 256, 3, 10, 4096, 2048, 4096 + 9 * 2048 + 100, 4, None),
    (64, 128, 256, 3, 10, 4096, 2048, 3600 * 4096, 4, None),
    (64, 128, 256, 3, 10, 4096, 2048, 40 * 4096, 4, [2 * (k + 1) for k in range(64)]),
    (32, 32, 32, 1, 8, 1024, 512, 1024 + 6 * 512 + 300, 2, [0, 3, -1]),
    (32, 32, 32, 1, 8, 1024, 512, 1024 + 40 * 512, 4, None),
    (32, 32, 32, 1, 8, 1024, 768, 1024 + 20 * 768 + 7, 2, [1, -2]),
    (32, 32, 32, 1, 8, 4096, 4096, 8 * 4096, 1, None),
]


@pytest.mark.parametrize("geo", GEOMETRIES)
@pytest.mark.parametrize("f8", [False, True])
def test_forward_addresses_stay_in_their_allocations(geo, f8):
    R, S, HC, stacks, lps, W, stride, n, nm, slides = geo
    if n > 10 * 4096 * 60 and slides is None:
        # the one-hour geometry: the same arithmetic on a window subset (the first and last CTAs' ranges)
        n = 40 * 4096
    got = replay(R, S, HC, f8, stacks, lps, W, stride, n, nm, slides)
    assert got > 0


def test_replay_catches_undersized_allocations():
    """The replay is a real check: one ring row or one projection element short is reported."""
    geo = (64, 128, 256, 3, 10, 1024, 512, 1024 + 5 * 512 + 17, 2, [1, 2, 5, -3, 0])
    R, S, HC, stacks, lps, W, stride, n, nm, slides = geo
    # 16 jobs on eight CTAs, two each: both rings of the last CTA are written up to their last row
    n16 = W + 7 * stride
    replay(R, S, HC, False, stacks, lps, W, stride, n16, nm, None, sms=8)
    with pytest.raises(AssertionError):
        replay(R, S, HC, False, stacks, lps, W, stride, n16, nm, None, sms=8, ring_short=128)
    with pytest.raises(AssertionError):
        replay(R, S, HC, False, stacks, lps, W, stride, n, nm, slides, proj_short=1)


@pytest.mark.parametrize("A,B,ppb", SLIDE_SHAPES)
def test_slide_heads_on_uneven_segments(A, B, ppb):
    """Segments of 1, 3, 6 and 13 windows (tiles straddle the boundaries), offsets with runs, gaps,
    negative values and offsets larger than a segment."""
    HC, W, nm = 256, 1024, 2
    seg_nw = [13, 1, 6, 3]
    slides = [1, 2, 3, 4, 5, 9, -3, -2, 0, 40, 41, 7]
    nw = sum(seg_nw)
    for sl in (slides, [2, 4, 6, 8, 10, 12, 14, 16, 18, 20, 3, -7], [3, 6, 9, 12, 0]):
        replay_slide_heads(256, W, seg_nw, nm, sl, A, B, ppb, 2 * nw * 256 * W, len(sl) * nm * nw * W)
    nw = sum(seg_nw)
    got = replay_slide_heads(HC, W, seg_nw, nm, slides, A, B, ppb, 2 * nw * HC * W, len(slides) * nm * nw * W)
    assert got > 0
    with pytest.raises(AssertionError):
        replay_slide_heads(HC, W, seg_nw, nm, slides, A, B, ppb, 2 * nw * HC * W - 8, len(slides) * nm * nw * W)


def test_slide_pieces():
    assert slide_pieces([1, 2, 3, 4, 5, 9, -3, -2, 0], 4) == [(0, 4), (4, 1), (5, 1), (6, 2), (8, 1)]
    assert slide_pieces(list(range(1, 65)), 8) == [(8 * i, 8) for i in range(8)]
    assert slide_pieces([], 4) == []
    offs = [2 * (k + 1) for k in range(64)]                 # 1 .. 64 s at 0.5 s stride
    assert slide_step(offs, 7199) == 2
    assert slide_pieces(offs, 4, 2) == [(4 * i, 4) for i in range(16)]
    assert slide_step([5, 1, 3], 100) == 2 and slide_step([4, 1], 100) == 1 and slide_step([1, 50], 40) == 1
