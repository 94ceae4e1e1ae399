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
    # slide heads: block (w, tile, offset group); Hanford rows of window w, Livingston rows of (w + k) mod nw
    if n_sl:
        bstride = nw * HC * W
        for w in range(nw):
            for k in slides:
                wl = (w + k) % nw
                inside(w * HC * W, HC * W, proj_alloc, "Hanford projections")
                inside(bstride + wl * HC * W, HC * W, proj_alloc, "Livingston projections")
            for si in range(n_sl):
                for mi in range(n_models):
                    inside(mi * nw * W + si * (n_models * nw * W) + w * W, W, out_alloc, "slide-head store")
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
