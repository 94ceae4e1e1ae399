"""The FP32 forms that the device trigger evaluation uses in place of the definition's FP64 steps
(numpy, no GPU):

* width test: for a float x and a double h, h < (double)x  <=>  x > hf, hf = the largest float <= h;
* half height: h = xp - (xp - base) / 2 evaluated in FP64 rounds down to the same float as
  RD(xp + base) * 0.5 evaluated in FP32, whenever |xp| and |base| lie in [2^-100, 2^100] within a
  factor 2^27 of each other (or one of them is 0): then xp - base and (xp + base) / 2 are exact in
  FP64;
* keep test: the interpolated width lies in (k_r - k_l - 2, k_r - k_l] for the integer stops of the
  width walks, so k_r - k_l < ceil(min_width) rejects without evaluating it."""
import numpy as np


def _rd_float(d):
    """Round FP64 values down to FP32."""
    f = np.asarray(d, dtype=np.float64).astype(np.float32)
    up = f.astype(np.float64) > d
    f[up] = np.nextafter(f[up], np.float32(-np.inf))
    return f


def _pairs(rng, n):
    xp = np.concatenate([rng.random(n), rng.standard_normal(n) * 10,
                         np.exp(rng.uniform(-60, 60, n)) * rng.choice([-1, 1], n)]).astype(np.float32)
    base = np.concatenate([rng.random(n), rng.standard_normal(n) * 10,
                           np.exp(rng.uniform(-60, 60, n)) * rng.choice([-1, 1], n)]).astype(np.float32)
    keep = base <= xp
    return xp[keep], base[keep]


def test_width_test_float_form():
    rng = np.random.default_rng(21)
    xp, base = _pairs(rng, 200_000)
    x64, b64 = xp.astype(np.float64), base.astype(np.float64)
    h = x64 - (x64 - b64) * 0.5
    hf = _rd_float(h)
    x = (x64 + rng.standard_normal(len(h)) * np.abs(x64 - b64)).astype(np.float32)
    assert np.array_equal(h < x.astype(np.float64), x > hf)
    # ties: x equal to the float just below or above h
    for xt in (hf, np.nextafter(hf, np.float32(np.inf))):
        assert np.array_equal(h < xt.astype(np.float64), xt > hf)


def test_half_height_float_form():
    rng = np.random.default_rng(22)
    xp, base = _pairs(rng, 300_000)
    aa, ab = np.abs(xp), np.abs(base)
    lo, hi = np.minimum(aa, ab), np.maximum(aa, ab)
    fast = (hi <= 2.0 ** 100) & np.where(lo == 0, (hi == 0) | (hi >= 2.0 ** -100),
                                         (lo >= 2.0 ** -100) & (hi <= lo * np.float32(2.0 ** 27)))
    assert fast.mean() > 0.5
    x64, b64 = xp.astype(np.float64), base.astype(np.float64)
    h = x64 - (x64 - b64) * 0.5
    hf_def = _rd_float(h)
    hf_fast = _rd_float(x64 + b64) * np.float32(0.5)
    assert np.array_equal(hf_fast[fast], hf_def[fast])


def test_width_bounds_by_integer_stops():
    """Width at half prominence written out (interpolation as in the definition) on random series:
    the width lies in (k_r - k_l - 2, k_r - k_l]."""
    rng = np.random.default_rng(23)
    for _ in range(200):
        x = rng.random(64)
        p = int(np.argmax(x[8:56])) + 8
        xp = x[p]
        lb = p
        for k in range(p, -1, -1):          # left base: minimum up to the first higher sample
            if x[k] > xp:
                break
            if x[k] < x[lb]:
                lb = k
        rb = p
        for k in range(p, 64):
            if x[k] > xp:
                break
            if x[k] < x[rb]:
                rb = k
        pr = xp - max(x[lb], x[rb])
        h = xp - pr * 0.5
        kl = p
        while lb < kl and h < x[kl]:
            kl -= 1
        lip = kl + ((h - x[kl]) / (x[kl + 1] - x[kl]) if x[kl] < h else 0.0)
        kr = p
        while kr < rb and h < x[kr]:
            kr += 1
        rip = kr - ((h - x[kr]) / (x[kr - 1] - x[kr]) if x[kr] < h else 0.0)
        wd = rip - lip
        assert kr - kl - 2 < wd <= kr - kl
