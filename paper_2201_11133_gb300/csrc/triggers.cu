// Trigger extraction on the device: stitched per-(slide, model) probability
// series -> peaks with SciPy find_peaks semantics (paper paragraph "AI ensemble
// construction"; section "Statistical Analysis": height threshold and width of
// at least 0.5 s) -> ensemble coincidence within 0.5 s (section "Event
// Detection").
//
// The stitched series is never materialised: sample g of a series is read
// from window 0 when g < window, else from window w = (g - window) / stride + 1
// at position g - w * stride (the last `stride` samples of every later window).
//
// Steps (all kernels, ordered so that results come out sorted by series and
// index without a sort):
//   1. a summary tree per series (256-sample blocks, then nodes of 32 nodes):
//      max, min, first and last argmin, so that the prominence and width
//      walks pass long stretches in a few steps;
//   2. candidate count per 8192-sample chunk -> exclusive scan -> ordered write
//      of every local maximum (plateau midpoint) whose height passes;
//   3. per candidate: prominence and width at half prominence in FP64 with
//      the same operation order as the definition (no contraction), keep
//      flag; one thread per candidate over a shared-memory window around its
//      chunk, one warp on the summary tree for the few whose walks leave it;
//   4. ordered compaction of kept peaks; per-series start offsets;
//   5. per model-0 peak: coincidence test against the other models' peaks.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "gwe_internal.h"

namespace gwe {
namespace {

constexpr int kBS = 256;       // samples per statistics block
constexpr int kFan = 32;       // children per node of the summary tree above the blocks
constexpr int kCH = 8192;      // samples per candidate chunk
constexpr int kT = 256;        // threads per block

struct Series {
    const float *base;
    int64_t n;       // stitched length
    int W, stride;
    __device__ __forceinline__ float at(int64_t g) const {
        if (g < W) return base[g];
        const uint64_t r = (uint64_t)(g - W);
        const int64_t w = (r < 0x100000000ull ? (int64_t)((uint32_t)r / (uint32_t)stride) : (int64_t)(r / (uint64_t)stride)) + 1;
        return base[w * W + (g - w * stride)];
    }
};

struct Geo {
    const float *prob;
    int64_t nw;
    int64_t series_nw;   // windows between the starts of consecutive series
    int W, stride;
    int64_t n;           // stitched length (same for every series)
    int64_t nblk;        // statistics blocks per series
    __device__ __forceinline__ Series series(int s) const {
        Series v;
        v.base = prob + (int64_t)s * series_nw * W;
        v.n = n; v.W = W; v.stride = stride;
        return v;
    }
};

// exclusive block scan of a 0/1 flag over kT threads; returns the rank and the block total
__device__ __forceinline__ int block_rank(int flag, int *sh, int &total) {
    const unsigned mask = __ballot_sync(0xffffffffu, flag);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int pre = __popc(mask & ((1u << lane) - 1u));
    if (lane == 0) sh[warp] = __popc(mask);
    __syncthreads();
    if (threadIdx.x == 0) {
        int s = 0;
        for (int w = 0; w < kT / 32; ++w) {
            const int v = sh[w];
            sh[w] = s;
            s += v;
        }
        sh[kT / 32] = s;
    }
    __syncthreads();
    const int r = sh[warp] + pre;
    total = sh[kT / 32];
    __syncthreads();
    return r;
}

// 1. block statistics: one warp per block of kBS samples
__global__ void k_stats(Geo g, float *bmax, float *bmin, int64_t *amin_lo, int64_t *amin_hi, int n_series) {
    const int lane = threadIdx.x & 31;
    const int64_t wid = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (wid >= g.nblk * n_series) return;
    const int s = (int)(wid / g.nblk);
    const int64_t blk = wid - (int64_t)s * g.nblk;
    const Series v = g.series(s);
    const int64_t lo = blk * kBS, hi = min(lo + kBS, v.n);
    float mx = -INFINITY, mn = INFINITY;
    int64_t ilo = INT64_MAX, ihi = -1;
    for (int64_t i = lo + lane; i < hi; i += 32) {
        const float x = v.at(i);
        mx = fmaxf(mx, x);
        if (x < mn) { mn = x; ilo = i; ihi = i; }
        else if (x == mn) { ilo = min(ilo, i); ihi = max(ihi, i); }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const float omx = __shfl_xor_sync(0xffffffffu, mx, o);
        const float omn = __shfl_xor_sync(0xffffffffu, mn, o);
        const long long olo = __shfl_xor_sync(0xffffffffu, (long long)ilo, o);
        const long long ohi = __shfl_xor_sync(0xffffffffu, (long long)ihi, o);
        mx = fmaxf(mx, omx);
        if (omn < mn) { mn = omn; ilo = olo; ihi = ohi; }
        else if (omn == mn) { ilo = min(ilo, (int64_t)olo); ihi = max(ihi, (int64_t)ohi); }
    }
    if (lane == 0) {
        bmax[wid] = mx; bmin[wid] = mn; amin_lo[wid] = ilo; amin_hi[wid] = ihi;
    }
}

// local maximum test at a left edge i over the chunk [lo, lo + kCH) held in xs (samples lo - 1 ..
// lo + kCH, those inside the series); returns the peak index (plateau midpoint) or -1.  thr: the
// height threshold (a float, so the float comparison is the definition's); the conditions are all
// required, so testing the height first does not change the result.
__device__ __forceinline__ int64_t peak_at(const Series &v, const float *xs, int64_t lo, int64_t i, float thr) {
    if (i < 1 || i > v.n - 2) return -1;
    const float xi = xs[i - lo + 1];
    if (!(xi >= thr)) return -1;
    if (!(xs[i - lo] < xi)) return -1;
    const int64_t top = lo + kCH;          // last sample held in xs (when inside the series)
    auto x = [&](int64_t k) -> float { return k <= top ? xs[k - lo + 1] : v.at(k); };
    int64_t ia = i + 1;
    while (ia < v.n - 1 && x(ia) == xi) ++ia;
    if (!(x(ia) < xi)) return -1;
    return (i + (ia - 1)) / 2;
}

// 2. candidates: mode 0 counts per chunk, mode 1 writes in order
__global__ void k_cand(Geo g, float thr, int mode, int64_t *counts, const int64_t *offsets, int64_t *cand_idx,
                       int *cand_ser, int64_t nchunk) {
    __shared__ int sh[kT / 32 + 1];
    __shared__ float xs[kCH + 2];
    const int s = blockIdx.y;
    const int64_t c = blockIdx.x;
    const Series v = g.series(s);
    const int64_t lo = c * kCH;
    for (int64_t k = lo - 1 + threadIdx.x; k <= lo + kCH; k += kT)
        if (k >= 0 && k < v.n) xs[k - lo + 1] = v.at(k);
    __syncthreads();
    int64_t run = (mode == 1) ? offsets[(int64_t)s * nchunk + c] : 0;
    for (int it = 0; it < kCH / kT; ++it) {
        const int64_t i = lo + (int64_t)it * kT + threadIdx.x;
        const int64_t pk = (i < v.n) ? peak_at(v, xs, lo, i, thr) : -1;
        int tot;
        const int r = block_rank(pk >= 0, sh, tot);
        if (mode == 1 && pk >= 0) {
            cand_idx[run + r] = pk;
            cand_ser[run + r] = s;
        }
        run += tot;
    }
    if (mode == 0 && threadIdx.x == 0) counts[(int64_t)s * nchunk + c] = run;
}

// exclusive scan of n int64 counts with one block of 1024 threads; out[n] = total
__global__ void k_scan(const int64_t *in, int64_t *out, int64_t n) {
    __shared__ int64_t sh[1024];
    int64_t carry = 0;
    for (int64_t base = 0; base < n; base += 1024) {
        const int64_t i = base + threadIdx.x;
        const int64_t v = (i < n) ? in[i] : 0;
        sh[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {
            const int64_t t = (threadIdx.x >= (unsigned)o) ? sh[threadIdx.x - o] : 0;
            __syncthreads();
            sh[threadIdx.x] += t;
            __syncthreads();
        }
        if (i < n) out[i] = carry + sh[threadIdx.x] - v;
        const int64_t tile = sh[1023];
        __syncthreads();
        carry += tile;
    }
    if (threadIdx.x == 0) out[n] = carry;
}

// 1b. statistics of the next tree level: node j summarises nodes [32 j, 32 j + 32) of the level
// below (one thread per node)
__global__ void k_stats_up(int64_t cnt_lo, int64_t cnt, int n_series, const float *bmax, const float *bmin,
                           const int64_t *alo, const int64_t *ahi, float *smax, float *smin, int64_t *slo,
                           int64_t *shi) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cnt * n_series) return;
    const int s = (int)(i / cnt);
    const int64_t j = i - (int64_t)s * cnt;
    const int64_t b0 = (int64_t)s * cnt_lo + j * kFan, b1 = (int64_t)s * cnt_lo + min((j + 1) * kFan, cnt_lo);
    float mx = -INFINITY, mn = INFINITY;
    int64_t lo = INT64_MAX, hi = -1;
    for (int64_t b = b0; b < b1; ++b) {
        mx = fmaxf(mx, bmax[b]);
        const float m = bmin[b];
        if (m < mn) { mn = m; lo = alo[b]; hi = ahi[b]; }
        else if (m == mn) { hi = ahi[b]; }
    }
    smax[i] = mx; smin[i] = mn; slo[i] = lo; shi[i] = hi;
}

constexpr unsigned kFull = 0xffffffffu;

// (value, lane) minimum over the warp; ties go to the lower lane
__device__ __forceinline__ void warp_argmin(float &m, int &l) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float om = __shfl_xor_sync(kFull, m, o);
        const int ol = __shfl_xor_sync(kFull, l, o);
        if (om < m || (om == m && ol < l)) { m = om; l = ol; }
    }
}

// Summary tree of the series: level 1 = blocks of kBS samples, level l + 1 = nodes of kFan level-l
// nodes, up to the first level with at most kFan nodes.  Per node: max, min, first and last argmin.
constexpr int kMaxLv = 8;
struct Tree {
    const float *MX[kMaxLv], *MN[kMaxLv];      // [series][cnt[l]] (index 0 unused)
    const int64_t *AL[kMaxLv], *AH[kMaxLv];
    int64_t cnt[kMaxLv];
    int top;
};
// one series' view of the tree (level l node j of series s at [s * cnt[l] + j]); the tree stays
// in the kernel's parameter space
struct STree {
    const Tree &t;
    int64_t s;
    int top;
    __device__ __forceinline__ float mx(int l, int64_t j) const { return t.MX[l][s * t.cnt[l] + j]; }
    __device__ __forceinline__ float mn(int l, int64_t j) const { return t.MN[l][s * t.cnt[l] + j]; }
    __device__ __forceinline__ int64_t al(int l, int64_t j) const { return t.AL[l][s * t.cnt[l] + j]; }
    __device__ __forceinline__ int64_t ah(int l, int64_t j) const { return t.AH[l][s * t.cnt[l] + j]; }
    __device__ __forceinline__ int64_t cnt(int l) const { return t.cnt[l]; }
};
__device__ __forceinline__ int64_t span_of(int l) { return (int64_t)kBS << (5 * (l - 1)); }

// The walks below give the same results as walking sample by sample (the definition).  A warp
// examines up to 32 consecutive samples or nodes per step (lane 0 nearest the peak): it climbs the
// tree through the siblings of the nodes that hold the peak, takes whole nodes from their summaries
// while the walk would pass all of them, and descends into the first node it would not pass.

// Prominence base on the left of peak p: minimum of the samples from p down to the first sample
// above xp (exclusive); on ties the largest index (the first met walking down).
__device__ void prom_left(const Series &v, const STree &u, int64_t p, float xp, int lane, float &lmin, int64_t &lb) {
    lmin = xp;
    lb = p;
    auto samples = [&](int64_t hi, int64_t lo) -> bool {
        for (int64_t base = hi; base >= lo; base -= 32) {
            const int64_t k = base - lane;
            const bool in = k >= lo;
            const float x = in ? v.at(k) : 0.f;
            const unsigned up = __ballot_sync(kFull, in && x > xp);
            const int nl = up ? __ffs(up) - 1 : 32;
            float m = (in && lane < nl) ? x : INFINITY;
            int l = lane;
            warp_argmin(m, l);
            if (m < lmin) { lmin = m; lb = base - l; }
            if (up) return true;
        }
        return false;
    };
    // nodes [lo, hi] of level lv, downwards; true once a sample above xp is met
    auto nodes = [&](int lv, int64_t hi, int64_t lo) -> bool {
        for (int64_t base = hi; base >= lo; base -= 32) {
            const int64_t j = base - lane;
            const bool in = j >= lo;
            const unsigned up = __ballot_sync(kFull, in && u.mx(lv, in ? j : lo) > xp);
            const int nl = up ? __ffs(up) - 1 : 32;
            float m = (in && lane < nl) ? u.mn(lv, j) : INFINITY;
            int l = lane;
            warp_argmin(m, l);
            if (m < lmin) { lmin = m; lb = u.ah(lv, base - l); }
            if (up) {
                // descend into node base - nl: its children from the top, down to the first one
                // above xp, then that block's samples
                int64_t nd = base - nl;
                for (int c = lv - 1; c >= 1; --c) {
                    const int64_t clo = nd * kFan, chi = min(clo + kFan, u.cnt(c)) - 1;
                    const int64_t jj = chi - lane;
                    const bool cin = jj >= clo;
                    const unsigned cup = __ballot_sync(kFull, cin && u.mx(c, cin ? jj : clo) > xp);
                    const int cn = cup ? __ffs(cup) - 1 : 32;
                    float cm = (cin && lane < cn) ? u.mn(c, jj) : INFINITY;
                    int cl = lane;
                    warp_argmin(cm, cl);
                    if (cm < lmin) { lmin = cm; lb = u.ah(c, chi - cl); }
                    nd = chi - cn;
                }
                return samples(nd * kBS + kBS - 1, nd * kBS);
            }
        }
        return false;
    };
    int64_t c = p / kBS;
    if (samples(p, c * kBS)) return;
    for (int lv = 1; lv <= u.top; ++lv, c /= kFan)
        if (nodes(lv, c - 1, lv == u.top ? 0 : (c / kFan) * kFan)) return;
}

// mirrored: samples from p up to the first sample above xp; on ties the smallest index
__device__ void prom_right(const Series &v, const STree &u, int64_t p, float xp, int lane, float &rmin,
                           int64_t &rb) {
    rmin = xp;
    rb = p;
    auto samples = [&](int64_t lo, int64_t hi) -> bool {
        for (int64_t base = lo; base <= hi; base += 32) {
            const int64_t k = base + lane;
            const bool in = k <= hi;
            const float x = in ? v.at(k) : 0.f;
            const unsigned up = __ballot_sync(kFull, in && x > xp);
            const int nl = up ? __ffs(up) - 1 : 32;
            float m = (in && lane < nl) ? x : INFINITY;
            int l = lane;
            warp_argmin(m, l);
            if (m < rmin) { rmin = m; rb = base + l; }
            if (up) return true;
        }
        return false;
    };
    auto nodes = [&](int lv, int64_t lo, int64_t hi) -> bool {
        for (int64_t base = lo; base <= hi; base += 32) {
            const int64_t j = base + lane;
            const bool in = j <= hi;
            const unsigned up = __ballot_sync(kFull, in && u.mx(lv, in ? j : hi) > xp);
            const int nl = up ? __ffs(up) - 1 : 32;
            float m = (in && lane < nl) ? u.mn(lv, j) : INFINITY;
            int l = lane;
            warp_argmin(m, l);
            if (m < rmin) { rmin = m; rb = u.al(lv, base + l); }
            if (up) {
                int64_t nd = base + nl;
                for (int c = lv - 1; c >= 1; --c) {
                    const int64_t clo = nd * kFan, chi = min(clo + kFan, u.cnt(c)) - 1;
                    const int64_t jj = clo + lane;
                    const bool cin = jj <= chi;
                    const unsigned cup = __ballot_sync(kFull, cin && u.mx(c, cin ? jj : chi) > xp);
                    const int cn = cup ? __ffs(cup) - 1 : 32;
                    float cm = (cin && lane < cn) ? u.mn(c, jj) : INFINITY;
                    int cl = lane;
                    warp_argmin(cm, cl);
                    if (cm < rmin) { rmin = cm; rb = u.al(c, clo + cl); }
                    nd = clo + cn;
                }
                return samples(nd * kBS, min(nd * kBS + kBS, v.n) - 1);
            }
        }
        return false;
    };
    int64_t c = p / kBS;
    if (samples(p, min((c + 1) * kBS, v.n) - 1)) return;
    for (int lv = 1; lv <= u.top; ++lv, c /= kFan)
        if (nodes(lv, c + 1, lv == u.top ? u.cnt(lv) - 1 : min((c / kFan + 1) * kFan, u.cnt(lv)) - 1)) return;
}

// Width walk on the left: the first k from p downwards with k <= lb or !(h < x[k]).  A node is
// passed when it lies above lb and all its samples are above h.
__device__ int64_t width_left(const Series &v, const STree &u, int64_t p, int64_t lb, double h, int lane) {
    int64_t k = lb;
    auto samples = [&](int64_t hi, int64_t lo) -> bool {   // lo >= lb
        for (int64_t base = hi; base >= lo; base -= 32) {
            const int64_t kk = base - lane;
            const bool in = kk >= lo;
            const bool stop = in && (kk <= lb || !(h < (double)v.at(kk)));
            const unsigned st = __ballot_sync(kFull, stop);
            if (st) { k = base - (__ffs(st) - 1); return true; }
        }
        return false;
    };
    auto passes = [&](int lv, int64_t j) -> bool { return j * span_of(lv) > lb && h < (double)u.mn(lv, j); };
    auto nodes = [&](int lv, int64_t hi, int64_t lo) -> bool {
        for (int64_t base = hi; base >= lo; base -= 32) {
            const int64_t j = base - lane;
            const unsigned st = __ballot_sync(kFull, j >= lo && !passes(lv, j));
            if (st) {
                int64_t nd = base - (__ffs(st) - 1);
                for (int c = lv - 1; c >= 1; --c) {
                    const int64_t clo = nd * kFan, chi = min(clo + kFan, u.cnt(c)) - 1;
                    const int64_t jj = chi - lane;
                    const unsigned cst = __ballot_sync(kFull, jj >= clo && !passes(c, jj));
                    nd = chi - (__ffs(cst) - 1);
                }
                return samples(nd * kBS + kBS - 1, max(nd * kBS, lb));
            }
        }
        return false;
    };
    int64_t c = p / kBS;
    if (samples(p, max(c * kBS, lb))) return k;
    for (int lv = 1; lv <= u.top; ++lv, c /= kFan)
        if (nodes(lv, c - 1, lv == u.top ? 0 : (c / kFan) * kFan)) return k;
    return k;
}

// Width walk on the right: the first k from p upwards with k >= rb or !(h < x[k]).
__device__ int64_t width_right(const Series &v, const STree &u, int64_t p, int64_t rb, double h, int lane) {
    int64_t k = rb;
    auto samples = [&](int64_t lo, int64_t hi) -> bool {   // hi <= rb
        for (int64_t base = lo; base <= hi; base += 32) {
            const int64_t kk = base + lane;
            const bool in = kk <= hi;
            const bool stop = in && (kk >= rb || !(h < (double)v.at(kk)));
            const unsigned st = __ballot_sync(kFull, stop);
            if (st) { k = base + (__ffs(st) - 1); return true; }
        }
        return false;
    };
    auto passes = [&](int lv, int64_t j) -> bool {
        return (j + 1) * span_of(lv) - 1 < rb && h < (double)u.mn(lv, j);
    };
    auto nodes = [&](int lv, int64_t lo, int64_t hi) -> bool {
        for (int64_t base = lo; base <= hi; base += 32) {
            const int64_t j = base + lane;
            const unsigned st = __ballot_sync(kFull, j <= hi && !passes(lv, j));
            if (st) {
                int64_t nd = base + (__ffs(st) - 1);
                for (int c = lv - 1; c >= 1; --c) {
                    const int64_t clo = nd * kFan, chi = min(clo + kFan, u.cnt(c)) - 1;
                    const int64_t jj = clo + lane;
                    const unsigned cst = __ballot_sync(kFull, jj <= chi && !passes(c, jj));
                    nd = clo + (__ffs(cst) - 1);
                }
                return samples(nd * kBS, min(nd * kBS + kBS - 1, rb));
            }
        }
        return false;
    };
    int64_t c = p / kBS;
    if (samples(p, min(c * kBS + kBS - 1, rb))) return k;
    for (int lv = 1; lv <= u.top; ++lv, c /= kFan)
        if (nodes(lv, c + 1, lv == u.top ? u.cnt(lv) - 1 : min((c / kFan + 1) * kFan, u.cnt(lv)) - 1)) return k;
    return k;
}

// 3b. prominence and width of the candidates whose walks leave the shared-memory window of
// k_eval_local (list[0 .. *count)), one warp each, on the summary tree
__global__ void k_eval_tree(Geo g, const int64_t *list, const int64_t *count, const int64_t *cand_idx,
                            const int *cand_ser, const Tree t, double min_width, int *keep, double *o_h, double *o_pr,
                            double *o_wd) {
    const int lane = threadIdx.x & 31;
    const int64_t nlong = *count;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t wi = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; wi < nlong; wi += nwarps) {
        const int64_t ci = list[wi];
        const int s = cand_ser[ci];
        const int64_t p = cand_idx[ci];
        const Series v = g.series(s);
        const STree u{t, (int64_t)s, t.top};
        const float xp = v.at(p);
        float lmin, rmin;
        int64_t lb, rb;
        prom_left(v, u, p, xp, lane, lmin, lb);
        prom_right(v, u, p, xp, lane, rmin, rb);
        const double dxp = (double)xp;
        const double base = (double)lmin > (double)rmin ? (double)lmin : (double)rmin;
        const double pr = __dsub_rn(dxp, base);
        const double h = __dsub_rn(dxp, __dmul_rn(pr, 0.5));
        // width at half prominence, interpolated between the samples on either side of h
        int64_t k = width_left(v, u, p, lb, h, lane);
        double lip = (double)k;
        {
            const double xk = (double)v.at(k);
            if (xk < h) lip = __dadd_rn(lip, __ddiv_rn(__dsub_rn(h, xk), __dsub_rn((double)v.at(k + 1), xk)));
        }
        k = width_right(v, u, p, rb, h, lane);
        double rip = (double)k;
        {
            const double xk = (double)v.at(k);
            if (xk < h) rip = __dsub_rn(rip, __ddiv_rn(__dsub_rn(h, xk), __dsub_rn((double)v.at(k - 1), xk)));
        }
        if (lane == 0) {
            const double wd = __dsub_rn(rip, lip);
            keep[ci] = (wd >= min_width) ? 1 : 0;
            o_h[ci] = dxp;
            o_pr[ci] = pr;
            o_wd[ci] = wd;
        }
    }
}

// order-preserving unsigned key of a float (-0 taken as +0): a < b  <=>  fkey(a) < fkey(b) for
// numbers; the series are probabilities or logits and hold no NaN (a NaN would compare as a number
// here, while the definition never takes it as a minimum)
__device__ __forceinline__ unsigned fkey(float x) {
    const unsigned u = __float_as_uint(x + 0.0f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// 3a. prominence and width of the candidates of one kCH-sample chunk (blockIdx.x) of series
// blockIdx.y over the chunk and kHalo samples on either side held in shared memory, one warp per
// candidate, 32 samples per step (lane 0 nearest the peak), with the results of the definition's
// sample-by-sample walks: the running minimum changes only at a strictly smaller sample, and the
// width test h < (double)x is x > hf with hf the largest float <= h.  A candidate whose
// prominence walk reaches the edge of the window (not the end of the series) goes to the list for
// k_eval_tree.
constexpr int kHalo = 2048;
__global__ void __launch_bounds__(kT) k_eval_local(Geo g, int64_t nchunk, const int64_t *offsets,
                                                     const int64_t *cand_idx, double min_width, int64_t mw_int,
                                                     int *keep,
                                                     double *o_h, double *o_pr, double *o_wd, int64_t *list,
                                                     unsigned long long *count) {
    __shared__ float sm[kCH + 2 * kHalo];
    const int s = blockIdx.y;
    const int64_t c = blockIdx.x;
    const int64_t beg = offsets[(int64_t)s * nchunk + c], end = offsets[(int64_t)s * nchunk + c + 1];
    if (beg == end) return;
    const Series v = g.series(s);
    const int64_t w0 = c * kCH > kHalo ? c * kCH - kHalo : 0;
    const int64_t w1 = c * kCH + kCH + kHalo < v.n ? c * kCH + kCH + kHalo : v.n;
    for (int64_t k = w0 + threadIdx.x; k < w1; k += kT) sm[k - w0] = v.at(k);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int nloc = (int)(w1 - w0);
    for (int64_t ci = beg + (threadIdx.x >> 5); ci < end; ci += kT / 32) {
        const int64_t p = cand_idx[ci];
        if (p >= w1) {   // the plateau midpoint of a candidate of this chunk lies beyond the window
            if (lane == 0) list[atomicAdd(count, 1ull)] = ci;
            continue;
        }
        const int pl = (int)(p - w0);
        const float xp = sm[pl];
        // prominence walks in window coordinates
        unsigned kmin = fkey(xp);
        int lbl = pl;
        bool done = w0 == 0;              // the walk may end at the series start
        for (int base = pl; base >= 0; base -= 32) {
            const int k = base - lane;
            const bool in = k >= 0;
            const float x = in ? sm[k] : 0.f;
            const unsigned up = __ballot_sync(kFull, in && x > xp);
            const int nl = up ? __ffs(up) - 1 : 32;
            const bool part = in && lane < nl;
            const unsigned key = part ? fkey(x) : 0xFFFFFFFFu;
            const unsigned mk = __reduce_min_sync(kFull, key);
            if (mk < kmin) {
                kmin = mk;
                lbl = base - (__ffs(__ballot_sync(kFull, part && key == mk)) - 1);
            }
            if (up) { done = true; break; }
        }
        if (done) {
            unsigned kr = fkey(xp);
            int rbl = pl;
            done = w1 == v.n;             // the walk may end at the series end
            for (int base = pl; base < nloc; base += 32) {
                const int k = base + lane;
                const bool in = k < nloc;
                const float x = in ? sm[k] : 0.f;
                const unsigned up = __ballot_sync(kFull, in && x > xp);
                const int nl = up ? __ffs(up) - 1 : 32;
                const bool part = in && lane < nl;
                const unsigned key = part ? fkey(x) : 0xFFFFFFFFu;
                const unsigned mk = __reduce_min_sync(kFull, key);
                if (mk < kr) {
                    kr = mk;
                    rbl = base + (__ffs(__ballot_sync(kFull, part && key == mk)) - 1);
                }
                if (up) { done = true; break; }
            }
            if (done) {
                const float lmin = sm[lbl], rmin = sm[rbl];
                const float bse = lmin > rmin ? lmin : rmin;
                // h = xp - (xp - base) / 2 (FP64, the definition) and hf, the largest float <= h.
                // When xp and base are within 2^27 of each other (and of moderate size), xp - base
                // and h = (xp + base) / 2 are exact in FP64, so hf = RD(xp + base) / 2 in FP32; only
                // the other cases evaluate h in FP64 here (FP64 is slow on this part).
                const float aa = fabsf(xp), ab = fabsf(bse);
                const float lo = fminf(aa, ab), hi = fmaxf(aa, ab);
                const bool exact = hi <= 0x1p100f && (lo == 0.f ? (hi == 0.f || hi >= 0x1p-100f)
                                                                : (lo >= 0x1p-100f && hi <= lo * 0x1p27f));
                float hf;
                if (exact) {
                    hf = __fmul_rn(__fadd_rd(xp, bse), 0.5f);
                } else {
                    const double pr0 = __dsub_rn((double)xp, (double)bse);
                    hf = __double2float_rd(__dsub_rn((double)xp, __dmul_rn(pr0, 0.5)));
                }
                // width walks: the first k from the peak with k at the base or !(h < x[k])
                int kl = lbl;
                for (int base = pl; base >= lbl; base -= 32) {
                    const int k = base - lane;
                    const unsigned st = __ballot_sync(kFull, k >= lbl && (k == lbl || !(sm[k] > hf)));
                    if (st) { kl = base - (__ffs(st) - 1); break; }
                }
                int kr2 = rbl;
                for (int base = pl; base <= rbl; base += 32) {
                    const int k = base + lane;
                    const unsigned st = __ballot_sync(kFull, k <= rbl && (k == rbl || !(sm[k] > hf)));
                    if (st) { kr2 = base + (__ffs(st) - 1); break; }
                }
                // the width lies in (kr2 - kl - 2, kr2 - kl]: below min_width when kr2 - kl < mw_int
                if (lane == 0 && (int64_t)(kr2 - kl) < mw_int) keep[ci] = 0;
                if (lane == 0 && (int64_t)(kr2 - kl) >= mw_int) {
                    const double dxp = (double)xp;
                    const double pr = __dsub_rn(dxp, (double)bse);
                    const double h = __dsub_rn(dxp, __dmul_rn(pr, 0.5));
                    double lip = (double)(w0 + kl);
                    {
                        const double xk = (double)sm[kl];
                        if (xk < h) lip = __dadd_rn(lip, __ddiv_rn(__dsub_rn(h, xk), __dsub_rn((double)sm[kl + 1], xk)));
                    }
                    double rip = (double)(w0 + kr2);
                    {
                        const double xk = (double)sm[kr2];
                        if (xk < h) rip = __dsub_rn(rip, __ddiv_rn(__dsub_rn(h, xk), __dsub_rn((double)sm[kr2 - 1], xk)));
                    }
                    const double wd = __dsub_rn(rip, lip);
                    keep[ci] = (wd >= min_width) ? 1 : 0;
                    o_h[ci] = dxp;
                    o_pr[ci] = pr;
                    o_wd[ci] = wd;
                }
                continue;
            }
        }
        if (lane == 0) list[atomicAdd(count, 1ull)] = ci;
    }
}

// ordered compaction of int flags: per 8192-element chunk counts, then writes
__global__ void k_flag_pass(const int *flags, int64_t n, int mode, int64_t *counts, const int64_t *offsets,
                            int64_t *sel) {
    __shared__ int sh[kT / 32 + 1];
    const int64_t lo = (int64_t)blockIdx.x * kCH;
    int64_t run = (mode == 1) ? offsets[blockIdx.x] : 0;
    for (int it = 0; it < kCH / kT; ++it) {
        const int64_t i = lo + (int64_t)it * kT + threadIdx.x;
        const int f = (i < n) ? flags[i] : 0;
        int tot;
        const int r = block_rank(f, sh, tot);
        if (mode == 1 && f) sel[run + r] = i;
        run += tot;
    }
    if (mode == 0 && threadIdx.x == 0) counts[blockIdx.x] = run;
}

__global__ void k_gather_peaks(int64_t npk, const int64_t *sel, const int64_t *cand_idx, const int *cand_ser,
                               const double *h, const double *pr, const double *wd, int64_t *p_idx, int *p_ser,
                               double *p_h, double *p_pr, double *p_wd) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npk) return;
    const int64_t c = sel[i];
    p_idx[i] = cand_idx[c]; p_ser[i] = cand_ser[c];
    p_h[i] = h[c]; p_pr[i] = pr[c]; p_wd[i] = wd[c];
}

__global__ void k_series_start(const int *p_ser, int64_t npk, int n_series, int64_t *start) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s > n_series) return;
    int64_t lo = 0, hi = npk;      // first index with p_ser >= s
    while (lo < hi) {
        const int64_t mid = (lo + hi) / 2;
        if (p_ser[mid] < s) lo = mid + 1; else hi = mid;
    }
    start[s] = lo;
}

__device__ __forceinline__ bool has_peak_in(const int64_t *pk, int64_t lo_i, int64_t hi_i, int64_t a, int64_t b) {
    int64_t lo = lo_i, hi = hi_i;   // first peak >= a
    while (lo < hi) {
        const int64_t mid = (lo + hi) / 2;
        if (pk[mid] < a) lo = mid + 1; else hi = mid;
    }
    return lo < hi_i && pk[lo] <= b;
}

// 5. coincidence: model-0 peak p0 is kept iff some window [a, a + coinc] with
//    a in [p0 - coinc, p0] holds a peak of every other model; the smallest
//    feasible a is p0 - coinc or (q - coinc) for a peak q in [p0, p0 + coinc].
__global__ void k_coinc(int64_t npk, const int64_t *p_idx, const int *p_ser, const int64_t *start, int n_models,
                        int64_t coinc, int *ens) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npk) return;
    const int s = p_ser[i];
    const int m = s % n_models;
    if (m != 0) { ens[i] = 0; return; }
    const int s0 = s;    // series of model 0 for this slide
    const int64_t p0 = p_idx[i];
    bool ok = false;
    for (int mc = -1; mc < n_models && !ok; ++mc) {
        int64_t qlo = 0, qhi = 1;
        if (mc >= 0) {
            const int64_t b0 = start[s0 + mc], b1 = start[s0 + mc + 1];
            // peaks q of model mc with q in [p0, p0 + coinc]
            int64_t lo = b0, hi = b1;
            while (lo < hi) {
                const int64_t mid = (lo + hi) / 2;
                if (p_idx[mid] < p0) lo = mid + 1; else hi = mid;
            }
            qlo = lo; qhi = b1;
        }
        for (int64_t q = qlo; q < qhi && !ok; ++q) {
            int64_t a;
            if (mc < 0) a = p0 - coinc;
            else {
                if (p_idx[q] > p0 + coinc) break;
                a = p_idx[q] - coinc;
            }
            bool all = true;
            for (int mm = 1; mm < n_models && all; ++mm)
                all = has_peak_in(p_idx, start[s0 + mm], start[s0 + mm + 1], a, a + coinc);
            ok = all;
        }
    }
    ens[i] = ok ? 1 : 0;
}

// Threshold sweep (section "Statistical Analysis": the ROC and false-alarm curves come from
// sweeping the height threshold over [0, 0.9998]).  A peak's prominence and width do not depend
// on the threshold, so with the peaks found once at the lowest threshold (and the width cut
// applied), model-0 peak p0 is an ensemble trigger at threshold thr iff h(p0) >= thr and some
// candidate window [a, a + coinc] of k_coinc holds, for every other model, a peak of height
// >= thr.  Its largest such threshold is
//   T(p0) = min(h(p0), max over candidate windows a of min over models m >= 1 of
//                      (largest height of model m's peaks in [a, a + coinc])),
// (the candidate windows of the peaks above any threshold are among those of all the peaks, and
// a window that serves at thr serves at every lower one), and it is a trigger at every
// threshold <= T(p0).  Each peak adds one to the histogram bin of its value: the number of
// thresholds <= value (thresholds ascending); count(thr_k) is then the sum of the bins above k.
__device__ __forceinline__ double max_height_in(const int64_t *pk, const double *ph, int64_t lo_i, int64_t hi_i,
                                                int64_t a, int64_t b) {
    int64_t lo = lo_i, hi = hi_i;   // first peak >= a
    while (lo < hi) {
        const int64_t mid = (lo + hi) / 2;
        if (pk[mid] < a) lo = mid + 1; else hi = mid;
    }
    double mx = -INFINITY;
    for (int64_t q = lo; q < hi_i && pk[q] <= b; ++q) mx = fmax(mx, ph[q]);
    return mx;
}

__device__ __forceinline__ int thr_bin(const double *thr, int K, double v) {
    int lo = 0, hi = K;             // number of thresholds <= v
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (thr[mid] <= v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// one thread per kept peak: model histogram bin of its height; model-0 peaks also the ensemble
// histogram bin of T(p0).  hist_m [series][K + 1], hist_e [slide][K + 1]
__global__ void k_sweep_hist(int64_t npk, const int64_t *p_idx, const int *p_ser, const double *p_h,
                             const int64_t *start, int n_models, int64_t coinc, const double *thr, int K,
                             unsigned long long *hist_m, unsigned long long *hist_e) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npk) return;
    const int s = p_ser[i];
    const int m = s % n_models;
    const double h0 = p_h[i];
    atomicAdd(&hist_m[(int64_t)s * (K + 1) + thr_bin(thr, K, h0)], 1ull);
    if (m != 0) return;
    const int64_t p0 = p_idx[i];
    double best = -INFINITY;
    for (int mc = -1; mc < n_models; ++mc) {
        int64_t qlo = 0, qhi = 1;
        if (mc >= 0) {
            const int64_t b0 = start[s + mc], b1 = start[s + mc + 1];
            int64_t lo = b0, hi = b1;   // peaks q of model mc with q in [p0, p0 + coinc]
            while (lo < hi) {
                const int64_t mid = (lo + hi) / 2;
                if (p_idx[mid] < p0) lo = mid + 1; else hi = mid;
            }
            qlo = lo;
            qhi = b1;
        }
        for (int64_t q = qlo; q < qhi; ++q) {
            int64_t a;
            if (mc < 0) {
                a = p0 - coinc;
            } else {
                if (p_idx[q] > p0 + coinc) break;
                a = p_idx[q] - coinc;
            }
            double v = INFINITY;
            for (int mm = 1; mm < n_models && v > best; ++mm)
                v = fmin(v, max_height_in(p_idx, p_h, start[s + mm], start[s + mm + 1], a, a + coinc));
            best = fmax(best, v);
        }
    }
    const double T = fmin(h0, best);
    atomicAdd(&hist_e[(int64_t)(s / n_models) * (K + 1) + thr_bin(thr, K, T)], 1ull);
}

// counts[row][k] = sum over bins b > k of hist[row][b]
__global__ void k_sweep_suffix(const unsigned long long *hist, int rows, int K, long long *counts) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    unsigned long long acc = 0;
    for (int k = K - 1; k >= 0; --k) {
        acc += hist[(int64_t)r * (K + 1) + k + 1];
        counts[(int64_t)r * K + k] = (long long)acc;
    }
}

struct TrigWs {
    std::mutex mu;
    DevBuf stats_mx, stats_mn, stats_lo, stats_hi, sb_mx, sb_mn, sb_lo, sb_hi, longs, nlong, counts, offsets, cand_idx, cand_ser, keep, h, pr, wd, sel,
        p_idx, p_ser, p_h, p_pr, p_wd, start, ens, sw_thr, sw_hist, sw_counts;
};

}  // namespace

// a threshold sweep request of triggers_collect: thresholds ascending (host, FP64 values of FP32
// thresholds), counts accumulated into the host arrays (per slide, and per slide and model)
struct SweepReq {
    std::vector<double> thr;
    int64_t *ens_counts = nullptr;     // [n_slides][K]
    int64_t *model_counts = nullptr;   // [n_slides][n_models][K] or NULL
};

namespace {
TrigWs &trig_ws() {
    static TrigWs *w = new TrigWs();   // kept until process exit
    return *w;
}

unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

namespace {

// all records of one segment's (slide, model) series, appended to recs
// With sw != NULL (threshold sweep, thr = the lowest threshold) the kept peaks go to the sweep
// histograms and their counts are added to sw's host arrays instead of records.
gwe_status triggers_collect(const float *prob, int n_models, int n_slides, int64_t nw, int64_t series_nw, int W,
                            int stride, float thr, double min_width, int64_t coinc, int flags,
                            std::vector<gwe_trigger> &recs, cudaStream_t st, const SweepReq *sw = nullptr) {
    TrigWs &ws = trig_ws();
    std::lock_guard<std::mutex> lock(ws.mu);
    const int ns = n_slides > 0 ? n_slides : 1;
    const int n_series = ns * n_models;
    if (nw <= 0) return GWE_OK;
    Geo g;
    g.prob = prob; g.nw = nw; g.series_nw = series_nw; g.W = W; g.stride = stride;
    g.n = (nw - 1) * (int64_t)stride + W;
    g.nblk = (g.n + kBS - 1) / kBS;
    const int64_t nstat = g.nblk * n_series;
    GWE_CUDA_TRY(ws.stats_mx.ensure(nstat * sizeof(float)));
    GWE_CUDA_TRY(ws.stats_mn.ensure(nstat * sizeof(float)));
    GWE_CUDA_TRY(ws.stats_lo.ensure(nstat * sizeof(int64_t)));
    GWE_CUDA_TRY(ws.stats_hi.ensure(nstat * sizeof(int64_t)));
    {
        ProfScope prof("k_trig_stats", st);
        k_stats<<<blocks_for(nstat, 8), 256, 0, st>>>(g, ws.stats_mx.as<float>(), ws.stats_mn.as<float>(),
                                                       ws.stats_lo.as<int64_t>(), ws.stats_hi.as<int64_t>(), n_series);
        note_launch();
    }
    // summary tree: level 1 = the block statistics, then levels of kFan nodes until at most kFan remain
    Tree tr{};
    tr.MX[1] = ws.stats_mx.as<float>();
    tr.MN[1] = ws.stats_mn.as<float>();
    tr.AL[1] = ws.stats_lo.as<int64_t>();
    tr.AH[1] = ws.stats_hi.as<int64_t>();
    tr.cnt[1] = g.nblk;
    int64_t upper = 0;
    for (int64_t c = g.nblk; c > kFan;) {
        c = (c + kFan - 1) / kFan;
        upper += c * n_series;
    }
    GWE_CUDA_TRY(ws.sb_mx.ensure(std::max<int64_t>(upper, 1) * sizeof(float)));
    GWE_CUDA_TRY(ws.sb_mn.ensure(std::max<int64_t>(upper, 1) * sizeof(float)));
    GWE_CUDA_TRY(ws.sb_lo.ensure(std::max<int64_t>(upper, 1) * sizeof(int64_t)));
    GWE_CUDA_TRY(ws.sb_hi.ensure(std::max<int64_t>(upper, 1) * sizeof(int64_t)));
    int top = 1;
    for (int64_t off = 0; tr.cnt[top] > kFan && top + 1 < kMaxLv; ++top) {
        const int64_t cn = (tr.cnt[top] + kFan - 1) / kFan;
        tr.MX[top + 1] = ws.sb_mx.as<float>() + off;
        tr.MN[top + 1] = ws.sb_mn.as<float>() + off;
        tr.AL[top + 1] = ws.sb_lo.as<int64_t>() + off;
        tr.AH[top + 1] = ws.sb_hi.as<int64_t>() + off;
        tr.cnt[top + 1] = cn;
        {
            ProfScope prof("k_trig_stats", st);
            k_stats_up<<<blocks_for(cn * n_series, 256), 256, 0, st>>>(
                tr.cnt[top], cn, n_series, tr.MX[top], tr.MN[top], tr.AL[top], tr.AH[top],
                const_cast<float *>(tr.MX[top + 1]), const_cast<float *>(tr.MN[top + 1]),
                const_cast<int64_t *>(tr.AL[top + 1]), const_cast<int64_t *>(tr.AH[top + 1]));
            note_launch();
        }
        off += cn * n_series;
    }
    tr.top = top;
    const int64_t nchunk = (g.n + kCH - 1) / kCH;
    const int64_t ncnt = nchunk * n_series;
    GWE_CUDA_TRY(ws.counts.ensure(ncnt * sizeof(int64_t)));
    GWE_CUDA_TRY(ws.offsets.ensure((ncnt + 1) * sizeof(int64_t)));
    const float dthr = thr;
    dim3 cgrid((unsigned)nchunk, (unsigned)n_series);
    {
        ProfScope prof("k_trig_cand", st);
        k_cand<<<cgrid, kT, 0, st>>>(g, dthr, 0, ws.counts.as<int64_t>(), nullptr, nullptr, nullptr, nchunk);
        note_launch();
    }
    {
        ProfScope prof("k_trig_scan", st);
        k_scan<<<1, 1024, 0, st>>>(ws.counts.as<int64_t>(), ws.offsets.as<int64_t>(), ncnt);
        note_launch();
    }
    int64_t ncand = 0;
    GWE_CUDA_TRY(cudaMemcpyAsync(&ncand, ws.offsets.as<int64_t>() + ncnt, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    GWE_CUDA_TRY(cudaStreamSynchronize(st));
    if (ncand > 0) {
        GWE_CUDA_TRY(ws.cand_idx.ensure(ncand * sizeof(int64_t)));
        GWE_CUDA_TRY(ws.cand_ser.ensure(ncand * sizeof(int)));
        GWE_CUDA_TRY(ws.keep.ensure(ncand * sizeof(int)));
        GWE_CUDA_TRY(ws.h.ensure(ncand * sizeof(double)));
        GWE_CUDA_TRY(ws.pr.ensure(ncand * sizeof(double)));
        GWE_CUDA_TRY(ws.wd.ensure(ncand * sizeof(double)));
        {
            ProfScope prof("k_trig_cand", st);
            k_cand<<<cgrid, kT, 0, st>>>(g, dthr, 1, nullptr, ws.offsets.as<int64_t>(), ws.cand_idx.as<int64_t>(),
                                         ws.cand_ser.as<int>(), nchunk);
            note_launch();
        }
        // an integer span below mw_int cannot reach min_width (NaN: nothing is kept)
        const int64_t mw_int = std::isnan(min_width) ? INT64_MAX
                               : (min_width <= 0.0 ? 0 : (min_width >= 9.0e18 ? INT64_MAX : (int64_t)std::ceil(min_width)));
        GWE_CUDA_TRY(ws.longs.ensure(ncand * sizeof(int64_t)));
        GWE_CUDA_TRY(ws.nlong.ensure(sizeof(unsigned long long)));
        GWE_CUDA_TRY(cudaMemsetAsync(ws.nlong.ptr, 0, sizeof(unsigned long long), st));
        {
            ProfScope prof("k_eval_local", st);
            k_eval_local<<<cgrid, kT, 0, st>>>(g, nchunk, ws.offsets.as<int64_t>(), ws.cand_idx.as<int64_t>(),
                                               min_width, mw_int, ws.keep.as<int>(), ws.h.as<double>(), ws.pr.as<double>(),
                                               ws.wd.as<double>(), ws.longs.as<int64_t>(),
                                               ws.nlong.as<unsigned long long>());
            note_launch();
        }
        {
            ProfScope prof("k_eval_tree", st);
            k_eval_tree<<<2048, 128, 0, st>>>(g, ws.longs.as<int64_t>(), ws.nlong.as<int64_t>(),
                                               ws.cand_idx.as<int64_t>(), ws.cand_ser.as<int>(), tr, min_width,
                                               ws.keep.as<int>(), ws.h.as<double>(), ws.pr.as<double>(),
                                               ws.wd.as<double>());
            note_launch();
        }
        const int64_t nfc = (ncand + kCH - 1) / kCH;
        GWE_CUDA_TRY(ws.counts.ensure(nfc * sizeof(int64_t)));
        GWE_CUDA_TRY(ws.offsets.ensure((nfc + 1) * sizeof(int64_t)));
        {
            ProfScope prof("k_trig_compact", st);
            k_flag_pass<<<(unsigned)nfc, kT, 0, st>>>(ws.keep.as<int>(), ncand, 0, ws.counts.as<int64_t>(), nullptr,
                                                      nullptr);
            note_launch();
        }
        {
            ProfScope prof("k_trig_scan", st);
            k_scan<<<1, 1024, 0, st>>>(ws.counts.as<int64_t>(), ws.offsets.as<int64_t>(), nfc);
            note_launch();
        }
        int64_t npk = 0;
        GWE_CUDA_TRY(cudaMemcpyAsync(&npk, ws.offsets.as<int64_t>() + nfc, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        GWE_CUDA_TRY(cudaStreamSynchronize(st));
        if (npk > 0) {
            GWE_CUDA_TRY(ws.sel.ensure(npk * sizeof(int64_t)));
            GWE_CUDA_TRY(ws.p_idx.ensure(npk * sizeof(int64_t)));
            GWE_CUDA_TRY(ws.p_ser.ensure(npk * sizeof(int)));
            GWE_CUDA_TRY(ws.p_h.ensure(npk * sizeof(double)));
            GWE_CUDA_TRY(ws.p_pr.ensure(npk * sizeof(double)));
            GWE_CUDA_TRY(ws.p_wd.ensure(npk * sizeof(double)));
            GWE_CUDA_TRY(ws.ens.ensure(npk * sizeof(int)));
            GWE_CUDA_TRY(ws.start.ensure((n_series + 1) * sizeof(int64_t)));
            {
                ProfScope prof("k_trig_compact", st);
                k_flag_pass<<<(unsigned)nfc, kT, 0, st>>>(ws.keep.as<int>(), ncand, 1, nullptr, ws.offsets.as<int64_t>(),
                                                          ws.sel.as<int64_t>());
                note_launch();
            }
            {
                ProfScope prof("k_trig_compact", st);
                k_gather_peaks<<<blocks_for(npk, 256), 256, 0, st>>>(
                    npk, ws.sel.as<int64_t>(), ws.cand_idx.as<int64_t>(), ws.cand_ser.as<int>(), ws.h.as<double>(),
                    ws.pr.as<double>(), ws.wd.as<double>(), ws.p_idx.as<int64_t>(), ws.p_ser.as<int>(),
                    ws.p_h.as<double>(), ws.p_pr.as<double>(), ws.p_wd.as<double>());
                note_launch();
            }
            {
                ProfScope prof("k_trig_compact", st);
                k_series_start<<<blocks_for(n_series + 1, 128), 128, 0, st>>>(ws.p_ser.as<int>(), npk, n_series,
                                                                             ws.start.as<int64_t>());
                note_launch();
            }
            if (sw) {
                const int K = (int)sw->thr.size();
                const int64_t hm = (int64_t)n_series * (K + 1), he = (int64_t)ns * (K + 1);
                GWE_CUDA_TRY(ws.sw_thr.ensure(K * sizeof(double)));
                GWE_CUDA_TRY(ws.sw_hist.ensure((hm + he) * sizeof(unsigned long long)));
                GWE_CUDA_TRY(ws.sw_counts.ensure((int64_t)(n_series + ns) * K * sizeof(long long)));
                GWE_CUDA_TRY(cudaMemcpyAsync(ws.sw_thr.ptr, sw->thr.data(), K * sizeof(double), cudaMemcpyHostToDevice, st));
                GWE_CUDA_TRY(cudaMemsetAsync(ws.sw_hist.ptr, 0, (hm + he) * sizeof(unsigned long long), st));
                unsigned long long *hist_m = ws.sw_hist.as<unsigned long long>(), *hist_e = hist_m + hm;
                long long *cnt = ws.sw_counts.as<long long>();
                {
                    ProfScope prof("k_sweep", st);
                    k_sweep_hist<<<blocks_for(npk, 128), 128, 0, st>>>(npk, ws.p_idx.as<int64_t>(), ws.p_ser.as<int>(),
                                                                       ws.p_h.as<double>(), ws.start.as<int64_t>(),
                                                                       n_models, coinc, ws.sw_thr.as<double>(), K,
                                                                       hist_m, hist_e);
                    note_launch();
                }
                {
                    ProfScope prof("k_sweep", st);
                    k_sweep_suffix<<<blocks_for(n_series + ns, 128), 128, 0, st>>>(hist_m, n_series + ns, K, cnt);
                    note_launch();
                }
                GWE_CUDA_TRY(cudaGetLastError());
                std::vector<long long> hc((size_t)(n_series + ns) * K);
                GWE_CUDA_TRY(cudaMemcpyAsync(hc.data(), cnt, hc.size() * sizeof(long long), cudaMemcpyDeviceToHost, st));
                GWE_CUDA_TRY(cudaStreamSynchronize(st));
                for (int64_t i = 0; i < (int64_t)ns * K; ++i) sw->ens_counts[i] += hc[(size_t)n_series * K + i];
                if (sw->model_counts)
                    for (int64_t i = 0; i < (int64_t)n_series * K; ++i) sw->model_counts[i] += hc[i];
                return GWE_OK;
            }
            {
                ProfScope prof("k_coinc", st);
                k_coinc<<<blocks_for(npk, 128), 128, 0, st>>>(npk, ws.p_idx.as<int64_t>(), ws.p_ser.as<int>(),
                                                              ws.start.as<int64_t>(), n_models, coinc, ws.ens.as<int>());
                note_launch();
            }
            GWE_CUDA_TRY(cudaGetLastError());
            std::vector<int64_t> idx(npk);
            std::vector<int> ser(npk), ens(npk);
            std::vector<double> hh(npk), pp(npk), ww(npk);
            GWE_CUDA_TRY(cudaMemcpyAsync(idx.data(), ws.p_idx.ptr, npk * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
            GWE_CUDA_TRY(cudaMemcpyAsync(ser.data(), ws.p_ser.ptr, npk * sizeof(int), cudaMemcpyDeviceToHost, st));
            GWE_CUDA_TRY(cudaMemcpyAsync(ens.data(), ws.ens.ptr, npk * sizeof(int), cudaMemcpyDeviceToHost, st));
            GWE_CUDA_TRY(cudaMemcpyAsync(hh.data(), ws.p_h.ptr, npk * sizeof(double), cudaMemcpyDeviceToHost, st));
            GWE_CUDA_TRY(cudaMemcpyAsync(pp.data(), ws.p_pr.ptr, npk * sizeof(double), cudaMemcpyDeviceToHost, st));
            GWE_CUDA_TRY(cudaMemcpyAsync(ww.data(), ws.p_wd.ptr, npk * sizeof(double), cudaMemcpyDeviceToHost, st));
            GWE_CUDA_TRY(cudaStreamSynchronize(st));
            // records: per slide, per-model peaks (model order, index order) then ensemble triggers
            int64_t i = 0;
            for (int si = 0; si < ns; ++si) {
                std::vector<gwe_trigger> ensr;
                while (i < npk && ser[i] / n_models == si) {
                    gwe_trigger t;
                    t.index = idx[i]; t.slide = si; t.model = ser[i] % n_models;
                    t.height = hh[i]; t.prominence = pp[i]; t.width = ww[i];
                    if (flags & GWE_TRIG_PER_MODEL) recs.push_back(t);
                    if (ens[i]) { t.model = -1; ensr.push_back(t); }
                    ++i;
                }
                recs.insert(recs.end(), ensr.begin(), ensr.end());
            }
        }
    }
    GWE_CUDA_TRY(cudaGetLastError());
    return GWE_OK;
}

gwe_status copy_out(const std::vector<gwe_trigger> &recs, const std::vector<int32_t> *segs, gwe_trigger *out,
                    int32_t *out_seg, int64_t cap, int64_t *n_out) {
    *n_out = (int64_t)recs.size();
    const int64_t k = std::min<int64_t>(cap, (int64_t)recs.size());
    if (k > 0 && out) std::copy(recs.begin(), recs.begin() + k, out);
    if (k > 0 && out_seg && segs) std::copy(segs->begin(), segs->begin() + k, out_seg);
    if ((int64_t)recs.size() > cap) {
        set_error("gwe_triggers: output capacity too small");
        return GWE_ERR_CAPACITY;
    }
    return GWE_OK;
}

}  // namespace

gwe_status triggers_run(const float *prob, int n_models, int n_slides, int64_t nw, int W, int stride, float thr,
                        double min_width, int64_t coinc, int flags, gwe_trigger *out, int64_t cap, int64_t *n_out,
                        cudaStream_t st) {
    *n_out = 0;
    std::vector<gwe_trigger> recs;
    gwe_status r = triggers_collect(prob, n_models, n_slides, nw, nw, W, stride, thr, min_width, coinc, flags, recs, st);
    if (r != GWE_OK) return r;
    return copy_out(recs, nullptr, out, nullptr, cap, n_out);
}

gwe_status triggers_sweep(const float *prob, int n_models, int n_slides, const int64_t *seg_nw, int n_seg, int W,
                          int stride, const float *thr, int n_thr, double min_width, int64_t coinc,
                          int64_t *ens_counts, int64_t *model_counts, cudaStream_t st) {
    const int ns = n_slides > 0 ? n_slides : 1;
    SweepReq sw;
    sw.thr.resize(n_thr);
    for (int k = 0; k < n_thr; ++k) sw.thr[k] = (double)thr[k];
    sw.ens_counts = ens_counts;
    sw.model_counts = model_counts;
    std::fill(ens_counts, ens_counts + (int64_t)ns * n_thr, 0);
    if (model_counts) std::fill(model_counts, model_counts + (int64_t)ns * n_models * n_thr, 0);
    int64_t nw_all = 0;
    for (int g = 0; g < n_seg; ++g) nw_all += seg_nw[g];
    std::vector<gwe_trigger> none;
    int64_t wo = 0;
    for (int g = 0; g < n_seg; ++g) {
        gwe_status r = triggers_collect(prob + wo * W, n_models, n_slides, seg_nw[g], nw_all, W, stride, thr[0],
                                        min_width, coinc, 0, none, st, &sw);
        if (r != GWE_OK) return r;
        wo += seg_nw[g];
    }
    return GWE_OK;
}

gwe_status triggers_run_segments(const float *prob, int n_models, int n_slides, const int64_t *seg_nw, int n_seg,
                                 int W, int stride, float thr, double min_width, int64_t coinc, int flags,
                                 gwe_trigger *out, int32_t *out_seg, int64_t cap, int64_t *n_out, cudaStream_t st) {
    *n_out = 0;
    int64_t nw_all = 0;
    for (int g = 0; g < n_seg; ++g) nw_all += seg_nw[g];
    std::vector<gwe_trigger> recs;
    std::vector<int32_t> segs;
    int64_t wo = 0;
    for (int g = 0; g < n_seg; ++g) {
        gwe_status r = triggers_collect(prob + wo * W, n_models, n_slides, seg_nw[g], nw_all, W, stride, thr,
                                        min_width, coinc, flags, recs, st);
        if (r != GWE_OK) return r;
        segs.resize(recs.size(), g);
        wo += seg_nw[g];
    }
    return copy_out(recs, &segs, out, out_seg, cap, n_out);
}

}  // namespace gwe
