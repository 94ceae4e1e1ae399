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
//   1. per 256-sample block of every series: max, min, first and last argmin
//      (lets the long prominence and width walks skip whole blocks);
//   2. candidate count per 8192-sample chunk -> exclusive scan -> ordered write
//      of every local maximum (plateau midpoint) whose height passes;
//   3. per candidate: prominence and width at half prominence in FP64 with the
//      same operation order as the definition (no contraction), keep flag;
//   4. ordered compaction of kept peaks; per-series start offsets;
//   5. per model-0 peak: coincidence test against the other models' peaks.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "gwe_internal.h"

namespace gwe {
namespace {

constexpr int kBS = 256;       // samples per statistics block
constexpr int kCH = 8192;      // samples per candidate chunk
constexpr int kT = 256;        // threads per block

struct Series {
    const float *base;
    int64_t n;       // stitched length
    int W, stride;
    __device__ __forceinline__ float at(int64_t g) const {
        if (g < W) return base[g];
        const int64_t w = (g - W) / stride + 1;
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

// local maximum test at a left edge i; returns the peak index (plateau midpoint) or -1
__device__ __forceinline__ int64_t peak_at(const Series &v, int64_t i, double thr) {
    if (i < 1 || i > v.n - 2) return -1;
    const float xi = v.at(i);
    if (!(v.at(i - 1) < xi)) return -1;
    int64_t ia = i + 1;
    while (ia < v.n - 1 && v.at(ia) == xi) ++ia;
    if (!(v.at(ia) < xi)) return -1;
    if (!((double)xi >= thr)) return -1;
    return (i + (ia - 1)) / 2;
}

// 2. candidates: mode 0 counts per chunk, mode 1 writes in order
__global__ void k_cand(Geo g, double thr, int mode, int64_t *counts, const int64_t *offsets, int64_t *cand_idx,
                       int *cand_ser, int64_t nchunk) {
    __shared__ int sh[kT / 32 + 1];
    const int s = blockIdx.y;
    const int64_t c = blockIdx.x;
    const Series v = g.series(s);
    const int64_t lo = c * kCH;
    int64_t run = (mode == 1) ? offsets[(int64_t)s * nchunk + c] : 0;
    for (int it = 0; it < kCH / kT; ++it) {
        const int64_t i = lo + (int64_t)it * kT + threadIdx.x;
        const int64_t pk = (i < v.n) ? peak_at(v, i, thr) : -1;
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

// 3. prominence and width of one candidate
__global__ void k_eval(Geo g, int64_t ncand, const int64_t *cand_idx, const int *cand_ser, const float *bmax,
                       const float *bmin, const int64_t *amin_lo, const int64_t *amin_hi, double min_width,
                       int *keep, double *o_h, double *o_pr, double *o_wd) {
    const int64_t ci = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (ci >= ncand) return;
    const int s = cand_ser[ci];
    const int64_t p = cand_idx[ci];
    const Series v = g.series(s);
    const float *BX = bmax + (int64_t)s * g.nblk;
    const float *BN = bmin + (int64_t)s * g.nblk;
    const int64_t *AL = amin_lo + (int64_t)s * g.nblk;
    const int64_t *AH = amin_hi + (int64_t)s * g.nblk;
    const float xp = v.at(p);
    const int64_t pb = p / kBS;

    // left: walk down while samples <= xp, tracking the strict minimum seen first
    float lmin = xp;
    int64_t lb = p;
    {
        bool stop = false;
        for (int64_t k = p; k >= pb * kBS; --k) {
            const float x = v.at(k);
            if (x > xp) { stop = true; break; }
            if (x < lmin) { lmin = x; lb = k; }
        }
        for (int64_t B = pb - 1; !stop && B >= 0; --B) {
            if (BX[B] <= xp) {
                if (BN[B] < lmin) { lmin = BN[B]; lb = AH[B]; }
            } else {
                for (int64_t k = B * kBS + kBS - 1; k >= B * kBS; --k) {
                    const float x = v.at(k);
                    if (x > xp) { stop = true; break; }
                    if (x < lmin) { lmin = x; lb = k; }
                }
            }
        }
    }
    // right: mirrored
    float rmin = xp;
    int64_t rb = p;
    {
        bool stop = false;
        const int64_t pend = min((pb + 1) * kBS, v.n);
        for (int64_t k = p; k < pend; ++k) {
            const float x = v.at(k);
            if (x > xp) { stop = true; break; }
            if (x < rmin) { rmin = x; rb = k; }
        }
        for (int64_t B = pb + 1; !stop && B < g.nblk; ++B) {
            if (BX[B] <= xp) {
                if (BN[B] < rmin) { rmin = BN[B]; rb = AL[B]; }
            } else {
                const int64_t e = min((B + 1) * kBS, v.n);
                for (int64_t k = B * kBS; k < e; ++k) {
                    const float x = v.at(k);
                    if (x > xp) { stop = true; break; }
                    if (x < rmin) { rmin = x; rb = k; }
                }
            }
        }
    }
    const double dxp = (double)xp;
    const double base = (double)lmin > (double)rmin ? (double)lmin : (double)rmin;
    const double pr = __dsub_rn(dxp, base);
    const double h = __dsub_rn(dxp, __dmul_rn(pr, 0.5));

    // width: walk from the peak towards each base while the samples stay above h
    int64_t k = p;
    {
        // samples of p's own block first, then whole blocks whose minimum is above h
        while (lb < k && h < (double)v.at(k)) {
            if (k % kBS == 0) {
                int64_t B = k / kBS - 1;
                while (B >= 0 && B * kBS > lb && h < (double)BN[B]) --B;
                // blocks B+1 .. k/kBS-1 are entirely above h and above lb
                const int64_t nk = (B + 1) * kBS - 1;
                if (nk < k - 1) { k = nk + 1; }
            }
            --k;
        }
    }
    double lip = (double)k;
    {
        const double xk = (double)v.at(k);
        if (xk < h) lip = __dadd_rn(lip, __ddiv_rn(__dsub_rn(h, xk), __dsub_rn((double)v.at(k + 1), xk)));
    }
    k = p;
    {
        while (k < rb && h < (double)v.at(k)) {
            if (k % kBS == kBS - 1) {
                int64_t B = k / kBS + 1;
                while (B < g.nblk && (B + 1) * kBS - 1 < rb && h < (double)BN[B]) ++B;
                const int64_t nk = B * kBS;   // first sample not skipped
                if (nk > k + 1) { k = nk - 1; }
            }
            ++k;
        }
    }
    double rip = (double)k;
    {
        const double xk = (double)v.at(k);
        if (xk < h) rip = __dsub_rn(rip, __ddiv_rn(__dsub_rn(h, xk), __dsub_rn((double)v.at(k - 1), xk)));
    }
    const double wd = __dsub_rn(rip, lip);
    keep[ci] = (wd >= min_width) ? 1 : 0;
    o_h[ci] = dxp;
    o_pr[ci] = pr;
    o_wd[ci] = wd;
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

struct TrigWs {
    std::mutex mu;
    DevBuf stats_mx, stats_mn, stats_lo, stats_hi, counts, offsets, cand_idx, cand_ser, keep, h, pr, wd, sel,
        p_idx, p_ser, p_h, p_pr, p_wd, start, ens;
};
TrigWs &trig_ws() {
    static TrigWs *w = new TrigWs();   // kept until process exit
    return *w;
}

unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

namespace {

// all records of one segment's (slide, model) series, appended to recs
gwe_status triggers_collect(const float *prob, int n_models, int n_slides, int64_t nw, int64_t series_nw, int W,
                            int stride, float thr, double min_width, int64_t coinc, int flags,
                            std::vector<gwe_trigger> &recs, cudaStream_t st) {
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
    k_stats<<<blocks_for(nstat, 8), 256, 0, st>>>(g, ws.stats_mx.as<float>(), ws.stats_mn.as<float>(),
                                                   ws.stats_lo.as<int64_t>(), ws.stats_hi.as<int64_t>(), n_series);
    note_launch();
    const int64_t nchunk = (g.n + kCH - 1) / kCH;
    const int64_t ncnt = nchunk * n_series;
    GWE_CUDA_TRY(ws.counts.ensure(ncnt * sizeof(int64_t)));
    GWE_CUDA_TRY(ws.offsets.ensure((ncnt + 1) * sizeof(int64_t)));
    const double dthr = (double)thr;
    dim3 cgrid((unsigned)nchunk, (unsigned)n_series);
    k_cand<<<cgrid, kT, 0, st>>>(g, dthr, 0, ws.counts.as<int64_t>(), nullptr, nullptr, nullptr, nchunk);
    note_launch();
    k_scan<<<1, 1024, 0, st>>>(ws.counts.as<int64_t>(), ws.offsets.as<int64_t>(), ncnt);
    note_launch();
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
        k_cand<<<cgrid, kT, 0, st>>>(g, dthr, 1, nullptr, ws.offsets.as<int64_t>(), ws.cand_idx.as<int64_t>(),
                                     ws.cand_ser.as<int>(), nchunk);
        note_launch();
        k_eval<<<blocks_for(ncand, 128), 128, 0, st>>>(
            g, ncand, ws.cand_idx.as<int64_t>(), ws.cand_ser.as<int>(), ws.stats_mx.as<float>(),
            ws.stats_mn.as<float>(), ws.stats_lo.as<int64_t>(), ws.stats_hi.as<int64_t>(), min_width,
            ws.keep.as<int>(), ws.h.as<double>(), ws.pr.as<double>(), ws.wd.as<double>());
        note_launch();
        const int64_t nfc = (ncand + kCH - 1) / kCH;
        GWE_CUDA_TRY(ws.counts.ensure(nfc * sizeof(int64_t)));
        GWE_CUDA_TRY(ws.offsets.ensure((nfc + 1) * sizeof(int64_t)));
        k_flag_pass<<<(unsigned)nfc, kT, 0, st>>>(ws.keep.as<int>(), ncand, 0, ws.counts.as<int64_t>(), nullptr,
                                                  nullptr);
        note_launch();
        k_scan<<<1, 1024, 0, st>>>(ws.counts.as<int64_t>(), ws.offsets.as<int64_t>(), nfc);
        note_launch();
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
            k_flag_pass<<<(unsigned)nfc, kT, 0, st>>>(ws.keep.as<int>(), ncand, 1, nullptr, ws.offsets.as<int64_t>(),
                                                      ws.sel.as<int64_t>());
            note_launch();
            k_gather_peaks<<<blocks_for(npk, 256), 256, 0, st>>>(
                npk, ws.sel.as<int64_t>(), ws.cand_idx.as<int64_t>(), ws.cand_ser.as<int>(), ws.h.as<double>(),
                ws.pr.as<double>(), ws.wd.as<double>(), ws.p_idx.as<int64_t>(), ws.p_ser.as<int>(),
                ws.p_h.as<double>(), ws.p_pr.as<double>(), ws.p_wd.as<double>());
            note_launch();
            k_series_start<<<blocks_for(n_series + 1, 128), 128, 0, st>>>(ws.p_ser.as<int>(), npk, n_series,
                                                                         ws.start.as<int64_t>());
            note_launch();
            k_coinc<<<blocks_for(npk, 128), 128, 0, st>>>(npk, ws.p_idx.as<int64_t>(), ws.p_ser.as<int>(),
                                                          ws.start.as<int64_t>(), n_models, coinc, ws.ens.as<int>());
            note_launch();
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
