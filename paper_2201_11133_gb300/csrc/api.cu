// C-ABI entry points of libgwe (declared in include/gwe.h): argument checks,
// model handles and dispatch to the precision-specific paths.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "gwe_internal.h"

namespace gwe {

static thread_local std::string g_err;

void set_error(const std::string &msg) { g_err = msg; }
void clear_error() { g_err.clear(); }

cudaError_t DevBuf::ensure(size_t want) {
    if (want <= bytes && ptr) return cudaSuccess;
    release();
    size_t sz = want < 256 ? 256 : want;
    cudaError_t e = cudaMalloc(&ptr, sz);
    if (e != cudaSuccess) {
        ptr = nullptr;
        bytes = 0;
        return e;
    }
    bytes = sz;
    return cudaSuccess;
}

void DevBuf::release() {
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    bytes = 0;
}

bool make_dims(const gwe_model_config *c, Dims *d) {
    if (!c) return false;
    if (c->n_models <= 0 || c->stacks <= 0 || c->layers_per_stack <= 0 || c->layers_per_stack > 24 ||
        c->kernel <= 0 || c->r_ch <= 0 || c->s_ch <= 0 || c->head_ch <= 0)
        return false;
    d->n_models = c->n_models;
    d->stacks = c->stacks;
    d->lps = c->layers_per_stack;
    d->k = c->kernel;
    d->R = c->r_ch;
    d->S = c->s_ch;
    d->Hc = c->head_ch;
    d->L = c->stacks * c->layers_per_stack;
    d->Pl = (int64_t)2 * d->R * d->k * d->R + 2 * d->R + (int64_t)d->R * d->R + d->R + (int64_t)d->S * d->R + d->S;
    d->Pb = 2 * d->R + (int64_t)d->L * d->Pl;
    d->head_off = 2 * d->Pb;
    d->P = d->head_off + (int64_t)d->Hc * 2 * d->S + 2 * d->Hc + 1;
    return true;
}

static cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

static gwe_status check_device() {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        set_error(std::string("no usable CUDA device: ") + cudaGetErrorString(e));
        return GWE_ERR_CUDA;
    }
    int major = 0, minor = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    if (major != 10 || minor != 3) {
        set_error("libgwe is built for sm_103a (GB300); current device is sm_" + std::to_string(major * 10 + minor));
        return GWE_ERR_CUDA;
    }
    return GWE_OK;
}

}  // namespace gwe

using namespace gwe;

extern "C" {

const char *gwe_last_error(void) { return g_err.c_str(); }

const char *gwe_version(void) { return "gwe 0.1 (sm_103a)"; }

int64_t gwe_param_count(const gwe_model_config *cfg) {
    Dims d;
    if (!make_dims(cfg, &d)) return -1;
    return d.P;
}

int64_t gwe_n_windows(int64_t n, int window, int stride) {
    if (window <= 0 || stride <= 0 || n < window) return 0;
    return (n - window) / stride + 1;
}

}  // extern "C"

namespace gwe {
namespace {

// Philox4x64-10 (Salmon, Moraes, Dror and Shaw, "Parallel random numbers: as easy as 1, 2, 3",
// SC 2011): ten rounds of two 64 x 64 -> 128-bit products with the published multipliers and
// Weyl key increments.  Host code only (weight initialisation).
void philox4x64_10(const uint64_t ctr_in[4], const uint64_t key_in[2], uint64_t out[4]) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
    uint64_t x0 = ctr_in[0], x1 = ctr_in[1], x2 = ctr_in[2], x3 = ctr_in[3];
    uint64_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        const unsigned __int128 p0 = (unsigned __int128)M0 * x0, p1 = (unsigned __int128)M1 * x2;
        const uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        const uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        const uint64_t y0 = hi1 ^ x1 ^ k0, y2 = hi0 ^ x3 ^ k1;
        x0 = y0;
        x1 = lo1;
        x2 = y2;
        x3 = lo0;
        k0 += W0;
        k1 += W1;
    }
    out[0] = x0;
    out[1] = x1;
    out[2] = x2;
    out[3] = x3;
}

// Standard normal number e of the stream (seed, model): block e / 2 of Philox4x64-10 with counter
// (e / 2, 0, 0, 0) and key (seed, model); words 2j, 2j + 1 (j = e mod 2) give u1 in (0, 1] and
// u2 in [0, 1) (53 bits each) and the Box-Muller cosine branch sqrt(-2 ln u1) cos(2 pi u2).
double philox_normal(uint64_t seed, uint64_t model, uint64_t e) {
    const uint64_t ctr[4] = {e >> 1, 0, 0, 0}, key[2] = {seed, model};
    uint64_t r[4];
    philox4x64_10(ctr, key, r);
    const int j = (int)(e & 1);
    const double u1 = (double)((r[2 * j] >> 11) + 1) * 0x1.0p-53;
    const double u2 = (double)(r[2 * j + 1] >> 11) * 0x1.0p-53;
    return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586476925286766559 * u2);
}

}  // namespace
}  // namespace gwe

extern "C" {

void gwe_philox4x64_10(const uint64_t *counter, const uint64_t *key, uint64_t *out) {
    philox4x64_10(counter, key, out);
}

gwe_status gwe_init_weights(const gwe_model_config *cfg, uint64_t seed, float *host_out) {
    clear_error();
    Dims d;
    GWE_ARG_CHECK(make_dims(cfg, &d), "invalid configuration");
    GWE_ARG_CHECK(host_out != nullptr, "host_out is NULL");
    // fan-in per weight tensor: inputs x kernel taps of the layer it feeds
    for (int mi = 0; mi < d.n_models; ++mi) {
        float *w = host_out + (int64_t)mi * d.P;
        std::fill(w, w + d.P, 0.f);
        auto fill = [&](int64_t off, int64_t n, int fan_in) {
            const double sc = 1.0 / std::sqrt((double)fan_in);
            for (int64_t e = off; e < off + n; ++e) w[e] = (float)(philox_normal(seed, (uint64_t)mi, (uint64_t)e) * sc);
        };
        for (int b = 0; b < 2; ++b) {
            fill(off_branch(d, b), d.R, 1);                                   // w_in (1 channel, 1 tap)
            for (int l = 0; l < d.L; ++l) {
                fill(off_wconv(d, b, l), (int64_t)2 * d.R * d.k * d.R, d.R * d.k);
                fill(off_wres(d, b, l), (int64_t)d.R * d.R, d.R);
                fill(off_wskip(d, b, l), (int64_t)d.S * d.R, d.R);
            }
        }
        fill(off_wh1(d), (int64_t)d.Hc * 2 * d.S, 2 * d.S);
        fill(off_wh2(d), d.Hc, d.Hc);
    }
    return GWE_OK;
}

gwe_status gwe_model_init_random(const gwe_model_config *cfg, uint64_t seed, int precision, gwe_model **out) {
    clear_error();
    GWE_ARG_CHECK(out != nullptr, "out is NULL");
    *out = nullptr;
    Dims d;
    GWE_ARG_CHECK(make_dims(cfg, &d), "invalid configuration");
    std::vector<float> hb;
    try {
        hb.resize((size_t)d.P * d.n_models);
    } catch (...) {
        set_error("host allocation failed");
        return GWE_ERR_OOM;
    }
    gwe_status st = gwe_init_weights(cfg, seed, hb.data());
    if (st != GWE_OK) return st;
    return gwe_model_create(cfg, hb.data(), precision, out);
}

gwe_status gwe_model_create(const gwe_model_config *cfg, const float *host_weights, int precision,
                            gwe_model **out) {
    clear_error();
    GWE_ARG_CHECK(out != nullptr, "out is NULL");
    *out = nullptr;
    Dims d;
    GWE_ARG_CHECK(make_dims(cfg, &d), "invalid configuration");
    GWE_ARG_CHECK(host_weights != nullptr, "host_weights is NULL");
    GWE_ARG_CHECK(precision == GWE_FP32 || precision == GWE_BF16 || precision == GWE_FP8, "unknown precision");
    if (d.k != 2) {
        set_error("only kernel size 2 is implemented");
        return GWE_ERR_UNSUPPORTED;
    }
    gwe_status st = check_device();
    if (st != GWE_OK) return st;
    gwe_model *m = new (std::nothrow) gwe_model();
    if (!m) {
        set_error("host allocation failed");
        return GWE_ERR_OOM;
    }
    m->cfg = *cfg;
    m->dims = d;
    m->precision = precision;
    cudaGetDevice(&m->device);
    st = gwe_model_set_weights(m, host_weights);
    if (st != GWE_OK) {
        gwe_model_destroy(m);
        return st;
    }
    *out = m;
    return GWE_OK;
}

gwe_status gwe_model_set_weights(gwe_model *m, const float *hb) {
    clear_error();
    GWE_ARG_CHECK(m != nullptr && hb != nullptr, "NULL argument");
    const size_t bytes = (size_t)m->dims.P * m->dims.n_models * sizeof(float);
    GWE_CUDA_TRY(m->w32.ensure(bytes));
    GWE_CUDA_TRY(cudaMemcpy(m->w32.ptr, hb, bytes, cudaMemcpyHostToDevice));
    ++m->wstamp;
    gwe_status st = fp32_prepare(m, hb);
    if (st != GWE_OK && m->precision == GWE_FP32) return st;
    if (m->precision == GWE_BF16 || m->precision == GWE_FP8) {
        if (st != GWE_OK) return st;   // the FP8 calibration runs on the FP32 path
        st = tc_prepare(m, hb, m->precision == GWE_FP8);
        if (st != GWE_OK) return st;
    }
    return GWE_OK;
}

gwe_status gwe_model_set_weights_device(gwe_model *m, const float *dev_weights, void *stream) {
    clear_error();
    GWE_ARG_CHECK(m != nullptr && dev_weights != nullptr, "NULL argument");
    cudaStream_t st = as_stream(stream);
    const size_t bytes = (size_t)m->dims.P * m->dims.n_models * sizeof(float);
    if (dev_weights != m->w32.as<float>())
        GWE_CUDA_TRY(cudaMemcpyAsync(m->w32.ptr, dev_weights, bytes, cudaMemcpyDeviceToDevice, st));
    ++m->wstamp;
    gwe_status r = fp32_repack_device(m, st);
    if (r != GWE_OK) return r;
    if (m->precision == GWE_BF16 || m->precision == GWE_FP8) return tc_rebuild_from_device(m, st);
    return GWE_OK;
}

gwe_status gwe_model_calibrate(gwe_model *m, const float *sH, const float *sL, int64_t n, int window, int stride,
                               void *stream) {
    clear_error();
    GWE_ARG_CHECK(m != nullptr, "model is NULL");
    GWE_ARG_CHECK(sH != nullptr && sL != nullptr, "NULL buffer");
    GWE_ARG_CHECK(window > 0 && stride > 0 && stride <= window, "bad window/stride");
    GWE_ARG_CHECK(n >= window, "n_samples < window");
    if (m->precision != GWE_FP8) {
        set_error("gwe_model_calibrate: only FP8 handles take activation scales");
        return GWE_ERR_UNSUPPORTED;
    }
    return tc_calibrate(m, sH, sL, n, window, stride, as_stream(stream));
}

gwe_status gwe_model_set_fp8_amax(gwe_model *m, const float *amax) {
    clear_error();
    GWE_ARG_CHECK(m != nullptr && amax != nullptr, "NULL argument");
    if (m->precision != GWE_FP8) {
        set_error("gwe_model_set_fp8_amax: not an FP8 handle");
        return GWE_ERR_UNSUPPORTED;
    }
    const int64_t n = (int64_t)m->dims.n_models * 2 * m->dims.L * m->dims.R;
    for (int64_t i = 0; i < n; ++i)
        GWE_ARG_CHECK(std::isfinite(amax[i]) && amax[i] >= 0.f, "amax entries must be finite and >= 0");
    return tc_set_amax(m, amax);
}

gwe_status gwe_model_set_f16_layers(gwe_model *m, int n) {
    clear_error();
    GWE_ARG_CHECK(m != nullptr, "model is NULL");
    if (m->precision != GWE_BF16) {
        set_error("gwe_model_set_f16_layers: not a GWE_BF16 handle");
        return GWE_ERR_UNSUPPORTED;
    }
    return tc_set_f16_layers(m, n);
}

int gwe_model_f16_layers(const gwe_model *m) {
    if (!m || m->precision != GWE_BF16) return 0;
    return tc_f16_layers(const_cast<gwe_model *>(m));
}

gwe_status gwe_model_get_fp8_amax(gwe_model *m, float *amax) {
    clear_error();
    GWE_ARG_CHECK(m != nullptr && amax != nullptr, "NULL argument");
    if (m->precision != GWE_FP8) {
        set_error("gwe_model_get_fp8_amax: not an FP8 handle");
        return GWE_ERR_UNSUPPORTED;
    }
    return tc_get_amax(m, amax);
}

void gwe_model_destroy(gwe_model *m) {
    if (!m) return;
    tc_release(m);
    fp32_backward_release(m);
    tc_backward_release(m->bwd_tc);
    m->w32.release();
    m->f32.buf.release();
    m->ws.x0.release();
    m->ws.x1.release();
    m->ws.skip.release();
    m->ws.proj.release();
    m->ws.logit.release();
    m->ws.aux.release();
    delete m;
}

static gwe_status dispatch_forward(gwe_model *m, const float *sH, const float *sL, const Segments &sg, int window,
                                   int stride, const int32_t *slides, int n_slides, float *out, bool logits,
                                   cudaStream_t st) {
    if (m->precision == GWE_FP32) return fp32_forward(m, sH, sL, sg, window, stride, slides, n_slides, out, logits, st);
    return tc_forward(m, sH, sL, sg, window, stride, slides, n_slides, out, logits, st);
}

static Segments one_segment(int64_t nw) {
    Segments sg;
    sg.s0.push_back(0);
    sg.nw.push_back(nw);
    return sg;
}

gwe_status gwe_forward(gwe_model *m, const float *sH, const float *sL, int64_t n, int window, int stride,
                       const int32_t *slides, int n_slides, float *out_prob, void *stream) {
    clear_error();
    GWE_ARG_CHECK(m != nullptr, "model is NULL");
    GWE_ARG_CHECK(sH != nullptr && sL != nullptr && out_prob != nullptr, "NULL buffer");
    GWE_ARG_CHECK(window > 0 && stride > 0, "window and stride must be positive");
    GWE_ARG_CHECK(stride <= window, "stride must not exceed window");
    GWE_ARG_CHECK(n >= window, "n_samples < window");
    GWE_ARG_CHECK(n_slides >= 0 && (n_slides == 0 || slides != nullptr), "slides is NULL with n_slides > 0");
    const int64_t nw = gwe_n_windows(n, window, stride);
    return dispatch_forward(m, sH, sL, one_segment(nw), window, stride, slides, n_slides, out_prob, false,
                            as_stream(stream));
}

gwe_status gwe_forward_segments(gwe_model *m, const float *sH, const float *sL, const int64_t *seg_start,
                                const int64_t *seg_len, int n_segments, int window, int stride, const int32_t *slides,
                                int n_slides, float *out_prob, void *stream) {
    clear_error();
    GWE_ARG_CHECK(m != nullptr, "model is NULL");
    GWE_ARG_CHECK(sH != nullptr && sL != nullptr && out_prob != nullptr, "NULL buffer");
    GWE_ARG_CHECK(seg_start != nullptr && seg_len != nullptr && n_segments > 0, "no segments");
    GWE_ARG_CHECK(window > 0 && stride > 0, "window and stride must be positive");
    GWE_ARG_CHECK(stride <= window, "stride must not exceed window");
    GWE_ARG_CHECK(n_slides >= 0 && (n_slides == 0 || slides != nullptr), "slides is NULL with n_slides > 0");
    Segments sg;
    for (int g = 0; g < n_segments; ++g) {
        GWE_ARG_CHECK(seg_start[g] >= 0 && seg_len[g] >= 0, "negative segment start or length");
        sg.s0.push_back(seg_start[g]);
        sg.nw.push_back(gwe_n_windows(seg_len[g], window, stride));
    }
    if (sg.total_windows() == 0) return GWE_OK;
    return dispatch_forward(m, sH, sL, sg, window, stride, slides, n_slides, out_prob, false, as_stream(stream));
}

gwe_status gwe_forward_logits(gwe_model *m, const float *xH, const float *xL, int batch, int window,
                              float *out_logit, void *stream) {
    clear_error();
    GWE_ARG_CHECK(m != nullptr, "model is NULL");
    GWE_ARG_CHECK(xH != nullptr && xL != nullptr && out_logit != nullptr, "NULL buffer");
    GWE_ARG_CHECK(batch > 0 && window > 0, "batch and window must be positive");
    return dispatch_forward(m, xH, xL, one_segment(batch), window, window, nullptr, 0, out_logit, true,
                            as_stream(stream));
}

gwe_status gwe_backward(gwe_model *m, int model_index, const float *xH, const float *xL, int batch, int window,
                        const float *dlogit, float *grad_w, float *grad_H, float *grad_L, void *stream) {
    clear_error();
    GWE_ARG_CHECK(m != nullptr, "model is NULL");
    GWE_ARG_CHECK(model_index >= 0 && model_index < m->dims.n_models, "model_index out of range");
    GWE_ARG_CHECK(xH != nullptr && xL != nullptr && dlogit != nullptr && grad_w != nullptr, "NULL buffer");
    GWE_ARG_CHECK(batch > 0 && window > 0, "batch and window must be positive");
    GWE_ARG_CHECK((int64_t)batch * window < ((int64_t)1 << 31), "batch * window too large");
    if (m->precision != GWE_FP32 && tc_backward_supported(m->dims)) {
        int sms = 0;
        GWE_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, m->device));
        return tc_backward(m, m->bwd_tc, model_index, xH, xL, batch, window, dlogit, grad_w, grad_H, grad_L, sms,
                           as_stream(stream));
    }
    return fp32_backward(m, model_index, xH, xL, batch, window, dlogit, grad_w, grad_H, grad_L, as_stream(stream));
}

gwe_status gwe_triggers(const float *prob, int n_models, int n_slides, int64_t n_windows, int window, int stride,
                        float height_thr, double min_width, int64_t coinc, int flags, gwe_trigger *out, int64_t cap,
                        int64_t *n_out, void *stream) {
    clear_error();
    GWE_ARG_CHECK(prob != nullptr && n_out != nullptr, "NULL argument");
    GWE_ARG_CHECK(n_models > 0 && n_slides >= 0 && n_windows >= 0, "bad counts");
    GWE_ARG_CHECK(window > 0 && stride > 0 && stride <= window, "bad window/stride");
    GWE_ARG_CHECK(coinc >= 0, "coinc must be >= 0");
    GWE_ARG_CHECK(cap >= 0 && (cap == 0 || out != nullptr), "out is NULL with cap > 0");
    return triggers_run(prob, n_models, n_slides, n_windows, window, stride, height_thr, min_width, coinc, flags, out,
                        cap, n_out, as_stream(stream));
}

gwe_status gwe_triggers_segments(const float *prob, int n_models, int n_slides, const int64_t *seg_len,
                                 int n_segments, int window, int stride, float height_thr, double min_width,
                                 int64_t coinc, int flags, gwe_trigger *out, int32_t *out_segment, int64_t cap,
                                 int64_t *n_out, void *stream) {
    clear_error();
    GWE_ARG_CHECK(prob != nullptr && n_out != nullptr && seg_len != nullptr, "NULL argument");
    GWE_ARG_CHECK(n_models > 0 && n_slides >= 0 && n_segments > 0, "bad counts");
    GWE_ARG_CHECK(window > 0 && stride > 0 && stride <= window, "bad window/stride");
    GWE_ARG_CHECK(coinc >= 0, "coinc must be >= 0");
    GWE_ARG_CHECK(cap >= 0 && (cap == 0 || out != nullptr), "out is NULL with cap > 0");
    std::vector<int64_t> nw(n_segments);
    for (int g = 0; g < n_segments; ++g) {
        GWE_ARG_CHECK(seg_len[g] >= 0, "negative segment length");
        nw[g] = gwe_n_windows(seg_len[g], window, stride);
    }
    return triggers_run_segments(prob, n_models, n_slides, nw.data(), n_segments, window, stride, height_thr,
                                 min_width, coinc, flags, out, out_segment, cap, n_out, as_stream(stream));
}

static gwe_status check_sweep(const float *thr, int n_thr, int64_t *ens_counts) {
    GWE_ARG_CHECK(thr != nullptr && n_thr > 0, "no thresholds");
    GWE_ARG_CHECK(ens_counts != nullptr, "ens_counts is NULL");
    for (int k = 0; k < n_thr; ++k) {
        GWE_ARG_CHECK(std::isfinite(thr[k]), "thresholds must be finite");
        GWE_ARG_CHECK(k == 0 || thr[k] >= thr[k - 1], "thresholds must be in ascending order");
    }
    return GWE_OK;
}

gwe_status gwe_trigger_sweep(const float *prob, int n_models, int n_slides, int64_t n_windows, int window,
                             int stride, const float *thresholds, int n_thr, double min_width, int64_t coinc,
                             int64_t *ens_counts, int64_t *model_counts, void *stream) {
    clear_error();
    GWE_ARG_CHECK(prob != nullptr, "prob is NULL");
    GWE_ARG_CHECK(n_models > 0 && n_slides >= 0 && n_windows >= 0, "bad counts");
    GWE_ARG_CHECK(window > 0 && stride > 0 && stride <= window, "bad window/stride");
    GWE_ARG_CHECK(coinc >= 0, "coinc must be >= 0");
    gwe_status r = check_sweep(thresholds, n_thr, ens_counts);
    if (r != GWE_OK) return r;
    return triggers_sweep(prob, n_models, n_slides, &n_windows, 1, window, stride, thresholds, n_thr, min_width, coinc,
                          ens_counts, model_counts, as_stream(stream));
}

gwe_status gwe_trigger_sweep_segments(const float *prob, int n_models, int n_slides, const int64_t *seg_len,
                                      int n_segments, int window, int stride, const float *thresholds, int n_thr,
                                      double min_width, int64_t coinc, int64_t *ens_counts, int64_t *model_counts,
                                      void *stream) {
    clear_error();
    GWE_ARG_CHECK(prob != nullptr && seg_len != nullptr, "NULL argument");
    GWE_ARG_CHECK(n_models > 0 && n_slides >= 0 && n_segments > 0, "bad counts");
    GWE_ARG_CHECK(window > 0 && stride > 0 && stride <= window, "bad window/stride");
    GWE_ARG_CHECK(coinc >= 0, "coinc must be >= 0");
    gwe_status r = check_sweep(thresholds, n_thr, ens_counts);
    if (r != GWE_OK) return r;
    std::vector<int64_t> nw(n_segments);
    for (int g = 0; g < n_segments; ++g) {
        GWE_ARG_CHECK(seg_len[g] >= 0, "negative segment length");
        nw[g] = gwe_n_windows(seg_len[g], window, stride);
    }
    return triggers_sweep(prob, n_models, n_slides, nw.data(), n_segments, window, stride, thresholds, n_thr,
                          min_width, coinc, ens_counts, model_counts, as_stream(stream));
}

gwe_status gwe_sync(gwe_model *m, void *stream) {
    clear_error();
    GWE_ARG_CHECK(m != nullptr, "model is NULL");
    cudaStream_t st = as_stream(stream);
    GWE_CUDA_TRY(cudaStreamSynchronize(st));
    GWE_CUDA_TRY(cudaGetLastError());
    if (m->precision != GWE_FP32) return tc_check(m, st);
    return GWE_OK;
}

gwe_status gwe_set_cross_window_reuse(int enable) {
    clear_error();
    GWE_ARG_CHECK(enable == 0 || enable == 1, "enable must be 0 or 1");
    set_cross_window_reuse(enable);
    return GWE_OK;
}

gwe_status gwe_debug_config(int drop, double wait_seconds) {
    clear_error();
    return debug_config(drop, wait_seconds);
}

gwe_status gwe_debug_ring_margin(int64_t bytes) {
    clear_error();
    return debug_ring_margin(bytes);
}

gwe_status gwe_whiten_ex(const float *strain, int64_t n, double fs, int seg_len, const gwe_whiten_options *opt,
                         float *out, void *stream) {
    clear_error();
    GWE_ARG_CHECK(strain != nullptr && out != nullptr && opt != nullptr, "NULL argument");
    GWE_ARG_CHECK(out != strain, "out must not alias strain");
    GWE_ARG_CHECK(fs > 0.0, "fs must be positive");
    GWE_ARG_CHECK(seg_len >= 16 && (seg_len & (seg_len - 1)) == 0, "seg_len must be a power of two >= 16");
    GWE_ARG_CHECK(n >= seg_len, "n_samples < seg_len");
    GWE_ARG_CHECK(opt->psd_average == GWE_PSD_MEAN || opt->psd_average == GWE_PSD_MEDIAN, "unknown psd_average");
    GWE_ARG_CHECK(opt->tukey_alpha >= 0.0 && opt->tukey_alpha <= 1.0, "tukey_alpha must lie in [0, 1]");
    GWE_ARG_CHECK(opt->f_low >= 0.0 && opt->f_low < fs / 2.0, "f_low must lie in [0, fs / 2)");
    return whiten_run(strain, n, fs, seg_len, *opt, out, as_stream(stream));
}

gwe_status gwe_whiten(const float *strain, int64_t n, double fs, int seg_len, int flags, float *out, void *stream) {
    clear_error();
    GWE_ARG_CHECK(flags == 0 || flags == GWE_PSD_MEDIAN, "flags must be 0 or GWE_PSD_MEDIAN");
    gwe_whiten_options o = whiten_defaults();
    o.psd_average = flags;
    return gwe_whiten_ex(strain, n, fs, seg_len, &o, out, stream);
}

}  // extern "C"
