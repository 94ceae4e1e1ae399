// Streaming search over long two-detector strain (the paper's month of data,
// section "Computational Efficiency": a month of Hanford + Livingston strain
// searched by the ensemble; section "Materials and Methods", paragraph "Data
// preparation": whitening with PSDs estimated from the data).
//
// The stream is cut into chunks of `chunk_windows` windows (the core).  Each
// chunk is processed on a span that adds `margin_windows` windows of context on
// both sides (for peak finding near the core's edges) and `guard_samples` raw
// samples beyond them (for the FFT whitening): the span's raw samples are
// brought to the device (pinned host input: copied on a second stream while
// the previous chunk computes), converted to FP32, whitened on the span, run
// through the ensemble forward, and the peaks / ensemble triggers of the
// span's stitched series are kept when their index lies in the core.  The
// cores partition the stream's stitched series, so every trigger is reported
// by exactly one chunk.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <string>
#include <vector>

#include "gwe_internal.h"

namespace gwe {
namespace {

template <class T>
__global__ void k_to_f32(const T *__restrict__ in, int64_t n, float scale, float *__restrict__ out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        out[i] = (float)in[i] * scale;
}

template <>
__global__ void k_to_f32<__half>(const __half *__restrict__ in, int64_t n, float scale, float *__restrict__ out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        out[i] = __half2float(in[i]) * scale;
}

struct SearchImpl {
    gwe_model *m = nullptr;
    gwe_search_config cfg{};
    cudaStream_t copy_st = nullptr;
    cudaEvent_t copied[2] = {nullptr, nullptr}, consumed[2] = {nullptr, nullptr};
    DevBuf raw[2][2];      // [buffer][detector] raw span (host input only)
    DevBuf x[2];           // FP32 span per detector
    DevBuf xw[2];          // whitened span per detector
    DevBuf prob;           // [n_models][span windows][window]
    std::vector<gwe_trigger> recs;
    ~SearchImpl() {
        for (int b = 0; b < 2; ++b) {
            if (copied[b]) cudaEventDestroy(copied[b]);
            if (consumed[b]) cudaEventDestroy(consumed[b]);
            raw[b][0].release();
            raw[b][1].release();
            x[b].release();
            xw[b].release();
        }
        prob.release();
        if (copy_st) cudaStreamDestroy(copy_st);
    }
};

// One chunk: windows [w_a, w_b) are its core, [w_lo, w_hi) the windows it computes, raw samples
// [x_a, x_b) the span it whitens.
struct Chunk {
    int64_t w_a, w_b, w_lo, w_hi, x_a, x_b;
};

Chunk chunk_of(const gwe_search_config &c, int64_t n, int64_t nw, int64_t i) {
    Chunk k;
    k.w_a = i * c.chunk_windows;
    k.w_b = std::min(nw, k.w_a + c.chunk_windows);
    k.w_lo = std::max<int64_t>(0, k.w_a - c.margin_windows);
    k.w_hi = std::min(nw, k.w_b + c.margin_windows);
    k.x_a = std::max<int64_t>(0, k.w_lo * c.stride - c.guard_samples);
    k.x_b = std::min(n, (k.w_hi - 1) * c.stride + c.window + c.guard_samples);
    return k;
}

size_t elem_bytes(int dtype) { return dtype == GWE_INPUT_F16 ? 2 : 4; }

gwe_status convert(const void *in, int dtype, int64_t n, float scale, float *out, cudaStream_t st) {
    const unsigned grid = (unsigned)std::min<int64_t>((n + 255) / 256, 152 * 16);
    if (dtype == GWE_INPUT_F16)
        k_to_f32<__half><<<grid, 256, 0, st>>>(reinterpret_cast<const __half *>(in), n, scale, out);
    else
        k_to_f32<float><<<grid, 256, 0, st>>>(reinterpret_cast<const float *>(in), n, scale, out);
    note_launch();
    GWE_CUDA_TRY(cudaGetLastError());
    return GWE_OK;
}

gwe_status prefetch(SearchImpl &S, const Chunk &k, const void *const in[2], int b) {
    const size_t eb = elem_bytes(S.cfg.input_dtype);
    const size_t bytes = (size_t)(k.x_b - k.x_a) * eb;
    GWE_CUDA_TRY(cudaStreamWaitEvent(S.copy_st, S.consumed[b], 0));
    for (int d = 0; d < 2; ++d) {
        GWE_CUDA_TRY(S.raw[b][d].ensure(bytes));
        GWE_CUDA_TRY(cudaMemcpyAsync(S.raw[b][d].ptr, reinterpret_cast<const uint8_t *>(in[d]) + (size_t)k.x_a * eb,
                                     bytes, cudaMemcpyHostToDevice, S.copy_st));
    }
    GWE_CUDA_TRY(cudaEventRecord(S.copied[b], S.copy_st));
    return GWE_OK;
}

int64_t chunk_count(const gwe_search_config &c, int64_t n) {
    if (n < c.window) return 0;
    const int64_t nw = (n - c.window) / c.stride + 1;
    return (nw + c.chunk_windows - 1) / c.chunk_windows;
}

// chunks [c_begin, c_end) of the stream (clipped to the stream's chunks)
gwe_status run(SearchImpl &S, const void *sH, const void *sL, int64_t n, int host_input, cudaStream_t st,
               int64_t c_begin, int64_t c_end) {
    const gwe_search_config &c = S.cfg;
    const Dims &d = S.m->dims;
    S.recs.clear();
    if (n < c.window) return GWE_OK;
    const int64_t nw = (n - c.window) / c.stride + 1;
    const int64_t n_chunks = std::min<int64_t>(c_end, chunk_count(c, n));
    if (c_begin >= n_chunks) return GWE_OK;
    const int64_t n_st = (nw - 1) * c.stride + c.window;   // stitched series length
    const void *in[2] = {sH, sL};
    const size_t eb = elem_bytes(c.input_dtype);
    // a device buffer must not be overwritten by the prefetch while a previous chunk still reads it
    for (int b = 0; b < 2; ++b) GWE_CUDA_TRY(cudaEventRecord(S.consumed[b], st));
    if (host_input) {
        gwe_status r = prefetch(S, chunk_of(c, n, nw, c_begin), in, (int)(c_begin & 1));
        if (r != GWE_OK) return r;
    }
    std::vector<gwe_trigger> part;
    for (int64_t i = c_begin; i < n_chunks; ++i) {
        const Chunk k = chunk_of(c, n, nw, i);
        const int b = (int)(i & 1);
        const int64_t span = k.x_b - k.x_a;
        if (span < c.welch_seg) {
            set_error("gwe_search_run: a chunk span is shorter than the Welch segment");
            return GWE_ERR_ARG;
        }
        if (host_input && i + 1 < n_chunks) {
            gwe_status r = prefetch(S, chunk_of(c, n, nw, i + 1), in, b ^ 1);
            if (r != GWE_OK) return r;
        }
        // raw span -> FP32 -> whitened, per detector
        for (int det = 0; det < 2; ++det) {
            const void *src;
            if (host_input) {
                if (det == 0) GWE_CUDA_TRY(cudaStreamWaitEvent(st, S.copied[b], 0));
                src = S.raw[b][det].ptr;
            } else {
                src = reinterpret_cast<const uint8_t *>(in[det]) + (size_t)k.x_a * eb;
            }
            GWE_CUDA_TRY(S.x[det].ensure(sizeof(float) * span));
            GWE_CUDA_TRY(S.xw[det].ensure(sizeof(float) * span));
            gwe_status r = convert(src, c.input_dtype, span, c.input_scale, S.x[det].as<float>(), st);
            if (r != GWE_OK) return r;
        }
        if (host_input) GWE_CUDA_TRY(cudaEventRecord(S.consumed[b], st));
        for (int det = 0; det < 2; ++det) {
            gwe_status r = whiten_run(S.x[det].as<float>(), span, c.fs, c.welch_seg, whiten_defaults(),
                                          S.xw[det].as<float>(), st);
            if (r != GWE_OK) return r;
        }
        // ensemble forward over the span's windows
        const int64_t nws = k.w_hi - k.w_lo;
        const int64_t off = k.w_lo * c.stride - k.x_a;
        GWE_CUDA_TRY(S.prob.ensure(sizeof(float) * (size_t)d.n_models * nws * c.window));
        Segments sg;
        sg.s0.push_back(0);
        sg.nw.push_back(nws);
        gwe_status r;
        if (S.m->precision == GWE_FP32)
            r = fp32_forward(S.m, S.xw[0].as<float>() + off, S.xw[1].as<float>() + off, sg, c.window, c.stride,
                             nullptr, 0, S.prob.as<float>(), false, st);
        else
            r = tc_forward(S.m, S.xw[0].as<float>() + off, S.xw[1].as<float>() + off, sg, c.window, c.stride, nullptr,
                           0, S.prob.as<float>(), false, st);
        if (r != GWE_OK) return r;
        // peaks and ensemble triggers of the span's stitched series; keep the core's
        int64_t cap = std::max<int64_t>(1024, (int64_t)part.capacity()), got = 0;
        for (int attempt = 0; attempt < 2; ++attempt) {
            part.resize(cap);
            r = triggers_run(S.prob.as<float>(), d.n_models, 0, nws, c.window, c.stride, c.height_thr, c.min_width,
                             c.coinc, c.trigger_flags, part.data(), cap, &got, st);
            if (r == GWE_ERR_CAPACITY) {
                cap = got;
                continue;
            }
            break;
        }
        if (r != GWE_OK) return r;
        const int64_t core_a = k.w_a == 0 ? 0 : k.w_a * c.stride + c.window - c.stride;
        const int64_t core_b = k.w_b == nw ? n_st : k.w_b * c.stride + c.window - c.stride;
        for (int64_t j = 0; j < got; ++j) {
            gwe_trigger t = part[j];
            t.index += k.w_lo * c.stride;
            if (t.index >= core_a && t.index < core_b) S.recs.push_back(t);
        }
    }
    return GWE_OK;
}

}  // namespace
}  // namespace gwe

struct gwe_search {
    gwe::SearchImpl *impl;
};

using namespace gwe;

extern "C" gwe_status gwe_search_create(gwe_model *m, const gwe_search_config *cfg, gwe_search **out) {
    clear_error();
    GWE_ARG_CHECK(out != nullptr, "out is NULL");
    *out = nullptr;
    GWE_ARG_CHECK(m != nullptr && cfg != nullptr, "NULL argument");
    const gwe_search_config &c = *cfg;
    GWE_ARG_CHECK(c.window > 0 && c.stride > 0 && c.stride <= c.window, "bad window/stride");
    GWE_ARG_CHECK(c.chunk_windows > 0 && c.margin_windows >= 0 && c.guard_samples >= 0, "bad chunking");
    GWE_ARG_CHECK(c.fs > 0.0, "fs must be positive");
    GWE_ARG_CHECK(c.welch_seg >= 16 && (c.welch_seg & (c.welch_seg - 1)) == 0, "welch_seg must be a power of two >= 16");
    GWE_ARG_CHECK(c.input_dtype == GWE_INPUT_F32 || c.input_dtype == GWE_INPUT_F16, "unknown input_dtype");
    GWE_ARG_CHECK(c.coinc >= 0, "coinc must be >= 0");
    gwe::SearchImpl *S = new gwe::SearchImpl();
    S->m = m;
    S->cfg = c;
    cudaError_t e = cudaStreamCreateWithFlags(&S->copy_st, cudaStreamNonBlocking);
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
        e = cudaEventCreateWithFlags(&S->copied[b], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S->consumed[b], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        delete S;
        set_error(std::string("gwe_search_create: ") + cudaGetErrorString(e));
        return GWE_ERR_CUDA;
    }
    *out = new gwe_search{S};
    return GWE_OK;
}

extern "C" gwe_status gwe_search_run(gwe_search *s, const void *strain_H, const void *strain_L, int64_t n_samples,
                                     int host_input, gwe_trigger *out, int64_t cap, int64_t *n_out, void *stream) {
    clear_error();
    GWE_ARG_CHECK(s != nullptr && s->impl != nullptr, "search is NULL");
    GWE_ARG_CHECK(strain_H != nullptr && strain_L != nullptr && n_out != nullptr, "NULL argument");
    GWE_ARG_CHECK(n_samples >= 0 && (host_input == 0 || host_input == 1), "bad n_samples or host_input");
    GWE_ARG_CHECK(cap >= 0 && (cap == 0 || out != nullptr), "out is NULL with cap > 0");
    *n_out = 0;
    gwe::SearchImpl &S = *s->impl;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    gwe_status r = gwe::run(S, strain_H, strain_L, n_samples, host_input, st, 0, INT64_MAX);
    // leave no copy in flight on the private stream, whatever happened
    cudaStreamSynchronize(S.copy_st);
    if (r != GWE_OK) return r;
    *n_out = (int64_t)S.recs.size();
    const int64_t k = std::min<int64_t>(cap, *n_out);
    if (k > 0) std::copy(S.recs.begin(), S.recs.begin() + k, out);
    if (*n_out > cap) {
        set_error("gwe_search_run: output capacity too small");
        return GWE_ERR_CAPACITY;
    }
    return GWE_OK;
}

extern "C" int64_t gwe_search_chunks(const gwe_search *s, int64_t n_samples) {
    if (!s || !s->impl || n_samples < 0) return 0;
    return gwe::chunk_count(s->impl->cfg, n_samples);
}

extern "C" gwe_status gwe_search_run_range(gwe_search *s, const void *strain_H, const void *strain_L,
                                           int64_t n_samples, int host_input, int64_t chunk_begin, int64_t chunk_end,
                                           gwe_trigger *out, int64_t cap, int64_t *n_out, void *stream) {
    clear_error();
    GWE_ARG_CHECK(s != nullptr && s->impl != nullptr, "search is NULL");
    GWE_ARG_CHECK(strain_H != nullptr && strain_L != nullptr && n_out != nullptr, "NULL argument");
    GWE_ARG_CHECK(n_samples >= 0 && (host_input == 0 || host_input == 1), "bad n_samples or host_input");
    GWE_ARG_CHECK(chunk_begin >= 0 && chunk_end >= chunk_begin, "bad chunk range");
    GWE_ARG_CHECK(cap >= 0 && (cap == 0 || out != nullptr), "out is NULL with cap > 0");
    *n_out = 0;
    gwe::SearchImpl &S = *s->impl;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    gwe_status r = gwe::run(S, strain_H, strain_L, n_samples, host_input, st, chunk_begin, chunk_end);
    cudaStreamSynchronize(S.copy_st);
    if (r != GWE_OK) return r;
    *n_out = (int64_t)S.recs.size();
    const int64_t k = std::min<int64_t>(cap, *n_out);
    if (k > 0) std::copy(S.recs.begin(), S.recs.begin() + k, out);
    if (*n_out > cap) {
        set_error("gwe_search_run_range: output capacity too small");
        return GWE_ERR_CAPACITY;
    }
    return GWE_OK;
}

extern "C" void gwe_search_destroy(gwe_search *s) {
    if (!s) return;
    delete s->impl;
    delete s;
}
