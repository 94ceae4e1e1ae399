// Internal declarations of libgwe (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/gwe.h"

namespace gwe {

// Thread-local error reporting.
void set_error(const std::string &msg);
void clear_error();

#define GWE_CUDA_TRY(expr)                                                                    \
    do {                                                                                      \
        cudaError_t _e = (expr);                                                              \
        if (_e != cudaSuccess) {                                                              \
            ::gwe::set_error(std::string(#expr) + ": " + cudaGetErrorString(_e));             \
            return (_e == cudaErrorMemoryAllocation) ? GWE_ERR_OOM : GWE_ERR_CUDA;            \
        }                                                                                     \
    } while (0)

#define GWE_ARG_CHECK(cond, msg)                                                              \
    do {                                                                                      \
        if (!(cond)) {                                                                        \
            ::gwe::set_error(std::string("argument error: ") + (msg));                        \
            return GWE_ERR_ARG;                                                               \
        }                                                                                     \
    } while (0)

// Sizes derived from a configuration.
struct Dims {
    int n_models, stacks, lps, k, R, S, Hc, L;
    int64_t P;    // parameters per model
    int64_t Pb;   // per branch
    int64_t Pl;   // per layer
    int64_t head_off;  // offset of w_h1 in a model blob
};
bool make_dims(const gwe_model_config *cfg, Dims *d);

// Offsets (in floats) inside one model's FP32 blob.
inline int64_t off_branch(const Dims &d, int b) { return (int64_t)b * d.Pb; }
inline int64_t off_layer(const Dims &d, int b, int l) { return off_branch(d, b) + 2 * d.R + (int64_t)l * d.Pl; }
inline int64_t off_wconv(const Dims &d, int b, int l) { return off_layer(d, b, l); }
inline int64_t off_bconv(const Dims &d, int b, int l) { return off_wconv(d, b, l) + (int64_t)2 * d.R * d.k * d.R; }
inline int64_t off_wres(const Dims &d, int b, int l) { return off_bconv(d, b, l) + 2 * d.R; }
inline int64_t off_bres(const Dims &d, int b, int l) { return off_wres(d, b, l) + (int64_t)d.R * d.R; }
inline int64_t off_wskip(const Dims &d, int b, int l) { return off_bres(d, b, l) + d.R; }
inline int64_t off_bskip(const Dims &d, int b, int l) { return off_wskip(d, b, l) + (int64_t)d.S * d.R; }
inline int64_t off_wh1(const Dims &d) { return d.head_off; }
inline int64_t off_bh1(const Dims &d) { return d.head_off + (int64_t)d.Hc * 2 * d.S; }
inline int64_t off_wh2(const Dims &d) { return off_bh1(d) + d.Hc; }
inline int64_t off_bh2(const Dims &d) { return off_wh2(d) + d.Hc; }

// Records CUDA events around one launch when profiling is enabled
// (gwe_profile_enable); a no-op otherwise.
struct ProfScope {
    int slot;
    cudaStream_t st;
    ProfScope(const char *name, cudaStream_t s);
    ~ProfScope();
};

// While alive, ProfScope records nothing on this thread (used around stream captures, where an
// event record would become part of the captured graph).
struct ProfSuspend {
    ProfSuspend();
    ~ProfSuspend();
};

// Counts the library's kernel launches (read with gwe_launch_count).
void note_launch(int n = 1);

// Grow-only device buffer.
struct DevBuf {
    void *ptr = nullptr;
    size_t bytes = 0;
    cudaError_t ensure(size_t want);
    void release();
    template <class T> T *as() const { return reinterpret_cast<T *>(ptr); }
};

// FP32 path: per model, per branch, per layer weights re-laid out for the
// SIMT kernels (transposed so that output channels are contiguous).
//   conv   [2R (k: lagged inputs then current inputs)][2R (out)]
//   rs     [R (k)][R + S (out: residual then skip)]
//   bias   b_conv[2R], b_res[R], b_skip[S]
// head, per branch X: w1t [S (k)][Hc (out)] = W_h1[:, X*S + k]^T.
struct Fp32Weights {
    DevBuf buf;
    int64_t layer_stride = 0;   // floats per (branch, layer) block
    int64_t conv_off = 0, rs_off = 0, bconv_off = 0, bres_off = 0, bskip_off = 0;
    int64_t model_stride = 0;   // floats per model
    int64_t win_off = 0;        // w_in[2][R], b_in[2][R] per model
    int64_t head_off = 0;       // w1t[2][S][Hc], b1[Hc], w2[Hc], b2[1] per model
};

struct Workspace {
    DevBuf x0, x1, skip, proj, logit;
    DevBuf aux;
};

}  // namespace gwe

struct gwe_model {
    gwe_model_config cfg;
    gwe::Dims dims;
    int precision = GWE_FP32;
    int device = 0;
    gwe::DevBuf w32;              // FP32 blob [n_models][P] as given
    gwe::Fp32Weights f32;         // FP32 kernel layout
    void *tc = nullptr;           // tensor-core path state (opaque, branch_tc.cu)
    void *bwd = nullptr;          // backward workspace (opaque, fp32_path.cu)
    void *bwd_tc = nullptr;       // tensor-core backward state (opaque, bwd_tc.cu)
    uint64_t wstamp = 0;          // incremented whenever the weights change
    gwe::Workspace ws;
};

namespace gwe {

// Science segments of one forward call: segment g starts at sample s0[g] of the strain arrays and
// holds nw[g] windows; the outputs of its windows follow those of segments 0 .. g-1.
struct Segments {
    std::vector<int64_t> s0, nw;
    int64_t total_windows() const {
        int64_t t = 0;
        for (int64_t v : nw) t += v;
        return t;
    }
};

// fp32_path.cu
gwe_status fp32_prepare(gwe_model *m, const float *host_blob);
// the FP32 kernel layout from the device FP32 blobs m->w32 (asynchronous on st; fp32_prepare must
// have run once for the handle)
gwe_status fp32_repack_device(gwe_model *m, cudaStream_t st);
// bwd_tc.cu: backward of one member with BF16 tensor-core GEMMs (FP32 accumulation)
bool tc_backward_supported(const Dims &d);
gwe_status tc_backward(gwe_model *m, void *&state, int model_index, const float *xH, const float *xL, int batch,
                       int W, const float *dlogit, float *grad_w, float *grad_H, float *grad_L, int sms,
                       cudaStream_t st);
void tc_backward_release(void *&state);
// Forward of all models over one segment; writes probabilities (or logits).
gwe_status fp32_forward(gwe_model *m, const float *sH, const float *sL, const Segments &sg, int window,
                        int stride, const int32_t *slides, int n_slides, float *out, bool logits, cudaStream_t st);

// Backward pass of one ensemble member (FP32, per-stack recomputation); grad_w is overwritten.
gwe_status fp32_backward(gwe_model *m, int model_index, const float *xH, const float *xL, int batch, int W,
                         const float *dlogit, float *grad_w, float *grad_H, float *grad_L, cudaStream_t st);
void fp32_backward_release(gwe_model *m);

// Largest |x_l[c]| per [model][branch][layer][channel] (device array `amax`) over the windows of
// one segment, from the FP32 forward; `keys` is 4 unsigned of device scratch.
gwe_status fp32_act_amax(gwe_model *m, const float *sH, const float *sL, int window, int stride, int64_t n_windows,
                         float *amax, unsigned *keys, cudaStream_t st);

// branch_tc.cu (tensor-core path: GWE_BF16, GWE_FP8)
gwe_status tc_check(gwe_model *m, cudaStream_t st);
gwe_status debug_config(int drop, double wait_seconds);
gwe_status debug_ring_margin(int64_t bytes);
void set_cross_window_reuse(int enable);
// f8: E4M3 convolutions, calibrated on synthetic unit-variance white noise until tc_calibrate runs
gwe_status tc_prepare(gwe_model *m, const float *host_blob, bool f8);
// rebuild the tensor-core images from the device FP32 blobs m->w32 (16-bit path: on the device,
// asynchronous on st; FP8: on the host, synchronous)
gwe_status tc_rebuild_from_device(gwe_model *m, cudaStream_t st);
gwe_status tc_calibrate(gwe_model *m, const float *sH, const float *sL, int64_t n_samples, int window, int stride,
                        cudaStream_t st);
gwe_status tc_set_amax(gwe_model *m, const float *host_amax);   // [n_models][2][L][R]
gwe_status tc_get_amax(gwe_model *m, float *host_amax);
// 16-bit path: layers l < n16 take FP16 conv operands, the rest BF16 (rebuilds the images)
gwe_status tc_set_f16_layers(gwe_model *m, int n16);
int tc_f16_layers(gwe_model *m);
void tc_release(gwe_model *m);
gwe_status tc_forward(gwe_model *m, const float *sH, const float *sL, const Segments &sg, int window, int stride,
                      const int32_t *slides, int n_slides, float *out, bool logits, cudaStream_t st);
bool tc_supported(const Dims &d);
// whether tc_forward_save can run for this handle and window length
bool tc_save_supported(gwe_model *m, int W);
// Fused forward of member mi over nwin back-to-back windows of W samples that also stores every
// stack's input x (FP32 [stack][branch][window][W][R]) and the pre-ReLU skip sum (FP32
// [branch][window][W][S]); logits go to `logits` ([nwin][W]).
gwe_status tc_forward_save(gwe_model *m, int mi, const float *xH, const float *xL, int nwin, int W, float *logits,
                           float *save_x, float *save_skip, cudaStream_t st);

// whiten.cu: Welch PSD (FP64 accumulation) and spectral whitening of one detector's strain
gwe_status whiten_run(const float *x, int64_t n, double fs, int seg, const gwe_whiten_options &opt, float *out,
                      cudaStream_t st);
// the defaults of gwe_whiten: mean PSD, no taper, f_low 15 Hz
inline gwe_whiten_options whiten_defaults() {
    gwe_whiten_options o;
    o.psd_average = GWE_PSD_MEAN;
    o.tukey_alpha = 0.0;
    o.f_low = 15.0;
    return o;
}

// triggers.cu
gwe_status triggers_run(const float *prob, int n_models, int n_slides, int64_t n_windows, int window,
                        int stride, float thr, double min_width, int64_t coinc, int flags, gwe_trigger *out,
                        int64_t cap, int64_t *n_out, cudaStream_t st);
// threshold sweep over the segments (n_seg = 1: one series of seg_nw[0] windows): ensemble-trigger
// counts per slide and threshold, optional per-model peak counts (host arrays, overwritten)
gwe_status triggers_sweep(const float *prob, int n_models, int n_slides, const int64_t *seg_nw, int n_seg, int W,
                          int stride, const float *thr, int n_thr, double min_width, int64_t coinc,
                          int64_t *ens_counts, int64_t *model_counts, cudaStream_t st);
// the same over the segments of a gwe_forward_segments output (segment g: seg_nw[g] windows);
// out_seg (optional) receives each record's segment
gwe_status triggers_run_segments(const float *prob, int n_models, int n_slides, const int64_t *seg_nw, int n_seg,
                                 int W, int stride, float thr, double min_width, int64_t coinc, int flags,
                                 gwe_trigger *out, int32_t *out_seg, int64_t cap, int64_t *n_out, cudaStream_t st);

}  // namespace gwe
