/*
 * gwe.h — C ABI of libgwe, the GB300 (sm_103a) implementation of the
 * inference and training hot path of the two-detector gravitational-wave
 * detector ensemble of arXiv:2201.11133 ("Inference-optimized AI and HPC for
 * gravitational wave detection at scale").
 *
 * The method (paper, section "Materials and Methods", paragraphs "AI
 * architecture" and "AI ensemble construction", caption of Fig. 1):
 *   - two WaveNet-style branches, one per detector (Hanford H1, Livingston L1),
 *     each a stack of dilated causal convolutions (kernel 2, dilation 2^j) with
 *     a gated tanh*sigmoid activation, residual and skip connections;
 *   - the two branch outputs are concatenated and fed to a pair of 1x1
 *     convolutions whose sigmoid output is a per-time-step probability that
 *     the input contains a waveform;
 *   - an ensemble of models with the same architecture and different random
 *     initialisation;
 *   - the probabilities of each model are searched with find_peaks (height
 *     threshold, width >= 0.5 s), and a trigger is kept when all models of the
 *     ensemble report one within 0.5 s (section "Event Detection");
 *   - background is estimated by time-sliding one detector against the other
 *     (section "Statistical Analysis").
 * Layer counts and widths are not stated in the paper; the caller chooses them
 * in gwe_model_config.
 *
 * Conventions shared by every call:
 *   - Pointers documented as "device" are CUDA device pointers owned by the
 *     caller; pointers documented as "host" are ordinary host memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls are asynchronous on that stream unless stated otherwise.
 *   - Argument errors are detected before any launch and return GWE_ERR_ARG.
 *     A CUDA error returns GWE_ERR_CUDA.  gwe_last_error() returns a
 *     thread-local description of the most recent failure.
 *   - No call falls back to the CPU: when no suitable GPU is present the call
 *     returns GWE_ERR_CUDA.
 *
 * Weight blob (FP32, one blob of gwe_param_count() floats per model, models
 * contiguous), in order:
 *   for branch b in {H, L}:
 *     w_in[R], b_in[R]                         input 1x1 conv (1 -> R)
 *     for layer l in 0 .. stacks*layers_per_stack-1, dilation 2^(l mod layers_per_stack):
 *       w_conv[2R][kernel][R]   (out, tap, in): tap kernel-1 multiplies x[t],
 *                               tap 0 the most lagged sample x[t-(kernel-1)d]
 *       b_conv[2R]              outputs 0..R-1 feed tanh, R..2R-1 the sigmoid gate
 *       w_res[R][R], b_res[R]   residual 1x1 conv (out, in)
 *       w_skip[S][R], b_skip[S] skip 1x1 conv (out, in)
 *   w_h1[Hc][2S], b_h1[Hc]      head conv 1 on ReLU([skip_H ; skip_L])
 *   w_h2[Hc],     b_h2[1]       head conv 2 on ReLU(conv 1) -> logit
 */
#ifndef GWE_H
#define GWE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gwe_model gwe_model;   /* opaque; owns device weights and workspace */

typedef enum {
    GWE_OK = 0,
    GWE_ERR_ARG = 1,          /* invalid argument or shape */
    GWE_ERR_CUDA = 2,         /* CUDA runtime / driver error, or no usable GPU */
    GWE_ERR_OOM = 3,          /* device allocation failed */
    GWE_ERR_TIMEOUT = 4,      /* a bounded device-side wait gave up */
    GWE_ERR_UNSUPPORTED = 5,  /* configuration not implemented for this precision */
    GWE_ERR_CAPACITY = 6      /* output buffer too small (count still reported) */
} gwe_status;

typedef enum {
    GWE_FP32 = 0,   /* FP32 SIMT path, accurate tanhf/expf */
    GWE_BF16 = 1,   /* BF16 operands on tcgen05 tensor cores, FP32 accumulate */
    GWE_FP8 = 2     /* FP8 E4M3 operands with per-channel scales, FP32 accumulate */
} gwe_precision;

typedef struct {
    int n_models;          /* ensemble size (paper: 4) */
    int stacks;            /* number of dilation stacks */
    int layers_per_stack;  /* dilations 1, 2, ..., 2^(layers_per_stack-1) */
    int kernel;            /* convolution kernel size (only 2 is implemented) */
    int r_ch;              /* residual channels R */
    int s_ch;              /* skip channels S */
    int head_ch;           /* head hidden channels Hc */
} gwe_model_config;

/* One peak or ensemble trigger (section "Event Detection"). */
typedef struct {
    int64_t index;       /* sample index in the stitched series (Hanford time) */
    int32_t slide;       /* ordinal of the time slide (0 when no slides) */
    int32_t model;       /* model index, or -1 for an ensemble trigger */
    double height;       /* probability at the peak (model 0's peak for ensemble triggers) */
    double prominence;   /* prominence of that peak */
    double width;        /* width at half prominence, in samples */
} gwe_trigger;

/* Parameters per model of a configuration (layout above); -1 if invalid. */
int64_t gwe_param_count(const gwe_model_config *cfg);

/* Number of windows of length `window` at `stride` in n_samples (tail dropped). */
int64_t gwe_n_windows(int64_t n_samples, int window, int stride);

/*
 * Create a model handle on the current CUDA device.
 *   cfg           configuration (copied).
 *   host_weights  host, FP32, n_models * gwe_param_count(cfg) floats, layout above
 *                 (copied; the caller keeps ownership).
 *   precision     gwe_precision of the forward path; the FP32 copy is always kept
 *                 (for gwe_backward and the FP32 path).
 *   out           receives the handle; release with gwe_model_destroy.
 * Returns GWE_ERR_UNSUPPORTED when kernel != 2 or when the precision does not
 * support the channel counts.
 */
gwe_status gwe_model_create(const gwe_model_config *cfg, const float *host_weights, int precision,
                            gwe_model **out);

/* Replace the weights of an existing handle (host FP32 blob, same layout);
 * derived low-precision copies are rebuilt.  Synchronous. */
gwe_status gwe_model_set_weights(gwe_model *model, const float *host_weights);

/*
 * Replace the weights from a device buffer (FP32 blob, same layout; for
 * example the master weights of a training loop).  The FP32 copy and the
 * derived layouts are rebuilt by kernels on `stream`, with no host round
 * trip, asynchronously; the new weights apply to every later launch on that
 * stream (launches on other streams must be ordered by the caller).  For a
 * GWE_FP8 handle the E4M3 images are built on the host (a synchronous copy to
 * the host).  dev_weights may be any device buffer of n_models *
 * gwe_param_count floats (it is copied).
 */
gwe_status gwe_model_set_weights_device(gwe_model *model, const float *dev_weights, void *stream);

/*
 * Seeded random initialisation (paper paragraph "AI ensemble construction":
 * the members share the architecture and differ in their random
 * initialisation).  Every weight tensor is drawn N(0, 1/fan_in), fan_in = input
 * channels x kernel taps of the layer (1 for the input projection, R*kernel for
 * a dilated convolution, R for the residual and skip projections, 2S for the
 * head's first convolution, Hc for its second); every bias is 0.
 * Weight number e of member m's blob (blob layout above) is the standard normal
 * sqrt(-2 ln u1) cos(2 pi u2) with u1 = ((r[2j] >> 11) + 1) 2^-53 and
 * u2 = (r[2j+1] >> 11) 2^-53, where r = Philox4x64-10(counter (e/2, 0, 0, 0),
 * key (seed, m)) and j = e mod 2, scaled by 1/sqrt(fan_in) in FP64 and rounded
 * to FP32.  The result does not depend on the machine.
 *   gwe_init_weights      host only (no GPU needed): writes n_models *
 *                         gwe_param_count(cfg) floats to host_out.
 *   gwe_model_init_random gwe_init_weights followed by gwe_model_create.
 * GWE_ERR_ARG for an invalid configuration or NULL output.
 */
gwe_status gwe_init_weights(const gwe_model_config *cfg, uint64_t seed, float *host_out);
gwe_status gwe_model_init_random(const gwe_model_config *cfg, uint64_t seed, int precision, gwe_model **out);

/* The counter-based generator of gwe_init_weights, Philox4x64-10 (Salmon et al.,
 * SC 2011): out[0..3] = Philox4x64-10(counter[0..3], key[0..1]).  Host only;
 * exported so that the stream can be checked against other implementations. */
void gwe_philox4x64_10(const uint64_t *counter, const uint64_t *key, uint64_t *out);

/*
 * Operand format of the dilated convolutions of a GWE_BF16 handle.  Layers
 * l < n take FP16 operands (both the activations and the weights; FP16 has
 * three more mantissa bits than BF16 and runs at the same tensor rate), layers
 * l >= n take BF16 operands; accumulation is FP32 either way.  Rounding errors
 * of the first layers pass through every later layer, so they weigh most in
 * the output: for the 30-layer R = 64 ensemble the default n = L/3 (10, the
 * first dilation stack) keeps the bulk of the convolutions (two thirds) in BF16
 * and brings the largest probability error against exact arithmetic from about
 * 9e-3 to about 6e-3 (the paper states no precision; the TensorRT engines it
 * deploys run FP16).  The default for every GWE_BF16 handle is floor(L/3).
 * set: 0 <= n <= L (GWE_ERR_ARG otherwise); synchronises the device and
 * rebuilds the weight images.  GWE_ERR_UNSUPPORTED for other precisions.
 * get: the current n (0 for other precisions or a NULL handle).
 */
gwe_status gwe_model_set_f16_layers(gwe_model *model, int n);
int gwe_model_f16_layers(const gwe_model *model);

/*
 * Activation scales of a GWE_FP8 handle (the paper's TensorRT paragraph runs
 * the network at reduced precision; it does not state how activations are
 * scaled, so this call is the library's own).  Runs the FP32 forward of every
 * model over the windows of one segment, records max |x_l[c]| per model,
 * branch, layer l and residual channel c, and rebuilds the E4M3 weights with
 * s_l[c] = 16 * max / 448 (values up to 16x the calibrated maximum stay in
 * range; larger ones saturate).  Until it is called, a GWE_FP8 handle uses
 * scales calibrated on 64 windows of synthetic unit-variance white Gaussian
 * noise (whitened strain has unit standard deviation).
 *   strain_H, strain_L  device, FP32, n_samples each (whitened strain).
 *   window, stride      as in gwe_forward.
 * Synchronous on `stream`.  GWE_ERR_UNSUPPORTED for a handle of another
 * precision; GWE_ERR_ARG if stride > window or n_samples < window.
 */
gwe_status gwe_model_calibrate(gwe_model *model, const float *strain_H, const float *strain_L, int64_t n_samples,
                               int window, int stride, void *stream);

/*
 * The calibration maxima of a GWE_FP8 handle, host FP32 [n_models][2 branches
 * (H, L)][L layers][R channels]: max |x_l[c]| of the input of layer l.
 * set: copies them (entries must be finite and >= 0; 0 means scale 1) and
 * rebuilds the E4M3 weights (synchronous), so that scales computed elsewhere,
 * for example by a reference implementation, can be applied.  get: copies the
 * current values out.  GWE_ERR_UNSUPPORTED for a handle of another precision.
 */
gwe_status gwe_model_set_fp8_amax(gwe_model *model, const float *host_amax);
gwe_status gwe_model_get_fp8_amax(gwe_model *model, float *host_amax);

void gwe_model_destroy(gwe_model *model);

/*
 * Ensemble forward over one segment of two-detector whitened strain
 * (section "Materials and Methods"; inference batch layout (batch, 4096, 2)
 * -> (batch, 4096, 1) of paragraph "Optimization with NVIDIA TensorRT").
 *   strain_H, strain_L  device, FP32, n_samples each.
 *   window, stride      window w covers samples [w*stride, w*stride + window);
 *                       n_windows = gwe_n_windows(n_samples, window, stride);
 *                       each window is an independent input with causal zero
 *                       padding at its start.
 *   slides              host, n_slides offsets in windows, or NULL / n_slides = 0
 *                       for zero lag only.  For slide k, Hanford window w is
 *                       paired with Livingston window (w + k) mod n_windows
 *                       (section "Statistical Analysis").
 *   out_prob            device, FP32 [max(n_slides,1)][n_models][n_windows][window],
 *                       per-sample probability of each model.
 * Uses the handle's precision.  Returns GWE_ERR_ARG if window <= 0, stride <= 0
 * or n_samples < window.
 */
gwe_status gwe_forward(gwe_model *model, const float *strain_H, const float *strain_L, int64_t n_samples,
                       int window, int stride, const int32_t *slides, int n_slides, float *out_prob,
                       void *stream);

/*
 * As gwe_forward for explicit windows (no slides), returning logits instead of
 * probabilities: x_H, x_L device FP32 [batch][window]; out_logit device FP32
 * [n_models][batch][window].  Used by the autograd wrapper (BCE on logits).
 */
gwe_status gwe_forward_logits(gwe_model *model, const float *x_H, const float *x_L, int batch, int window,
                              float *out_logit, void *stream);

/*
 * Backward pass of one model (training; paper paragraph "AI ensemble
 * construction": per-time-step labels, BCE on logits).
 *   model_index  which ensemble member.
 *   x_H, x_L     device FP32 [batch][window] inputs of the forward.
 *   dlogit       device FP32 [batch][window], dLoss/dlogit.
 *   grad_weights device FP32 [gwe_param_count], overwritten with dLoss/dweights
 *                (summed over the batch), blob layout.
 *   grad_H, grad_L device FP32 [batch][window] dLoss/dstrain, or NULL.
 * The forward keeps only each stack's input and the final skip sums; the
 * backward recomputes one stack at a time from its input (per-stack
 * recomputation) and walks it backwards.  An FP32 handle runs FP32 SIMT
 * kernels on the FP32 weights (windows in chunks of 16, about 0.3 GB of
 * workspace per chunk for the 30-layer R = 64 model).  A GWE_BF16 or GWE_FP8
 * handle runs every contraction (recomputed forward, dz, dgrad, weight
 * gradients) as a BF16 tensor-core GEMM with FP32 accumulation on BF16 copies
 * of the FP32 weights, keeps dL/dx, the residual stream and the skip sums in
 * FP32, and uses the FP32 kernels for the head, the biases and the input
 * projection (windows in chunks of 128, about 13.5 GB of workspace per chunk
 * for the 30-layer R = 64, S = 128, Hc = 256 model); the head's contractions
 * run on the tensor cores too when Hc <= 256 and 2 S <= 256 (u with FP16
 * operands as in the forward, dh with BF16 operands, dW_h1 from BF16 hi/lo
 * splits of both operands); its gradients differ from the FP32 ones by the
 * 16-bit rounding of the operands.  Weight gradients are reduced with atomic
 * additions, so their summation order is not fixed.  The workspace is owned
 * by the handle.  GWE_ERR_UNSUPPORTED for channel counts the kernels do not
 * cover; GWE_ERR_TIMEOUT if a device-side wait of the tensor-core kernels
 * gave up.
 */
gwe_status gwe_backward(gwe_model *model, int model_index, const float *x_H, const float *x_L, int batch,
                        int window, const float *dlogit, float *grad_weights, float *grad_H, float *grad_L,
                        void *stream);

/*
 * Operand staging of the tensor-core backward's GEMMs, from now on
 * (process-wide).  on = 1 (the default): the row GEMMs' A tiles and both
 * operands of the weight-gradient GEMMs arrive by tensor-map copies
 * (cp.async.bulk.tensor with the 128-byte swizzle) where the shapes allow
 * (segments of a multiple of 64 channels; windows a multiple of 128 samples
 * for the row GEMMs, of 64 for the weight gradients; 64 or 128 channels per
 * weight-gradient operand); elsewhere, and everywhere with on = 0, per-thread
 * 16-byte copies stage them.  Both give the same row-GEMM products, so
 * dLoss/dstrain is the same bit for bit; the weight gradients differ only in
 * the order of their atomic partial sums.  GWE_ERR_ARG unless on is 0 or 1.
 */
gwe_status gwe_set_tensor_map_copies(int on);

/*
 * Ensemble forward over a batch of science segments of uneven length in one
 * pass (section "Statistical Analysis": the data come as segments, and time
 * slides pair windows within a segment).  Equivalent to one gwe_forward per
 * segment with the outputs concatenated, but every kernel launch covers all
 * segments (the persistent tensor-core kernel walks the windows of all
 * segments and models; cross-window reuse stops at segment boundaries).
 *   strain_H, strain_L  device FP32; segment g is samples
 *                       [seg_start[g], seg_start[g] + seg_len[g]) of both.
 *   seg_start, seg_len  host int64 [n_segments]; a segment shorter than one
 *                       window has no windows.
 *   slides              as in gwe_forward; Livingston windows wrap within
 *                       each segment: (w + k) mod n_windows(segment).
 *   out_prob            device FP32 [max(n_slides,1)][n_models][N][window],
 *                       N = sum over segments of gwe_n_windows(seg_len[g]);
 *                       segment g's windows follow those of segments < g.
 * GWE_ERR_ARG for n_segments < 1, a negative start or length, or the
 * conditions of gwe_forward.
 */
gwe_status gwe_forward_segments(gwe_model *model, const float *strain_H, const float *strain_L,
                                const int64_t *seg_start, const int64_t *seg_len, int n_segments, int window,
                                int stride, const int32_t *slides, int n_slides, float *out_prob, void *stream);

/*
 * Wait for the work queued on `stream` and report device-side failures of the
 * handle's kernels: GWE_ERR_TIMEOUT when a bounded wait inside a tensor-core
 * kernel gave up (its outputs are then invalid), GWE_ERR_CUDA for a CUDA
 * error.  Clears the recorded failure.
 */
gwe_status gwe_sync(gwe_model *model, void *stream);

/*
 * Cross-window reuse of the tensor-core forward, on by default (process-wide
 * switch; the paper has no counterpart: its TensorRT engine recomputes every
 * window).  Consecutive windows of a segment overlap by window - stride
 * samples; where a layer's output at a position does not reach back to the
 * window start (position >= receptive field of the layers so far - 1), it
 * equals the previous window's output stride samples later, and the library
 * takes it from there instead of recomputing it.  The results are
 * bit-identical either way.  Applies when stride is a multiple of 128 with
 * window/2 <= stride < window (the paper's 0.5 s stride on 1 s windows
 * saves 21 % of the layer work of the 30-layer model); otherwise every
 * window is computed in full.  enable: 1 on, 0 off; GWE_ERR_ARG otherwise.
 */
gwe_status gwe_set_cross_window_reuse(int enable);

/*
 * Allocation-free ensemble forward (the paper has no counterpart: this is an
 * interface for callers, not a step of the method).  It computes exactly what
 * gwe_forward computes for zero lag on the tensor-core path, but it never
 * allocates device memory: its scratch (the per-CTA history of lagged rows,
 * a block of zero rows and an error word) sits in one fixed 24 MiB array
 * compiled into the library, instead of buffers the handle grows on demand.
 * It serves callers that must not call cudaMalloc while they stream: for
 * example a low-latency trigger pipeline sharing the GPU with other work, for
 * which cudaMalloc's implicit device-wide synchronisation would stall the
 * other work, or a process whose device memory is fully reserved up front by
 * a framework's pool.  The handle itself is still created (and allocated)
 * once, beforehand, with gwe_model_create.
 *   model       handle created with precision GWE_BF16 or GWE_FP8.
 *   strain_H/L  device, FP32, n_samples each; out_prob device, FP32
 *               [n_models][n_windows][window] (caller-owned, as for gwe_forward).
 *   status      device pointer to one int owned by the caller, or NULL.  It is
 *               set to 0 on the stream, then to a nonzero wait-site code if a
 *               bounded device-side wait of the kernel gave up (the outputs are
 *               then invalid).  With NULL the code goes to the handle's own
 *               error word (allocated with the handle), and gwe_sync on the
 *               handle returns GWE_ERR_TIMEOUT, as for the other calls.
 * Limits: window must be a multiple of 128; the number of CTAs is reduced so
 * that their lag rings fit the array (the 30-layer, R = 64 configuration
 * needs 768 KiB per CTA in BF16 and 384 KiB in FP8, so at most 32 or 64 CTAs
 * run and the call is slower than gwe_forward); a configuration whose
 * single-CTA ring exceeds the array is
 * rejected with GWE_ERR_ARG.
 * The first call on each device looks up the array's device address for that
 * device (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  The address is kept per device and CUDA context:
 * after cudaDeviceReset the next call looks it up again.  Every call on a
 * device shares the one array (the previous call's lag rows stay in it) and
 * clears its zero rows on the stream; calls whose executions overlap on the GPU
 * (for example on two streams) race on it, so serialise them.
 */
gwe_status gwe_forward_static(gwe_model *model, const float *strain_H, const float *strain_L, int64_t n_samples,
                              int window, int stride, float *out_prob, int *status, void *stream);

/* Opaque forward plan (gwe_plan_create). */
typedef struct gwe_plan gwe_plan;

/* Flags of gwe_plan_create. */
#define GWE_PLAN_AUTOTUNE 1   /* choose the slide heads' launch shape by timing the candidates */

/*
 * Forward plan: the batched ensemble forward over many science segments of
 * uneven length times many time-slide offsets (section "Statistical
 * Analysis": background from time-shifted Livingston data; the same
 * computation as gwe_forward_segments with these arguments), prepared once and
 * recorded into one CUDA graph, so that every execution is a single graph
 * launch of the persistent tensor-core kernel(s) and the slide heads.
 *   model            GWE_BF16 or GWE_FP8 handle (GWE_ERR_UNSUPPORTED otherwise).
 *   strain_H/L, seg_start, seg_len, n_segments, window, stride, slides,
 *   n_slides, out_prob   as for gwe_forward_segments.  The device buffers are
 *                    bound at creation: every execution reads the strain
 *                    buffers as they are then and overwrites out_prob; refill
 *                    the strain in place between executions.  window must be a
 *                    multiple of 128.
 *   flags            0 or GWE_PLAN_AUTOTUNE.  With GWE_PLAN_AUTOTUNE and
 *                    n_slides > 0 the plan times every candidate launch shape of
 *                    the slide heads (2 or 4 Hanford windows per block; pieces
 *                    of up to 4 or 8 consecutive offsets; all pieces per block
 *                    or a quarter of them) on these buffers with CUDA events
 *                    and keeps the fastest; the choice is cached per geometry
 *                    for the process.  Without it, the shape set by
 *                    gwe_set_slide_shape (4 windows, pieces of up to 8
 *                    offsets, all pieces per block unless changed).  Every shape computes
 *                    the same sums in the same order: the output does not
 *                    depend on the shape.
 *   stream           creation runs (and synchronises) on this stream; the graph
 *                    is recorded on a private stream.
 *   out              receives the plan.
 * The plan owns its lag rings, carry buffer, slide projections (2 x windows x
 * Hc x window FP16) and tables; the handle's weights are used in place (so
 * gwe_model_set_weights and FP8 calibration take effect in later executions).
 * Executions of one plan, and other calls on the same handle, must not overlap
 * on the GPU.  A device-side wait that times out is reported by gwe_sync on
 * the handle.
 */
gwe_status gwe_plan_create(gwe_model *model, const float *strain_H, const float *strain_L, const int64_t *seg_start,
                           const int64_t *seg_len, int n_segments, int window, int stride, const int32_t *slides,
                           int n_slides, float *out_prob, int flags, void *stream, gwe_plan **out);

/* Launch the plan's graph on `stream` (asynchronous). */
gwe_status gwe_plan_execute(gwe_plan *plan, void *stream);

/*
 * The launch shape the plan uses for the slide heads: Hanford windows per
 * block, the longest run of consecutive offsets a block pairs with them (a
 * piece), and pieces per block; the number of kernels in its graph; and
 * (after autotuning) the time of one model's slide heads with the chosen shape
 * and with the default shape, in milliseconds (0 when not tuned).  NULL
 * outputs are skipped.
 */
gwe_status gwe_plan_shape(const gwe_plan *plan, int *window_tile, int *offset_tile, int *pieces_per_block,
                          int *n_kernels, double *tuned_ms, double *default_ms);

/*
 * Slide-head launch shape of the launches that are not autotuned, from now on
 * (process-wide): gwe_forward and gwe_forward_segments with slides, and plans
 * created without GWE_PLAN_AUTOTUNE.  Hanford windows per block (2 or 4), the
 * longest offset piece (4 or 8) and pieces per block (0: all).  The default is
 * (4, 8, 0).  The output does not depend on the shape.  GWE_ERR_ARG for other
 * values.
 */
gwe_status gwe_set_slide_shape(int window_tile, int offset_tile, int pieces_per_block);

/* Release a plan (after its executions have completed). */
void gwe_plan_destroy(gwe_plan *plan);

/* Flags of gwe_triggers. */
#define GWE_TRIG_PER_MODEL 1   /* also return every model's kept peaks (model >= 0) */

/*
 * Peak finding and ensemble coincidence on the device (paper paragraph "AI
 * ensemble construction": find_peaks; section "Event Detection": all models
 * coincident within 0.5 s; section "Statistical Analysis": ROC threshold and
 * width >= 0.5 s).
 *   prob         device FP32 [n_slides][n_models][n_windows][window] as written by
 *                gwe_forward (probabilities or logits; no NaN).
 *   Each (slide, model) series is stitched: window 0 gives samples [0, window),
 *   every later window w its last `stride` samples.  Peaks follow SciPy's
 *   find_peaks(x, height=height_thr, width=min_width) semantics (rel_height 0.5,
 *   no window limit), bit-exact for identical probabilities.  An ensemble
 *   trigger is a model-0 peak p0 for which every other model has a peak such
 *   that max - min of the chosen indices and p0 is <= coinc samples.
 *   out          host array of `cap` records, sorted by (slide, model, index);
 *                ensemble records have model = -1 and follow the per-model ones
 *                of the same slide.
 *   n_out        host, receives the total number of records (may exceed cap, in
 *                which case GWE_ERR_CAPACITY is returned and `cap` records written).
 * Synchronises `stream` before returning.
 */
gwe_status gwe_triggers(const float *prob, int n_models, int n_slides, int64_t n_windows, int window,
                        int stride, float height_thr, double min_width, int64_t coinc, int flags,
                        gwe_trigger *out, int64_t cap, int64_t *n_out, void *stream);

/*
 * Peaks and ensemble triggers of every segment of a gwe_forward_segments
 * output: the same as gwe_triggers applied to each segment's windows (series
 * never span segments; `index` is relative to the segment's first sample).
 *   seg_len      host int64 [n_segments], the lengths given to gwe_forward_segments.
 *   out_segment  host int32 [cap] or NULL: the segment of each record.
 * Records are ordered by segment, then as in gwe_triggers.  Synchronises `stream`.
 */
gwe_status gwe_triggers_segments(const float *prob, int n_models, int n_slides, const int64_t *seg_len,
                                 int n_segments, int window, int stride, float height_thr, double min_width,
                                 int64_t coinc, int flags, gwe_trigger *out, int32_t *out_segment, int64_t cap,
                                 int64_t *n_out, void *stream);

/*
 * Threshold sweep of the trigger statistics in one pass (section "Statistical
 * Analysis": the ROC curve and the false-alarm rate come from sweeping the
 * probability threshold, over [0, 0.9998] in the paper, on the zero-lag and
 * the time-slid outputs; the paper post-processes ~500 GB per searched month
 * on CPUs, section "Computational Efficiency").  The result is exactly what
 * gwe_triggers would report once per threshold with the same min_width and
 * coinc, counted instead of listed: peaks are found once at the lowest
 * threshold (prominence and width do not depend on the threshold), and each
 * model-0 peak's largest threshold at which it is still an ensemble trigger is
 * computed on the device.
 *   prob, n_models, n_slides, n_windows, window, stride, min_width, coinc
 *                as gwe_triggers (one segment).
 *   thresholds   host FP32 [n_thr], finite and in ascending order (a peak is
 *                kept at threshold t when its height >= t, as in gwe_triggers).
 *   ens_counts   host int64 [max(n_slides,1)][n_thr]: number of ensemble
 *                triggers of each slide at each threshold (overwritten).
 *   model_counts host int64 [max(n_slides,1)][n_models][n_thr] or NULL: number
 *                of kept peaks of each model (overwritten).
 * Synchronises `stream`.  GWE_ERR_ARG for unsorted or non-finite thresholds.
 * The _segments form takes the segments of a gwe_forward_segments output (as
 * gwe_triggers_segments) and sums the counts over them.
 */
gwe_status gwe_trigger_sweep(const float *prob, int n_models, int n_slides, int64_t n_windows, int window,
                             int stride, const float *thresholds, int n_thr, double min_width, int64_t coinc,
                             int64_t *ens_counts, int64_t *model_counts, void *stream);
gwe_status gwe_trigger_sweep_segments(const float *prob, int n_models, int n_slides, const int64_t *seg_len,
                                      int n_segments, int window, int stride, const float *thresholds, int n_thr,
                                      double min_width, int64_t coinc, int64_t *ens_counts, int64_t *model_counts,
                                      void *stream);

/* Input sample types of gwe_search_run. */
#define GWE_INPUT_F32 0
#define GWE_INPUT_F16 1

/* Parameters of a streaming search (gwe_search_create). */
typedef struct {
    int window, stride;        /* window and stride in samples (paper: 4096, 2048) */
    int chunk_windows;         /* windows per chunk core */
    int margin_windows;        /* windows of context computed on each side of a core */
    int64_t guard_samples;     /* raw samples whitened beyond the margins on each side */
    double fs;                 /* sample rate, Hz */
    int welch_seg;             /* Welch segment length (power of two; 16384 = 4 s at 4096 Hz) */
    int input_dtype;           /* GWE_INPUT_F32 or GWE_INPUT_F16 */
    float input_scale;         /* samples are multiplied by this after conversion to FP32 */
    float height_thr;          /* peak height threshold (as gwe_triggers) */
    double min_width;          /* minimum peak width in samples (as gwe_triggers) */
    int64_t coinc;             /* coincidence span in samples (as gwe_triggers) */
    int trigger_flags;         /* 0 or GWE_TRIG_PER_MODEL */
} gwe_search_config;

/* Opaque streaming search (gwe_search_create). */
typedef struct gwe_search gwe_search;

/*
 * Streaming search over one long stream of raw two-detector strain (section
 * "Computational Efficiency": a month of Hanford and Livingston data searched
 * by the ensemble; section "Materials and Methods", paragraph "Data
 * preparation": whitening with PSDs estimated from the data).  The stream's
 * windows (window w = samples [w*stride, w*stride + window)) are cut into
 * chunks of chunk_windows windows (the cores).  Each chunk computes the
 * windows of its core plus margin_windows windows on each side, on a span of
 * raw samples that reaches guard_samples further on each side (clipped to the
 * stream): the span is converted to FP32 (times input_scale), whitened as
 * gwe_whiten does with the span as its segment (PSD and standard deviation of
 * the span), run through the handle's ensemble forward, and peak finding and
 * ensemble coincidence (as gwe_triggers) run on the stitched series of the
 * span's windows.  A record is kept when its index lies in the core's part of
 * the stream's stitched series (window 0 gives samples [0, window), window w
 * its last stride samples): the cores partition the series, so each trigger
 * comes from one chunk.  Peaks whose bases or half-height crossings reach
 * beyond a span can differ from peak finding on the whole series; the margins
 * bound that.  The model handle must not be used by other calls meanwhile.
 *   cfg     parameters; validated here (GWE_ERR_ARG).
 */
gwe_status gwe_search_create(gwe_model *model, const gwe_search_config *cfg, gwe_search **out);

/*
 * Run the search over n_samples samples per detector.
 *   strain_H/L   the raw strain, input_dtype elements: device memory
 *                (host_input = 0), or host memory (host_input = 1; pinned
 *                memory lets the copy of the next chunk's span overlap the
 *                current chunk's work, which runs on `stream`).
 *   out, cap     host array of records, index in the stream's stitched
 *                series, slide 0; ordered by chunk, then as gwe_triggers.
 *   n_out        total number of records (GWE_ERR_CAPACITY if above cap).
 * Synchronous (returns after the last chunk).  GWE_ERR_ARG when a chunk's
 * span is shorter than welch_seg.
 */
gwe_status gwe_search_run(gwe_search *search, const void *strain_H, const void *strain_L, int64_t n_samples,
                          int host_input, gwe_trigger *out, int64_t cap, int64_t *n_out, void *stream);

/*
 * Checkpoint and resume of a long search (a month of data is searched chunk by
 * chunk; the paper's run spans many nodes and hours, section "Computational
 * Efficiency").  The chunks' cores partition the stream, so the records of
 * chunks [a, b) followed by those of [b, c) are exactly the records of [a, c):
 * a caller that stores the records found so far and the next chunk index can
 * stop after any range and continue later with the same configuration and
 * strain.
 *   gwe_search_chunks     number of chunks of a stream of n_samples samples
 *                         (0 if the stream is shorter than one window).
 *   gwe_search_run_range  as gwe_search_run for chunks [chunk_begin,
 *                         min(chunk_end, gwe_search_chunks)) only; records in
 *                         chunk order.  GWE_ERR_ARG for a negative or reversed
 *                         range.
 */
int64_t gwe_search_chunks(const gwe_search *search, int64_t n_samples);
gwe_status gwe_search_run_range(gwe_search *search, const void *strain_H, const void *strain_L, int64_t n_samples,
                                int host_input, int64_t chunk_begin, int64_t chunk_end, gwe_trigger *out, int64_t cap,
                                int64_t *n_out, void *stream);

/* Release a search. */
void gwe_search_destroy(gwe_search *search);

/* PSD averages of the whitening front end. */
#define GWE_PSD_MEAN 0     /* mean of |X|^2 over the Welch segments */
#define GWE_PSD_MEDIAN 1   /* median over the segments, divided by the median's bias */

/* Options of gwe_whiten_ex. */
typedef struct {
    int psd_average;       /* GWE_PSD_MEAN or GWE_PSD_MEDIAN */
    double tukey_alpha;    /* taper fraction in [0, 1] of a Tukey window on the strain before its
                              transform (0: none) */
    double f_low;          /* the whitened spectrum is zero below this frequency, Hz (>= 0; default 15) */
} gwe_whiten_options;

/*
 * Whitening front end (paper section "Materials and Methods", paragraph "Data
 * preparation": the strain is whitened with power spectral densities
 * estimated from the data, then normalised to unit standard deviation).
 * Welch PSD: segments of seg_len samples at 50 % overlap, each minus its mean,
 * periodic Hann window, one-sided density; |X|^2 of the segments averaged by
 * the mean or (GWE_PSD_MEDIAN, robust against loud short glitches such as the
 * ones the paper's section "Event Detection" discusses) by the median over
 * segments divided by 1 - 1/2 + 1/3 - ... (the bias of the median of
 * exponentially distributed values; over the largest odd number of terms <= the
 * number of segments).  The segment transforms are FP32; FP64 is used only for
 * |X|^2 and its accumulation or selection over segments.  The strain (times a
 * Tukey window when tukey_alpha > 0) is transformed (FP32), divided by
 * sqrt(fs * PSD / 2), the PSD interpolated linearly onto the data's frequency
 * grid, zeroed below f_low, transformed back and scaled to unit standard
 * deviation (FP32 compensated sums).  The FFTs are cuFFT calls; everything
 * else is this library's kernels.
 *   strain   device FP32 [n] (one detector; not modified).
 *   n        samples; >= seg_len.
 *   fs       sample rate in Hz (> 0).
 *   seg_len  Welch segment length, a power of two >= 16 (16384 = 4 s at 4096 Hz).
 *   flags    (gwe_whiten) 0, or GWE_PSD_MEDIAN for the median average; no taper,
 *            f_low = 15 Hz.
 *   options  (gwe_whiten_ex) as above.
 *   out      device FP32 [n], whitened strain; must not alias strain.
 * Asynchronous on `stream`; plans and work buffers are cached in the library
 * (one whitening at a time per process).  GWE_ERR_ARG for invalid arguments;
 * GWE_ERR_UNSUPPORTED for a median over more than 16384 segments.
 */
gwe_status gwe_whiten(const float *strain, int64_t n, double fs, int seg_len, int flags, float *out, void *stream);
gwe_status gwe_whiten_ex(const float *strain, int64_t n, double fs, int seg_len, const gwe_whiten_options *options,
                         float *out, void *stream);

/*
 * Per-kernel device timing.  gwe_profile_enable(1) clears the accumulators and
 * makes the library record a pair of CUDA events on the launch stream around
 * each of its main kernel launches; gwe_profile_enable(0) stops it.
 * gwe_profile_read(i, ...) synchronises on the recorded events of the i-th
 * kernel name and returns its name (copied into `name`, at most name_cap
 * bytes including the terminator), the summed device time in milliseconds and
 * the number of launches; GWE_ERR_ARG when i is out of range.  Host-side only;
 * the paper has no counterpart (it is the measurement harness).
 */
gwe_status gwe_profile_enable(int on);
gwe_status gwe_profile_read(int idx, char *name, int name_cap, double *total_ms, int64_t *launches);

/* Total number of kernels this library has launched in the process (all calls). */
int64_t gwe_launch_count(void);

/*
 * Failure-detection test hook (the paper has no counterpart).  Every wait
 * inside the tensor-core kernels is bounded; wait_seconds sets that bound
 * (default 4 s, at most 60).  drop = 1 makes the Hanford branch's producer warp
 * issue nothing, so a consumer's wait runs out: the kernel records the wait
 * site, every role drains the copies and MMAs it issued and leaves, TMEM is
 * freed, and gwe_sync returns GWE_ERR_TIMEOUT; the CUDA context stays usable.
 * drop = 0 restores normal operation.  Process-wide; not for production use.
 */
gwe_status gwe_debug_config(int drop, double wait_seconds);

/*
 * Address checks of the tensor-core forward (the paper has no counterpart).
 * The kernel checks every lag-copy source and history-row store it computes
 * against the size of its lag ring, and every projection store against the
 * projection buffer; an address outside is not accessed: the kernel records
 * the site (41: lag source, 42: history store, 43: projection store) in the
 * handle's error word, stops the copies of the branch concerned, and gwe_sync
 * returns GWE_ERR_CUDA with the site in gwe_last_error().  Test hook: with
 * bytes > 0 the checks treat the ring as that many bytes smaller than it is,
 * so that the path can be exercised without any out-of-range access; 0
 * restores normal operation.  Process-wide; GWE_ERR_ARG for bytes < 0.
 */
gwe_status gwe_debug_ring_margin(int64_t bytes);

/* Thread-local description of the last error ("" if none). */
const char *gwe_last_error(void);

/* Library version string. */
const char *gwe_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GWE_H */
