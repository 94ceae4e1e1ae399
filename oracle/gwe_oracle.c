/*
 * FP64 CPU oracle for the two-detector WaveNet-ensemble detector of
 * "Inference-optimized AI and HPC for gravitational wave detection at scale"
 * (arXiv:2201.11133).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain, obviously-correct
 * definition that the CUDA library is checked against.  Only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark may load it.  It
 * shares no code, header, table or constant with the CUDA library.
 *
 * What it computes (paper section "AI architecture" and the caption of Fig. 1;
 * layer sizes are the configuration's, the paper gives none):
 *   per model m, per window, per detector branch X in {H, L}:
 *     x0[t]      = w_in * s_X[t] + b_in                       (1x1 conv, 1 -> R)
 *     for each layer l (dilation d_l = 2^(l mod layers_per_stack)):
 *       a[t]     = sum_j Wconv_l[:, j, :] x_l[t - (k-1-j) d_l] + b_conv   (causal, zero before t=0)
 *       z[t]     = tanh(a[t][0:R]) * sigmoid(a[t][R:2R])      (gated activation)
 *       x_{l+1}  = x_l + W_res z + b_res                       (residual)
 *       skip_X  += W_skip z + b_skip                           (skip sum)
 *   head (the "pair of convolutional layers" on the concatenated branches):
 *     h     = ReLU([skip_H ; skip_L])
 *     u     = ReLU(W_h1 h + b_h1)
 *     logit = w_h2 . u + b_h2,   p = 1 / (1 + exp(-logit))   (per-time-step probability)
 *
 * Post-processing (paper section "AI ensemble construction" and section
 * "Event Detection"): stitch the overlapping window outputs into one series,
 * find its peaks (local maxima, height threshold, prominence, width at half
 * prominence, minimum width 0.5 s) and keep the times at which every model of
 * the ensemble has a peak within one 0.5 s window.
 *
 * Weight blob layout (one FP64 blob per model; the CUDA library takes the same
 * layout in FP32), in order:
 *   for branch b in {H, L}:
 *     w_in[R], b_in[R]
 *     for layer l: w_conv[2R][k][R] (out, tap, in; tap k-1 multiplies x[t],
 *                  tap 0 the most-lagged sample), b_conv[2R],
 *                  w_res[R][R] (out, in), b_res[R], w_skip[S][R], b_skip[S]
 *   w_h1[Hc][2S] (input order [skip_H ; skip_L]), b_h1[Hc], w_h2[Hc], b_h2[1]
 *
 * Configuration vector cfg[7] = {n_models, stacks, layers_per_stack, kernel,
 * R, S, Hc}.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int n_models, stacks, lps, k, R, S, Hc;
    int L;          /* total layers */
    int64_t P;      /* parameters per model */
    int64_t Pb;     /* parameters per branch */
    int64_t Pl;     /* parameters per layer */
} ocfg;

static ocfg ocfg_make(const int *c) {
    ocfg o;
    o.n_models = c[0]; o.stacks = c[1]; o.lps = c[2]; o.k = c[3];
    o.R = c[4]; o.S = c[5]; o.Hc = c[6];
    o.L = o.stacks * o.lps;
    o.Pl = (int64_t)2 * o.R * o.k * o.R + 2 * o.R + (int64_t)o.R * o.R + o.R
         + (int64_t)o.S * o.R + o.S;
    o.Pb = 2 * o.R + o.L * o.Pl;
    o.P = 2 * o.Pb + (int64_t)o.Hc * 2 * o.S + 2 * o.Hc + 1;
    return o;
}

/* pointers to one layer's parameters inside a branch */
typedef struct {
    const double *w_conv, *b_conv, *w_res, *b_res, *w_skip, *b_skip;
} olayer;

static int dil(const ocfg *c, int l) { return 1 << (l % c->lps); }

static const double *branch_base(const ocfg *c, const double *w, int b) { return w + (int64_t)b * c->Pb; }

static olayer layer_ptrs(const ocfg *c, const double *wb, int l) {
    olayer p;
    const double *q = wb + 2 * c->R + (int64_t)l * c->Pl;
    p.w_conv = q; q += (int64_t)2 * c->R * c->k * c->R;
    p.b_conv = q; q += 2 * c->R;
    p.w_res = q;  q += (int64_t)c->R * c->R;
    p.b_res = q;  q += c->R;
    p.w_skip = q; q += (int64_t)c->S * c->R;
    p.b_skip = q;
    return p;
}

static const double *head_base(const ocfg *c, const double *w) { return w + 2 * c->Pb; }

static double sigm(double x) { return 1.0 / (1.0 + exp(-x)); }

int64_t orc_param_count(const int *cfg) { ocfg c = ocfg_make(cfg); return c.P; }

/* ---------------------------------------------------------------------------
 * FP8 reading (for error statements of the reduced-precision path).  The
 * paper's TensorRT deployment quantises "where appropriate" without saying
 * how; the library's FP8 path takes this reading, emulated here exactly in
 * FP64 except for the quantisation itself:
 *   E4M3: sign, 4 exponent bits (bias 7), 3 mantissa bits, no infinities,
 *   largest finite value 448, subnormals k * 2^-9.  Conversion rounds to the
 *   nearest value, ties to the even mantissa, and saturates at +-448.
 *   Activation scale of input channel i of layer l: s_i = margin * amax_l[i] / 448
 *   (1 when amax_l[i] is 0), amax_l[i] the calibrated max |x_l[i]|.
 *   The scales are folded into the weights: W'[o][j][i] = W[o][j][i] s_i, and
 *   every output row o takes its own scale w_o = max |W'[o][.][.]| / 448 (1 if 0).
 *   a[t][o] = w_o * sum_{j,i} e4m3(W'[o][j][i] / w_o) e4m3(x[t - lag_j][i] / s_i) + b[o].
 * ------------------------------------------------------------------------- */
double orc_e4m3(double v) {
    if (v != v) return v;
    double a = fabs(v);
    if (a >= 448.0) return v < 0 ? -448.0 : 448.0;
    if (a == 0.0) return v;
    int ex;
    frexp(a, &ex);                   /* a = m 2^ex, m in [0.5, 1): binade [2^(ex-1), 2^ex) */
    int e = ex - 1;
    if (e < -6) e = -6;              /* subnormal range shares the spacing of the lowest binade */
    double q = ldexp(1.0, e - 3);    /* spacing: 3 mantissa bits */
    double n = nearbyint(a / q);     /* a / q is exact (power-of-two divisor); ties to even */
    double r = n * q;
    if (r > 448.0) r = 448.0;
    return v < 0 ? -r : r;
}

/* e4m3 operands of one layer: q_x [W][R] = e4m3(x / s), q_w [2R][k][R], w_o [2R] */
static void quant_layer(const ocfg *c, const double *w_conv, const double *x, int W, const double *amax,
                        double margin, double *qx, double *qw, double *wo) {
    const int R = c->R, K = c->k;
    double *sc = (double *)malloc(sizeof(double) * R);
    for (int i = 0; i < R; i++) sc[i] = amax[i] > 0 ? margin * amax[i] / 448.0 : 1.0;
    for (int t = 0; t < W; t++)
        for (int i = 0; i < R; i++) qx[(int64_t)t * R + i] = orc_e4m3(x[(int64_t)t * R + i] / sc[i]);
    for (int o = 0; o < 2 * R; o++) {
        double mx = 0.0;
        for (int j = 0; j < K; j++)
            for (int i = 0; i < R; i++) {
                double v = fabs(w_conv[((int64_t)o * K + j) * R + i] * sc[i]);
                if (v > mx) mx = v;
            }
        wo[o] = mx > 0 ? mx / 448.0 : 1.0;
        for (int j = 0; j < K; j++)
            for (int i = 0; i < R; i++) {
                int64_t k = ((int64_t)o * K + j) * R + i;
                qw[k] = orc_e4m3(w_conv[k] * sc[i] / wo[o]);
            }
    }
    free(sc);
}

/* ---------------------------------------------------------------------------
 * One branch over one window of W samples.  Optional traces:
 *   xs [L+1][W][R]  residual-stream inputs of every layer (xs[L] = final)
 *   as [L][W][2R]   pre-activations
 *   zs [L][W][R]    gate outputs
 * skip [W][S] receives the skip sum.
 * ------------------------------------------------------------------------- */
static void branch_fwd(const ocfg *c, const double *wb, const double *s, int W,
                       double *skip, double *xs, double *as, double *zs, const double *amax, double margin) {
    /* amax: NULL for exact arithmetic, else [L][R] and the convolutions take the FP8 reading */
    const int R = c->R, S = c->S, K = c->k, L = c->L;
    double *x = (double *)malloc(sizeof(double) * W * R);
    double *xn = (double *)malloc(sizeof(double) * W * R);
    double *a = (double *)malloc(sizeof(double) * W * 2 * R);
    double *z = (double *)malloc(sizeof(double) * W * R);
    double *qx = amax ? (double *)malloc(sizeof(double) * W * R) : NULL;
    double *qw = amax ? (double *)malloc(sizeof(double) * 2 * R * K * R) : NULL;
    double *wo = amax ? (double *)malloc(sizeof(double) * 2 * R) : NULL;
    const double *w_in = wb, *b_in = wb + R;
    for (int t = 0; t < W; t++)
        for (int ch = 0; ch < R; ch++) x[t * R + ch] = w_in[ch] * s[t] + b_in[ch];
    memset(skip, 0, sizeof(double) * W * S);
    for (int l = 0; l < L; l++) {
        olayer p = layer_ptrs(c, wb, l);
        int d = dil(c, l);
        if (xs) memcpy(xs + (int64_t)l * W * R, x, sizeof(double) * W * R);
        /* dilated causal convolution, direct sum */
        if (amax) {
            quant_layer(c, p.w_conv, x, W, amax + (int64_t)l * R, margin, qx, qw, wo);
            for (int t = 0; t < W; t++) {
                for (int o = 0; o < 2 * R; o++) {
                    double acc = 0.0;
                    for (int j = 0; j < K; j++) {
                        int tt = t - (K - 1 - j) * d;
                        if (tt < 0) continue;
                        const double *wr = qw + ((int64_t)o * K + j) * R;
                        const double *xr = qx + (int64_t)tt * R;
                        for (int i = 0; i < R; i++) acc += wr[i] * xr[i];
                    }
                    a[(int64_t)t * 2 * R + o] = wo[o] * acc + p.b_conv[o];
                }
            }
        } else {
            for (int t = 0; t < W; t++) {
                for (int o = 0; o < 2 * R; o++) {
                    double acc = p.b_conv[o];
                    for (int j = 0; j < K; j++) {
                        int tt = t - (K - 1 - j) * d;
                        if (tt < 0) continue;
                        const double *wr = p.w_conv + ((int64_t)o * K + j) * R;
                        const double *xr = x + (int64_t)tt * R;
                        for (int i = 0; i < R; i++) acc += wr[i] * xr[i];
                    }
                    a[(int64_t)t * 2 * R + o] = acc;
                }
            }
        }
        if (as) memcpy(as + (int64_t)l * W * 2 * R, a, sizeof(double) * W * 2 * R);
        /* gate */
        for (int t = 0; t < W; t++)
            for (int ch = 0; ch < R; ch++)
                z[t * R + ch] = tanh(a[(int64_t)t * 2 * R + ch]) * sigm(a[(int64_t)t * 2 * R + R + ch]);
        if (zs) memcpy(zs + (int64_t)l * W * R, z, sizeof(double) * W * R);
        /* residual and skip 1x1 projections */
        for (int t = 0; t < W; t++) {
            const double *zr = z + (int64_t)t * R;
            for (int o = 0; o < R; o++) {
                double acc = p.b_res[o];
                const double *wr = p.w_res + (int64_t)o * R;
                for (int i = 0; i < R; i++) acc += wr[i] * zr[i];
                xn[t * R + o] = x[t * R + o] + acc;
            }
            for (int o = 0; o < S; o++) {
                double acc = p.b_skip[o];
                const double *wr = p.w_skip + (int64_t)o * R;
                for (int i = 0; i < R; i++) acc += wr[i] * zr[i];
                skip[(int64_t)t * S + o] += acc;
            }
        }
        double *tmp = x; x = xn; xn = tmp;
    }
    if (xs) memcpy(xs + (int64_t)L * W * R, x, sizeof(double) * W * R);
    free(x); free(xn); free(a); free(z); free(qx); free(qw); free(wo);
}

/* head over W samples: u_pre [W][Hc] optional trace, logit [W] */
static void head_fwd(const ocfg *c, const double *w, const double *skH, const double *skL, int W,
                     double *logit, double *upre) {
    const int S = c->S, Hc = c->Hc;
    const double *hb = head_base(c, w);
    const double *w1 = hb, *b1 = hb + (int64_t)Hc * 2 * S, *w2 = b1 + Hc, *b2 = w2 + Hc;
    double *h = (double *)malloc(sizeof(double) * 2 * S);
    for (int t = 0; t < W; t++) {
        for (int i = 0; i < S; i++) {
            double vh = skH[(int64_t)t * S + i], vl = skL[(int64_t)t * S + i];
            h[i] = vh > 0 ? vh : 0.0;
            h[S + i] = vl > 0 ? vl : 0.0;
        }
        double lg = b2[0];
        for (int j = 0; j < Hc; j++) {
            double acc = b1[j];
            const double *wr = w1 + (int64_t)j * 2 * S;
            for (int i = 0; i < 2 * S; i++) acc += wr[i] * h[i];
            if (upre) upre[(int64_t)t * Hc + j] = acc;
            lg += w2[j] * (acc > 0 ? acc : 0.0);
        }
        logit[t] = lg;
    }
    free(h);
}

static double *to_double(const double *w, int64_t n) {
    double *d = (double *)malloc(sizeof(double) * n);
    memcpy(d, w, sizeof(double) * n);
    return d;
}

/* ---------------------------------------------------------------------------
 * Forward of one model over B explicit windows (xh, xl: [B][W]); logits out.
 * ------------------------------------------------------------------------- */
void orc_forward_windows(const int *cfg, const double *wblob, const double *xh, const double *xl,
                         int B, int W, double *logit, int nthreads) {
    ocfg c = ocfg_make(cfg);
    double *w = to_double(wblob, c.P);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int b = 0; b < B; b++) {
        double *skH = (double *)malloc(sizeof(double) * W * c.S);
        double *skL = (double *)malloc(sizeof(double) * W * c.S);
        branch_fwd(&c, branch_base(&c, w, 0), xh + (int64_t)b * W, W, skH, NULL, NULL, NULL, NULL, 0.0);
        branch_fwd(&c, branch_base(&c, w, 1), xl + (int64_t)b * W, W, skL, NULL, NULL, NULL, NULL, 0.0);
        head_fwd(&c, w, skH, skL, W, logit + (int64_t)b * W, NULL);
        free(skH); free(skL);
    }
    free(w);
}

/* Branch trace for the pinning tests (one branch, one window). */
void orc_branch_trace(const int *cfg, const double *wblob, int branch, const double *s, int W,
                      double *xs, double *as, double *zs, double *skip) {
    ocfg c = ocfg_make(cfg);
    double *w = to_double(wblob, c.P);
    branch_fwd(&c, branch_base(&c, w, branch), s, W, skip, xs, as, zs, NULL, 0.0);
    free(w);
}

/* ---------------------------------------------------------------------------
 * FP8 reading: forward of one model over B explicit windows with E4M3
 * convolution operands (see orc_e4m3); amax [2][L][R] per branch, layer and
 * input channel; logits out.
 * ------------------------------------------------------------------------- */
void orc_forward_windows_q8(const int *cfg, const double *wblob, const double *amax, double margin,
                            const double *xh, const double *xl, int B, int W, double *logit, int nthreads) {
    ocfg c = ocfg_make(cfg);
    double *w = to_double(wblob, c.P);
    const int64_t ab = (int64_t)c.L * c.R;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int b = 0; b < B; b++) {
        double *skH = (double *)malloc(sizeof(double) * W * c.S);
        double *skL = (double *)malloc(sizeof(double) * W * c.S);
        branch_fwd(&c, branch_base(&c, w, 0), xh + (int64_t)b * W, W, skH, NULL, NULL, NULL, amax, margin);
        branch_fwd(&c, branch_base(&c, w, 1), xl + (int64_t)b * W, W, skL, NULL, NULL, NULL, amax + ab, margin);
        head_fwd(&c, w, skH, skL, W, logit + (int64_t)b * W, NULL);
        free(skH); free(skL);
    }
    free(w);
}

/* Calibration for the FP8 reading: amax [L][R] = max over the B windows s [B][W] and time of
 * |x_l[t][i]|, the input of layer l of branch `branch` (exact arithmetic). */
void orc_act_amax(const int *cfg, const double *wblob, int branch, const double *s, int B, int W, double *amax,
                  int nthreads) {
    ocfg c = ocfg_make(cfg);
    double *w = to_double(wblob, c.P);
    const int64_t per = (int64_t)(c.L + 1) * W * c.R;
    double *part = (double *)calloc((size_t)B * c.L * c.R, sizeof(double));
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int b = 0; b < B; b++) {
        double *xs = (double *)malloc(sizeof(double) * per);
        double *sk = (double *)malloc(sizeof(double) * W * c.S);
        branch_fwd(&c, branch_base(&c, w, branch), s + (int64_t)b * W, W, sk, xs, NULL, NULL, NULL, 0.0);
        double *pb = part + (int64_t)b * c.L * c.R;
        for (int l = 0; l < c.L; l++)
            for (int t = 0; t < W; t++)
                for (int i = 0; i < c.R; i++) {
                    double v = fabs(xs[((int64_t)l * W + t) * c.R + i]);
                    if (v > pb[l * c.R + i]) pb[l * c.R + i] = v;
                }
        free(xs); free(sk);
    }
    for (int k = 0; k < c.L * c.R; k++) {
        double m = 0.0;
        for (int b = 0; b < B; b++)
            if (part[(int64_t)b * c.L * c.R + k] > m) m = part[(int64_t)b * c.L * c.R + k];
        amax[k] = m;
    }
    free(part);
    free(w);
}

/* Number of windows of length W at the given stride in n samples (tail dropped). */
int64_t orc_n_windows(int64_t n, int W, int stride) {
    if (n < W || W <= 0 || stride <= 0) return 0;
    return (n - W) / stride + 1;
}

/* ---------------------------------------------------------------------------
 * Ensemble forward over one stream segment with time slides.
 * H window w is paired with L window (w + slide) mod n_w (slides in windows;
 * zero lag is slide 0).  prob [n_slides][n_models][n_w][W].
 * Each window is an independent input with causal zero padding at its start
 * (the inference batch of shape (batch, 4096, 2) in the section on TensorRT).
 * ------------------------------------------------------------------------- */
void orc_forward_stream(const int *cfg, const double *wblobs, const float *sH, const float *sL,
                        int64_t n, int W, int stride, const int *slides, int n_slides,
                        double *prob, int nthreads) {
    ocfg c = ocfg_make(cfg);
    int64_t nw = orc_n_windows(n, W, stride);
    if (nw == 0) return;
    int ns = n_slides > 0 ? n_slides : 1;
    double *w = to_double(wblobs, c.P * c.n_models);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    /* every (slide, model, window) triple is independent */
    int64_t total = (int64_t)ns * c.n_models * nw;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t it = 0; it < total; it++) {
        int64_t wi = it % nw;
        int m = (int)((it / nw) % c.n_models);
        int si = (int)(it / (nw * c.n_models));
        int64_t sl = (n_slides > 0 && slides) ? slides[si] : 0;
        int64_t wl = ((wi + sl) % nw + nw) % nw;
        const double *wm = w + (int64_t)m * c.P;
        double *xh = (double *)malloc(sizeof(double) * W);
        double *xl = (double *)malloc(sizeof(double) * W);
        for (int t = 0; t < W; t++) {
            xh[t] = sH[wi * stride + t];
            xl[t] = sL[wl * stride + t];
        }
        double *skH = (double *)malloc(sizeof(double) * W * c.S);
        double *skL = (double *)malloc(sizeof(double) * W * c.S);
        double *lg = (double *)malloc(sizeof(double) * W);
        branch_fwd(&c, branch_base(&c, wm, 0), xh, W, skH, NULL, NULL, NULL, NULL, 0.0);
        branch_fwd(&c, branch_base(&c, wm, 1), xl, W, skL, NULL, NULL, NULL, NULL, 0.0);
        head_fwd(&c, wm, skH, skL, W, lg, NULL);
        double *out = prob + (((int64_t)si * c.n_models + m) * nw + wi) * W;
        for (int t = 0; t < W; t++) out[t] = sigm(lg[t]);
        free(xh); free(xl); free(skH); free(skL); free(lg);
    }
    free(w);
}

/* ---------------------------------------------------------------------------
 * Backward (reverse-mode chain rule, FP64, everything stored).
 * Given dL/dlogit [B][W] returns dL/dweights (blob layout, one model, summed
 * over the batch) and dL/dstrain for both detectors (nullable).
 * ------------------------------------------------------------------------- */
static void branch_bwd(const ocfg *c, const double *wb, const double *s, int W,
                       const double *xs, const double *as, const double *zs,
                       const double *dskip, double *gwb, double *ds) {
    const int R = c->R, S = c->S, K = c->k, L = c->L;
    double *dx = (double *)calloc((size_t)W * R, sizeof(double));     /* dL/dx_{l+1} */
    double *dxn = (double *)malloc(sizeof(double) * W * R);
    double *dz = (double *)malloc(sizeof(double) * W * R);
    double *da = (double *)malloc(sizeof(double) * W * 2 * R);
    for (int l = L - 1; l >= 0; l--) {
        olayer p = layer_ptrs(c, wb, l);
        double *g = gwb + 2 * R + (int64_t)l * c->Pl;
        double *g_wconv = g, *g_bconv = g_wconv + (int64_t)2 * R * K * R;
        double *g_wres = g_bconv + 2 * R, *g_bres = g_wres + (int64_t)R * R;
        double *g_wskip = g_bres + R, *g_bskip = g_wskip + (int64_t)S * R;
        int d = dil(c, l);
        const double *x = xs + (int64_t)l * W * R;
        const double *a = as + (int64_t)l * W * 2 * R;
        const double *z = zs + (int64_t)l * W * R;
        /* residual and skip projections */
        for (int t = 0; t < W; t++) {
            const double *dr = dx + (int64_t)t * R;       /* dL/dr = dL/dx_{l+1} */
            const double *dq = dskip + (int64_t)t * S;    /* dL/dq = dL/dskip */
            const double *zr = z + (int64_t)t * R;
            for (int o = 0; o < R; o++) {
                g_bres[o] += dr[o];
                for (int i = 0; i < R; i++) g_wres[(int64_t)o * R + i] += dr[o] * zr[i];
            }
            for (int o = 0; o < S; o++) {
                g_bskip[o] += dq[o];
                for (int i = 0; i < R; i++) g_wskip[(int64_t)o * R + i] += dq[o] * zr[i];
            }
            for (int i = 0; i < R; i++) {
                double acc = 0.0;
                for (int o = 0; o < R; o++) acc += p.w_res[(int64_t)o * R + i] * dr[o];
                for (int o = 0; o < S; o++) acc += p.w_skip[(int64_t)o * R + i] * dq[o];
                dz[(int64_t)t * R + i] = acc;
            }
        }
        /* gate backward */
        for (int t = 0; t < W; t++)
            for (int ch = 0; ch < R; ch++) {
                double f = a[(int64_t)t * 2 * R + ch], gg = a[(int64_t)t * 2 * R + R + ch];
                double th = tanh(f), sg = sigm(gg), dzz = dz[(int64_t)t * R + ch];
                da[(int64_t)t * 2 * R + ch] = dzz * sg * (1.0 - th * th);
                da[(int64_t)t * 2 * R + R + ch] = dzz * th * sg * (1.0 - sg);
            }
        /* convolution backward: weight gradient and input gradient */
        memcpy(dxn, dx, sizeof(double) * W * R);   /* residual path */
        for (int t = 0; t < W; t++) {
            const double *dar = da + (int64_t)t * 2 * R;
            for (int o = 0; o < 2 * R; o++) {
                g_bconv[o] += dar[o];
                for (int j = 0; j < K; j++) {
                    int tt = t - (K - 1 - j) * d;
                    if (tt < 0) continue;
                    const double *wr = p.w_conv + ((int64_t)o * K + j) * R;
                    double *gwr = g_wconv + ((int64_t)o * K + j) * R;
                    const double *xr = x + (int64_t)tt * R;
                    double *dxr = dxn + (int64_t)tt * R;
                    for (int i = 0; i < R; i++) {
                        gwr[i] += dar[o] * xr[i];
                        dxr[i] += wr[i] * dar[o];
                    }
                }
            }
        }
        double *tmp = dx; dx = dxn; dxn = tmp;
    }
    /* input projection */
    const double *w_in = wb;
    double *g_win = gwb, *g_bin = gwb + R;
    for (int t = 0; t < W; t++) {
        double acc = 0.0;
        for (int ch = 0; ch < R; ch++) {
            g_win[ch] += dx[(int64_t)t * R + ch] * s[t];
            g_bin[ch] += dx[(int64_t)t * R + ch];
            acc += w_in[ch] * dx[(int64_t)t * R + ch];
        }
        if (ds) ds[t] = acc;
    }
    free(dx); free(dxn); free(dz); free(da);
}

static void window_bwd(const ocfg *c, const double *w, const double *xh, const double *xl, int W,
                       const double *dlogit, double *gw, double *dh, double *dl) {
    const int R = c->R, S = c->S, Hc = c->Hc, L = c->L;
    double *xs[2], *as[2], *zs[2], *sk[2], *dsk[2];
    const double *in[2] = {xh, xl};
    for (int b = 0; b < 2; b++) {
        xs[b] = (double *)malloc(sizeof(double) * (size_t)(L + 1) * W * R);
        as[b] = (double *)malloc(sizeof(double) * (size_t)L * W * 2 * R);
        zs[b] = (double *)malloc(sizeof(double) * (size_t)L * W * R);
        sk[b] = (double *)malloc(sizeof(double) * (size_t)W * S);
        dsk[b] = (double *)calloc((size_t)W * S, sizeof(double));
        branch_fwd(c, branch_base(c, w, b), in[b], W, sk[b], xs[b], as[b], zs[b], NULL, 0.0);
    }
    double *lg = (double *)malloc(sizeof(double) * W);
    double *upre = (double *)malloc(sizeof(double) * (size_t)W * Hc);
    head_fwd(c, w, sk[0], sk[1], W, lg, upre);
    /* head backward */
    const double *hb = head_base(c, w);
    const double *w1 = hb, *w2 = hb + (int64_t)Hc * 2 * S + Hc;
    double *ghb = gw + 2 * c->Pb;
    double *g_w1 = ghb, *g_b1 = ghb + (int64_t)Hc * 2 * S, *g_w2 = g_b1 + Hc, *g_b2 = g_w2 + Hc;
    for (int t = 0; t < W; t++) {
        double gl = dlogit[t];
        g_b2[0] += gl;
        for (int j = 0; j < Hc; j++) {
            double up = upre[(int64_t)t * Hc + j];
            double u = up > 0 ? up : 0.0;
            g_w2[j] += gl * u;
            double dup = up > 0 ? gl * w2[j] : 0.0;
            g_b1[j] += dup;
            for (int i = 0; i < 2 * S; i++) {
                int b = i / S, ii = i % S;
                double sv = sk[b][(int64_t)t * S + ii];
                double h = sv > 0 ? sv : 0.0;
                g_w1[(int64_t)j * 2 * S + i] += dup * h;
                if (sv > 0) dsk[b][(int64_t)t * S + ii] += w1[(int64_t)j * 2 * S + i] * dup;
            }
        }
    }
    double *dsv[2] = {dh, dl};
    for (int b = 0; b < 2; b++)
        branch_bwd(c, branch_base(c, w, b), in[b], W, xs[b], as[b], zs[b], dsk[b],
                   gw + (int64_t)b * c->Pb, dsv[b]);
    for (int b = 0; b < 2; b++) { free(xs[b]); free(as[b]); free(zs[b]); free(sk[b]); free(dsk[b]); }
    free(lg); free(upre);
}

void orc_backward(const int *cfg, const double *wblob, const double *xh, const double *xl, int B, int W,
                  const double *dlogit, double *grad_w, double *grad_h, double *grad_l, int nthreads) {
    ocfg c = ocfg_make(cfg);
    double *w = to_double(wblob, c.P);
    memset(grad_w, 0, sizeof(double) * c.P);
    double *gws = (double *)calloc((size_t)B * c.P, sizeof(double));
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int b = 0; b < B; b++)
        window_bwd(&c, w, xh + (int64_t)b * W, xl + (int64_t)b * W, W, dlogit + (int64_t)b * W,
                   gws + (int64_t)b * c.P, grad_h ? grad_h + (int64_t)b * W : NULL,
                   grad_l ? grad_l + (int64_t)b * W : NULL);
    for (int b = 0; b < B; b++)    /* fixed summation order */
        for (int64_t i = 0; i < c.P; i++) grad_w[i] += gws[(int64_t)b * c.P + i];
    free(gws); free(w);
}

/* ---------------------------------------------------------------------------
 * Binary cross-entropy on logits, mean over all n samples:
 *   loss = mean( max(z,0) - z*y + log(1 + exp(-|z|)) ),  dL/dz = (sigmoid(z) - y) / n
 * Labels follow the paper: steps up to and including the merger are
 * "waveform" (1), later steps "noise" (0).
 * ------------------------------------------------------------------------- */
double orc_bce(const double *z, const double *y, int64_t n, double *dz) {
    double loss = 0.0;
    for (int64_t i = 0; i < n; i++) {
        double zi = z[i];
        loss += (zi > 0 ? zi : 0.0) - zi * y[i] + log1p(exp(-fabs(zi)));
        if (dz) dz[i] = (sigm(zi) - y[i]) / (double)n;
    }
    return loss / (double)n;
}

/* ---------------------------------------------------------------------------
 * Stitching of overlapping window outputs into one series.  The paper does not
 * say how; the reading taken here: window 0 gives samples [0, W), every later
 * window w gives its last `stride` samples, i.e. global samples
 * [w*stride + W - stride, w*stride + W).  Length (n_w - 1)*stride + W.
 * ------------------------------------------------------------------------- */
int64_t orc_stitch(const float *prob, int64_t nw, int W, int stride, float *out) {
    if (nw <= 0) return 0;
    int64_t len = (nw - 1) * stride + W;
    for (int t = 0; t < W; t++) out[t] = prob[t];
    for (int64_t w = 1; w < nw; w++)
        for (int t = W - stride; t < W; t++) out[w * stride + t] = prob[w * W + t];
    return len;
}

/* ---------------------------------------------------------------------------
 * Peak finding with the semantics of SciPy's find_peaks(x, height=thr,
 * width=min_width) (rel_height 0.5, no window limit), restated:
 *  1. a local maximum is a maximal run x[i..j] of equal values with
 *     x[i-1] < x[i] and x[j+1] < x[j]; its index is (i + j) / 2 (floor);
 *     the first and last samples are never maxima;
 *  2. keep it if x[peak] >= thr;
 *  3. prominence: walk left from the peak while samples are <= x[peak],
 *     tracking the strict minimum (left base = its first occurrence seen
 *     from the peak); the same to the right; prom = x[peak] - max(the two
 *     minima);
 *  4. width at half prominence: reference level h = x[peak] - prom/2; walk
 *     from the peak towards each base while x > h, interpolate linearly
 *     where the walk stopped below h; width = right - left;
 *  5. keep it if width >= min_width.
 * All arithmetic of 3-5 in FP64 on the FP32 samples.
 * Returns the number of peaks found (writes at most cap).
 * ------------------------------------------------------------------------- */
int64_t orc_find_peaks(const float *xf, int64_t n, double thr, double min_width, int64_t *peak,
                       double *height, double *prom, double *width, int64_t cap) {
    int64_t cnt = 0;
    int64_t i = 1;
    while (i < n - 1) {
        if ((double)xf[i - 1] < (double)xf[i]) {
            int64_t ia = i + 1;
            while (ia < n - 1 && xf[ia] == xf[i]) ia++;
            if ((double)xf[ia] < (double)xf[i]) {
                int64_t p = (i + (ia - 1)) / 2;
                double xp = xf[p];
                i = ia;
                if (xp >= thr) {
                    /* prominence */
                    double lmin = xp, rmin = xp;
                    int64_t lb = p, rb = p, k;
                    for (k = p; k >= 0 && (double)xf[k] <= xp; k--)
                        if ((double)xf[k] < lmin) { lmin = xf[k]; lb = k; }
                    for (k = p; k <= n - 1 && (double)xf[k] <= xp; k++)
                        if ((double)xf[k] < rmin) { rmin = xf[k]; rb = k; }
                    double pr = xp - (lmin > rmin ? lmin : rmin);
                    /* width at half prominence */
                    double h = xp - pr * 0.5;
                    k = p;
                    while (lb < k && h < (double)xf[k]) k--;
                    double lip = (double)k;
                    if ((double)xf[k] < h) lip += (h - (double)xf[k]) / ((double)xf[k + 1] - (double)xf[k]);
                    k = p;
                    while (k < rb && h < (double)xf[k]) k++;
                    double rip = (double)k;
                    if ((double)xf[k] < h) rip -= (h - (double)xf[k]) / ((double)xf[k - 1] - (double)xf[k]);
                    double wd = rip - lip;
                    if (wd >= min_width) {
                        if (cnt < cap) {
                            peak[cnt] = p; height[cnt] = xp; prom[cnt] = pr; width[cnt] = wd;
                        }
                        cnt++;
                    }
                }
                continue;   /* i already advanced past the run */
            }
        }
        i++;
    }
    return cnt;
}

/* ---------------------------------------------------------------------------
 * Ensemble coincidence.  The paper keeps triggers "reported by all AI models
 * in the ensemble" and "coincident within a time window of 0.5 seconds".
 * Reading: a peak p0 of model 0 is an ensemble trigger iff there is a choice
 * of one peak per other model such that max - min over the chosen indices and
 * p0 is <= coinc.  Peak lists are sorted ascending.  Writes the indices (into
 * model 0's list) of the accepted model-0 peaks; returns their number.
 *
 * Direct test: a window [a, a + coinc] containing p0 must hold at least one
 * peak of every model; the smallest feasible a is p0 - coinc or q - coinc for
 * some peak q, so those candidates are tried.
 * ------------------------------------------------------------------------- */
static int has_peak_in(const int64_t *pk, int64_t np, int64_t lo, int64_t hi) {
    for (int64_t i = 0; i < np; i++)
        if (pk[i] >= lo && pk[i] <= hi) return 1;
    return 0;
}

int64_t orc_coincidence(const int64_t *const *peaks, const int64_t *npk, int n_models, int64_t coinc,
                        int64_t *out_idx) {
    int64_t cnt = 0;
    for (int64_t i0 = 0; i0 < npk[0]; i0++) {
        int64_t p0 = peaks[0][i0];
        int ok = 0;
        /* candidate window starts */
        for (int m = -1; m < n_models && !ok; m++) {
            int64_t ncand = (m < 0) ? 1 : npk[m];
            for (int64_t q = 0; q < ncand && !ok; q++) {
                int64_t a = (m < 0) ? p0 - coinc : peaks[m][q] - coinc;
                if (a < p0 - coinc || a > p0) continue;
                int all = 1;
                for (int mm = 1; mm < n_models && all; mm++)
                    all = has_peak_in(peaks[mm], npk[mm], a, a + coinc);
                ok = all;
            }
        }
        if (ok) out_idx[cnt++] = i0;
    }
    return cnt;
}
