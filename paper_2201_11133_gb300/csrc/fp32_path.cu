// FP32 SIMT forward path of the two-branch WaveNet detector ensemble
// (arXiv:2201.11133, section "Materials and Methods", paragraph "AI
// architecture" and Fig. 1).  This is the plain FP32 path that the tensor-core
// paths are compared against; it uses accurate tanhf / expf.
//
// Structure (one launch per layer over a chunk of windows, both branches):
//   layer kernel   a = Wconv [x(t-d); x(t)] + b  -> z = tanh(a_f) sigmoid(a_g)
//                  x_{l+1} = x_l + W_res z + b_res,  skip += W_skip z + b_skip
//                  (layer 0 also forms x_0 = w_in s + b_in from the strain)
//   head projection (the head's first 1x1 conv is linear in [skip_H ; skip_L],
//                  so it splits per branch): P_X = W_h1[:, X] ReLU(skip_X) (+ b_h1 for H)
//   combine        logit = b_h2 + w_h2 . ReLU(P_H(w) + P_L(w')) with w' = w + slide,
//                  probability = sigmoid(logit)
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "gwe_internal.h"

namespace gwe {
namespace {

constexpr int kTM = 64;        // time rows per block
constexpr int LF_FROM_STRAIN = 1, LF_SKIP_INIT = 2, LF_NO_SKIP = 4;
constexpr int kThreads = 256;  // 16 x 16 thread grid: 4 rows x (N/16) columns per thread

template <int R, int S>
struct LayerShape {
    static constexpr int N1 = 2 * R;
    static constexpr int J1 = N1 / 16;
    static constexpr int N2 = R + S;
    static constexpr int J2 = N2 / 16;
    static constexpr int LD = R + 1;
    static constexpr int WFLOATS = 4 * R * R + R * N2;   // conv + [res|skip] weights
    static constexpr size_t SMEM = sizeof(float) * (size_t)(WFLOATS + 3 * kTM * LD);
};

template <int R, int S>
__global__ void __launch_bounds__(kThreads, 1)
k_fp32_layer(const float *__restrict__ xin, float *__restrict__ xout, float *__restrict__ skip,
             const float *__restrict__ wl_base, int64_t branch_stride, const float *__restrict__ win,
             const float *__restrict__ sH, const float *__restrict__ sL, int64_t w0, int stride, int W,
             int C, int d, int flags, float *__restrict__ a_out) {
    // flags: LF_FROM_STRAIN x_l is the input projection of the strain (else read xin);
    //        LF_SKIP_INIT skip = q (else skip += q); LF_NO_SKIP skip is not written.
    // a_out (optional): the pre-activations a = conv + b_conv, [rows][2R].
    const int first = flags & LF_FROM_STRAIN;
    using Sh = LayerShape<R, S>;
    extern __shared__ float4 smem4[];
    float *smem = reinterpret_cast<float *>(smem4);
    float *wc = smem;                       // [2R (k)][2R (out)]
    float *wrs = wc + 4 * R * R;            // [R (k)][R+S (out)]
    float *xc = wrs + R * Sh::N2;           // [TM][R+1] current rows
    float *xl = xc + kTM * Sh::LD;          // [TM][R+1] rows lagged by d
    float *zz = xl + kTM * Sh::LD;          // [TM][R+1] gate output
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int bw = blockIdx.y, b = bw / C, c = bw - b * C;
    const int t0 = blockIdx.x * kTM;
    const float *wl = wl_base + (int64_t)b * branch_stride;

    {
        const float4 *src = reinterpret_cast<const float4 *>(wl);
        float4 *dst = reinterpret_cast<float4 *>(wc);
        for (int i = tid; i < Sh::WFLOATS / 4; i += kThreads) dst[i] = src[i];
    }
    const float *bconv = wl + Sh::WFLOATS;
    const float *bres = bconv + 2 * R;
    const float *bskip = bres + R;
    const int64_t xrow0 = (int64_t)bw * W;   // row index of (window-branch, t = 0)

    if (first) {
        const float *s = (b ? sL : sH) + (w0 + c) * (int64_t)stride;
        const float *wi = win + b * R;
        const float *bi = win + 2 * R + b * R;
        for (int i = tid; i < kTM * R; i += kThreads) {
            const int r = i / R, ch = i - r * R, t = t0 + r, tl = t - d;
            xc[r * Sh::LD + ch] = (t < W) ? wi[ch] * s[t] + bi[ch] : 0.f;
            xl[r * Sh::LD + ch] = (tl >= 0 && tl < W) ? wi[ch] * s[tl] + bi[ch] : 0.f;
        }
    } else {
        for (int i = tid; i < kTM * R; i += kThreads) {
            const int r = i / R, ch = i - r * R, t = t0 + r, tl = t - d;
            xc[r * Sh::LD + ch] = (t < W) ? xin[(xrow0 + t) * R + ch] : 0.f;
            xl[r * Sh::LD + ch] = (tl >= 0 && tl < W) ? xin[(xrow0 + tl) * R + ch] : 0.f;
        }
    }
    __syncthreads();

    // dilated causal convolution as a [TM x 2R] x [2R x 2R] product
    float acc[4][Sh::J1];
#pragma unroll
    for (int j = 0; j < Sh::J1; ++j) {
        const float bj = bconv[tx + 16 * j];
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[i][j] = bj;
    }
#pragma unroll 4
    for (int k = 0; k < R; ++k) {
        float a[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = xl[(ty + 16 * i) * Sh::LD + k];
#pragma unroll
        for (int j = 0; j < Sh::J1; ++j) {
            const float wv = wc[k * Sh::N1 + tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i) acc[i][j] = fmaf(a[i], wv, acc[i][j]);
        }
    }
#pragma unroll 4
    for (int k = 0; k < R; ++k) {
        float a[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = xc[(ty + 16 * i) * Sh::LD + k];
#pragma unroll
        for (int j = 0; j < Sh::J1; ++j) {
            const float wv = wc[(R + k) * Sh::N1 + tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i) acc[i][j] = fmaf(a[i], wv, acc[i][j]);
        }
    }
    if (a_out) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int t = t0 + ty + 16 * i;
            if (t >= W) continue;
#pragma unroll
            for (int j = 0; j < Sh::J1; ++j) a_out[(xrow0 + t) * (2 * R) + tx + 16 * j] = acc[i][j];
        }
    }
    // gate: column ch (< R) is the tanh input, column ch + R its sigmoid gate
#pragma unroll
    for (int j = 0; j < Sh::J1 / 2; ++j) {
        const int ch = tx + 16 * j;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float f = acc[i][j], g = acc[i][j + Sh::J1 / 2];
            zz[(ty + 16 * i) * Sh::LD + ch] = tanhf(f) * (1.f / (1.f + expf(-g)));
        }
    }
    __syncthreads();

    // residual and skip projections: [TM x R] x [R x (R+S)]
    float acc2[4][Sh::J2];
#pragma unroll
    for (int j = 0; j < Sh::J2; ++j) {
        const int col = tx + 16 * j;
        const float bj = (col < R) ? bres[col] : bskip[col - R];
#pragma unroll
        for (int i = 0; i < 4; ++i) acc2[i][j] = bj;
    }
#pragma unroll 4
    for (int k = 0; k < R; ++k) {
        float a[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = zz[(ty + 16 * i) * Sh::LD + k];
#pragma unroll
        for (int j = 0; j < Sh::J2; ++j) {
            const float wv = wrs[k * Sh::N2 + tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i) acc2[i][j] = fmaf(a[i], wv, acc2[i][j]);
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int r = ty + 16 * i, t = t0 + r;
        if (t >= W) continue;
#pragma unroll
        for (int j = 0; j < Sh::J2; ++j) {
            const int col = tx + 16 * j;
            if (col < R) {
                xout[(xrow0 + t) * R + col] = xc[r * Sh::LD + col] + acc2[i][j];
            } else if (!(flags & LF_NO_SKIP)) {
                float *sp = skip + (xrow0 + t) * S + (col - R);
                *sp = (flags & LF_SKIP_INIT) ? acc2[i][j] : (*sp + acc2[i][j]);
            }
        }
    }
}

// P_X[t][j] = sum_k W_h1[j][X*S + k] ReLU(skip_X[t][k]) (+ b_h1[j] for X = H)
template <int S, int HC>
struct HeadShape {
    static constexpr int J = HC / 16;
    static constexpr int LD = S + 1;
    static constexpr size_t SMEM = sizeof(float) * (size_t)(S * HC + kTM * LD);
};

template <int S, int HC>
__global__ void __launch_bounds__(kThreads, 1)
k_fp32_headproj(const float *__restrict__ skip, float *__restrict__ proj, const float *__restrict__ head,
                int W, int C) {
    using Sh = HeadShape<S, HC>;
    extern __shared__ float4 smem4[];
    float *smem = reinterpret_cast<float *>(smem4);
    float *w1 = smem;               // [S (k)][HC (out)]
    float *hs = w1 + S * HC;        // [TM][S+1]
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int bw = blockIdx.y, b = bw / C;
    const int t0 = blockIdx.x * kTM;
    {
        const float4 *src = reinterpret_cast<const float4 *>(head + (int64_t)b * S * HC);
        float4 *dst = reinterpret_cast<float4 *>(w1);
        for (int i = tid; i < S * HC / 4; i += kThreads) dst[i] = src[i];
    }
    const float *b1 = head + 2 * S * HC;
    const int64_t row0 = (int64_t)bw * W;
    for (int i = tid; i < kTM * S; i += kThreads) {
        const int r = i / S, k = i - r * S, t = t0 + r;
        const float v = (t < W) ? skip[(row0 + t) * S + k] : 0.f;
        hs[r * Sh::LD + k] = v > 0.f ? v : 0.f;
    }
    __syncthreads();
    float acc[4][Sh::J];
#pragma unroll
    for (int j = 0; j < Sh::J; ++j) {
        const float bj = (b == 0) ? b1[tx + 16 * j] : 0.f;
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[i][j] = bj;
    }
#pragma unroll 4
    for (int k = 0; k < S; ++k) {
        float a[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = hs[(ty + 16 * i) * Sh::LD + k];
#pragma unroll
        for (int j = 0; j < Sh::J; ++j) {
            const float wv = w1[k * HC + tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i) acc[i][j] = fmaf(a[i], wv, acc[i][j]);
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int t = t0 + ty + 16 * i;
        if (t >= W) continue;
#pragma unroll
        for (int j = 0; j < Sh::J; ++j) proj[(row0 + t) * HC + tx + 16 * j] = acc[i][j];
    }
}

// One warp per output sample: logit = b2 + sum_j w2[j] ReLU(PH[j] + PL[j]).
__global__ void k_fp32_combine(const float *__restrict__ PH, const float *__restrict__ PL,
                               const float *__restrict__ w2, const float *__restrict__ b2, float *__restrict__ out,
                               int W, int C, int64_t nw_total, int64_t w0, int64_t slide, int Hc, int logits) {
    const int lane = threadIdx.x & 31;
    const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= (int64_t)C * W) return;
    const int64_t c = row / W;
    const int t = (int)(row - c * W);
    int64_t cl = c + slide;      // paired Livingston window (all windows resident when slides are used)
    cl %= nw_total;
    if (cl < 0) cl += nw_total;
    const float *ph = PH + row * Hc;
    const float *pl = PL + (cl * W + t) * Hc;
    float acc = 0.f;
    for (int j = lane; j < Hc; j += 32) {
        const float u = ph[j] + pl[j];
        acc = fmaf(w2[j], u > 0.f ? u : 0.f, acc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
        const float lg = acc + b2[0];
        out[(w0 + c) * W + t] = logits ? lg : 1.f / (1.f + expf(-lg));
    }
}

template <int R, int S>
void launch_layer(const float *xin, float *xout, float *skip, const float *wl, int64_t bstride, const float *win,
                  const float *sH, const float *sL, int64_t w0, int stride, int W, int C, int d, int flags,
                  cudaStream_t st, float *a_out = nullptr) {
    using Sh = LayerShape<R, S>;
    dim3 grid((W + kTM - 1) / kTM, 2 * C);
    ProfScope prof("k_fp32_layer", st);
    k_fp32_layer<R, S><<<grid, kThreads, Sh::SMEM, st>>>(xin, xout, skip, wl, bstride, win, sH, sL, w0, stride, W,
                                                         C, d, flags, a_out);
    note_launch();
}

template <int S, int HC>
void launch_headproj(const float *skip, float *proj, const float *head, int W, int C, cudaStream_t st) {
    using Sh = HeadShape<S, HC>;
    dim3 grid((W + kTM - 1) / kTM, 2 * C);
    k_fp32_headproj<S, HC><<<grid, kThreads, Sh::SMEM, st>>>(skip, proj, head, W, C);
    note_launch();
}

template <int R, int S>
cudaError_t set_layer_attr() {
    return cudaFuncSetAttribute(k_fp32_layer<R, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)LayerShape<R, S>::SMEM);
}
template <int S, int HC>
cudaError_t set_head_attr() {
    return cudaFuncSetAttribute(k_fp32_headproj<S, HC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)HeadShape<S, HC>::SMEM);
}

enum Variant { kSmall = 0, kLarge = 1, kNone = -1 };

Variant variant_of(const Dims &d) {
    if (d.k != 2) return kNone;
    if (d.R == 32 && d.S == 32 && d.Hc == 32) return kSmall;
    if (d.R == 64 && d.S == 128 && d.Hc == 256) return kLarge;
    return kNone;
}

int64_t round4(int64_t x) { return (x + 3) & ~int64_t(3); }

// The FP32 kernel layout (fp32_prepare's host loops) from the device blobs: one thread per blob
// element writes it to its place; padding stays as cleared.
struct F32Geo {
    int R, S, Hc, L, n_models;
    int64_t P, Pb, Pl, head_blob;
    int64_t layer_stride, conv_off, rs_off, bconv_off, bres_off, bskip_off, layers_off, head_off, model_stride;
};

__global__ void k_pack_fp32(const float *__restrict__ blob, F32Geo g, float *__restrict__ out) {
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= g.P * g.n_models) return;
    const int mi = (int)(gid / g.P);
    const int64_t e = gid % g.P;
    const int R = g.R, S = g.S, Hc = g.Hc;
    float *dst = out + (int64_t)mi * g.model_stride;
    const float v = blob[gid];
    if (e < 2 * g.Pb) {
        const int b = (int)(e / g.Pb);
        int64_t r = e % g.Pb;
        if (r < R) { dst[b * R + r] = v; return; }                      // w_in
        if (r < 2 * R) { dst[2 * R + b * R + (r - R)] = v; return; }    // b_in
        r -= 2 * R;
        const int l = (int)(r / g.Pl);
        int64_t q = r % g.Pl;
        float *ly = dst + g.layers_off + ((int64_t)b * g.L + l) * g.layer_stride;
        if (q < 4LL * R * R) {                                         // conv (o, tap, i)
            const int o = (int)(q / (2 * R)), tap = (int)((q / R) % 2), i = (int)(q % R);
            ly[g.conv_off + (int64_t)(tap * R + i) * 2 * R + o] = v;
            return;
        }
        if ((q -= 4LL * R * R) < 2 * R) { ly[g.bconv_off + q] = v; return; }
        if ((q -= 2 * R) < (int64_t)R * R) {                           // w_res (o, k)
            ly[g.rs_off + (q % R) * (R + S) + q / R] = v;
            return;
        }
        if ((q -= (int64_t)R * R) < R) { ly[g.bres_off + q] = v; return; }
        if ((q -= R) < (int64_t)S * R) {                               // w_skip (o, k)
            ly[g.rs_off + (q % R) * (R + S) + R + q / R] = v;
            return;
        }
        q -= (int64_t)S * R;
        ly[g.bskip_off + q] = v;
        return;
    }
    int64_t h = e - 2 * g.Pb;
    float *hd = dst + g.head_off;
    if (h < (int64_t)Hc * 2 * S) {                                     // w_h1 (j, b * S + k)
        const int j = (int)(h / (2 * S)), c = (int)(h % (2 * S));
        hd[(int64_t)c * Hc + j] = v;
        return;
    }
    h -= (int64_t)Hc * 2 * S;
    hd[2LL * S * Hc + h] = v;                                          // b_h1, w_h2, b_h2
}

}  // namespace

gwe_status fp32_repack_device(gwe_model *m, cudaStream_t st) {
    const Dims &d = m->dims;
    Fp32Weights &f = m->f32;
    if (!f.buf.ptr || f.model_stride == 0) {
        set_error("FP32 layout not prepared");
        return GWE_ERR_UNSUPPORTED;
    }
    F32Geo g;
    g.R = d.R;
    g.S = d.S;
    g.Hc = d.Hc;
    g.L = d.L;
    g.n_models = d.n_models;
    g.P = d.P;
    g.Pb = d.Pb;
    g.Pl = d.Pl;
    g.head_blob = d.head_off;
    g.layer_stride = f.layer_stride;
    g.conv_off = f.conv_off;
    g.rs_off = f.rs_off;
    g.bconv_off = f.bconv_off;
    g.bres_off = f.bres_off;
    g.bskip_off = f.bskip_off;
    g.layers_off = round4(4 * d.R);
    g.head_off = f.head_off;
    g.model_stride = f.model_stride;
    GWE_CUDA_TRY(cudaMemsetAsync(f.buf.ptr, 0, sizeof(float) * f.model_stride * d.n_models, st));
    const int64_t n = d.P * d.n_models;
    k_pack_fp32<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(m->w32.as<float>(), g, f.buf.as<float>());
    note_launch();
    GWE_CUDA_TRY(cudaGetLastError());
    return GWE_OK;
}

gwe_status fp32_prepare(gwe_model *m, const float *hb) {
    const Dims &d = m->dims;
    if (variant_of(d) == kNone) {
        set_error("FP32 path supports (R, S, Hc) = (32, 32, 32) or (64, 128, 256) with kernel 2");
        return GWE_ERR_UNSUPPORTED;
    }
    const int R = d.R, S = d.S, Hc = d.Hc, L = d.L;
    Fp32Weights &f = m->f32;
    f.conv_off = 0;
    f.rs_off = 4LL * R * R;
    f.bconv_off = f.rs_off + (int64_t)R * (R + S);
    f.bres_off = f.bconv_off + 2 * R;
    f.bskip_off = f.bres_off + R;
    f.layer_stride = round4(f.bskip_off + S);
    f.win_off = 0;
    const int64_t layers_off = round4(4 * R);
    f.head_off = layers_off + 2LL * L * f.layer_stride;
    f.model_stride = round4(f.head_off + 2LL * S * Hc + 2 * Hc + 1);
    std::vector<float> h((size_t)(f.model_stride * d.n_models), 0.f);
    for (int mi = 0; mi < d.n_models; ++mi) {
        const float *src = hb + (int64_t)mi * d.P;
        float *dst = h.data() + (int64_t)mi * f.model_stride;
        for (int b = 0; b < 2; ++b) {
            const float *bb = src + off_branch(d, b);
            for (int ch = 0; ch < R; ++ch) {
                dst[b * R + ch] = bb[ch];
                dst[2 * R + b * R + ch] = bb[R + ch];
            }
            for (int l = 0; l < L; ++l) {
                float *ly = dst + layers_off + ((int64_t)b * L + l) * f.layer_stride;
                const float *wc = src + off_wconv(d, b, l);
                for (int o = 0; o < 2 * R; ++o)
                    for (int tap = 0; tap < 2; ++tap)
                        for (int i = 0; i < R; ++i)
                            ly[f.conv_off + (int64_t)(tap * R + i) * 2 * R + o] = wc[((int64_t)o * 2 + tap) * R + i];
                const float *wr = src + off_wres(d, b, l);
                const float *ws = src + off_wskip(d, b, l);
                for (int k = 0; k < R; ++k) {
                    for (int o = 0; o < R; ++o) ly[f.rs_off + (int64_t)k * (R + S) + o] = wr[(int64_t)o * R + k];
                    for (int o = 0; o < S; ++o) ly[f.rs_off + (int64_t)k * (R + S) + R + o] = ws[(int64_t)o * R + k];
                }
                for (int o = 0; o < 2 * R; ++o) ly[f.bconv_off + o] = src[off_bconv(d, b, l) + o];
                for (int o = 0; o < R; ++o) ly[f.bres_off + o] = src[off_bres(d, b, l) + o];
                for (int o = 0; o < S; ++o) ly[f.bskip_off + o] = src[off_bskip(d, b, l) + o];
            }
        }
        float *hd = dst + f.head_off;
        const float *w1 = src + off_wh1(d);
        for (int b = 0; b < 2; ++b)
            for (int k = 0; k < S; ++k)
                for (int j = 0; j < Hc; ++j)
                    hd[((int64_t)b * S + k) * Hc + j] = w1[(int64_t)j * 2 * S + b * S + k];
        for (int j = 0; j < Hc; ++j) {
            hd[2LL * S * Hc + j] = src[off_bh1(d) + j];
            hd[2LL * S * Hc + Hc + j] = src[off_wh2(d) + j];
        }
        hd[2LL * S * Hc + 2 * Hc] = src[off_bh2(d)];
    }
    GWE_CUDA_TRY(f.buf.ensure(h.size() * sizeof(float)));
    GWE_CUDA_TRY(cudaMemcpy(f.buf.ptr, h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice));
    if (variant_of(d) == kSmall) {
        GWE_CUDA_TRY((set_layer_attr<32, 32>()));
        GWE_CUDA_TRY((set_head_attr<32, 32>()));
    } else {
        GWE_CUDA_TRY((set_layer_attr<64, 128>()));
        GWE_CUDA_TRY((set_head_attr<128, 256>()));
    }
    return GWE_OK;
}

namespace {

// one segment of nw windows; series (slide, model) of out start every out_nw windows
gwe_status fp32_forward_segment(gwe_model *m, const float *sH, const float *sL, int W, int stride, int64_t nw,
                                const int32_t *slides, int n_slides, float *out, int64_t out_nw, bool logits,
                                cudaStream_t st) {
    const Dims &d = m->dims;
    const Variant v = variant_of(d);
    if (v == kNone) {
        set_error("FP32 path: unsupported configuration");
        return GWE_ERR_UNSUPPORTED;
    }
    const int R = d.R, S = d.S, Hc = d.Hc, L = d.L;
    // With slides every Livingston window must be resident; otherwise chunk the windows.
    const int64_t chunk = (n_slides > 0) ? nw : std::min<int64_t>(nw, 128);
    GWE_ARG_CHECK(chunk * W < (int64_t)1 << 31, "too many windows for one FP32 slide pass");
    const size_t rows = (size_t)(2 * chunk) * W;
    GWE_CUDA_TRY(m->ws.x0.ensure(rows * R * sizeof(float)));
    GWE_CUDA_TRY(m->ws.x1.ensure(rows * R * sizeof(float)));
    GWE_CUDA_TRY(m->ws.skip.ensure(rows * S * sizeof(float)));
    GWE_CUDA_TRY(m->ws.proj.ensure(rows * Hc * sizeof(float)));
    const Fp32Weights &f = m->f32;
    const int ns = n_slides > 0 ? n_slides : 1;
    for (int mi = 0; mi < d.n_models; ++mi) {
        const float *wm = f.buf.as<float>() + (int64_t)mi * f.model_stride;
        const float *layers = wm + ((4 * R + 3) & ~3);
        const float *head = wm + f.head_off;
        for (int64_t w0 = 0; w0 < nw; w0 += chunk) {
            const int C = (int)std::min<int64_t>(chunk, nw - w0);
            float *xin = m->ws.x0.as<float>();
            float *xout = m->ws.x1.as<float>();
            for (int l = 0; l < L; ++l) {
                const int dl = 1 << (l % d.lps);
                const float *wl = layers + (int64_t)l * f.layer_stride;
                const int64_t bstride = (int64_t)L * f.layer_stride;
                const int flags = l == 0 ? (LF_FROM_STRAIN | LF_SKIP_INIT) : 0;
                if (v == kSmall)
                    launch_layer<32, 32>(xin, xout, m->ws.skip.as<float>(), wl, bstride, wm, sH, sL, w0, stride, W, C,
                                         dl, flags, st);
                else
                    launch_layer<64, 128>(xin, xout, m->ws.skip.as<float>(), wl, bstride, wm, sH, sL, w0, stride, W,
                                          C, dl, flags, st);
                std::swap(xin, xout);
            }
            float *proj = m->ws.proj.as<float>();
            if (v == kSmall)
                launch_headproj<32, 32>(m->ws.skip.as<float>(), proj, head, W, C, st);
            else
                launch_headproj<128, 256>(m->ws.skip.as<float>(), proj, head, W, C, st);
            const float *w2 = head + 2LL * S * Hc + Hc;
            const float *b2 = w2 + Hc;
            for (int si = 0; si < ns; ++si) {
                const int64_t k = (n_slides > 0) ? slides[si] : 0;
                float *o = out + ((int64_t)si * d.n_models + mi) * out_nw * W;
                const int64_t nrows = (int64_t)C * W;
                const int warps = 8;
                const int64_t blocks = (nrows + warps - 1) / warps;
                k_fp32_combine<<<(unsigned)blocks, warps * 32, 0, st>>>(proj, proj + (size_t)C * W * Hc, w2, b2, o, W,
                                                                         C, nw, w0, k, Hc, logits ? 1 : 0);
                note_launch();
            }
            GWE_CUDA_TRY(cudaGetLastError());
        }
    }
    return GWE_OK;
}

}  // namespace

gwe_status fp32_forward(gwe_model *m, const float *sH, const float *sL, const Segments &sg, int W, int stride,
                        const int32_t *slides, int n_slides, float *out, bool logits, cudaStream_t st) {
    const int64_t nw_all = sg.total_windows();
    int64_t wo = 0;
    for (size_t g = 0; g < sg.s0.size(); ++g) {
        if (sg.nw[g] > 0) {
            gwe_status r = fp32_forward_segment(m, sH + sg.s0[g], sL + sg.s0[g], W, stride, sg.nw[g], slides, n_slides,
                                                out + wo * W, nw_all, logits, st);
            if (r != GWE_OK) return r;
        }
        wo += sg.nw[g];
    }
    return GWE_OK;
}

// ============================================================================ activation statistics
// Largest |x_l[c]| per (model, branch, layer, channel) over a set of windows, from the FP32
// forward: the calibration the FP8 tensor-core path takes its activation scales from.
namespace {

// monotone unsigned key of a float (ordered like the float), for atomic min / max
__device__ __forceinline__ unsigned f_key(float f) {
    const unsigned u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float f_unkey(unsigned k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// keys[2b], keys[2b+1]: keys of the minimum and maximum of strain b over [0, n)
__global__ void k_strain_minmax(const float *__restrict__ sH, const float *__restrict__ sL, int64_t n,
                                unsigned *__restrict__ keys) {
    const int b = blockIdx.y;
    const float *s = b ? sL : sH;
    unsigned kmin = 0xffffffffu, kmax = 0u;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned k = f_key(s[i]);
        kmin = min(kmin, k);
        kmax = max(kmax, k);
    }
    kmin = __reduce_min_sync(0xffffffffu, kmin);
    kmax = __reduce_max_sync(0xffffffffu, kmax);
    if ((threadIdx.x & 31) == 0) {
        atomicMin(keys + 2 * b, kmin);
        atomicMax(keys + 2 * b + 1, kmax);
    }
}

// x_0 = w_in s + b_in is affine in s: its largest magnitude over the samples is taken at the
// smallest or the largest sample.  amax[b * bstride + c] (layer 0) = that maximum.
__global__ void k_amax_x0(const unsigned *__restrict__ keys, const float *__restrict__ win, int R,
                          float *__restrict__ amax, int64_t bstride) {
    const int b = blockIdx.x, c = threadIdx.x;
    if (c >= R) return;
    const float w = win[b * R + c], bi = win[2 * R + b * R + c];
    const float lo = f_unkey(keys[2 * b]), hi = f_unkey(keys[2 * b + 1]);
    const float m = fmaxf(fabsf(fmaf(w, lo, bi)), fabsf(fmaf(w, hi, bi)));
    float *a = amax + b * bstride + c;
    *a = fmaxf(*a, m);
}

// amax[b * bstride + c] = max(itself, max over the rows of branch b of |x[row][c]|)
__global__ void k_amax_cols(const float *__restrict__ x, int64_t rows_per_branch, int R, float *__restrict__ amax,
                            int64_t bstride) {
    __shared__ unsigned sh[256];
    const int b = blockIdx.y;
    const int c = threadIdx.x % R, sub = threadIdx.x / R, nsub = blockDim.x / R;
    if (threadIdx.x < R) sh[threadIdx.x] = 0u;
    __syncthreads();
    float m = 0.f;
    const float *xb = x + (int64_t)b * rows_per_branch * R;
    for (int64_t row = (int64_t)blockIdx.x * nsub + sub; row < rows_per_branch; row += (int64_t)gridDim.x * nsub)
        m = fmaxf(m, fabsf(xb[row * R + c]));
    atomicMax(sh + c, __float_as_uint(m));   // non-negative floats order like their bits
    __syncthreads();
    if (threadIdx.x < R) atomicMax(reinterpret_cast<unsigned *>(amax + b * bstride + threadIdx.x), sh[threadIdx.x]);
}

}  // namespace

gwe_status fp32_act_amax(gwe_model *m, const float *sH, const float *sL, int W, int stride, int64_t nw,
                         float *amax, unsigned *keys, cudaStream_t st) {
    const Dims &d = m->dims;
    const Variant v = variant_of(d);
    if (v == kNone) {
        set_error("FP32 path: unsupported configuration");
        return GWE_ERR_UNSUPPORTED;
    }
    const int R = d.R, L = d.L;
    const int64_t chunk = std::min<int64_t>(nw, 128);
    const size_t rows = (size_t)(2 * chunk) * W;
    GWE_CUDA_TRY(m->ws.x0.ensure(rows * R * sizeof(float)));
    GWE_CUDA_TRY(m->ws.x1.ensure(rows * R * sizeof(float)));
    const Fp32Weights &f = m->f32;
    const int64_t bstride = (int64_t)L * R;   // amax layout [model][branch][layer][channel]
    GWE_CUDA_TRY(cudaMemsetAsync(amax, 0, sizeof(float) * d.n_models * 2 * bstride, st));
    const unsigned init[4] = {0xffffffffu, 0u, 0xffffffffu, 0u};
    GWE_CUDA_TRY(cudaMemcpyAsync(keys, init, sizeof(init), cudaMemcpyHostToDevice, st));
    GWE_CUDA_TRY(cudaStreamSynchronize(st));   // `init` is pageable stack memory
    const int64_t n_used = (nw - 1) * (int64_t)stride + W;
    k_strain_minmax<<<dim3(256, 2), 256, 0, st>>>(sH, sL, n_used, keys);
    note_launch();
    for (int mi = 0; mi < d.n_models; ++mi) {
        const float *wm = f.buf.as<float>() + (int64_t)mi * f.model_stride;
        const float *layers = wm + ((4 * R + 3) & ~3);
        float *am = amax + (int64_t)mi * 2 * bstride;
        k_amax_x0<<<2, 64, 0, st>>>(keys, wm, R, am, bstride);
        note_launch();
        for (int64_t w0 = 0; w0 < nw; w0 += chunk) {
            const int C = (int)std::min<int64_t>(chunk, nw - w0);
            float *xin = m->ws.x0.as<float>();
            float *xout = m->ws.x1.as<float>();
            for (int l = 0; l + 1 < L; ++l) {
                const int dl = 1 << (l % d.lps);
                const float *wl = layers + (int64_t)l * f.layer_stride;
                const int64_t lstride = (int64_t)L * f.layer_stride;
                const int flags = (l == 0 ? LF_FROM_STRAIN : 0) | LF_NO_SKIP;
                if (v == kSmall)
                    launch_layer<32, 32>(xin, xout, nullptr, wl, lstride, wm, sH, sL, w0, stride, W, C, dl, flags, st);
                else
                    launch_layer<64, 128>(xin, xout, nullptr, wl, lstride, wm, sH, sL, w0, stride, W, C, dl, flags, st);
                const int64_t rpb = (int64_t)C * W;
                const unsigned blocks = (unsigned)std::min<int64_t>(1024, (rpb + 255) / 256);
                k_amax_cols<<<dim3(blocks, 2), 256, 0, st>>>(xout, rpb, R, am + (int64_t)(l + 1) * R, bstride);
                note_launch();
                std::swap(xin, xout);
            }
        }
        GWE_CUDA_TRY(cudaGetLastError());
    }
    return GWE_OK;
}

// ============================================================================ backward (FP32)
// Reverse-mode pass of one model over a batch of explicit windows (paper paragraph "AI ensemble
// construction": per-time-step labels, binary cross-entropy on the logits), in FP32 with
// per-stack recomputation: the forward keeps only each stack's input and the final skip sums;
// the backward re-runs one stack at a time (saving x_l and a_l of its layers) and walks it
// backwards.  Per layer (dilation d), rows t of one window, with dskip the gradient of the skip
// sum (the same for every layer of the branch):
//   dz    = W_res^T dx_{l+1} + W_skip^T dskip
//   da_f  = dz s (1 - tanh(f)^2),  da_g = dz tanh(f) s (1 - s),  s = sigmoid(g)
//   dx_l  = dx_{l+1} + W1^T da(t) + W0^T da(t + d)      (zero beyond the window end)
//   dW0  += da(t) x_l(t - d)^T, dW1 += da(t) x_l(t)^T, dW_res += dx_{l+1} z^T, dW_skip += dskip z^T
// and the biases take the column sums.  Weight gradients are reduced over rows in blocks that
// each own a slice of rows, then added atomically (summation order is not fixed).
namespace {

constexpr int BT = 64;   // rows and columns per block tile
constexpr int BK = 32;   // K slice staged in shared memory

struct BSrc {
    const float *A;      // A[row][k] of branch 0; branch b adds b * a_boff
    int lda;
    int shift;           // use row t + shift of the same window (zero outside [0, W))
    int relu;            // apply ReLU to A on load
    const float *Wt;     // Wt[k][n] of branch 0; branch b adds b * w_boff
    int ldw;
    int K;
};

struct BRows {
    BSrc s[2];
    int nsrc;
    int N;               // output columns
    int W, C;            // window length; windows per branch (grid.y = nbranch * C)
    int64_t a_boff, w_boff, y_boff;   // per-branch offsets (elements)
    float *Y;            // output [row][ldy] of branch 0
    int ldy;
    // epilogue operands
    const float *aux0;   // EP_DZ: a [row][2R]; EP_ADD: residual [row][N]; EP_HEAD_U: b1; EP_HEAD_DH: skip (both branches)
    const float *aux1;   // EP_HEAD_U: w2
    const float *aux2;   // EP_HEAD_U: dlogit [row]
    float *out1;         // EP_DZ: z [row][R]; EP_HEAD_U: ReLU(u) [row][N]; EP_HEAD_DH: dskip (both branches)
    int64_t aux_boff;    // per-branch offset of aux0 / out1 rows (EP_DZ) or branch block size (EP_HEAD_DH)
};

enum { EP_DZ = 0, EP_ADD = 1, EP_HEAD_U = 2, EP_HEAD_DH = 3 };

__device__ __forceinline__ float sigm_f(float x) { return 1.f / (1.f + expf(-x)); }

template <int EP>
__global__ void __launch_bounds__(256) k_bwd_rows(const BRows p) {
    __shared__ float As[BK][BT + 1];
    __shared__ float Ws[BK][BT];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int bw = blockIdx.y, b = bw / p.C;
    const int t0 = blockIdx.x * BT, n0 = blockIdx.z * BT;
    const int64_t row0 = (int64_t)(bw - b * p.C) * p.W;   // first row of this window within its branch
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    for (int si = 0; si < p.nsrc; ++si) {
        const BSrc &sc = p.s[si];
        const float *A = sc.A + b * p.a_boff;
        const float *Wt = sc.Wt + b * p.w_boff;
        for (int k0 = 0; k0 < sc.K; k0 += BK) {
            for (int i = tid; i < BT * BK; i += 256) {
                const int r = i / BK, k = i - r * BK, t = t0 + r + sc.shift;
                float v = 0.f;
                if (t >= 0 && t < p.W && k0 + k < sc.K) v = A[(row0 + t) * sc.lda + k0 + k];
                if (sc.relu) v = fmaxf(v, 0.f);
                As[k][r] = v;
            }
            for (int i = tid; i < BK * BT; i += 256) {
                const int k = i / BT, n = i - k * BT;
                Ws[k][n] = (k0 + k < sc.K && n0 + n < p.N) ? Wt[(int64_t)(k0 + k) * sc.ldw + n0 + n] : 0.f;
            }
            __syncthreads();
#pragma unroll 8
            for (int k = 0; k < BK; ++k) {
                float a[4], w[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) a[i] = As[k][ty + 16 * i];
#pragma unroll
                for (int j = 0; j < 4; ++j) w[j] = Ws[k][tx + 16 * j];
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], w[j], acc[i][j]);
            }
            __syncthreads();
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int t = t0 + ty + 16 * i;
        if (t >= p.W) continue;
        const int64_t row = row0 + t;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = n0 + tx + 16 * j;
            if (n >= p.N) continue;
            const float v = acc[i][j];
            if (EP == EP_DZ) {
                // n is a residual channel c (N = R); a holds [f | g] per row
                const int R = p.N;
                const float *a = p.aux0 + b * p.aux_boff * 2 + row * 2 * R;
                const float f = a[n], g = a[R + n];
                const float th = tanhf(f), sg = sigm_f(g);
                float *da = p.Y + b * p.y_boff + row * p.ldy;
                da[n] = v * sg * (1.f - th * th);
                da[R + n] = v * th * sg * (1.f - sg);
                p.out1[b * p.aux_boff + row * R + n] = th * sg;
            } else if (EP == EP_ADD) {
                p.Y[b * p.y_boff + row * p.ldy + n] = v + p.aux0[b * p.y_boff + row * p.ldy + n];
            } else if (EP == EP_HEAD_U) {
                const float u = v + p.aux0[n];
                const float dl = p.aux2[row];
                p.Y[row * p.ldy + n] = (u > 0.f) ? dl * p.aux1[n] : 0.f;
                p.out1[row * p.ldy + n] = fmaxf(u, 0.f);
            } else {   // EP_HEAD_DH: n < 2S -> branch n / S, skip channel n % S
                const int S = p.N / 2;
                const int bb = n / S, ch = n - bb * S;
                const int64_t idx = bb * p.aux_boff + row * S + ch;
                p.out1[idx] = (p.aux0[idx] > 0.f) ? v : 0.f;
            }
        }
    }
}

// dW[n][k] += sum_r G(r)[n] X(r)[k] (X optional) and db[n] += sum_r G(r)[n] (db optional), over
// the rows of each branch; X(r) is row t + shift of the same window (zero outside [0, W)).
struct BWg {
    const float *G; int ldg; int N; int64_t g_boff;
    const float *X; int ldx; int K; int shift; int xrelu; int64_t x_boff;
    float *dW; int ldw; int64_t w_boff;
    float *db; int64_t db_boff;
    int W, C, splits;
};

__global__ void __launch_bounds__(256) k_wgrad(const BWg p) {
    __shared__ float Gs[BK][BT];
    __shared__ float Xs[BK][BT];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int b = blockIdx.z / p.splits, sp = blockIdx.z - b * p.splits;
    const int k0 = blockIdx.x * BT, n0 = blockIdx.y * BT;
    const int64_t rows = (int64_t)p.C * p.W;
    const int64_t chunk = (rows + p.splits - 1) / p.splits;
    const int64_t r_begin = sp * chunk, r_end = min(rows, r_begin + chunk);
    const float *G = p.G + b * p.g_boff;
    const float *X = p.X ? p.X + b * p.x_boff : nullptr;
    const bool do_bias = p.db && blockIdx.x == 0;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    float bacc = 0.f;
    for (int64_t r0 = r_begin; r0 < r_end; r0 += BK) {
        for (int i = tid; i < BK * BT; i += 256) {
            const int r = i / BT, c = i - r * BT;
            const int64_t row = r0 + r;
            float gv = 0.f, xv = 0.f;
            if (row < r_end) {
                if (n0 + c < p.N) gv = G[row * p.ldg + n0 + c];
                if (X && k0 + c < p.K) {
                    const int64_t w = row / p.W;
                    const int t = (int)(row - w * p.W) + p.shift;
                    if (t >= 0 && t < p.W) xv = X[(w * p.W + t) * p.ldx + k0 + c];
                    if (p.xrelu) xv = fmaxf(xv, 0.f);
                }
            }
            Gs[r][c] = gv;
            Xs[r][c] = xv;
        }
        __syncthreads();
        if (X) {
#pragma unroll 8
            for (int r = 0; r < BK; ++r) {
                float g[4], x[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) g[i] = Gs[r][ty + 16 * i];
#pragma unroll
                for (int j = 0; j < 4; ++j) x[j] = Xs[r][tx + 16 * j];
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(g[i], x[j], acc[i][j]);
            }
        }
        if (do_bias && tid < BT)
            for (int r = 0; r < BK; ++r) bacc += Gs[r][tid];
        __syncthreads();
    }
    if (X) {
        float *dW = p.dW + b * p.w_boff;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int n = n0 + ty + 16 * i;
            if (n >= p.N) continue;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int k = k0 + tx + 16 * j;
                if (k < p.K) atomicAdd(dW + (int64_t)n * p.ldw + k, acc[i][j]);
            }
        }
    }
    if (do_bias && tid < BT && n0 + tid < p.N) atomicAdd(p.db + b * p.db_boff + n0 + tid, bacc);
}

// Weighted column sums of a row-major FP32 matrix, for the reductions with few outputs (dw_h2 and
// db_h2; the input projection's gradients): out_w[n] += sum_r G[r][n] x[r], out_b[n] += sum_r G[r][n],
// out_x += sum_r x[r] (each output optional), N a multiple of 4 up to 256, rows of G 16-byte aligned.
// 256 threads = row lanes x N/4 float4 columns; a block sums a contiguous range of rows (loads of
// several rows in flight per thread), adds its row lanes in shared memory and issues one atomic per
// output.
__global__ void __launch_bounds__(256) k_colsum(const float *__restrict__ G, int ldg, int N, const float *__restrict__ x,
                                                int64_t rows, int64_t rows_per_block, float *out_w, float *out_b,
                                                float *out_x) {
    __shared__ float4 sw[256], sb[256];
    __shared__ float sx[256];
    const int NQ = N / 4, RP = 256 / NQ;
    const int tid = threadIdx.x, q = tid % NQ, rl = tid / NQ;
    const int64_t r0 = (int64_t)blockIdx.x * rows_per_block, r1 = min(rows, r0 + rows_per_block);
    float4 aw = make_float4(0.f, 0.f, 0.f, 0.f), ab = aw;
    float ax = 0.f;
    if (rl < RP) {
#pragma unroll 4
        for (int64_t r = r0 + rl; r < r1; r += RP) {
            const float4 g = __ldg(reinterpret_cast<const float4 *>(G + r * ldg) + q);
            const float xv = x ? __ldg(x + r) : 0.f;
            aw.x = fmaf(g.x, xv, aw.x);
            aw.y = fmaf(g.y, xv, aw.y);
            aw.z = fmaf(g.z, xv, aw.z);
            aw.w = fmaf(g.w, xv, aw.w);
            ab.x += g.x;
            ab.y += g.y;
            ab.z += g.z;
            ab.w += g.w;
            ax += xv;
        }
    }
    sw[tid] = aw;
    sb[tid] = ab;
    sx[tid] = (rl < RP && q == 0) ? ax : 0.f;
    __syncthreads();
    if (tid < NQ) {
        float4 w = sw[tid], bsum = sb[tid];
        for (int k = 1; k < RP; ++k) {
            const float4 a = sw[k * NQ + tid], c = sb[k * NQ + tid];
            w.x += a.x;
            w.y += a.y;
            w.z += a.z;
            w.w += a.w;
            bsum.x += c.x;
            bsum.y += c.y;
            bsum.z += c.z;
            bsum.w += c.w;
        }
        if (out_w) {
            atomicAdd(out_w + 4 * tid, w.x);
            atomicAdd(out_w + 4 * tid + 1, w.y);
            atomicAdd(out_w + 4 * tid + 2, w.z);
            atomicAdd(out_w + 4 * tid + 3, w.w);
        }
        if (out_b) {
            atomicAdd(out_b + 4 * tid, bsum.x);
            atomicAdd(out_b + 4 * tid + 1, bsum.y);
            atomicAdd(out_b + 4 * tid + 2, bsum.z);
            atomicAdd(out_b + 4 * tid + 3, bsum.w);
        }
    }
    if (out_x && tid == 0) {
        float t = 0.f;
        for (int k = 0; k < RP; ++k) t += sx[k * NQ];
        atomicAdd(out_x, t);
    }
}

// x_0 = w_in s + b_in for both branches; rows of branch b follow branch b-1
__global__ void k_input_proj(const float *__restrict__ sH, const float *__restrict__ sL,
                             const float *__restrict__ blob, int64_t Pb, int R, int64_t rows, float *__restrict__ x0) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 2 * rows * R) return;
    const int64_t row = i / R;
    const int c = (int)(i - row * R);
    const int b = row >= rows;
    const float s = b ? sL[row - rows] : sH[row];
    const float *w = blob + b * Pb;
    x0[i] = fmaf(w[c], s, w[R + c]);
}

// ds[t] = sum_c w_in[c] dx_0[t][c]
__global__ void k_dstrain(const float *__restrict__ dx0, const float *__restrict__ w_in, int R, int64_t rows,
                          float *__restrict__ ds) {
    const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= rows) return;
    float acc = 0.f;
    for (int c = lane; c < R; c += 32) acc = fmaf(w_in[c], dx0[row * R + c], acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) ds[row] = acc;
}

template <int EP>
void launch_rows(const BRows &p, int nbranch, cudaStream_t st) {
    dim3 grid((p.W + BT - 1) / BT, nbranch * p.C, (p.N + BT - 1) / BT);
    k_bwd_rows<EP><<<grid, 256, 0, st>>>(p);
    note_launch();
}

void launch_wgrad(const BWg &p, int nbranch, cudaStream_t st) {
    const int kt = p.X ? (p.K + BT - 1) / BT : 1;
    dim3 grid(kt, (p.N + BT - 1) / BT, p.splits * nbranch);
    ProfScope prof("k_wgrad", st);
    k_wgrad<<<grid, 256, 0, st>>>(p);
    note_launch();
}

// k_colsum where the shapes allow it (N a multiple of 4 up to 256, 16-byte aligned rows); false otherwise
bool launch_colsum(const float *G, int ldg, int N, const float *x, int64_t rows, float *out_w, float *out_b,
                   float *out_x, cudaStream_t st) {
    if (N <= 0 || N % 4 || N > 256 || ldg % 4 || (reinterpret_cast<uintptr_t>(G) & 15) || rows <= 0) return false;
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>(1024, rows / 512));
    const int64_t rpb = (rows + blocks - 1) / blocks;
    ProfScope prof("k_wgrad", st);
    k_colsum<<<(unsigned)blocks, 256, 0, st>>>(G, ldg, N, x, rows, rpb, out_w, out_b, out_x);
    note_launch();
    return true;
}

BWg wg(const float *G, int ldg, int N, int64_t g_boff, const float *X, int ldx, int K, int shift, int64_t x_boff,
       float *dW, int ldw, int64_t w_boff, float *db, int64_t db_boff, int W, int C) {
    BWg p;
    p.G = G; p.ldg = ldg; p.N = N; p.g_boff = g_boff;
    p.X = X; p.ldx = ldx; p.K = K; p.shift = shift; p.xrelu = 0; p.x_boff = x_boff;
    p.dW = dW; p.ldw = ldw; p.w_boff = w_boff;
    p.db = db; p.db_boff = db_boff;
    p.W = W; p.C = C;
    const int64_t rows = (int64_t)C * W;
    p.splits = (int)std::max<int64_t>(1, std::min<int64_t>(64, rows / 2048));
    return p;
}

// Reductions with one or a few outputs (K <= 1, N <= 256: dw_h2, db_h2, the input projection's
// gradients) have too few tiles for the default 64 row splits to fill the GPU: split the rows into
// up to 1024 ranges of at least 512 rows (each adds its partial sums atomically).
BWg wide(BWg p) {
    const int64_t rows = (int64_t)p.C * p.W;
    p.splits = (int)std::max<int64_t>(1, std::min<int64_t>(1024, rows / 512));
    return p;
}

BSrc src(const float *A, int lda, int shift, int relu, const float *Wt, int ldw, int K) {
    BSrc s;
    s.A = A; s.lda = lda; s.shift = shift; s.relu = relu; s.Wt = Wt; s.ldw = ldw; s.K = K;
    return s;
}

}  // namespace

namespace {

struct BwdWs {
    DevBuf xsave, xrec, arec, skip, dskip, dxa, dxb, da, z, ru, du, dummy;
};

}  // namespace

void fp32_backward_release(gwe_model *m) {
    BwdWs *w = reinterpret_cast<BwdWs *>(m->bwd);
    if (!w) return;
    DevBuf *all[] = {&w->xsave, &w->xrec, &w->arec, &w->skip, &w->dskip, &w->dxa, &w->dxb, &w->da, &w->z, &w->ru,
                     &w->du, &w->dummy};
    for (DevBuf *b : all) b->release();
    delete w;
    m->bwd = nullptr;
}

// Pieces of the backward pass shared with the tensor-core backward (bwd_tc.cu): the head, the
// bias sums, the input projection and its backward.  Arrays hold both branches, branch 1 after
// branch 0 (rb rows each).
gwe_status fp32_input_proj(gwe_model *m, int mi, const float *sH, const float *sL, int64_t rb, float *x0,
                           cudaStream_t st) {
    const Dims &d = m->dims;
    const float *blob = m->w32.as<float>() + (int64_t)mi * d.P;
    const int64_t n = 2 * rb * d.R;
    k_input_proj<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(sH, sL, blob, d.Pb, d.R, rb, x0);
    note_launch();
    GWE_CUDA_TRY(cudaGetLastError());
    return GWE_OK;
}

gwe_status fp32_head_backward(gwe_model *m, int mi, const float *skip, int64_t rb, int W, int C, const float *dlogit,
                              float *dskip, float *gw, cudaStream_t st) {
    const Dims &d = m->dims;
    const int S = d.S, Hc = d.Hc;
    BwdWs *w = reinterpret_cast<BwdWs *>(m->bwd);
    if (!w) {
        w = new BwdWs();
        m->bwd = w;
    }
    GWE_CUDA_TRY(w->ru.ensure(sizeof(float) * rb * Hc));
    GWE_CUDA_TRY(w->du.ensure(sizeof(float) * rb * Hc));
    float *ru = w->ru.as<float>(), *du = w->du.as<float>();
    const float *blob = m->w32.as<float>() + (int64_t)mi * d.P;
    const Fp32Weights &f = m->f32;
    const float *head = f.buf.as<float>() + (int64_t)mi * f.model_stride + f.head_off;
    BRows p{};
    p.nsrc = 2;
    p.s[0] = src(skip, S, 0, 1, head, Hc, S);
    p.s[1] = src(skip + rb * S, S, 0, 1, head + (int64_t)S * Hc, Hc, S);
    p.N = Hc; p.W = W; p.C = C;
    p.Y = du; p.ldy = Hc;
    p.aux0 = blob + off_bh1(d); p.aux1 = blob + off_wh2(d); p.aux2 = dlogit;
    p.out1 = ru;
    launch_rows<EP_HEAD_U>(p, 1, st);
    BRows q{};
    q.nsrc = 1;
    q.s[0] = src(du, Hc, 0, 0, blob + off_wh1(d), 2 * S, Hc);
    q.N = 2 * S; q.W = W; q.C = C;
    q.aux0 = skip; q.out1 = dskip; q.aux_boff = rb * S;
    launch_rows<EP_HEAD_DH>(q, 1, st);
    float *g1 = gw + off_wh1(d);
    BWg p1 = wg(du, Hc, Hc, 0, skip, S, S, 0, 0, g1, 2 * S, 0, gw + off_bh1(d), 0, W, C);
    p1.xrelu = 1;
    launch_wgrad(p1, 1, st);
    BWg p2 = wg(du, Hc, Hc, 0, skip + rb * S, S, S, 0, 0, g1 + S, 2 * S, 0, nullptr, 0, W, C);
    p2.xrelu = 1;
    launch_wgrad(p2, 1, st);
    launch_wgrad(wide(wg(ru, Hc, Hc, 0, dlogit, 1, 1, 0, 0, gw + off_wh2(d), 1, 0, nullptr, 0, W, C)), 1, st);
    launch_wgrad(wide(wg(dlogit, 1, 1, 0, nullptr, 0, 0, 0, 0, nullptr, 0, 0, gw + off_bh2(d), 0, W, C)), 1, st);
    GWE_CUDA_TRY(cudaGetLastError());
    return GWE_OK;
}

// the head's second layer: dw_h2 = sum over rows of dlogit ReLU(u + b_h1), db_h2 = sum of dlogit
// (ru = ReLU(u + b_h1) [row][Hc]; one pass over ru, or one launch each for widths k_colsum does not take)
gwe_status fp32_head_w2_grad(gwe_model *m, const float *ru, int W, int C, const float *dlogit, float *gw,
                             cudaStream_t st) {
    const Dims &d = m->dims;
    const int Hc = d.Hc;
    if (!launch_colsum(ru, Hc, Hc, dlogit, (int64_t)C * W, gw + off_wh2(d), nullptr, gw + off_bh2(d), st)) {
        launch_wgrad(wide(wg(ru, Hc, Hc, 0, dlogit, 1, 1, 0, 0, gw + off_wh2(d), 1, 0, nullptr, 0, W, C)), 1, st);
        launch_wgrad(wide(wg(dlogit, 1, 1, 0, nullptr, 0, 0, 0, 0, nullptr, 0, 0, gw + off_bh2(d), 0, W, C)), 1, st);
    }
    GWE_CUDA_TRY(cudaGetLastError());
    return GWE_OK;
}

gwe_status fp32_bias_grad(const float *G, int ldg, int N, int64_t g_boff, float *db, int64_t db_boff, int W, int C,
                          int nbranch, cudaStream_t st) {
    launch_wgrad(wg(G, ldg, N, g_boff, nullptr, 0, 0, 0, 0, nullptr, 0, 0, db, db_boff, W, C), nbranch, st);
    GWE_CUDA_TRY(cudaGetLastError());
    return GWE_OK;
}

gwe_status fp32_input_backward(gwe_model *m, int mi, const float *dx0, int64_t rb, const float *sH, const float *sL,
                               int W, int C, float *gw, float *gH, float *gL, cudaStream_t st) {
    const Dims &d = m->dims;
    const int R = d.R;
    const float *blob = m->w32.as<float>() + (int64_t)mi * d.P;
    // dw_in = sum_r dx_0[r] s[r], db_in = sum_r dx_0[r], per branch
    if (!launch_colsum(dx0, R, R, sH, rb, gw + off_branch(d, 0), gw + off_branch(d, 0) + R, nullptr, st))
        launch_wgrad(wide(wg(dx0, R, R, 0, sH, 1, 1, 0, 0, gw + off_branch(d, 0), 1, 0, gw + off_branch(d, 0) + R, 0,
                             W, C)),
                     1, st);
    if (!launch_colsum(dx0 + rb * R, R, R, sL, rb, gw + off_branch(d, 1), gw + off_branch(d, 1) + R, nullptr, st))
        launch_wgrad(wide(wg(dx0 + rb * R, R, R, 0, sL, 1, 1, 0, 0, gw + off_branch(d, 1), 1, 0,
                             gw + off_branch(d, 1) + R, 0, W, C)),
                     1, st);
    const unsigned nb = (unsigned)((rb + 7) / 8);
    if (gH) {
        k_dstrain<<<nb, 256, 0, st>>>(dx0, blob + off_branch(d, 0), R, rb, gH);
        note_launch();
    }
    if (gL) {
        k_dstrain<<<nb, 256, 0, st>>>(dx0 + rb * R, blob + off_branch(d, 1), R, rb, gL);
        note_launch();
    }
    GWE_CUDA_TRY(cudaGetLastError());
    return GWE_OK;
}

gwe_status fp32_backward(gwe_model *m, int mi, const float *xH, const float *xL, int batch, int W,
                         const float *dlogit, float *gw, float *gH, float *gL, cudaStream_t st) {
    const Dims &d = m->dims;
    const Variant v = variant_of(d);
    if (v == kNone) {
        set_error("backward: unsupported configuration");
        return GWE_ERR_UNSUPPORTED;
    }
    const int R = d.R, S = d.S, Hc = d.Hc, L = d.L, lps = d.lps, stacks = d.stacks;
    BwdWs *w = reinterpret_cast<BwdWs *>(m->bwd);
    if (!w) {
        w = new BwdWs();
        m->bwd = w;
    }
    const int C = std::min(batch, 16);                       // windows per chunk
    const size_t rows = (size_t)C * W, rows2 = 2 * rows;      // per branch, both branches
    GWE_CUDA_TRY(w->xsave.ensure(sizeof(float) * stacks * rows2 * R));
    GWE_CUDA_TRY(w->xrec.ensure(sizeof(float) * (lps + 1) * rows2 * R));
    GWE_CUDA_TRY(w->arec.ensure(sizeof(float) * lps * rows2 * 2 * R));
    GWE_CUDA_TRY(w->skip.ensure(sizeof(float) * rows2 * S));
    GWE_CUDA_TRY(w->dskip.ensure(sizeof(float) * rows2 * S));
    GWE_CUDA_TRY(w->dxa.ensure(sizeof(float) * rows2 * R));
    GWE_CUDA_TRY(w->dxb.ensure(sizeof(float) * rows2 * R));
    GWE_CUDA_TRY(w->da.ensure(sizeof(float) * rows2 * 2 * R));
    GWE_CUDA_TRY(w->z.ensure(sizeof(float) * rows2 * R));
    GWE_CUDA_TRY(w->ru.ensure(sizeof(float) * rows * Hc));
    GWE_CUDA_TRY(w->du.ensure(sizeof(float) * rows * Hc));
    GWE_CUDA_TRY(w->dummy.ensure(sizeof(float) * 64));
    GWE_CUDA_TRY(cudaMemsetAsync(gw, 0, sizeof(float) * d.P, st));

    const float *blob = m->w32.as<float>() + (int64_t)mi * d.P;          // FP32 weights, blob layout
    const Fp32Weights &f = m->f32;
    const float *wm = f.buf.as<float>() + (int64_t)mi * f.model_stride;   // FP32 kernel layout
    const float *layers = wm + ((4 * R + 3) & ~3);
    const float *head = wm + f.head_off;
    const int64_t bstride = (int64_t)L * f.layer_stride;
    float *xsave = w->xsave.as<float>(), *xrec = w->xrec.as<float>(), *arec = w->arec.as<float>();
    float *skip = w->skip.as<float>(), *dskip = w->dskip.as<float>();
    float *da = w->da.as<float>(), *z = w->z.as<float>(), *ru = w->ru.as<float>(), *du = w->du.as<float>();
    const int64_t Pb = d.Pb;

    for (int c0 = 0; c0 < batch; c0 += C) {
        const int Cc = std::min(C, batch - c0);
        const int64_t rb = (int64_t)Cc * W;      // rows per branch in this chunk
        const float *sH = xH + (int64_t)c0 * W, *sL = xL + (int64_t)c0 * W;
        // ---- forward, keeping each stack's input and the final skip sums
        {
            float *xa = xrec, *xb = xrec + rows2 * R;
            const int64_t n = 2 * rb * R;
            k_input_proj<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(sH, sL, blob, Pb, R, rb, xa);
            note_launch();
            for (int l = 0; l < L; ++l) {
                if (l % lps == 0)
                    GWE_CUDA_TRY(cudaMemcpyAsync(xsave + (size_t)(l / lps) * rows2 * R, xa, sizeof(float) * 2 * rb * R,
                                                 cudaMemcpyDeviceToDevice, st));
                const float *wl = layers + (int64_t)l * f.layer_stride;
                const int flags = (l == 0) ? LF_SKIP_INIT : 0;
                if (v == kSmall)
                    launch_layer<32, 32>(xa, xb, skip, wl, bstride, wm, sH, sL, 0, W, W, Cc, 1 << (l % lps), flags, st);
                else
                    launch_layer<64, 128>(xa, xb, skip, wl, bstride, wm, sH, sL, 0, W, W, Cc, 1 << (l % lps), flags, st);
                std::swap(xa, xb);
            }
        }
        // ---- head: u = W1 [ReLU(s_H); ReLU(s_L)] + b1, du = dlogit w2 [u > 0]; dskip
        {
            BRows p{};
            p.nsrc = 2;
            p.s[0] = src(skip, S, 0, 1, head, Hc, S);                          // W1t rows of branch H
            p.s[1] = src(skip + rb * S, S, 0, 1, head + (int64_t)S * Hc, Hc, S); // branch L
            p.N = Hc; p.W = W; p.C = Cc;
            p.Y = du; p.ldy = Hc;
            p.aux0 = blob + off_bh1(d); p.aux1 = blob + off_wh2(d); p.aux2 = dlogit + (int64_t)c0 * W;
            p.out1 = ru;
            launch_rows<EP_HEAD_U>(p, 1, st);
            BRows q{};
            q.nsrc = 1;
            q.s[0] = src(du, Hc, 0, 0, blob + off_wh1(d), 2 * S, Hc);
            q.N = 2 * S; q.W = W; q.C = Cc;
            q.aux0 = skip; q.out1 = dskip; q.aux_boff = rb * S;
            launch_rows<EP_HEAD_DH>(q, 1, st);
            // dW1[:, branch half] = sum_r du[r] ReLU(s_branch[r])^T, db1 = sum_r du[r]
            float *g1 = gw + off_wh1(d);
            BWg p1 = wg(du, Hc, Hc, 0, skip, S, S, 0, 0, g1, 2 * S, 0, gw + off_bh1(d), 0, W, Cc);
            p1.xrelu = 1;
            launch_wgrad(p1, 1, st);
            BWg p2 = wg(du, Hc, Hc, 0, skip + rb * S, S, S, 0, 0, g1 + S, 2 * S, 0, nullptr, 0, W, Cc);
            p2.xrelu = 1;
            launch_wgrad(p2, 1, st);
            // dw2[j] = sum_r ReLU(u)[r][j] dlogit[r]; db2 = sum_r dlogit[r]
            launch_wgrad(wg(ru, Hc, Hc, 0, dlogit + (int64_t)c0 * W, 1, 1, 0, 0, gw + off_wh2(d), 1, 0, nullptr, 0, W, Cc),
                         1, st);
            launch_wgrad(wg(dlogit + (int64_t)c0 * W, 1, 1, 0, nullptr, 0, 0, 0, 0, nullptr, 0, 0, gw + off_bh2(d), 0, W,
                            Cc), 1, st);
        }
        // ---- branches, stack by stack in reverse, recomputing each stack from its input
        float *dx_hi = w->dxa.as<float>(), *dx_lo = w->dxb.as<float>();   // dL/dx_{l+1}, dL/dx_l
        GWE_CUDA_TRY(cudaMemsetAsync(dx_hi, 0, sizeof(float) * 2 * rb * R, st));
        const int64_t xb_off = rb * R;               // branch offsets in [branch][rows][C] arrays
        for (int k = stacks - 1; k >= 0; --k) {
            GWE_CUDA_TRY(cudaMemcpyAsync(xrec, xsave + (size_t)k * rows2 * R, sizeof(float) * 2 * rb * R,
                                         cudaMemcpyDeviceToDevice, st));
            for (int j = 0; j < lps; ++j) {
                const int l = k * lps + j;
                const float *wl = layers + (int64_t)l * f.layer_stride;
                float *xin = xrec + (size_t)j * rows2 * R, *xout = xrec + (size_t)(j + 1) * rows2 * R;
                float *aout = arec + (size_t)j * rows2 * 2 * R;
                if (v == kSmall)
                    launch_layer<32, 32>(xin, xout, w->dummy.as<float>(), wl, bstride, wm, sH, sL, 0, W, W, Cc, 1 << j,
                                         LF_NO_SKIP, st, aout);
                else
                    launch_layer<64, 128>(xin, xout, w->dummy.as<float>(), wl, bstride, wm, sH, sL, 0, W, W, Cc, 1 << j,
                                          LF_NO_SKIP, st, aout);
            }
            for (int j = lps - 1; j >= 0; --j) {
                const int l = k * lps + j, dl = 1 << j;
                const float *xl = xrec + (size_t)j * rows2 * R;
                const float *al = arec + (size_t)j * rows2 * 2 * R;
                // dz and the gate backward -> da, z
                BRows p{};
                p.nsrc = 2;
                p.s[0] = src(dx_hi, R, 0, 0, blob + off_wres(d, 0, l), R, R);
                p.s[1] = src(dskip, S, 0, 0, blob + off_wskip(d, 0, l), R, S);
                p.N = R; p.W = W; p.C = Cc;
                p.a_boff = 0; p.w_boff = Pb; p.y_boff = rb * 2 * R;
                p.Y = da; p.ldy = 2 * R;
                p.aux0 = al; p.out1 = z; p.aux_boff = rb * R;
                // per-branch A offsets differ between the two sources; run one branch per launch
                for (int b = 0; b < 2; ++b) {
                    BRows pb = p;
                    pb.s[0].A = dx_hi + b * xb_off;
                    pb.s[1].A = dskip + b * rb * S;
                    pb.s[0].Wt = blob + off_wres(d, b, l);
                    pb.s[1].Wt = blob + off_wskip(d, b, l);
                    pb.w_boff = 0;
                    pb.Y = da + b * rb * 2 * R; pb.y_boff = 0;
                    pb.aux0 = al + b * rb * 2 * R; pb.out1 = z + b * rb * R; pb.aux_boff = 0;
                    launch_rows<EP_DZ>(pb, 1, st);
                }
                // weight gradients of this layer (both branches: offsets per branch)
                launch_wgrad(wg(dx_hi, R, R, xb_off, z, R, R, 0, rb * R, gw + off_wres(d, 0, l), R, Pb,
                                gw + off_bres(d, 0, l), Pb, W, Cc), 2, st);
                launch_wgrad(wg(dskip, S, S, rb * S, z, R, R, 0, rb * R, gw + off_wskip(d, 0, l), R, Pb,
                                gw + off_bskip(d, 0, l), Pb, W, Cc), 2, st);
                launch_wgrad(wg(da, 2 * R, 2 * R, rb * 2 * R, xl, R, R, -dl, rb * R, gw + off_wconv(d, 0, l), 2 * R, Pb,
                                gw + off_bconv(d, 0, l), Pb, W, Cc), 2, st);
                launch_wgrad(wg(da, 2 * R, 2 * R, rb * 2 * R, xl, R, R, 0, rb * R, gw + off_wconv(d, 0, l) + R, 2 * R, Pb,
                                nullptr, 0, W, Cc), 2, st);
                // dx_l = dx_{l+1} + W1^T da(t) + W0^T da(t + d)
                BRows q{};
                q.nsrc = 2;
                q.s[0] = src(da, 2 * R, 0, 0, blob + off_wconv(d, 0, l) + R, 2 * R, 2 * R);
                q.s[1] = src(da, 2 * R, dl, 0, blob + off_wconv(d, 0, l), 2 * R, 2 * R);
                q.N = R; q.W = W; q.C = Cc;
                q.a_boff = rb * 2 * R; q.w_boff = Pb; q.y_boff = rb * R;
                q.Y = dx_lo; q.ldy = R; q.aux0 = dx_hi;
                launch_rows<EP_ADD>(q, 2, st);
                std::swap(dx_hi, dx_lo);
            }
        }
        // ---- input projection: dw_in, db_in and dL/dstrain
        {
            launch_wgrad(wg(dx_hi, R, R, 0, sH, 1, 1, 0, 0, gw + off_branch(d, 0), 1, 0, gw + off_branch(d, 0) + R, 0,
                            W, Cc), 1, st);
            launch_wgrad(wg(dx_hi + xb_off, R, R, 0, sL, 1, 1, 0, 0, gw + off_branch(d, 1), 1, 0,
                            gw + off_branch(d, 1) + R, 0, W, Cc), 1, st);
            const unsigned nb = (unsigned)((rb + 7) / 8);
            if (gH) {
                k_dstrain<<<nb, 256, 0, st>>>(dx_hi, blob + off_branch(d, 0), R, rb, gH + (int64_t)c0 * W);
                note_launch();
            }
            if (gL) {
                k_dstrain<<<nb, 256, 0, st>>>(dx_hi + xb_off, blob + off_branch(d, 1), R, rb, gL + (int64_t)c0 * W);
                note_launch();
            }
        }
        GWE_CUDA_TRY(cudaGetLastError());
    }
    return GWE_OK;
}

}  // namespace gwe
