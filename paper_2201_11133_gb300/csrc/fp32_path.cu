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
             int C, int d, int first) {
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
            } else {
                float *sp = skip + (xrow0 + t) * S + (col - R);
                *sp = first ? acc2[i][j] : (*sp + acc2[i][j]);
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
                  const float *sH, const float *sL, int64_t w0, int stride, int W, int C, int d, int first,
                  cudaStream_t st) {
    using Sh = LayerShape<R, S>;
    dim3 grid((W + kTM - 1) / kTM, 2 * C);
    ProfScope prof("k_fp32_layer", st);
    k_fp32_layer<R, S><<<grid, kThreads, Sh::SMEM, st>>>(xin, xout, skip, wl, bstride, win, sH, sL, w0, stride, W,
                                                         C, d, first);
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

}  // namespace

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

gwe_status fp32_forward(gwe_model *m, const float *sH, const float *sL, int64_t n_samples, int W, int stride,
                        int64_t nw, const int32_t *slides, int n_slides, float *out, bool logits, cudaStream_t st) {
    (void)n_samples;
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
                if (v == kSmall)
                    launch_layer<32, 32>(xin, xout, m->ws.skip.as<float>(), wl, bstride, wm, sH, sL, w0, stride, W, C,
                                         dl, l == 0, st);
                else
                    launch_layer<64, 128>(xin, xout, m->ws.skip.as<float>(), wl, bstride, wm, sH, sL, w0, stride, W,
                                          C, dl, l == 0, st);
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
                float *o = out + ((int64_t)si * d.n_models + mi) * nw * W;
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

}  // namespace gwe
