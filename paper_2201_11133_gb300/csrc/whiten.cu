// Whitening front end (paper section "Materials and Methods", paragraph "Data
// preparation": strain whitened with PSDs estimated from the data, then
// normalised to unit standard deviation).
//
//   Welch PSD: segments of `seg` samples at 50 % overlap, each minus its own
//   mean, times the periodic Hann window; one-sided density
//   S_k = c_k A_s(|X_s[k]|^2) / (fs sum w^2), c_k = 2 except DC and Nyquist,
//   with A the mean over segments, or the median divided by the median's bias
//   for exponentially distributed values (robust against loud short glitches).
//   The segment transforms are FP32 (cuFFT, batched); FP64 is used only for
//   |X|^2 and its accumulation (mean) or selection (median) over segments.
//   Whitening: X = rfft(x w_T) (FP32; w_T a Tukey taper, 1 without one), S
//   interpolated linearly at f_k = k fs / n, Y_k = X_k / sqrt(fs S / 2), zero
//   below f_low, y = irfft(Y), y / std(y).  Means, the window, the division and
//   the moments are FP32 (compensated sums).
#include <cuda_runtime.h>
#include <cufft.h>

#include <cmath>
#include <map>
#include <mutex>
#include <utility>

#include "gwe_internal.h"

namespace gwe {
namespace {

// compensated (Kahan) FP32 accumulation
struct Kahan {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float v) {
        const float y = v - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
};

// block sum of one value per thread (256 threads), FP32 tree; valid in thread 0
__device__ __forceinline__ float block_sum256(float v, float *sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    const float r = sh[0];
    __syncthreads();
    return r;
}

__global__ void k_seg_mean(const float *__restrict__ x, int64_t step, int seg, float *__restrict__ mean) {
    __shared__ float sh[256];
    const int s = blockIdx.x;
    const float *xs = x + (int64_t)s * step;
    Kahan acc;
    for (int i = threadIdx.x; i < seg; i += 256) acc.add(xs[i]);
    const float tot = block_sum256(acc.s, sh);
    if (threadIdx.x == 0) mean[s] = tot / (float)seg;
}

// buf[s][i] = (x[s*step + i] - mean_s) * (0.5 - 0.5 cos(2 pi i / seg))
__global__ void k_seg_window(const float *__restrict__ x, int64_t step, int seg, int n_seg,
                             const float *__restrict__ mean, float *__restrict__ buf) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)n_seg * seg) return;
    const int s = (int)(idx / seg), i = (int)(idx - (int64_t)s * seg);
    const float w = 0.5f - 0.5f * cospif(2.0f * (float)i / (float)seg);
    buf[idx] = (x[(int64_t)s * step + i] - mean[s]) * w;
}

// psd[k] = c_k * median_s |X_s[k]|^2 * norm   (|X|^2 in FP64, exact selection): one block per bin,
// the n_seg values sorted in shared memory (bitonic, padded to P = next power of two with +inf)
__global__ void k_psd_median(const cufftComplex *__restrict__ X, int nbin, int n_seg, int P, double norm,
                             double *__restrict__ psd) {
    extern __shared__ double v[];
    const int k = blockIdx.x;
    for (int s = threadIdx.x; s < P; s += blockDim.x) {
        if (s < n_seg) {
            const cufftComplex c = X[(int64_t)s * nbin + k];
            v[s] = (double)c.x * (double)c.x + (double)c.y * (double)c.y;
        } else {
            v[s] = INFINITY;
        }
    }
    __syncthreads();
    for (int size = 2; size <= P; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = threadIdx.x; t < P / 2; t += blockDim.x) {
                const int i = 2 * t - (t & (stride - 1));   // lower element of the pair
                const int j = i + stride;
                const bool up = (i & size) == 0;
                const double a = v[i], b = v[j];
                if ((a > b) == up) {
                    v[i] = b;
                    v[j] = a;
                }
            }
            __syncthreads();
        }
    }
    if (threadIdx.x == 0) {
        const double med = (n_seg & 1) ? v[n_seg / 2] : 0.5 * (v[n_seg / 2 - 1] + v[n_seg / 2]);
        const double ck = (k == 0 || k == nbin - 1) ? 1.0 : 2.0;
        psd[k] = ck * med * norm;
    }
}

// psd[k] = c_k * sum_s |X_s[k]|^2 * norm   (FP64 accumulation)
__global__ void k_psd(const cufftComplex *__restrict__ X, int nbin, int n_seg, double norm, double *__restrict__ psd) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nbin) return;
    double acc = 0.0;
    for (int s = 0; s < n_seg; ++s) {
        const cufftComplex c = X[(int64_t)s * nbin + k];
        acc += (double)c.x * (double)c.x + (double)c.y * (double)c.y;
    }
    const double ck = (k == 0 || k == nbin - 1) ? 1.0 : 2.0;
    psd[k] = ck * acc * norm;
}

// out[i] = x[i] * w_T[i], the Tukey taper of `width` = alpha (n - 1) / 2 samples at each end
__global__ void k_taper(const float *__restrict__ x, int64_t n, float width, float *__restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float w = 1.f;
    const float fi = (float)i, fj = (float)(n - 1 - i);
    if (fi < width) w = 0.5f * (1.f + cospif(fi / width - 1.f));
    else if (fj < width) w = 0.5f * (1.f + cospif(fj / width - 1.f));
    out[i] = x[i] * w;
}

// Y_k = X_k / sqrt(fs S(f_k) / 2) for k >= k_low (f_k >= f_low), else 0; S interpolated linearly
// between Welch bins j0 = k seg / n and j0 + 1 (index arithmetic in integers, the rest FP32)
__global__ void k_whiten_spec(cufftComplex *__restrict__ X, int64_t nbin, int64_t n, float half_fs, int seg,
                              int64_t k_low, const double *__restrict__ psd) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nbin) return;
    cufftComplex c = X[k];
    if (k < k_low) {
        c.x = 0.f;
        c.y = 0.f;
    } else {
        const int64_t num = k * (int64_t)seg;
        const int64_t j0 = num / n;
        const int last = seg / 2;
        float s;
        if (j0 >= last) {
            s = (float)psd[last];
        } else {
            const float fr = (float)(num - j0 * n) / (float)n;
            s = (float)psd[j0] * (1.f - fr) + (float)psd[j0 + 1] * fr;
        }
        const float sc = 1.f / sqrtf(half_fs * s);
        c.x *= sc;
        c.y *= sc;
    }
    X[k] = c;
}

// per-block sums of y and y^2 (FP32, compensated), then one block combines them
__global__ void k_moments(const float *__restrict__ y, int64_t n, float *__restrict__ part) {
    __shared__ float sh[256];
    Kahan a, b;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float v = y[i];
        a.add(v);
        b.add(v * v);
    }
    const float sa = block_sum256(a.s, sh);
    const float sb = block_sum256(b.s, sh);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = sa;
        part[2 * blockIdx.x + 1] = sb;
    }
}

__global__ void k_moments_final(const float *__restrict__ part, int nb, float *__restrict__ sums) {
    __shared__ float sh[256];
    Kahan a, b;
    for (int i = threadIdx.x; i < nb; i += 256) {
        a.add(part[2 * i]);
        b.add(part[2 * i + 1]);
    }
    const float sa = block_sum256(a.s, sh);
    const float sb = block_sum256(b.s, sh);
    if (threadIdx.x == 0) {
        sums[0] = sa;
        sums[1] = sb;
    }
}

__global__ void k_scale(float *__restrict__ y, int64_t n, const float *__restrict__ sums) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float mean = sums[0] / (float)n;
    const float var = sums[1] / (float)n - mean * mean;
    y[i] = y[i] / sqrtf(var);
}

struct WhitenWs {
    std::mutex mu;
    DevBuf seg_buf, seg_spec, spec, mean, psd, sums, part;
    std::map<std::pair<int64_t, int>, cufftHandle> r2c;   // (length, batch) -> plan
    std::map<int64_t, cufftHandle> c2r;
};

WhitenWs &whiten_ws() {
    static WhitenWs *w = new WhitenWs();   // plans and buffers are kept until process exit
    return *w;
}

gwe_status plan_r2c(WhitenWs &w, int64_t len, int batch, cufftHandle *out) {
    auto key = std::make_pair(len, batch);
    auto it = w.r2c.find(key);
    if (it != w.r2c.end()) {
        *out = it->second;
        return GWE_OK;
    }
    cufftHandle h;
    long long nn[1] = {(long long)len};
    size_t ws = 0;
    if (cufftCreate(&h) != CUFFT_SUCCESS ||
        cufftMakePlanMany64(h, 1, nn, nullptr, 1, len, nullptr, 1, len / 2 + 1, CUFFT_R2C, batch, &ws) !=
            CUFFT_SUCCESS) {
        set_error("gwe_whiten: cuFFT R2C plan failed");
        return GWE_ERR_CUDA;
    }
    w.r2c[key] = h;
    *out = h;
    return GWE_OK;
}

gwe_status plan_c2r(WhitenWs &w, int64_t len, cufftHandle *out) {
    auto it = w.c2r.find(len);
    if (it != w.c2r.end()) {
        *out = it->second;
        return GWE_OK;
    }
    cufftHandle h;
    long long nn[1] = {(long long)len};
    size_t ws = 0;
    if (cufftCreate(&h) != CUFFT_SUCCESS ||
        cufftMakePlanMany64(h, 1, nn, nullptr, 1, len / 2 + 1, nullptr, 1, len, CUFFT_C2R, 1, &ws) != CUFFT_SUCCESS) {
        set_error("gwe_whiten: cuFFT C2R plan failed");
        return GWE_ERR_CUDA;
    }
    w.c2r[len] = h;
    *out = h;
    return GWE_OK;
}

unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

gwe_status whiten_run(const float *x, int64_t n, double fs, int seg, const gwe_whiten_options &opt, float *out,
                      cudaStream_t st) {
    WhitenWs &w = whiten_ws();
    std::lock_guard<std::mutex> lock(w.mu);
    const int64_t step = seg / 2;
    const int n_seg = (int)((n - step) / step);
    const int nbin = seg / 2 + 1;
    const int64_t nspec = n / 2 + 1;
    GWE_CUDA_TRY(w.mean.ensure(sizeof(float) * n_seg));
    GWE_CUDA_TRY(w.seg_buf.ensure(sizeof(float) * (size_t)n_seg * seg));
    GWE_CUDA_TRY(w.seg_spec.ensure(sizeof(cufftComplex) * (size_t)n_seg * nbin));
    GWE_CUDA_TRY(w.psd.ensure(sizeof(double) * nbin));
    GWE_CUDA_TRY(w.spec.ensure(sizeof(cufftComplex) * (size_t)nspec));
    GWE_CUDA_TRY(w.sums.ensure(sizeof(float) * 2));
    constexpr int kMomBlocks = 1024;
    GWE_CUDA_TRY(w.part.ensure(sizeof(float) * 2 * kMomBlocks));
    int P = 1;
    while (P < n_seg) P <<= 1;
    if (opt.psd_average == GWE_PSD_MEDIAN && (size_t)P * sizeof(double) > 200 * 1024) {
        set_error("gwe_whiten: the median PSD supports at most 16384 Welch segments");
        return GWE_ERR_UNSUPPORTED;
    }
    cufftHandle p_seg, p_full, p_inv;
    gwe_status s = plan_r2c(w, seg, n_seg, &p_seg);
    if (s == GWE_OK) s = plan_r2c(w, n, 1, &p_full);
    if (s == GWE_OK) s = plan_c2r(w, n, &p_inv);
    if (s != GWE_OK) return s;
    // every whitening kernel and transform below, as one profiling entry
    ProfScope prof("k_whiten", st);
    // Welch PSD
    k_seg_mean<<<n_seg, 256, 0, st>>>(x, step, seg, w.mean.as<float>());
    note_launch();
    k_seg_window<<<nblk((int64_t)n_seg * seg, 256), 256, 0, st>>>(x, step, seg, n_seg, w.mean.as<float>(),
                                                                  w.seg_buf.as<float>());
    note_launch();
    if (cufftSetStream(p_seg, st) != CUFFT_SUCCESS ||
        cufftExecR2C(p_seg, w.seg_buf.as<cufftReal>(), w.seg_spec.as<cufftComplex>()) != CUFFT_SUCCESS) {
        set_error("gwe_whiten: cuFFT segment transform failed");
        return GWE_ERR_CUDA;
    }
    const double sum_w2 = 0.375 * seg;          // sum of the periodic Hann window squared
    if (opt.psd_average == GWE_PSD_MEDIAN) {
        // bias of the median of n_seg exponentially distributed values: 1 - 1/2 + 1/3 - ... over the
        // largest odd number of terms <= n_seg
        const int terms = (n_seg & 1) ? n_seg : n_seg - 1;
        double bias = 0.0;
        for (int i = 1; i <= terms; ++i) bias += ((i & 1) ? 1.0 : -1.0) / (double)i;
        if (terms <= 0) bias = 1.0;
        const size_t sm = (size_t)P * sizeof(double);
        if (sm > 48 * 1024)
            GWE_CUDA_TRY(cudaFuncSetAttribute(k_psd_median, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        k_psd_median<<<nbin, 256, sm, st>>>(w.seg_spec.as<cufftComplex>(), nbin, n_seg, P,
                                            1.0 / (bias * fs * sum_w2), w.psd.as<double>());
    } else {
        k_psd<<<nblk(nbin, 256), 256, 0, st>>>(w.seg_spec.as<cufftComplex>(), nbin, n_seg,
                                               1.0 / ((double)n_seg * fs * sum_w2), w.psd.as<double>());
    }
    note_launch();
    // spectral division of the whole segment (Tukey-tapered copy in `out` when a taper is asked for)
    const float *src = x;
    if (opt.tukey_alpha > 0.0) {
        const float width = (float)(opt.tukey_alpha * (double)(n - 1) / 2.0);
        k_taper<<<nblk(n, 256), 256, 0, st>>>(x, n, width, out);
        note_launch();
        src = out;
    }
    if (cufftSetStream(p_full, st) != CUFFT_SUCCESS ||
        cufftExecR2C(p_full, const_cast<cufftReal *>(src), w.spec.as<cufftComplex>()) != CUFFT_SUCCESS) {
        set_error("gwe_whiten: cuFFT forward transform failed");
        return GWE_ERR_CUDA;
    }
    // first bin at or above f_low: k >= f_low n / fs (host arithmetic)
    const int64_t k_low = (int64_t)std::ceil(opt.f_low * (double)n / fs);
    k_whiten_spec<<<nblk(nspec, 256), 256, 0, st>>>(w.spec.as<cufftComplex>(), nspec, n, (float)(0.5 * fs), seg,
                                                    k_low, w.psd.as<double>());
    note_launch();
    if (cufftSetStream(p_inv, st) != CUFFT_SUCCESS ||
        cufftExecC2R(p_inv, w.spec.as<cufftComplex>(), out) != CUFFT_SUCCESS) {
        set_error("gwe_whiten: cuFFT inverse transform failed");
        return GWE_ERR_CUDA;
    }
    // unit standard deviation
    k_moments<<<kMomBlocks, 256, 0, st>>>(out, n, w.part.as<float>());
    k_moments_final<<<1, 256, 0, st>>>(w.part.as<float>(), kMomBlocks, w.sums.as<float>());
    k_scale<<<nblk(n, 256), 256, 0, st>>>(out, n, w.sums.as<float>());
    note_launch(3);
    GWE_CUDA_TRY(cudaGetLastError());
    return GWE_OK;
}

}  // namespace gwe
