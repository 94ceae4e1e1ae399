// Whitening front end (paper section "Materials and Methods", paragraph "Data
// preparation": strain whitened with PSDs estimated from the data, then
// normalised to unit standard deviation).
//
//   Welch PSD: segments of `seg` samples at 50 % overlap, each minus its own
//   mean (FP64), times the periodic Hann window; one-sided density
//   S_k = c_k mean_s |X_s[k]|^2 / (fs sum w^2), c_k = 2 except DC and Nyquist.
//   The segment transforms are FP32 (cuFFT, batched); the |X|^2 accumulation
//   over segments and everything derived from it is FP64.
//   Whitening: X = rfft(x) (FP32), S interpolated linearly at f_k = k fs / n,
//   Y_k = X_k / sqrt(fs S / 2), zero below 15 Hz, y = irfft(Y), y / std(y)
//   (the sums for the standard deviation in FP64).
#include <cuda_runtime.h>
#include <cufft.h>

#include <map>
#include <mutex>
#include <utility>

#include "gwe_internal.h"

namespace gwe {
namespace {

constexpr double kFLow = 15.0;

__global__ void k_seg_mean(const float *__restrict__ x, int64_t step, int seg, double *__restrict__ mean) {
    __shared__ double sh[256];
    const int s = blockIdx.x;
    const float *xs = x + (int64_t)s * step;
    double acc = 0.0;
    for (int i = threadIdx.x; i < seg; i += 256) acc += (double)xs[i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) mean[s] = sh[0] / seg;
}

// buf[s][i] = (x[s*step + i] - mean_s) * (0.5 - 0.5 cos(2 pi i / seg))
__global__ void k_seg_window(const float *__restrict__ x, int64_t step, int seg, int n_seg,
                             const double *__restrict__ mean, float *__restrict__ buf) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)n_seg * seg) return;
    const int s = (int)(idx / seg), i = (int)(idx - (int64_t)s * seg);
    const double w = 0.5 - 0.5 * cospi(2.0 * i / seg);
    buf[idx] = (float)(((double)x[(int64_t)s * step + i] - mean[s]) * w);
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

// Y_k = X_k / sqrt(fs S(f_k) / 2) for f_k >= 15 Hz, else 0
__global__ void k_whiten_spec(cufftComplex *__restrict__ X, int64_t nbin, int64_t n, double fs, int seg,
                              const double *__restrict__ psd) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nbin) return;
    const double f = (double)k * fs / (double)n;
    cufftComplex c = X[k];
    if (f < kFLow) {
        c.x = 0.f;
        c.y = 0.f;
    } else {
        const double jf = f * seg / fs;
        int64_t j0 = (int64_t)floor(jf);
        const int last = seg / 2;
        double s;
        if (j0 >= last) {
            s = psd[last];
        } else {
            const double fr = jf - (double)j0;
            s = psd[j0] * (1.0 - fr) + psd[j0 + 1] * fr;
        }
        const double sc = 1.0 / sqrt(fs * s / 2.0);
        c.x = (float)((double)c.x * sc);
        c.y = (float)((double)c.y * sc);
    }
    X[k] = c;
}

__global__ void k_moments(const float *__restrict__ y, int64_t n, double *__restrict__ sums) {
    __shared__ double s1[256], s2[256];
    double a = 0.0, b = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = y[i];
        a += v;
        b += v * v;
    }
    s1[threadIdx.x] = a;
    s2[threadIdx.x] = b;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            s1[threadIdx.x] += s1[threadIdx.x + o];
            s2[threadIdx.x] += s2[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        atomicAdd(sums, s1[0]);
        atomicAdd(sums + 1, s2[0]);
    }
}

__global__ void k_scale(float *__restrict__ y, int64_t n, const double *__restrict__ sums) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double mean = sums[0] / (double)n;
    const double var = sums[1] / (double)n - mean * mean;
    y[i] = (float)((double)y[i] / sqrt(var));
}

struct WhitenWs {
    std::mutex mu;
    DevBuf seg_buf, seg_spec, spec, mean, psd, sums;
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

gwe_status whiten_run(const float *x, int64_t n, double fs, int seg, float *out, cudaStream_t st) {
    WhitenWs &w = whiten_ws();
    std::lock_guard<std::mutex> lock(w.mu);
    const int64_t step = seg / 2;
    const int n_seg = (int)((n - step) / step);
    const int nbin = seg / 2 + 1;
    const int64_t nspec = n / 2 + 1;
    GWE_CUDA_TRY(w.mean.ensure(sizeof(double) * n_seg));
    GWE_CUDA_TRY(w.seg_buf.ensure(sizeof(float) * (size_t)n_seg * seg));
    GWE_CUDA_TRY(w.seg_spec.ensure(sizeof(cufftComplex) * (size_t)n_seg * nbin));
    GWE_CUDA_TRY(w.psd.ensure(sizeof(double) * nbin));
    GWE_CUDA_TRY(w.spec.ensure(sizeof(cufftComplex) * (size_t)nspec));
    GWE_CUDA_TRY(w.sums.ensure(sizeof(double) * 2));
    cufftHandle p_seg, p_full, p_inv;
    gwe_status s = plan_r2c(w, seg, n_seg, &p_seg);
    if (s == GWE_OK) s = plan_r2c(w, n, 1, &p_full);
    if (s == GWE_OK) s = plan_c2r(w, n, &p_inv);
    if (s != GWE_OK) return s;
    // every whitening kernel and transform below, as one profiling entry
    ProfScope prof("k_whiten", st);
    // Welch PSD
    k_seg_mean<<<n_seg, 256, 0, st>>>(x, step, seg, w.mean.as<double>());
    note_launch();
    k_seg_window<<<nblk((int64_t)n_seg * seg, 256), 256, 0, st>>>(x, step, seg, n_seg, w.mean.as<double>(),
                                                                  w.seg_buf.as<float>());
    note_launch();
    if (cufftSetStream(p_seg, st) != CUFFT_SUCCESS ||
        cufftExecR2C(p_seg, w.seg_buf.as<cufftReal>(), w.seg_spec.as<cufftComplex>()) != CUFFT_SUCCESS) {
        set_error("gwe_whiten: cuFFT segment transform failed");
        return GWE_ERR_CUDA;
    }
    const double sum_w2 = 0.375 * seg;          // sum of the periodic Hann window squared
    k_psd<<<nblk(nbin, 256), 256, 0, st>>>(w.seg_spec.as<cufftComplex>(), nbin, n_seg,
                                           1.0 / ((double)n_seg * fs * sum_w2), w.psd.as<double>());
    note_launch();
    // spectral division of the whole segment
    if (cufftSetStream(p_full, st) != CUFFT_SUCCESS ||
        cufftExecR2C(p_full, const_cast<cufftReal *>(x), w.spec.as<cufftComplex>()) != CUFFT_SUCCESS) {
        set_error("gwe_whiten: cuFFT forward transform failed");
        return GWE_ERR_CUDA;
    }
    k_whiten_spec<<<nblk(nspec, 256), 256, 0, st>>>(w.spec.as<cufftComplex>(), nspec, n, fs, seg, w.psd.as<double>());
    note_launch();
    if (cufftSetStream(p_inv, st) != CUFFT_SUCCESS ||
        cufftExecC2R(p_inv, w.spec.as<cufftComplex>(), out) != CUFFT_SUCCESS) {
        set_error("gwe_whiten: cuFFT inverse transform failed");
        return GWE_ERR_CUDA;
    }
    // unit standard deviation
    GWE_CUDA_TRY(cudaMemsetAsync(w.sums.ptr, 0, sizeof(double) * 2, st));
    k_moments<<<1024, 256, 0, st>>>(out, n, w.sums.as<double>());
    note_launch();
    k_scale<<<nblk(n, 256), 256, 0, st>>>(out, n, w.sums.as<double>());
    note_launch();
    GWE_CUDA_TRY(cudaGetLastError());
    return GWE_OK;
}

}  // namespace gwe
