// Backward pass of one ensemble member on the tensor cores (paper paragraph "AI ensemble
// construction": per-sample labels, binary cross-entropy on the logits), BF16 operands with FP32
// accumulation and an FP32 chain of dL/dx, with per-stack recomputation.
//
// The same reverse-mode algebra as the FP32 path (fp32_path.cu), with every contraction a tcgen05
// GEMM over 128-row tiles (row = one time sample of one window of one branch):
//   forward   a   = [x(t-d) | x(t)] . Wconv^T + b_conv          (N = 2R, K = 2R)
//             z   = tanh(a_f) sigmoid(a_g)
//             [r | q] = z . [W_res ; W_skip]^T                   (N = R (+ S), K = R)
//             x_{l+1} = x_l + r + b_res,  skip += q + b_skip
//   backward  dz  = [dx_{l+1} | dskip] . [W_res | W_skip]          (N = R, K = R + S)
//             da  = gate backward of dz at a                      (fused in the dz epilogue)
//             dx_l = dx_{l+1} + [da(t) | da(t+d)] . [W1 ; W0]      (N = R, K = 4R)
//             dWconv += da^T [x(t-d) | x(t)], dW_res += dx_{l+1}^T z, dW_skip += dskip^T z
//                                                                 (weight gradients: M = output
//                                                                  channels, K = rows)
// Row GEMMs stage their A tile (thread = row, window boundaries zero-filled) and keep the
// layer's B image in shared memory; the MMA accumulates in TMEM and the epilogue (thread = row)
// applies the fused step.  Weight-gradient GEMMs stage G^T and X^T tiles (transposed while
// staging), accumulate over a range of row tiles in TMEM and add their partial sums atomically.
// The head, the biases, the input projection and dL/dstrain use the FP32 kernels.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "gwe_internal.h"
#include "tc_ptx.cuh"

namespace gwe {
namespace {

using namespace tc;

constexpr int kRows = 128;              // rows per tile (the MMA's M)
constexpr uint64_t kWaitNs = 4000000000ull;

// one K-range of a row GEMM's A operand: columns [0, C) of a row-major BF16 array, taken at row
// t + shift of the same window (zero outside [0, W))
struct RowSeg {
    const __nv_bfloat16 *p;
    int64_t boff;      // elements between the branches' arrays
    int ld;            // elements per row
    int C;             // columns (multiple of 8)
    int shift;
};

enum { EPI_CONV = 0, EPI_RES = 1, EPI_DZ = 2, EPI_DGRAD = 3 };

struct RowGemm {
    RowSeg seg[2];
    int nseg;
    int K, N;                         // K = sum of the segments' C; N = MMA columns
    int bn;                           // rows of the B image (>= N; the MMA uses its first N rows)
    const uint8_t *bimg;              // B image [bn rows][K] (chunk layout) of branch 0
    int64_t bimg_boff;                // bytes to branch 1's image
    int64_t rows;                     // rows per branch
    int W;
    int nbranch;
    int64_t n_tiles;                  // nbranch * ceil(rows / 128)
    int *err;
    int R;                            // residual channels
    const float *bias;                // per-branch bias of the epilogue (blob), branch 1 at + bias_boff
    const float *bias2;               // EPI_RES with skip: b_skip
    int64_t bias_boff;
    const float *aux;                 // EPI_RES: x_l; EPI_DGRAD: dx_{l+1}   (FP32)
    const __half *gate;               // EPI_DZ: [tanh(f) | sigmoid(g)] per row (FP16), written by EPI_CONV
    __half *gate_out;                 // EPI_CONV: where to write it (or null)
    int64_t gate_boff;
    int64_t aux_boff;
    float *o32;                       // EPI_RES: x_{l+1}; EPI_DGRAD: dx_l
    int64_t o32_boff;
    __nv_bfloat16 *o16;               // EPI_CONV: z; EPI_RES: x_{l+1}; EPI_DZ: da; EPI_DGRAD: dx_l
    int64_t o16_boff;
    float *skip;                      // EPI_RES with N > R: skip sum [row][S] (accumulated)
    int64_t skip_boff;
    int skip_init;                    // 1: skip = q + b_skip (first layer)
};

struct WgGemm {
    const __nv_bfloat16 *G;           // [row][ldg], columns [0, M) used
    int64_t g_boff;
    int ldg, M;                       // M <= 128 (rows M..127 of the MMA are zero)
    RowSeg xs[2];                     // X: N columns
    int nxs, N;
    int64_t rows;                     // rows per branch
    int W;
    int tiles_per_cta;
    int64_t tiles;                    // row tiles per branch
    float *dW;                        // dW[m][n] at dW + m * ldw + n, branch 1 at + w_boff
    int ldw;
    int64_t w_boff;
    float *db;                        // or null: db[m] += sum over rows of G[row][m] (column nx of X is 1)
    int nx;                           // columns of X from the segments (N = nx, or nx + 16 with db)
    int *err;
};

__device__ __forceinline__ uint32_t tmem_cols_for(int n) {
    uint32_t c = 32;
    while ((int)c < n) c <<= 1;
    return c;
}

// 8 BF16 values of row `row` (window-relative t) from segment s at chunk c, zero outside the window
__device__ __forceinline__ uint4 seg_load(const RowSeg &s, int b, int64_t row, int W, int c) {
    const int64_t w = row / W;
    const int t = (int)(row - w * W) + s.shift;
    if (t < 0 || t >= W) return make_uint4(0, 0, 0, 0);
    const __nv_bfloat16 *src = s.p + b * s.boff + (w * W + t) * (int64_t)s.ld + 8 * c;
    return __ldg(reinterpret_cast<const uint4 *>(src));
}

__device__ __forceinline__ float sigm(float x) { return 1.f / (1.f + expf(-x)); }

// 16-byte global -> shared copy in flight until cp_async_wait_all; zero-filled when !valid
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, bool valid) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(valid ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// address of 8 BF16 values of row `row` of segment s at chunk c, and whether they lie in the window
__device__ __forceinline__ const __nv_bfloat16 *seg_addr(const RowSeg &s, int b, int64_t row, int W, int c,
                                                          bool &valid) {
    const int64_t w = row / W;
    const int t = (int)(row - w * W) + s.shift;
    valid = t >= 0 && t < W;
    return valid ? s.p + b * s.boff + (w * W + t) * (int64_t)s.ld + 8 * c : s.p;
}

// 16 consecutive values of one row (16-byte aligned): FP32 loads and stores, BF16 stores
__device__ __forceinline__ void ld16_f32(const float *src, float (&v)[16]) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float4 t = *reinterpret_cast<const float4 *>(src + 4 * q);
        v[4 * q] = t.x;
        v[4 * q + 1] = t.y;
        v[4 * q + 2] = t.z;
        v[4 * q + 3] = t.w;
    }
}
__device__ __forceinline__ void st16_f32(float *dst, const float (&v)[16]) {
#pragma unroll
    for (int q = 0; q < 4; ++q)
        *reinterpret_cast<float4 *>(dst + 4 * q) = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
}
__device__ __forceinline__ void st16_f16(__half *dst, const float (&v)[16]) {
    uint32_t w[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const __half2 h = __floats2half2_rn(v[2 * q], v[2 * q + 1]);
        w[q] = *reinterpret_cast<const uint32_t *>(&h);
    }
    *reinterpret_cast<uint4 *>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
    *reinterpret_cast<uint4 *>(dst + 8) = make_uint4(w[4], w[5], w[6], w[7]);
}
__device__ __forceinline__ void ld16_f16(const __half *src, float (&v)[16]) {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const uint4 t = *reinterpret_cast<const uint4 *>(src + 8 * q);
        const uint32_t w[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float2 f = __half22float2(*reinterpret_cast<const __half2 *>(&w[i]));
            v[8 * q + 2 * i] = f.x;
            v[8 * q + 2 * i + 1] = f.y;
        }
    }
}
__device__ __forceinline__ void st16_bf16(__nv_bfloat16 *dst, const float (&v)[16]) {
    uint32_t w[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
        w[q] = *reinterpret_cast<const uint32_t *>(&h);
    }
    *reinterpret_cast<uint4 *>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
    *reinterpret_cast<uint4 *>(dst + 8) = make_uint4(w[4], w[5], w[6], w[7]);
}

// D = A . B^T over the row tiles of both branches, fused epilogue EPI.
template <int EPI>
__global__ void __launch_bounds__(128) k_tc_rows(const RowGemm p) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    __shared__ uint64_t bar[2];
    __shared__ uint32_t tslot;
    __shared__ int abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int KC = p.K / 8;                                   // 16-byte chunks per row
    const uint32_t a_bytes = (uint32_t)kRows * p.K * 2;   // B image follows the A tile
    uint8_t *sA = smem, *sB = smem + a_bytes;
    const uint32_t ncols = tmem_cols_for(p.N);
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 0) tmem_alloc(&tslot, ncols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tslot;
    const int64_t tpb = (p.rows + kRows - 1) / kRows;         // tiles per branch
    int cur_b = -1;
    uint32_t ph = 0;
    bool ok = true;
    const uint32_t idesc = idesc_f16(128, p.N, 1);
    for (int64_t tile = blockIdx.x; tile < p.n_tiles && ok; tile += gridDim.x) {
        const int b = (int)(tile / tpb);
        const int64_t r0 = (tile - (int64_t)b * tpb) * kRows;
        // the branch's B image (once per branch change; every earlier MMA has completed here)
        if (b != cur_b) {
            const uint8_t *src = p.bimg + b * p.bimg_boff;
            const int n16 = p.bn * p.K * 2 / 16;
            for (int i = tid; i < n16; i += 128) cp_async16(smem_u32(sB + 16 * i), src + 16 * i, true);
            cur_b = b;
        }
        // A tile: thread = row, chunk-column layout; every copy of the tile in flight at once
        const int64_t row = r0 + tid;
        int c = 0;
        for (int si = 0; si < p.nseg; ++si) {
            const RowSeg &s = p.seg[si];
            for (int cc = 0; cc < s.C / 8; ++cc, ++c) {
                bool valid = false;
                const __nv_bfloat16 *src = row < p.rows ? seg_addr(s, b, row, p.W, cc, valid) : s.p;
                cp_async16(smem_u32(sA + (size_t)c * kRows * 16 + tid * 16), src, valid && row < p.rows);
            }
        }
        cp_async_wait_all();
        fence_proxy_async_smem();
        tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
            for (int ks = 0; ks < KC / 2; ++ks) {
                const uint64_t ad = sdesc(a0 + ks * 2 * kRows * 16, kRows * 16, 128);
                const uint64_t bd = sdesc(b0 + ks * 2 * p.bn * 16, p.bn * 16, 128);
                mma_f16(tmem, ad, bd, idesc, ks > 0 ? 1u : 0u);
            }
            mma_commit(&bar[0]);
        }
        const bool w_ok = mbar_wait(&bar[0], ph & 1, &abort_flag, p.err, 60 + EPI, kWaitNs);
        ++ph;
        if (__syncthreads_or(!w_ok)) {
            ok = false;
            break;
        }
        tc_fence_after();
        // epilogue: thread = row (TMEM lane = warp * 32 + lane = tid)
        const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);
        const bool live = row < p.rows;
        const int64_t orow = row;
        if (EPI == EPI_CONV) {
            const int R = p.R;
            const float *bc = p.bias + b * p.bias_boff;
            for (int c0 = 0; c0 < R; c0 += 16) {
                uint32_t fr[16], gr[16];
                tmem_ld16(tl + c0, fr);
                tmem_ld16(tl + R + c0, gr);
                tmem_ld_wait();
                if (!live) continue;
                float th[16], sg[16], z[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    th[j] = tanhf(__uint_as_float(fr[j]) + __ldg(bc + c0 + j));
                    sg[j] = sigm(__uint_as_float(gr[j]) + __ldg(bc + R + c0 + j));
                    z[j] = th[j] * sg[j];
                }
                if (p.gate_out) {   // the backward's gate cache: tanh(f), sigmoid(g) in FP16
                    __half *go = p.gate_out + b * p.gate_boff + orow * 2 * R;
                    st16_f16(go + c0, th);
                    st16_f16(go + R + c0, sg);
                }
                st16_bf16(p.o16 + b * p.o16_boff + orow * R + c0, z);
            }
        } else if (EPI == EPI_RES) {
            const int R = p.R;
            const float *br = p.bias + b * p.bias_boff;
            for (int c0 = 0; c0 < R; c0 += 16) {
                uint32_t rr[16];
                tmem_ld16(tl + c0, rr);
                tmem_ld_wait();
                if (!live) continue;
                float v[16];
                ld16_f32(p.aux + b * p.aux_boff + orow * R + c0, v);
#pragma unroll
                for (int j = 0; j < 16; ++j) v[j] += __uint_as_float(rr[j]) + __ldg(br + c0 + j);
                st16_f32(p.o32 + b * p.o32_boff + orow * R + c0, v);
                st16_bf16(p.o16 + b * p.o16_boff + orow * R + c0, v);
            }
            const int S = p.N - R;
            const float *bs = p.bias2 ? p.bias2 + b * p.bias_boff : nullptr;
            for (int c0 = 0; c0 < S; c0 += 16) {
                uint32_t qr[16];
                tmem_ld16(tl + R + c0, qr);
                tmem_ld_wait();
                if (!live) continue;
                float *so = p.skip + b * p.skip_boff + orow * S + c0;
                float v[16];
                if (p.skip_init) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) v[j] = 0.f;
                } else {
                    ld16_f32(so, v);
                }
#pragma unroll
                for (int j = 0; j < 16; ++j) v[j] += __uint_as_float(qr[j]) + __ldg(bs + c0 + j);
                st16_f32(so, v);
            }
        } else if (EPI == EPI_DZ) {
            const int R = p.R;
            for (int c0 = 0; c0 < R; c0 += 16) {
                uint32_t dr[16];
                tmem_ld16(tl + c0, dr);
                tmem_ld_wait();
                if (!live) continue;
                const __half *gc = p.gate + b * p.gate_boff + orow * 2 * R;
                float th[16], sg[16], df[16], dg[16];
                ld16_f16(gc + c0, th);
                ld16_f16(gc + R + c0, sg);
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const float dz = __uint_as_float(dr[j]);
                    df[j] = dz * sg[j] * (1.f - th[j] * th[j]);
                    dg[j] = dz * th[j] * sg[j] * (1.f - sg[j]);
                }
                __nv_bfloat16 *d16 = p.o16 + b * p.o16_boff + orow * 2 * R;
                st16_bf16(d16 + c0, df);
                st16_bf16(d16 + R + c0, dg);
            }
        } else {   // EPI_DGRAD
            const int R = p.R;
            for (int c0 = 0; c0 < R; c0 += 16) {
                uint32_t dr[16];
                tmem_ld16(tl + c0, dr);
                tmem_ld_wait();
                if (!live) continue;
                float v[16];
                ld16_f32(p.aux + b * p.aux_boff + orow * R + c0, v);
#pragma unroll
                for (int j = 0; j < 16; ++j) v[j] += __uint_as_float(dr[j]);
                st16_f32(p.o32 + b * p.o32_boff + orow * R + c0, v);
                st16_bf16(p.o16 + b * p.o16_boff + orow * R + c0, v);
            }
        }
        // every thread's TMEM reads and shared-memory use of this tile end before the next tile
        tc_fence_before();
        __syncthreads();
    }
    // no MMA of this thread may be in flight when TMEM is released
    if (tid == 0) {
        mma_commit(&bar[1]);
        mbar_wait_drain(&bar[1], 0, p.err, 70 + EPI, kWaitNs);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, ncols);
    }
}

// dW += G^T X over the row tiles [blockIdx.x * tiles_per_cta, ...) of branch blockIdx.y.
template <int N>
__global__ void __launch_bounds__(128) k_tc_wgrad(const WgGemm p) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    __shared__ uint64_t bar[2];
    __shared__ uint32_t tslot;
    __shared__ int abort_flag;
    constexpr uint32_t NCOLS = N <= 32 ? 32 : (N <= 64 ? 64 : (N <= 128 ? 128 : 256));
    const int tid = threadIdx.x, warp = tid >> 5;
    uint8_t *sA = smem;                       // G^T: [128 rows = channels][K = 128 rows of the tile]
    uint8_t *sB = smem + 128 * 128 * 2;       // X^T: [N][128]
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 0) tmem_alloc(&tslot, NCOLS);
    // rows M..127 of G^T stay zero for every tile
    for (int i = tid; i < 128 * 128 * 2 / 16; i += 128) reinterpret_cast<uint4 *>(sA)[i] = make_uint4(0, 0, 0, 0);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tslot;
    const int b = blockIdx.y;
    const int64_t t_begin = (int64_t)blockIdx.x * p.tiles_per_cta;
    const int64_t t_end = std::min<int64_t>(p.tiles, t_begin + p.tiles_per_cta);
    const uint32_t idesc = idesc_f16(128, N, 1);
    uint32_t ph = 0;
    int issued = 0;
    bool ok = true;
    for (int64_t tile = t_begin; tile < t_end; ++tile) {
        const int64_t row = tile * kRows + tid;   // thread = row of the tile = K index of the MMA
        const bool live = row < p.rows;
        // G^T: element (m, k = tid) at chunk k / 8, row m, position k % 8
        const uint32_t kofs = (uint32_t)(tid >> 3) * 128 * 16 + (uint32_t)(tid & 7) * 2;
        const __nv_bfloat16 *g = p.G + b * p.g_boff + row * p.ldg;
        {
            uint4 v[16];                      // M <= 128: at most 16 chunks, all loads issued first
#pragma unroll
            for (int q = 0; q < 16; ++q)
                v[q] = (live && 8 * q < p.M) ? __ldg(reinterpret_cast<const uint4 *>(g + 8 * q)) : make_uint4(0, 0, 0, 0);
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                if (8 * q >= p.M) break;
                const uint16_t *e = reinterpret_cast<const uint16_t *>(&v[q]);
#pragma unroll
                for (int i = 0; i < 8; ++i) *reinterpret_cast<uint16_t *>(sA + kofs + (8 * q + i) * 16) = e[i];
            }
        }
        // X^T: element (n, k = tid) at chunk k / 8, row n, position k % 8
        const uint32_t kofsb = (uint32_t)(tid >> 3) * N * 16 + (uint32_t)(tid & 7) * 2;
        {
            uint4 v[N / 8];                   // all X chunks of the row, loads issued first
            const int c0 = p.xs[0].C / 8;     // chunks of the first segment; the rest from the second
            const int cx = p.nx / 8;          // beyond: the ones column (BF16 1.0 at column nx) and zeros
#pragma unroll
            for (int k = 0; k < N / 8; ++k)
                v[k] = !live ? make_uint4(0, 0, 0, 0)
                             : (k < c0 ? seg_load(p.xs[0], b, row, p.W, k)
                                       : (k < cx ? seg_load(p.xs[1], b, row, p.W, k - c0)
                                                 : make_uint4(k == cx ? 0x3F80u : 0u, 0, 0, 0)));
#pragma unroll
            for (int k = 0; k < N / 8; ++k) {
                const uint16_t *e = reinterpret_cast<const uint16_t *>(&v[k]);
#pragma unroll
                for (int i = 0; i < 8; ++i) *reinterpret_cast<uint16_t *>(sB + kofsb + (8 * k + i) * 16) = e[i];
            }
        }
        fence_proxy_async_smem();
        tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
#pragma unroll
            for (int ks = 0; ks < 8; ++ks) {
                const uint64_t ad = sdesc(a0 + ks * 2 * 128 * 16, 128 * 16, 128);
                const uint64_t bd = sdesc(b0 + ks * 2 * N * 16, N * 16, 128);
                mma_f16(tmem, ad, bd, idesc, (issued > 0 || ks > 0) ? 1u : 0u);
            }
            mma_commit(&bar[0]);
        }
        ++issued;
        // the tile's shared memory is rewritten by the next tile: wait for the MMAs to read it
        const bool w_ok = mbar_wait(&bar[0], ph & 1, &abort_flag, p.err, 80, kWaitNs);
        ++ph;
        if (__syncthreads_or(!w_ok)) {
            ok = false;
            break;
        }
    }
    if (ok && issued > 0) {
        tc_fence_after();
        // D[m][n] in TMEM lane m: warps whose lanes hold m < M add their rows
        const int m = tid;
        const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);
        for (int c0 = 0; c0 < N; c0 += 16) {
            uint32_t v[16];
            tmem_ld16(tl + c0, v);
            tmem_ld_wait();
            if (m < p.M) {
                float *dw = p.dW + b * p.w_boff + (int64_t)m * p.ldw + c0;
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    if (c0 + j < p.nx)
                        atomicAdd(dw + j, __uint_as_float(v[j]));
                    else if (c0 + j == p.nx && p.db)
                        atomicAdd(p.db + b * p.w_boff + m, __uint_as_float(v[j]));
                }
            }
        }
    }
    if (tid == 0) {
        mma_commit(&bar[1]);
        mbar_wait_drain(&bar[1], 0, p.err, 81, kWaitNs);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, NCOLS);
    }
}

__global__ void k_f32_to_bf16(const float *__restrict__ in, __nv_bfloat16 *__restrict__ out, int64_t n) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        out[i] = __float2bfloat16_rn(in[i]);
}

// ---------------------------------------------------------------------------- host side

// B images of one model (BF16, chunk layout [N rows][K]): per layer and branch
//   conv [2R][2R]      row o = Wconv[o][tap][i] at k = tap * R + i
//   rs   [R + S][R]    rows W_res then W_skip (forward)
//   dz   [R][R + S]    row i: W_res[o][i] at k = o, W_skip[o][i] at k = R + o
//   dgr  [R][4R]       row i: Wconv[o][1][i] at k = o, Wconv[o][0][i] at k = 2R + o
struct TcBwd {
    DevBuf img;
    std::vector<uint8_t> host;
    size_t conv_b = 0, rs_b = 0, dz_b = 0, dg_b = 0, layer_b = 0;
    int model = -1;
    uint64_t stamp = 0;
    DevBuf xsave, skip, dskip32, dskip16, x32, x16, gate16, z16, dx32[2], dx16[2], da16, err;
};

inline size_t choff(int rows, int n, int k) { return (size_t)(k / 8) * rows * 16 + (size_t)n * 16 + (k % 8) * 2; }

void put_bf16(std::vector<uint8_t> &v, size_t off, float x) {
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    std::memcpy(v.data() + off, &h, 2);
}

void build_bwd_images(const Dims &d, const float *blob, TcBwd &t) {
    const int R = d.R, S = d.S, L = d.L;
    t.conv_b = (size_t)2 * R * 2 * R * 2;
    t.rs_b = (size_t)(R + S) * R * 2;
    t.dz_b = (size_t)R * (R + S) * 2;
    t.dg_b = (size_t)R * 4 * R * 2;
    t.layer_b = t.conv_b + t.rs_b + t.dz_b + t.dg_b;
    t.host.assign(t.layer_b * 2 * L, 0);
    for (int b = 0; b < 2; ++b)
        for (int l = 0; l < L; ++l) {
            const size_t base = t.layer_b * ((size_t)l * 2 + b);
            const float *wc = blob + off_wconv(d, b, l);      // [2R][2][R]
            const float *wr = blob + off_wres(d, b, l);       // [R][R]
            const float *ws = blob + off_wskip(d, b, l);      // [S][R]
            for (int o = 0; o < 2 * R; ++o)
                for (int k = 0; k < 2 * R; ++k) put_bf16(t.host, base + choff(2 * R, o, k), wc[o * 2 * R + k]);
            const size_t rs = base + t.conv_b;
            for (int o = 0; o < R + S; ++o)
                for (int i = 0; i < R; ++i)
                    put_bf16(t.host, rs + choff(R + S, o, i), o < R ? wr[o * R + i] : ws[(o - R) * R + i]);
            const size_t dz = rs + t.rs_b;
            for (int i = 0; i < R; ++i)
                for (int k = 0; k < R + S; ++k)
                    put_bf16(t.host, dz + choff(R, i, k), k < R ? wr[k * R + i] : ws[(k - R) * R + i]);
            const size_t dg = dz + t.dz_b;
            for (int i = 0; i < R; ++i)
                for (int k = 0; k < 4 * R; ++k) {
                    const int o = k % (2 * R), tap = k < 2 * R ? 1 : 0;
                    put_bf16(t.host, dg + choff(R, i, k), wc[(o * 2 + tap) * R + i]);
                }
        }
}

int g_rows_smem_set = 0;

gwe_status set_attrs() {
    if (g_rows_smem_set) return GWE_OK;
    const int big = 200 * 1024;
    GWE_CUDA_TRY(cudaFuncSetAttribute(k_tc_rows<EPI_CONV>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    GWE_CUDA_TRY(cudaFuncSetAttribute(k_tc_rows<EPI_RES>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    GWE_CUDA_TRY(cudaFuncSetAttribute(k_tc_rows<EPI_DZ>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    GWE_CUDA_TRY(cudaFuncSetAttribute(k_tc_rows<EPI_DGRAD>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    GWE_CUDA_TRY(cudaFuncSetAttribute(k_tc_wgrad<48>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    GWE_CUDA_TRY(cudaFuncSetAttribute(k_tc_wgrad<80>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    GWE_CUDA_TRY(cudaFuncSetAttribute(k_tc_wgrad<144>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    g_rows_smem_set = 1;
    return GWE_OK;
}

RowSeg seg(const __nv_bfloat16 *p, int64_t boff, int ld, int C, int shift) {
    RowSeg s;
    s.p = p;
    s.boff = boff;
    s.ld = ld;
    s.C = C;
    s.shift = shift;
    return s;
}

template <int EPI>
gwe_status run_rows(RowGemm p, int sms, cudaStream_t st) {
    const int64_t tpb = (p.rows + kRows - 1) / kRows;
    p.n_tiles = tpb * p.nbranch;
    if (p.bn < p.N) p.bn = p.N;
    // at least 80 KB of shared memory per CTA, so that at most two CTAs (2 x <= 256 TMEM columns)
    // share an SM and no TMEM allocation has to wait
    const size_t smem = std::max<size_t>((size_t)kRows * p.K * 2 + (size_t)p.bn * p.K * 2 + 128, 80 * 1024);
    const int grid = (int)std::min<int64_t>(p.n_tiles, (int64_t)sms * (smem <= 100 * 1024 ? 2 : 1));
    ProfScope prof("k_tc_rows", st);
    k_tc_rows<EPI><<<grid, 128, smem, st>>>(p);
    note_launch();
    GWE_CUDA_TRY(cudaGetLastError());
    return GWE_OK;
}

gwe_status run_wgrad(WgGemm p, int sms, cudaStream_t st) {
    p.tiles = (p.rows + kRows - 1) / kRows;
    // about four CTAs per SM over both branches, at least 8 tiles each
    const int64_t want = std::max<int64_t>(1, (int64_t)sms * 2);
    p.tiles_per_cta = (int)std::max<int64_t>(8, (p.tiles + want - 1) / want);
    dim3 grid((unsigned)((p.tiles + p.tiles_per_cta - 1) / p.tiles_per_cta), 2);
    // with 256 TMEM columns (N > 128) at most two CTAs may share an SM: ask for at least 80 KB
    const size_t smem = std::max<size_t>((size_t)128 * 128 * 2 + (size_t)p.N * 128 * 2 + 128,
                                         p.N > 128 ? 80 * 1024 : 0);
    ProfScope prof("k_tc_wgrad", st);
    // N = nx + 16: the segments' columns, then the ones column for the bias gradient (nx = 32, 64, 128)
    if (p.N == 48)
        k_tc_wgrad<48><<<grid, 128, smem, st>>>(p);
    else if (p.N == 80)
        k_tc_wgrad<80><<<grid, 128, smem, st>>>(p);
    else if (p.N == 144)
        k_tc_wgrad<144><<<grid, 128, smem, st>>>(p);
    else {
        set_error("tensor-core backward: unsupported weight-gradient width");
        return GWE_ERR_UNSUPPORTED;
    }
    note_launch();
    GWE_CUDA_TRY(cudaGetLastError());
    return GWE_OK;
}

}  // namespace

bool tc_backward_supported(const Dims &d) {
    return d.k == 2 && d.R % 16 == 0 && d.S % 16 == 0 && 2 * d.R <= 128 && d.R + d.S <= 256 && d.S <= 128 &&
           d.R >= 16;
}

void tc_backward_release(void *&state) {
    TcBwd *t = reinterpret_cast<TcBwd *>(state);
    if (!t) return;
    DevBuf *all[] = {&t->img, &t->xsave, &t->skip, &t->dskip32, &t->dskip16, &t->x32, &t->x16, &t->gate16, &t->z16,
                     &t->dx32[0], &t->dx32[1], &t->dx16[0], &t->dx16[1], &t->da16, &t->err};
    for (DevBuf *b : all) b->release();
    delete t;
    state = nullptr;
}

// The FP32 head backward, bias sums, input projection and dstrain of fp32_path.cu.
gwe_status fp32_head_backward(gwe_model *m, int mi, const float *skip, int64_t rb, int W, int C, const float *dlogit,
                              float *dskip, float *gw, cudaStream_t st);
gwe_status fp32_bias_grad(const float *G, int ldg, int N, int64_t g_boff, float *db, int64_t db_boff, int W, int C,
                          int nbranch, cudaStream_t st);
gwe_status fp32_input_backward(gwe_model *m, int mi, const float *dx0, int64_t rb, const float *sH, const float *sL,
                               int W, int C, float *gw, float *gH, float *gL, cudaStream_t st);
gwe_status fp32_input_proj(gwe_model *m, int mi, const float *sH, const float *sL, int64_t rb, float *x0,
                           cudaStream_t st);

gwe_status tc_backward(gwe_model *m, void *&state, int mi, const float *xH, const float *xL, int batch, int W,
                       const float *dlogit, float *gw, float *gH, float *gL, int sms, cudaStream_t st) {
    const Dims &d = m->dims;
    if (!tc_backward_supported(d)) {
        set_error("tensor-core backward: unsupported channel counts");
        return GWE_ERR_UNSUPPORTED;
    }
    gwe_status r = set_attrs();
    if (r != GWE_OK) return r;
    TcBwd *t = reinterpret_cast<TcBwd *>(state);
    if (!t) {
        t = new TcBwd();
        state = t;
    }
    const int R = d.R, S = d.S, L = d.L, lps = d.lps, stacks = d.stacks;
    const float *blob = m->w32.as<float>() + (int64_t)mi * d.P;
    // B images from the current FP32 weights (rebuilt when the weights or the member change)
    const uint64_t stamp = m->wstamp;
    if (t->model != mi || t->stamp != stamp || t->host.empty()) {
        std::vector<float> hb((size_t)d.P);
        GWE_CUDA_TRY(cudaMemcpy(hb.data(), blob, sizeof(float) * d.P, cudaMemcpyDeviceToHost));
        build_bwd_images(d, hb.data(), *t);
        GWE_CUDA_TRY(t->img.ensure(t->host.size()));
        GWE_CUDA_TRY(cudaMemcpy(t->img.ptr, t->host.data(), t->host.size(), cudaMemcpyHostToDevice));
        t->model = mi;
        t->stamp = stamp;
    }
    const int C = std::min(batch, 64);                       // windows per chunk
    const size_t rows = (size_t)C * W, rows2 = 2 * rows;
    GWE_CUDA_TRY(t->err.ensure(256));
    GWE_CUDA_TRY(cudaMemsetAsync(t->err.ptr, 0, sizeof(int), st));
    GWE_CUDA_TRY(t->xsave.ensure(sizeof(float) * stacks * rows2 * R));
    GWE_CUDA_TRY(t->skip.ensure(sizeof(float) * rows2 * S));
    GWE_CUDA_TRY(t->dskip32.ensure(sizeof(float) * rows2 * S));
    GWE_CUDA_TRY(t->dskip16.ensure(2 * rows2 * S));
    GWE_CUDA_TRY(t->x32.ensure(sizeof(float) * (lps + 1) * rows2 * R));
    GWE_CUDA_TRY(t->x16.ensure(2 * (lps + 1) * rows2 * R));
    GWE_CUDA_TRY(t->gate16.ensure(2 * lps * rows2 * 2 * R));
    GWE_CUDA_TRY(t->z16.ensure(2 * lps * rows2 * R));
    for (int i = 0; i < 2; ++i) {
        GWE_CUDA_TRY(t->dx32[i].ensure(sizeof(float) * rows2 * R));
        GWE_CUDA_TRY(t->dx16[i].ensure(2 * rows2 * R));
    }
    GWE_CUDA_TRY(t->da16.ensure(2 * rows2 * 2 * R));
    GWE_CUDA_TRY(cudaMemsetAsync(gw, 0, sizeof(float) * d.P, st));
    const int64_t Pb = d.Pb;
    int *err = t->err.as<int>();
    const uint8_t *img = t->img.as<uint8_t>();
    auto limg = [&](int l, int b) { return img + t->layer_b * ((size_t)l * 2 + b); };
    float *x32 = t->x32.as<float>(), *xsave = t->xsave.as<float>();
    __half *gate16 = t->gate16.as<__half>();
    __nv_bfloat16 *x16 = t->x16.as<__nv_bfloat16>(), *z16 = t->z16.as<__nv_bfloat16>();

    for (int c0 = 0; c0 < batch; c0 += C) {
        const int Cc = std::min(C, batch - c0);
        const int64_t rb = (int64_t)Cc * W;          // rows per branch
        const int64_t xo = rb * R;                   // branch offset of [row][R] arrays (this chunk)
        const float *sH = xH + (int64_t)c0 * W, *sL = xL + (int64_t)c0 * W;
        // one layer's forward: conv (a optional) then res (+ skip when skip_mode >= 0)
        auto layer_fwd = [&](int l, float *xin32, __nv_bfloat16 *xin16, float *xout32, __nv_bfloat16 *xout16,
                             __half *gout, __nv_bfloat16 *zout, int skip_mode) -> gwe_status {
            const int dl = 1 << (l % lps);
            RowGemm p{};
            p.seg[0] = seg(xin16, xo, R, R, -dl);
            p.seg[1] = seg(xin16, xo, R, R, 0);
            p.nseg = 2;
            p.K = 2 * R;
            p.N = 2 * R;
            p.bimg = limg(l, 0);
            p.bimg_boff = (int64_t)(limg(l, 1) - limg(l, 0));
            p.rows = rb;
            p.W = W;
            p.nbranch = 2;
            p.err = err;
            p.R = R;
            p.bias = blob + off_bconv(d, 0, l);
            p.bias_boff = Pb;
            p.gate_out = gout;
            p.gate_boff = rb * 2 * R;
            p.o16 = zout;
            p.o16_boff = xo;
            gwe_status e = run_rows<EPI_CONV>(p, sms, st);
            if (e != GWE_OK) return e;
            RowGemm q{};
            q.seg[0] = seg(zout, xo, R, R, 0);
            q.nseg = 1;
            q.K = R;
            q.N = skip_mode >= 0 ? R + S : R;
            q.bn = R + S;
            q.bimg = limg(l, 0) + t->conv_b;
            q.bimg_boff = p.bimg_boff;
            q.rows = rb;
            q.W = W;
            q.nbranch = 2;
            q.err = err;
            q.R = R;
            q.bias = blob + off_bres(d, 0, l);
            q.bias2 = blob + off_bskip(d, 0, l);
            q.bias_boff = Pb;
            q.aux = xin32;
            q.aux_boff = xo;
            q.o32 = xout32;
            q.o32_boff = xo;
            q.o16 = xout16;
            q.o16_boff = xo;
            q.skip = t->skip.as<float>();
            q.skip_boff = rb * S;
            q.skip_init = skip_mode == 1;
            return run_rows<EPI_RES>(q, sms, st);
        };
        // ---- forward keeping each stack's input and the skip sums
        {
            float *xa32 = x32, *xb32 = x32 + rows2 * R;
            __nv_bfloat16 *xa16 = x16, *xb16 = x16 + rows2 * R;
            r = fp32_input_proj(m, mi, sH, sL, rb, xa32, st);
            if (r != GWE_OK) return r;
            k_f32_to_bf16<<<1024, 256, 0, st>>>(xa32, xa16, 2 * rb * R);
            note_launch();
            for (int l = 0; l < L; ++l) {
                if (l % lps == 0)
                    GWE_CUDA_TRY(cudaMemcpyAsync(xsave + (size_t)(l / lps) * rows2 * R, xa32, sizeof(float) * 2 * rb * R,
                                                 cudaMemcpyDeviceToDevice, st));
                r = layer_fwd(l, xa32, xa16, xb32, xb16, nullptr, z16, l == 0 ? 1 : 0);
                if (r != GWE_OK) return r;
                std::swap(xa32, xb32);
                std::swap(xa16, xb16);
            }
        }
        // ---- head (FP32): dskip
        r = fp32_head_backward(m, mi, t->skip.as<float>(), rb, W, Cc, dlogit + (int64_t)c0 * W, t->dskip32.as<float>(),
                               gw, st);
        if (r != GWE_OK) return r;
        k_f32_to_bf16<<<1024, 256, 0, st>>>(t->dskip32.as<float>(), t->dskip16.as<__nv_bfloat16>(), 2 * rb * S);
        note_launch();
        // ---- branches, stack by stack in reverse
        int hi = 0;   // dx buffers: [hi] = dL/dx_{l+1}
        GWE_CUDA_TRY(cudaMemsetAsync(t->dx32[hi].ptr, 0, sizeof(float) * 2 * rb * R, st));
        GWE_CUDA_TRY(cudaMemsetAsync(t->dx16[hi].ptr, 0, 2 * 2 * rb * R, st));
        for (int k = stacks - 1; k >= 0; --k) {
            GWE_CUDA_TRY(cudaMemcpyAsync(x32, xsave + (size_t)k * rows2 * R, sizeof(float) * 2 * rb * R,
                                         cudaMemcpyDeviceToDevice, st));
            k_f32_to_bf16<<<1024, 256, 0, st>>>(x32, x16, 2 * rb * R);
            note_launch();
            for (int j = 0; j < lps; ++j) {
                const int l = k * lps + j;
                r = layer_fwd(l, x32 + (size_t)j * rows2 * R, x16 + (size_t)j * rows2 * R,
                              x32 + (size_t)(j + 1) * rows2 * R, x16 + (size_t)(j + 1) * rows2 * R,
                              gate16 + (size_t)j * rows2 * 2 * R, z16 + (size_t)j * rows2 * R, -1);
                if (r != GWE_OK) return r;
            }
            for (int j = lps - 1; j >= 0; --j) {
                const int l = k * lps + j, dl = 1 << j;
                const __nv_bfloat16 *xl16 = x16 + (size_t)j * rows2 * R;
                const __nv_bfloat16 *zl16 = z16 + (size_t)j * rows2 * R;
                const __half *gl = gate16 + (size_t)j * rows2 * 2 * R;
                float *dxh32 = t->dx32[hi].as<float>(), *dxl32 = t->dx32[hi ^ 1].as<float>();
                __nv_bfloat16 *dxh16 = t->dx16[hi].as<__nv_bfloat16>(), *dxl16 = t->dx16[hi ^ 1].as<__nv_bfloat16>();
                // dz = [dx_{l+1} | dskip] . [W_res | W_skip], gate backward -> da
                {
                    RowGemm p{};
                    p.seg[0] = seg(dxh16, xo, R, R, 0);
                    p.seg[1] = seg(t->dskip16.as<__nv_bfloat16>(), rb * S, S, S, 0);
                    p.nseg = 2;
                    p.K = R + S;
                    p.N = R;
                    p.bimg = limg(l, 0) + t->conv_b + t->rs_b;
                    p.bimg_boff = (int64_t)(limg(l, 1) - limg(l, 0));
                    p.rows = rb;
                    p.W = W;
                    p.nbranch = 2;
                    p.err = err;
                    p.R = R;
                    p.gate = gl;
                    p.gate_boff = rb * 2 * R;
                    p.o16 = t->da16.as<__nv_bfloat16>();
                    p.o16_boff = rb * 2 * R;
                    r = run_rows<EPI_DZ>(p, sms, st);
                    if (r != GWE_OK) return r;
                }
                // weight gradients of this layer
                {
                    WgGemm g{};
                    g.G = t->da16.as<__nv_bfloat16>();
                    g.g_boff = rb * 2 * R;
                    g.ldg = 2 * R;
                    g.M = 2 * R;
                    g.xs[0] = seg(xl16, xo, R, R, -dl);
                    g.xs[1] = seg(xl16, xo, R, R, 0);
                    g.nxs = 2;
                    g.nx = 2 * R;
                    g.N = 2 * R + 16;
                    g.db = gw + off_bconv(d, 0, l);
                    g.rows = rb;
                    g.W = W;
                    g.dW = gw + off_wconv(d, 0, l);
                    g.ldw = 2 * R;
                    g.w_boff = Pb;
                    g.err = err;
                    r = run_wgrad(g, sms, st);
                    if (r != GWE_OK) return r;
                    WgGemm gr = g;
                    gr.G = dxh16;
                    gr.g_boff = xo;
                    gr.ldg = R;
                    gr.M = R;
                    gr.xs[0] = seg(zl16, xo, R, R, 0);
                    gr.nxs = 1;
                    gr.nx = R;
                    gr.N = R + 16;
                    gr.dW = gw + off_wres(d, 0, l);
                    gr.db = gw + off_bres(d, 0, l);
                    gr.ldw = R;
                    r = run_wgrad(gr, sms, st);
                    if (r != GWE_OK) return r;
                    WgGemm gs = gr;
                    gs.G = t->dskip16.as<__nv_bfloat16>();
                    gs.g_boff = rb * S;
                    gs.ldg = S;
                    gs.M = S;
                    gs.dW = gw + off_wskip(d, 0, l);
                    gs.db = gw + off_bskip(d, 0, l);
                    r = run_wgrad(gs, sms, st);
                    if (r != GWE_OK) return r;
                }
                // dx_l = dx_{l+1} + [da(t) | da(t + d)] . [W1 ; W0]
                {
                    RowGemm p{};
                    p.seg[0] = seg(t->da16.as<__nv_bfloat16>(), rb * 2 * R, 2 * R, 2 * R, 0);
                    p.seg[1] = seg(t->da16.as<__nv_bfloat16>(), rb * 2 * R, 2 * R, 2 * R, dl);
                    p.nseg = 2;
                    p.K = 4 * R;
                    p.N = R;
                    p.bimg = limg(l, 0) + t->conv_b + t->rs_b + t->dz_b;
                    p.bimg_boff = (int64_t)(limg(l, 1) - limg(l, 0));
                    p.rows = rb;
                    p.W = W;
                    p.nbranch = 2;
                    p.err = err;
                    p.R = R;
                    p.aux = dxh32;
                    p.aux_boff = xo;
                    p.o32 = dxl32;
                    p.o32_boff = xo;
                    p.o16 = dxl16;
                    p.o16_boff = xo;
                    r = run_rows<EPI_DGRAD>(p, sms, st);
                    if (r != GWE_OK) return r;
                }
                hi ^= 1;
            }
        }
        r = fp32_input_backward(m, mi, t->dx32[hi].as<float>(), rb, sH, sL, W, Cc, gw, gH ? gH + (int64_t)c0 * W : nullptr,
                                gL ? gL + (int64_t)c0 * W : nullptr, st);
        if (r != GWE_OK) return r;
    }
    // a device-side wait that gave up leaves its site in the error word
    int e = 0;
    GWE_CUDA_TRY(cudaMemcpyAsync(&e, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    GWE_CUDA_TRY(cudaStreamSynchronize(st));
    if (e != 0) {
        set_error("tensor-core backward: a device-side wait timed out (site " + std::to_string(e) + ")");
        return GWE_ERR_TIMEOUT;
    }
    return GWE_OK;
}

}  // namespace gwe
