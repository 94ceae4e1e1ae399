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
// Row GEMMs bring in their A tile (tensor-map copies with the 128-byte swizzle where the shapes
// allow, else per-thread copies; window boundaries zero-filled) and keep the layer's B image in
// shared memory; the MMA accumulates in TMEM and the epilogue (thread = row)
// applies the fused step.  Weight-gradient GEMMs bring in G^T and X^T tiles (tensor-map copies with
// the 128-byte swizzle where every operand has 64 or 128 channels, else per-thread copies),
// accumulate over a range of row tiles in TMEM and add their partial sums atomically.
// The stack inputs and skip sums that the per-stack recomputation starts from come, for BF16
// handles, from the fused forward kernel (one launch per chunk, training save mode); otherwise from
// a forward pass of row GEMMs.  The head, the input projection and dL/dstrain use the FP32 kernels.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <vector>

#include "gwe_internal.h"
#include "tc_ptx.cuh"

namespace gwe {
namespace {

using namespace tc;

constexpr int kRows = 128;              // rows per tile (the MMA's M)
constexpr int kWgThreads = 512;         // weight-gradient GEMM: 4 threads per staged row
constexpr uint64_t kWaitNs = 4000000000ull;
// 1: operands by tensor-map copies where the shapes allow (gwe_set_tensor_map_copies)
std::atomic<int> g_tma_copies{1};

// one K-range of a row GEMM's A operand: columns [0, C) of a row-major BF16 array, taken at row
// t + shift of the same window (zero outside [0, W))
struct RowSeg {
    const __nv_bfloat16 *p;
    int64_t boff;      // elements between the branches' arrays
    int ld;            // elements per row
    int C;             // columns (multiple of 8)
    int shift;
};

// EPI_HEAD_U: u = [h_H | h_L] . W_h1^T (N = Hc, K = 2S), du = (u + b_h1 > 0) ? dlogit w_h2 : 0, ReLU(u + b_h1);
// EPI_HEAD_DH: dh = du . W_h1 (N = 2S, K = Hc), dskip_b = (h_b > 0) ? dh_b : 0 (thread half = branch)
enum { EPI_CONV = 0, EPI_RES = 1, EPI_DZ = 2, EPI_DGRAD = 3, EPI_HEAD_U = 4, EPI_HEAD_DH = 5 };

// ---------------------------------------------------------------- tensor-map copies
// Tiled global -> shared copies through a tensor map (a kernel parameter), completion counted in
// bytes on the mbarrier at `bar`; out-of-range coordinates are zero-filled.
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, uint32_t bar, int c0, int c1,
                                            int c2) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], "
        "[%2];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(c0), "r"(c1), "r"(c2)
        : "memory");
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap *map, uint32_t bar, int c0, int c1,
                                            int c2, int c3) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5, "
        "%6}], [%2];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
        : "memory");
}

// shared-memory descriptor of an operand in the 128-byte swizzled layout (layout type 2)
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr, uint32_t lbo_bytes, uint32_t sbo_bytes) {
    return sdesc(saddr, lbo_bytes, sbo_bytes) | (2ull << 61);
}

struct RowGemm {
    CUtensorMap a_map[2];             // a_tma: the segments as {C channels, W, windows, branches}
    int a_tma;                        // 1: A tiles by tensor-map copies (128-byte swizzle, K-major)
    int a_nb[2];                      // 2 when the branches have their own segment array, else 1
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
    const __nv_bfloat16 *mask16;      // EPI_HEAD_DH: h = ReLU(skip) [branch][row][S] (BF16)
    __nv_bfloat16 *o16_lo;            // EPI_HEAD_U: du - BF16(du) in BF16
    int64_t mask_boff;
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
    int db_nb;                        // branches that add their sums to db (at db + b * w_boff); 0 = all
    int nx;                           // columns of X from the segments (N = nx, or nx + 16 with db)
    int *err;
};

__device__ __forceinline__ uint32_t tmem_cols_for(int n) {
    uint32_t c = 32;
    while ((int)c < n) c <<= 1;
    return c;
}

__device__ __forceinline__ float tanh_approx(float x) {
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// 16-byte global -> shared copy in flight until cp_async_wait_all; zero-filled when !valid
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, bool valid) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(valid ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_group() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// address of 8 BF16 values of row `row` of segment s at chunk c, and whether they lie in the window
__device__ __forceinline__ const __nv_bfloat16 *seg_addr(const RowSeg &s, int b, int64_t row, int W, int c,
                                                          bool &valid) {
    const int64_t w = row / W;
    const int t = (int)(row - w * W) + s.shift;
    valid = t >= 0 && t < W;
    return valid ? s.p + b * s.boff + (w * W + t) * (int64_t)s.ld + 8 * c : s.p;
}

// 16 consecutive values of one row (16-byte aligned): FP32, FP16 and BF16 stores
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

// Warp-cooperative stores of 16 consecutive values per lane's row (lane = row, rows 32 lanes apart in
// memory by the array's row pitch): the values go through a per-warp staging area in shared memory
// (80-byte row pitch, so that eight consecutive rows hit distinct banks) and come back out so that
// each store instruction writes whole 32-byte sectors of 8 rows (FP32) or 16 rows (16-bit) instead of
// half sectors of 32 rows.  Rows whose `live` is false are not stored.  Every lane of the warp calls.
constexpr uint32_t kWarpStage = 32 * 80;   // bytes of staging per warp
__device__ __forceinline__ uint4 lds128(uint32_t addr) {
    uint4 v;
    asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(addr));
    return v;
}
__device__ __forceinline__ void wst16_f32(float *dst, const float (&v)[16], bool live, uint32_t stg, int lane) {
#pragma unroll
    for (int q = 0; q < 4; ++q)
        asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(stg + lane * 80 + q * 16),
                     "r"(__float_as_uint(v[4 * q])), "r"(__float_as_uint(v[4 * q + 1])),
                     "r"(__float_as_uint(v[4 * q + 2])), "r"(__float_as_uint(v[4 * q + 3]))
                     : "memory");
    __syncwarp();
    const unsigned long long d = reinterpret_cast<unsigned long long>(dst);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int rr = 8 * i + (lane >> 2), c = lane & 3;
        const unsigned long long dr = __shfl_sync(0xffffffffu, d, rr);
        const int lv = __shfl_sync(0xffffffffu, live ? 1 : 0, rr);
        const uint4 x = lds128(stg + rr * 80 + c * 16);
        if (lv) *reinterpret_cast<uint4 *>(reinterpret_cast<float *>(dr) + 4 * c) = x;
    }
    __syncwarp();
}
__device__ __forceinline__ void wst16_w(void *dst, const uint32_t (&w)[8], bool live, uint32_t stg, int lane) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(stg + lane * 80), "r"(w[0]), "r"(w[1]), "r"(w[2]),
                 "r"(w[3])
                 : "memory");
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(stg + lane * 80 + 16), "r"(w[4]), "r"(w[5]),
                 "r"(w[6]), "r"(w[7])
                 : "memory");
    __syncwarp();
    const unsigned long long d = reinterpret_cast<unsigned long long>(dst);
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int rr = 16 * i + (lane >> 1), c = lane & 1;
        const unsigned long long dr = __shfl_sync(0xffffffffu, d, rr);
        const int lv = __shfl_sync(0xffffffffu, live ? 1 : 0, rr);
        const uint4 x = lds128(stg + rr * 80 + c * 16);
        if (lv) *reinterpret_cast<uint4 *>(reinterpret_cast<uint8_t *>(dr) + 16 * c) = x;
    }
    __syncwarp();
}
// The same through a narrower staging area (48-byte row pitch, 32 bytes per row and pass: eight
// FP32 or sixteen 16-bit values), for the dgrad epilogue, whose tiles leave only 12 KB of shared
// memory at two CTAs per SM; each store instruction writes whole sectors of 16 rows.
constexpr uint32_t kWarpStageNarrow = 32 * 48;
__device__ __forceinline__ void wst32b_p48(void *dst, uint4 lo, uint4 hi, bool live, uint32_t stg, int lane) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(stg + lane * 48), "r"(lo.x), "r"(lo.y), "r"(lo.z),
                 "r"(lo.w)
                 : "memory");
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(stg + lane * 48 + 16), "r"(hi.x), "r"(hi.y),
                 "r"(hi.z), "r"(hi.w)
                 : "memory");
    __syncwarp();
    const unsigned long long d = reinterpret_cast<unsigned long long>(dst);
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int rr = 16 * i + (lane >> 1), c = lane & 1;
        const unsigned long long dr = __shfl_sync(0xffffffffu, d, rr);
        const int lv = __shfl_sync(0xffffffffu, live ? 1 : 0, rr);
        const uint4 x = lds128(stg + rr * 48 + c * 16);
        if (lv) *reinterpret_cast<uint4 *>(reinterpret_cast<uint8_t *>(dr) + 16 * c) = x;
    }
    __syncwarp();
}
__device__ __forceinline__ void pack16_bf16(const float (&v)[16], uint32_t (&w)[8]) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
        w[q] = *reinterpret_cast<const uint32_t *>(&h);
    }
}
__device__ __forceinline__ void pack16_f16(const float (&v)[16], uint32_t (&w)[8]) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const __half2 h = __floats2half2_rn(v[2 * q], v[2 * q + 1]);
        w[q] = *reinterpret_cast<const uint32_t *>(&h);
    }
}

// D = A . B^T over the row tiles of both branches, fused epilogue EPI.
// 256 threads: thread (r = tid % 128, h = tid / 128) owns row r of the tile and half h of the
// epilogue's channels (TMEM lanes of warp w: 32 (w % 4) ..).  Per tile the epilogue's global
// operands are loaded into registers before the MMA is waited for, and the next tile's A copies
// (and B image, at a branch change) are issued as soon as the MMA has read shared memory, so that
// they are in flight while the epilogue runs.  With p.a_tma thread 0 issues the A tile as
// tensor-map boxes (one per 64-channel block, 128-byte swizzle, completion on bar[2]) and waits for
// them before the MMAs; otherwise every thread stages its share with 16-byte copies.
template <int EPI>
__global__ void __launch_bounds__(256, 2) k_tc_rows(const __grid_constant__ RowGemm p) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    __shared__ uint64_t bar[3];   // MMA done; final drain; A tile landed (tensor-map copies)
    __shared__ uint32_t tslot;
    __shared__ int abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int r = tid & 127, h = tid >> 7;
    const int KC = p.K / 8;                                   // 16-byte chunks per row
    const uint32_t a_bytes = (uint32_t)kRows * p.K * 2;   // B image follows the A tile
    uint8_t *sA = smem, *sB = smem + a_bytes;
    // epilogues with staged (coalesced) stores: a per-warp staging area after the B image
    const uint32_t stg = smem_u32(smem + a_bytes + (uint32_t)p.bn * p.K * 2) +
                         (tid >> 5) * (EPI == EPI_DGRAD ? kWarpStageNarrow : kWarpStage);
    const int lane = tid & 31;
    const uint32_t ncols = tmem_cols_for(p.N);
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_init(&bar[2], 1);
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
    uint32_t a_issued = 0, a_landed = 0;                      // thread 0: tensor-map A tiles
    // cp.async copies of one tile: B image at a branch change, A tile in chunk-column layout
    // (chunks 2j and 2j + 1 of row tid / 2 by threads tid & ~1 and tid | 1, so that a lane pair
    // reads one 32-byte sector; window boundaries zero-filled)
    auto issue_tile = [&](int64_t tile) {
        const int b = (int)(tile / tpb);
        const int64_t r0 = (tile - (int64_t)b * tpb) * kRows;
        if (b != cur_b) {
            const uint8_t *src = p.bimg + b * p.bimg_boff;
            const int n16 = p.bn * p.K * 2 / 16;
            for (int i = tid; i < n16; i += 256) cp_async16(smem_u32(sB + 16 * i), src + 16 * i, true);
            cur_b = b;
        }
        if (p.a_tma) {
            // one thread: each 64-channel block of the segments as 128 rows of 128 bytes (128-byte
            // swizzle), block j at sA + j * 16 KB; the tile lies in one window (W % 128 == 0)
            if (tid == 0) {
                const int w = (int)(r0 / p.W), t0 = (int)(r0 - (int64_t)w * p.W);
                const uint32_t a = smem_u32(sA), fb = smem_u32(&bar[2]);
                mbar_arrive_expect_tx(&bar[2], (uint32_t)kRows * p.K * 2);
                int blk = 0;
                for (int si = 0; si < p.nseg; ++si)
                    for (int j = 0; j < p.seg[si].C / 64; ++j, ++blk)
                        tma_load_4d(a + blk * (kRows * 128), &p.a_map[si], fb, 64 * j, t0 + p.seg[si].shift, w,
                                    p.a_nb[si] > 1 ? b : 0);
                ++a_issued;
            }
            return;
        }
        const int cr = tid >> 1, par = tid & 1;
        const int64_t row = r0 + cr;
        int c = 0;
        for (int si = 0; si < p.nseg; ++si) {
            const RowSeg &s = p.seg[si];
            for (int cc = 0; cc < s.C / 8; ++cc, ++c) {
                if ((c & 1) != par) continue;
                bool valid = false;
                const __nv_bfloat16 *src = row < p.rows ? seg_addr(s, b, row, p.W, cc, valid) : s.p;
                cp_async16(smem_u32(sA + (size_t)c * kRows * 16 + cr * 16), src, valid && row < p.rows);
            }
        }
    };
    if (blockIdx.x < p.n_tiles) issue_tile(blockIdx.x);
    uint32_t ph = 0;
    bool ok = true;
    const uint32_t idesc = idesc_f16(128, p.N, EPI == EPI_HEAD_U ? 0 : 1);   // u: FP16 operands, else BF16
    const int R = p.R, hr = R / 2, ch0 = h * hr;   // this thread's channels [ch0, ch0 + hr), hr <= 32
    const uint32_t tl = tmem + ((uint32_t)((warp & 3) * 32) << 16);
    for (int64_t tile = blockIdx.x; tile < p.n_tiles && ok; tile += gridDim.x) {
        const int b = (int)(tile / tpb);
        const int64_t row = (tile - (int64_t)b * tpb) * kRows + r;
        const bool live = row < p.rows;
        // the epilogue's global operands, in flight during the A copies and the MMA
        float4 pa[8];                                         // EPI_RES, EPI_DGRAD: aux[row][ch0 ..]
        uint4 pg[8];                                          // EPI_DZ: tanh(f), then sigmoid(g), [ch0 ..]
        if (EPI == EPI_RES || EPI == EPI_DGRAD) {
            const float *src = p.aux + b * p.aux_boff + row * R + ch0;
#pragma unroll
            for (int q = 0; q < 8; ++q)
                pa[q] = (live && 4 * q < hr) ? __ldg(reinterpret_cast<const float4 *>(src + 4 * q))
                                             : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        if (EPI == EPI_DZ) {
            const __half *src = p.gate + b * p.gate_boff + row * 2 * R + ch0;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const bool in = live && 8 * q < hr;
                pg[q] = in ? __ldg(reinterpret_cast<const uint4 *>(src + 8 * q)) : make_uint4(0, 0, 0, 0);
                pg[4 + q] = in ? __ldg(reinterpret_cast<const uint4 *>(src + R + 8 * q)) : make_uint4(0, 0, 0, 0);
            }
        }
        cp_async_wait_all();
        fence_proxy_async_smem();
        tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            // a wait that gives up sets abort_flag, so that every thread's MMA wait below gives up too
            const bool a_ok = !p.a_tma || mbar_wait(&bar[2], a_landed & 1, &abort_flag, p.err, 90 + EPI, kWaitNs);
            if (a_ok) {
                a_landed += p.a_tma ? 1 : 0;
                tc_fence_after();
                const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
                for (int ks = 0; ks < KC / 2; ++ks) {
                    // K-major A with the 128-byte swizzle: K step ks at byte 32 (ks % 4) of 64-channel
                    // block ks / 4 (8-row groups 1024 bytes apart); else the chunk-column layout
                    const uint64_t ad = p.a_tma ? sdesc_sw128(a0 + (ks >> 2) * (kRows * 128) + (ks & 3) * 32, 16, 1024)
                                                : sdesc(a0 + ks * 2 * kRows * 16, kRows * 16, 128);
                    const uint64_t bd = sdesc(b0 + ks * 2 * p.bn * 16, p.bn * 16, 128);
                    mma_f16(tmem, ad, bd, idesc, ks > 0 ? 1u : 0u);
                }
                mma_commit(&bar[0]);
            }
        }
        const bool w_ok = mbar_wait(&bar[0], ph & 1, &abort_flag, p.err, 60 + EPI, kWaitNs);
        ++ph;
        if (__syncthreads_or(!w_ok)) {
            ok = false;
            break;
        }
        tc_fence_after();
        // the MMA has read the A tile and the B image: the next tile's copies may overwrite them
        if (tile + gridDim.x < p.n_tiles) issue_tile(tile + gridDim.x);
        if (EPI == EPI_CONV) {
            const float *bc = p.bias + b * p.bias_boff;
#pragma unroll
            for (int g = 0; g < 2; ++g) {
                if (16 * g >= hr) break;
                const int c0 = ch0 + 16 * g;
                uint32_t fr[16], gr[16];
                tmem_ld16(tl + c0, fr);
                tmem_ld16(tl + R + c0, gr);
                tmem_ld_wait();
                float th[16], sg[16], z[16];
                // the forward kernel's gate arithmetic: tanh.approx, and sigmoid(g) = 0.5 tanh(g/2) + 0.5
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    th[j] = tanh_approx(__uint_as_float(fr[j]) + __ldg(bc + c0 + j));
                    sg[j] = fmaf(tanh_approx(0.5f * (__uint_as_float(gr[j]) + __ldg(bc + R + c0 + j))), 0.5f, 0.5f);
                    z[j] = th[j] * sg[j];
                }
                uint32_t w[8];
                if (p.gate_out) {   // the backward's gate cache: tanh(f), sigmoid(g) in FP16
                    __half *go = p.gate_out + b * p.gate_boff + row * 2 * R;
                    pack16_f16(th, w);
                    wst16_w(go + c0, w, live, stg, lane);
                    pack16_f16(sg, w);
                    wst16_w(go + R + c0, w, live, stg, lane);
                }
                pack16_bf16(z, w);
                wst16_w(p.o16 + b * p.o16_boff + row * R + c0, w, live, stg, lane);
            }
        } else if (EPI == EPI_RES) {
            const float *br = p.bias + b * p.bias_boff;
            const int S = p.N - R, hs = S / 2, s0 = h * hs;   // skip channels [s0, s0 + hs), hs <= 64
            float *so = S > 0 ? p.skip + b * p.skip_boff + row * S + s0 : nullptr;
#pragma unroll
            for (int g = 0; g < 2; ++g) {
                if (16 * g >= hr) break;
                const int c0 = ch0 + 16 * g;
                uint32_t rr[16];
                tmem_ld16(tl + c0, rr);
                tmem_ld_wait();
                float v[16];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    v[4 * q] = pa[4 * g + q].x;
                    v[4 * q + 1] = pa[4 * g + q].y;
                    v[4 * q + 2] = pa[4 * g + q].z;
                    v[4 * q + 3] = pa[4 * g + q].w;
                }
#pragma unroll
                for (int j = 0; j < 16; ++j) v[j] += __uint_as_float(rr[j]) + __ldg(br + c0 + j);
                wst16_f32(p.o32 + b * p.o32_boff + row * R + c0, v, live, stg, lane);
                uint32_t w[8];
                pack16_bf16(v, w);
                wst16_w(p.o16 + b * p.o16_boff + row * R + c0, w, live, stg, lane);
            }
            const float *bs = p.bias2 ? p.bias2 + b * p.bias_boff : nullptr;
            // the skip sums of this thread's half, all loads in flight together
            float4 ps[16];
#pragma unroll
            for (int q = 0; q < 16; ++q)
                ps[q] = (live && S > 0 && !p.skip_init && 4 * q < hs) ? *reinterpret_cast<const float4 *>(so + 4 * q)
                                                                       : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int g = 0; g < 4; ++g) {
                if (16 * g >= hs) break;
                uint32_t qr[16];
                tmem_ld16(tl + R + s0 + 16 * g, qr);
                tmem_ld_wait();
                if (!live) continue;
                float v[16];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    v[4 * q] = ps[4 * g + q].x;
                    v[4 * q + 1] = ps[4 * g + q].y;
                    v[4 * q + 2] = ps[4 * g + q].z;
                    v[4 * q + 3] = ps[4 * g + q].w;
                }
#pragma unroll
                for (int j = 0; j < 16; ++j) v[j] += __uint_as_float(qr[j]) + __ldg(bs + s0 + 16 * g + j);
                st16_f32(so + 16 * g, v);
            }
        } else if (EPI == EPI_DZ) {
#pragma unroll
            for (int g = 0; g < 2; ++g) {
                if (16 * g >= hr) break;
                const int c0 = ch0 + 16 * g;
                uint32_t dr[16];
                tmem_ld16(tl + c0, dr);
                tmem_ld_wait();
                float th[16], sg[16], df[16], dg[16];
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const uint32_t wt[4] = {pg[2 * g + q].x, pg[2 * g + q].y, pg[2 * g + q].z, pg[2 * g + q].w};
                    const uint32_t ws[4] = {pg[4 + 2 * g + q].x, pg[4 + 2 * g + q].y, pg[4 + 2 * g + q].z,
                                            pg[4 + 2 * g + q].w};
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const float2 ft = __half22float2(*reinterpret_cast<const __half2 *>(&wt[i]));
                        const float2 fs = __half22float2(*reinterpret_cast<const __half2 *>(&ws[i]));
                        th[8 * q + 2 * i] = ft.x;
                        th[8 * q + 2 * i + 1] = ft.y;
                        sg[8 * q + 2 * i] = fs.x;
                        sg[8 * q + 2 * i + 1] = fs.y;
                    }
                }
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const float dz = __uint_as_float(dr[j]);
                    df[j] = dz * sg[j] * (1.f - th[j] * th[j]);
                    dg[j] = dz * th[j] * sg[j] * (1.f - sg[j]);
                }
                __nv_bfloat16 *d16 = p.o16 + b * p.o16_boff + row * 2 * R;
                uint32_t w[8];
                pack16_bf16(df, w);
                wst16_w(d16 + c0, w, live, stg, lane);
                pack16_bf16(dg, w);
                wst16_w(d16 + R + c0, w, live, stg, lane);
            }
        } else if (EPI == EPI_HEAD_U) {
            // this thread's u channels [h N/2, h N/2 + N/2) of its row
            const int hn = p.N / 2, u0 = h * hn;
            const float dl = live ? __ldg(p.aux + row) : 0.f;
            for (int g = 0; g < hn / 16; ++g) {
                const int c0 = u0 + 16 * g;
                uint32_t ur[16];
                tmem_ld16(tl + c0, ur);
                tmem_ld_wait();
                if (!live) continue;
                float du[16], ru[16], lo[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const float u = __uint_as_float(ur[j]) + __ldg(p.bias + c0 + j);
                    du[j] = u > 0.f ? dl * __ldg(p.bias2 + c0 + j) : 0.f;
                    ru[j] = fmaxf(u, 0.f);
                    lo[j] = du[j] - __bfloat162float(__float2bfloat16_rn(du[j]));
                }
                st16_bf16(p.o16 + row * p.N + c0, du);
                st16_bf16(p.o16_lo + row * p.N + c0, lo);
                st16_f32(p.o32 + row * p.N + c0, ru);
            }
        } else if (EPI == EPI_HEAD_DH) {
            // thread half h = branch h: dskip_h[row][c] for c < S = N / 2
            const int S = p.N / 2;
            for (int g = 0; g < S / 16; ++g) {
                const int c0 = 16 * g;
                uint32_t dr[16];
                tmem_ld16(tl + h * S + c0, dr);
                tmem_ld_wait();
                if (!live) continue;
                const __nv_bfloat16 *mk = p.mask16 + h * p.mask_boff + row * S + c0;
                const uint4 m0 = *reinterpret_cast<const uint4 *>(mk), m1 = *reinterpret_cast<const uint4 *>(mk + 8);
                const uint32_t mw[8] = {m0.x, m0.y, m0.z, m0.w, m1.x, m1.y, m1.z, m1.w};
                float v[16];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const float2 hv = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&mw[q]));
                    v[2 * q] = hv.x > 0.f ? __uint_as_float(dr[2 * q]) : 0.f;
                    v[2 * q + 1] = hv.y > 0.f ? __uint_as_float(dr[2 * q + 1]) : 0.f;
                }
                st16_f32(p.o32 + h * p.o32_boff + row * S + c0, v);
                st16_bf16(p.o16 + h * p.o16_boff + row * S + c0, v);
            }
        } else {   // EPI_DGRAD
#pragma unroll
            for (int g = 0; g < 2; ++g) {
                if (16 * g >= hr) break;
                const int c0 = ch0 + 16 * g;
                uint32_t dr[16];
                tmem_ld16(tl + c0, dr);
                tmem_ld_wait();
                float v[16];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    v[4 * q] = pa[4 * g + q].x + __uint_as_float(dr[4 * q]);
                    v[4 * q + 1] = pa[4 * g + q].y + __uint_as_float(dr[4 * q + 1]);
                    v[4 * q + 2] = pa[4 * g + q].z + __uint_as_float(dr[4 * q + 2]);
                    v[4 * q + 3] = pa[4 * g + q].w + __uint_as_float(dr[4 * q + 3]);
                }
                // staged: FP32 values 0-7, then 8-15, then the sixteen BF16 values
                float *o32 = p.o32 + b * p.o32_boff + row * R + c0;
                wst32b_p48(o32, make_uint4(__float_as_uint(v[0]), __float_as_uint(v[1]), __float_as_uint(v[2]),
                                           __float_as_uint(v[3])),
                           make_uint4(__float_as_uint(v[4]), __float_as_uint(v[5]), __float_as_uint(v[6]),
                                      __float_as_uint(v[7])),
                           live, stg, lane);
                wst32b_p48(o32 + 8, make_uint4(__float_as_uint(v[8]), __float_as_uint(v[9]), __float_as_uint(v[10]),
                                               __float_as_uint(v[11])),
                           make_uint4(__float_as_uint(v[12]), __float_as_uint(v[13]), __float_as_uint(v[14]),
                                      __float_as_uint(v[15])),
                           live, stg, lane);
                uint32_t w[8];
                pack16_bf16(v, w);
                wst32b_p48(p.o16 + b * p.o16_boff + row * R + c0, make_uint4(w[0], w[1], w[2], w[3]),
                           make_uint4(w[4], w[5], w[6], w[7]), live, stg, lane);
            }
        }
        // every thread's TMEM reads of this tile end before the next tile's MMA
        tc_fence_before();
        __syncthreads();
    }
    // copies issued for a tile that an aborted loop never reached complete before the CTA exits
    cp_async_wait_all();
    if (tid == 0 && a_issued > a_landed) mbar_wait_drain(&bar[2], (a_issued - 1) & 1, p.err, 100 + EPI, kWaitNs);
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
// Both operands are MN-major: rows of G and X are copied unchanged (8 channels per 16 bytes),
// element (mn, k) of a stage at (mn / 8) * 2048 + k * 16 + (mn % 8) * 2, i.e. 8-channel groups
// 2048 bytes apart and 8-row K groups 128 bytes apart.  In the descriptor of a non-swizzled
// MN-major operand the stride byte offset is the step between 8-channel groups and the leading
// byte offset the step between 8-row K groups.  Two stages: the copies of tile i + 1 are in flight while
// the MMAs of tile i run.  Channels M..127 of A are zero; columns nx..N-1 of B are [1, 0, ...],
// so that column nx of D is the column sum of G (the bias gradient).
template <int N, int NS>
__global__ void __launch_bounds__(kWgThreads) k_tc_wgrad(const WgGemm p) {
    constexpr uint32_t A_BYTES = 16 * 2048, B_BYTES = (N / 8) * 2048, STAGE = A_BYTES + B_BYTES;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    __shared__ uint64_t bar[NS + 1];
    __shared__ uint32_t tslot;
    __shared__ int abort_flag;
    constexpr uint32_t NCOLS = N <= 32 ? 32 : (N <= 64 ? 64 : (N <= 128 ? 128 : 256));
    const int tid = threadIdx.x, warp = tid >> 5;
    if (tid == 0) {
        for (int i = 0; i < NS + 1; ++i) mbar_init(&bar[i], 1);
        abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 0) tmem_alloc(&tslot, NCOLS);
    // constant parts of both stages (row k = tid < 128): A channel groups >= M / 8 zero, B groups
    // from nx / 8 on: 1.0 at column nx, zeros after it
    for (int s = 0; s < NS && tid < kRows; ++s) {
        uint8_t *a = smem + s * STAGE, *bb = a + A_BYTES;
        for (int mi = p.M / 8; mi < 16; ++mi) *reinterpret_cast<uint4 *>(a + mi * 2048 + tid * 16) = make_uint4(0, 0, 0, 0);
        for (int ni = p.nx / 8; ni < N / 8; ++ni)
            *reinterpret_cast<uint4 *>(bb + ni * 2048 + tid * 16) = make_uint4(ni == p.nx / 8 ? 0x3F80u : 0u, 0, 0, 0);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tslot;
    const int b = blockIdx.y;
    const int64_t t_begin = (int64_t)blockIdx.x * p.tiles_per_cta;
    const int64_t t_end = std::min<int64_t>(p.tiles, t_begin + p.tiles_per_cta);
    const int64_t n = t_end - t_begin;
    // copies of one tile into stage s: row tid / TPR, 16-byte channel groups of index = tid % TPR
    // modulo TPR (consecutive threads on consecutive groups of one row)
    auto issue = [&](int64_t tile, int s) {
        constexpr int TPR = kWgThreads / kRows;
        uint8_t *a = smem + s * STAGE, *bb = a + A_BYTES;
        const int par = tid % TPR;
        const int k = tid / TPR;
        const int64_t row = tile * kRows + k;
        const bool live = row < p.rows;
        const __nv_bfloat16 *g = p.G + b * p.g_boff + (live ? row : 0) * p.ldg;
        for (int mi = par; mi < p.M / 8; mi += TPR) cp_async16(smem_u32(a + mi * 2048 + k * 16), g + 8 * mi, live);
        int ni = 0;
        for (int si = 0; si < p.nxs; ++si) {
            const RowSeg &sg = p.xs[si];
            bool valid = false;
            const __nv_bfloat16 *x0 = live ? seg_addr(sg, b, row, p.W, 0, valid) : sg.p;
            for (int cc = 0; cc < sg.C / 8; ++cc, ++ni) {
                if (ni % TPR != par) continue;
                cp_async16(smem_u32(bb + ni * 2048 + k * 16), valid ? x0 + 8 * cc : sg.p, valid);
            }
        }
        cp_async_commit();
    };
    const uint32_t idesc = idesc_f16(128, N, 1) | (1u << 15) | (1u << 16);   // A and B MN-major
    for (int s = 0; s < NS; ++s)
        if (s < n) issue(t_begin + s, s);
    bool ok = true;
    for (int64_t i = 0; i < n; ++i) {
        const int s = (int)(i % NS);
        // groups committed after tile i's: the tiles issued ahead of it, at most NS - 1
        const int64_t ahead = std::min<int64_t>(n - 1, i + NS - 1) - i;
        if (ahead >= 2)
            cp_async_wait_group<2>();
        else if (ahead == 1)
            cp_async_wait_group<1>();
        else
            cp_async_wait_group<0>();
        fence_proxy_async_smem();
        tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            const uint32_t a0 = smem_u32(smem + s * STAGE), b0 = a0 + A_BYTES;
#pragma unroll
            for (int ks = 0; ks < 8; ++ks) {
                const uint64_t ad = sdesc(a0 + ks * 256, 128, 2048);
                const uint64_t bd = sdesc(b0 + ks * 256, 128, 2048);
                mma_f16(tmem, ad, bd, idesc, (i > 0 || ks > 0) ? 1u : 0u);
            }
            mma_commit(&bar[s]);
        }
        if (i + NS < n) {
            // stage s takes tile i + NS once the MMAs of tile i have read it
            const bool w_ok = mbar_wait(&bar[s], (uint32_t)(i / NS) & 1, &abort_flag, p.err, 80, kWaitNs);
            if (__syncthreads_or(!w_ok)) {
                ok = false;
                break;
            }
            issue(t_begin + i + NS, s);
        }
    }
    cp_async_wait_all();
    // every MMA of the CTA has completed (and written D) once this commit arrives
    bool d_ok = true;
    if (tid == 0) {
        mma_commit(&bar[NS]);
        d_ok = mbar_wait_drain(&bar[NS], 0, p.err, 81, kWaitNs);
    }
    if (__syncthreads_or(!d_ok)) ok = false;
    if (ok && n > 0 && warp < 4) {
        tc_fence_after();
        // D[m][n] in TMEM lane m: warps 0-3 (lanes 0-127) whose lanes hold m < M add their rows
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
                    else if (c0 + j == p.nx && p.db && (p.db_nb == 0 || b < p.db_nb))
                        atomicAdd(p.db + b * p.w_boff + m, __uint_as_float(v[j]));
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, NCOLS);
    }
}

// ---------------------------------------------------------------- weight gradients through TMA
// dW += G^T X as in k_tc_wgrad, with the operands brought in by tensor-map copies
// (cp.async.bulk.tensor) instead of per-thread 16-byte copies: one thread issues a tile's copies,
// another its MMAs, and the copies of up to `stages` tiles are in flight at once.  A tile is
// kTmaRows rows of one window.  Each 64-channel block of a tile lands as kTmaRows rows of 128 bytes
// with the 128-byte swizzle (16-byte chunk j of row k at chunk position j ^ (k % 8)), which is the
// canonical MN-major operand layout with that swizzle: 64-channel blocks kTmaBlk bytes apart (the
// descriptor's leading byte offset) and 8-row K groups 1024 bytes apart (its stride byte offset).
// A = G^T takes blocks 0 and 1 (block 1 stays zero when M = 64); B = X^T takes the segments'
// nx / 64 blocks and a last block holding the ones column (column nx) for the bias gradient.
// Rows outside [0, W) of a shifted segment are zero-filled by the copy (out-of-range coordinates).
constexpr int kTmaRows = 64;
constexpr int kTmaBlk = kTmaRows * 128;
constexpr int kTmaMaxStages = 6;
constexpr size_t kTmaSmem = 226 * 1024;   // dynamic shared memory of the tensor-map weight-gradient kernels

struct WgTma {
    CUtensorMap g_map;        // G: {M channels, rows, branches}
    CUtensorMap x_map[2];     // segments: {C channels, W, windows, branches}
    int g_blocks;             // M / 64
    int g_nb;                 // 2 when the branches read their own G, else 1
    int x_blocks[2];          // C / 64 of each segment
    int x_shift[2];
    int x_nb[2];
    int nxs;
    int W;
    int64_t tiles;            // kTmaRows-row tiles per branch
    int tiles_per_cta;
    int stages;
    int M, nx, ldw;
    float *dW;                // dW[m][n] at dW + m * ldw + n (16-byte aligned rows), branch 1 at + w_boff
    int64_t w_boff;
    float *db;
    int db_nb;
    int *err;
};

// NB: B blocks (nx / 64 + 1); N = nx + 16
template <int NB>
__global__ void __launch_bounds__(128, 1) k_tc_wgrad_tma(const __grid_constant__ WgTma p) {
    constexpr int N = (NB - 1) * 64 + 16;
    constexpr uint32_t NCOLS = N <= 128 ? 128 : 256;
    constexpr uint32_t A_BYTES = 2 * kTmaBlk, STAGE = (2 + NB) * kTmaBlk;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    __shared__ uint64_t full[kTmaMaxStages], empty[kTmaMaxStages], done;
    __shared__ uint32_t tslot;
    __shared__ int abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int ns = p.stages;
    if (tid == 0) {
        for (int s = 0; s < ns; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&done, 1);
        abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 0) tmem_alloc(&tslot, NCOLS);
    // constant blocks of every stage (never written by the copies): A block 1 when M = 64 (zeros);
    // B's last block: 1.0 at its column 0 (logical chunk 0 of row k sits at position k % 8)
    for (int s = 0; s < ns; ++s) {
        uint8_t *st = smem + s * STAGE;
        if (p.g_blocks == 1)
            for (int i = tid; i < kTmaBlk / 16; i += 128) *reinterpret_cast<uint4 *>(st + kTmaBlk + i * 16) = make_uint4(0, 0, 0, 0);
        uint8_t *ones = st + A_BYTES + (NB - 1) * kTmaBlk;
        for (int i = tid; i < kTmaBlk / 16; i += 128)
            *reinterpret_cast<uint4 *>(ones + i * 16) = make_uint4((i % 8) == ((i / 8) % 8) ? 0x3F80u : 0u, 0, 0, 0);
    }
    // the constant blocks are read by the tensor cores (async proxy)
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tslot;
    const int b = blockIdx.y;
    const int64_t t_begin = (int64_t)blockIdx.x * p.tiles_per_cta;
    const int64_t n = std::max<int64_t>(0, std::min<int64_t>(p.tiles, t_begin + p.tiles_per_cta) - t_begin);
    int xb = 0;
    for (int si = 0; si < p.nxs; ++si) xb += p.x_blocks[si];
    const uint32_t tile_bytes = (uint32_t)(p.g_blocks + xb) * kTmaBlk;
    bool ok = true;
    if (tid == 0 && n > 0) {
        // producer: stage s takes tile i once the MMAs of tile i - ns have read it
        int64_t armed = 0;
        for (int64_t i = 0; i < n; ++i) {
            const int s = (int)(i % ns);
            const uint32_t u = (uint32_t)(i / ns);
            if (i >= ns && !mbar_wait(&empty[s], (u - 1) & 1, &abort_flag, p.err, 82, kWaitNs)) {
                ok = false;
                break;
            }
            const int64_t row0 = (t_begin + i) * kTmaRows;
            const int w = (int)(row0 / p.W), t0 = (int)(row0 - (int64_t)w * p.W);
            const uint32_t a = smem_u32(smem + s * STAGE), bb = a + A_BYTES, fb = smem_u32(&full[s]);
            mbar_arrive_expect_tx(&full[s], tile_bytes);
            for (int j = 0; j < p.g_blocks; ++j) tma_load_3d(a + j * kTmaBlk, &p.g_map, fb, 64 * j, (int)row0, p.g_nb > 1 ? b : 0);
            int blk = 0;
            for (int si = 0; si < p.nxs; ++si)
                for (int j = 0; j < p.x_blocks[si]; ++j, ++blk)
                    tma_load_4d(bb + blk * kTmaBlk, &p.x_map[si], fb, 64 * j, t0 + p.x_shift[si], w,
                                p.x_nb[si] > 1 ? b : 0);
            armed = i + 1;
        }
        // copies armed for tiles that an aborted MMA thread never consumed land before the CTA exits
        for (int64_t i = std::max<int64_t>(0, armed - ns); i < armed; ++i)
            mbar_wait_drain(&full[i % ns], (uint32_t)(i / ns) & 1, p.err, 85, kWaitNs);
    } else if (tid == 32 && n > 0) {
        // MMA issuer: K = 16 rows per instruction, 2048 bytes per step within each block
        const uint32_t idesc = idesc_f16(128, N, 1) | (1u << 15) | (1u << 16);   // A and B MN-major
        for (int64_t i = 0; i < n; ++i) {
            const int s = (int)(i % ns);
            if (!mbar_wait(&full[s], (uint32_t)(i / ns) & 1, &abort_flag, p.err, 83, kWaitNs)) {
                ok = false;
                break;
            }
            tc_fence_after();
            const uint32_t a = smem_u32(smem + s * STAGE), bb = a + A_BYTES;
#pragma unroll
            for (int ks = 0; ks < kTmaRows / 16; ++ks)
                mma_f16(tmem, sdesc_sw128(a + ks * 2048, kTmaBlk, 1024), sdesc_sw128(bb + ks * 2048, kTmaBlk, 1024),
                        idesc, (i > 0 || ks > 0) ? 1u : 0u);
            mma_commit(&empty[s]);
        }
        // arrives once every MMA issued above has completed (also after an abort)
        mma_commit(&done);
    }
    __syncwarp();
    bool d_ok = true;
    if (n > 0) d_ok = mbar_wait_drain(&done, 0, p.err, 84, kWaitNs);
    const bool bad = __syncthreads_or(!ok || !d_ok);
    if (!bad && n > 0) {
        tc_fence_after();
        // D[m][c] in TMEM lane m = tid; columns [0, nx) into dW (four columns per atomic), column nx into db
        const int m = tid;
        const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
        for (int c0 = 0; c0 < N; c0 += 16) {
            uint32_t v[16];
            tmem_ld16(tl + c0, v);
            tmem_ld_wait();
            if (m >= p.M) continue;
            if (c0 < p.nx) {
                float4 *dw = reinterpret_cast<float4 *>(p.dW + b * p.w_boff + (int64_t)m * p.ldw + c0);
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    atomicAdd(dw + q, make_float4(__uint_as_float(v[4 * q]), __uint_as_float(v[4 * q + 1]),
                                                  __uint_as_float(v[4 * q + 2]), __uint_as_float(v[4 * q + 3])));
            } else if (c0 == p.nx && p.db && (p.db_nb == 0 || b < p.db_nb)) {
                atomicAdd(p.db + b * p.w_boff + m, __uint_as_float(v[0]));
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, NCOLS);
    }
}

// h = ReLU(skip) (skip: the pre-ReLU skip sums with their biases, both branches) in FP16, the
// forward kernel's head operand, and in BF16 (hi, and lo = BF16(h - hi)), the weight-gradient
// operands; hi is also the dskip mask
__global__ void k_relu_h(const float *__restrict__ in, __half *__restrict__ hf, __nv_bfloat16 *__restrict__ hb,
                         __nv_bfloat16 *__restrict__ hb_lo, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n / 4; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 v = reinterpret_cast<const float4 *>(in)[i];
        const float a0 = fmaxf(v.x, 0.f), a1 = fmaxf(v.y, 0.f), a2 = fmaxf(v.z, 0.f), a3 = fmaxf(v.w, 0.f);
        const __half2 f0 = __floats2half2_rn(a0, a1), f1 = __floats2half2_rn(a2, a3);
        const __nv_bfloat162 b0 = __floats2bfloat162_rn(a0, a1), b1 = __floats2bfloat162_rn(a2, a3);
        reinterpret_cast<uint2 *>(hf)[i] = make_uint2(*reinterpret_cast<const uint32_t *>(&f0),
                                                      *reinterpret_cast<const uint32_t *>(&f1));
        reinterpret_cast<uint2 *>(hb)[i] = make_uint2(*reinterpret_cast<const uint32_t *>(&b0),
                                                      *reinterpret_cast<const uint32_t *>(&b1));
        // the rounding remainders h - BF16(h), in BF16 (the lo term of the weight gradient's split)
        const float2 r0 = __bfloat1622float2(b0), r1 = __bfloat1622float2(b1);
        const __nv_bfloat162 l0 = __floats2bfloat162_rn(a0 - r0.x, a1 - r0.y), l1 = __floats2bfloat162_rn(a2 - r1.x, a3 - r1.y);
        reinterpret_cast<uint2 *>(hb_lo)[i] = make_uint2(*reinterpret_cast<const uint32_t *>(&l0),
                                                         *reinterpret_cast<const uint32_t *>(&l1));
    }
}

// B images of the head's first convolution W_h1 [Hc][2S] (chunk-column layout): the u image
// [Hc rows: u channel j][2S K: h channel c] in FP16 (the forward kernel's head operands) and the dh
// image [2S rows: c][Hc K: j] in BF16
__global__ void k_pack_head(const float *__restrict__ w1, int Hc, int S2, __half *__restrict__ u_img,
                            __nv_bfloat16 *__restrict__ dh_img) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)Hc * S2) return;
    const int j = (int)(e / S2), c = (int)(e % S2);
    u_img[((size_t)(c / 8) * Hc * 16 + (size_t)j * 16 + (c % 8) * 2) / 2] = __float2half_rn(w1[e]);
    dh_img[((size_t)(j / 8) * S2 * 16 + (size_t)c * 16 + (j % 8) * 2) / 2] = __float2bfloat16_rn(w1[e]);
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
    size_t conv_b = 0, rs_b = 0, dz_b = 0, dg_b = 0, layer_b = 0;
    int model = -1;
    uint64_t stamp = 0;
    DevBuf xsave, skip, dskip32, dskip16, x32, x16, gate16, z16, dx32[2], dx16[2], da16, err;
    DevBuf head_img, hf16, hb16, hblo16, du16, dulo16, ru32;   // tensor-core head backward
};

__host__ __device__ inline size_t choff(int rows, int n, int k) { return (size_t)(k / 8) * rows * 16 + (size_t)n * 16 + (k % 8) * 2; }

// BF16 B images of one member's branch layers, gathered on the device from its FP32 blob
// (one thread per image element), per (layer, branch) in this order:
//   conv  [2R rows: conv output o][2R K: tap * R + input i]         (recomputed forward)
//   rs    [R + S rows: residual then skip output][R K: input i]     (recomputed forward)
//   dz    [R rows: input i][R + S K: residual then skip output]     (dz = [dx | dskip] . [Wres ; Wskip])
//   dg    [R rows: input i][4R K: (tap 1 outputs, tap 0 outputs)]   (dx = [da(t) | da(t + d)] . [W1 ; W0])
// each in the chunk-column layout of choff.
struct BwdGeo {
    int R, S, L;
    int64_t Pb, Pl;            // floats per branch / per layer of the blob
    size_t conv_b, rs_b, dz_b, dg_b, layer_b;
};

__global__ void k_pack_bwd(const float *__restrict__ blob, BwdGeo g, __nv_bfloat16 *__restrict__ img) {
    const int64_t per = (int64_t)(g.layer_b / 2);       // elements per (layer, branch)
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= per * 2 * g.L) return;
    const int lb = (int)(e / per);
    const int l = lb >> 1, b = lb & 1;
    int64_t q = e % per;
    const int R = g.R, S = g.S;
    const float *lay = blob + (int64_t)b * g.Pb + 2 * R + (int64_t)l * g.Pl;
    const float *wc = lay;                                             // [2R][2][R]
    const float *wr = lay + (int64_t)2 * R * 2 * R + 2 * R;            // [R][R]
    const float *ws = wr + (int64_t)R * R + R;                         // [S][R]
    size_t off = g.layer_b * (size_t)lb;
    float v;
    if (q < 4LL * R * R) {                                             // conv: (o, k)
        const int o = (int)(q / (2 * R)), k = (int)(q % (2 * R));
        v = wc[(int64_t)o * 2 * R + k];
        off += choff(2 * R, o, k);
    } else if ((q -= 4LL * R * R) < (int64_t)(R + S) * R) {            // rs: (o, i)
        const int o = (int)(q / R), i = (int)(q % R);
        v = o < R ? wr[(int64_t)o * R + i] : ws[(int64_t)(o - R) * R + i];
        off += g.conv_b + choff(R + S, o, i);
    } else if ((q -= (int64_t)(R + S) * R) < (int64_t)R * (R + S)) {   // dz: (i, k)
        const int i = (int)(q / (R + S)), k = (int)(q % (R + S));
        v = k < R ? wr[(int64_t)k * R + i] : ws[(int64_t)(k - R) * R + i];
        off += g.conv_b + g.rs_b + choff(R, i, k);
    } else {                                                           // dg: (i, k)
        q -= (int64_t)R * (R + S);
        const int i = (int)(q / (4 * R)), k = (int)(q % (4 * R));
        const int o = k % (2 * R), tap = k < 2 * R ? 1 : 0;
        v = wc[((int64_t)o * 2 + tap) * R + i];
        off += g.conv_b + g.rs_b + g.dz_b + choff(R, i, k);
    }
    img[off / 2] = __float2bfloat16_rn(v);
}

int g_rows_smem_set = 0;

gwe_status set_attrs() {
    if (g_rows_smem_set) return GWE_OK;
    const int big = 200 * 1024;
    GWE_CUDA_TRY(cudaFuncSetAttribute(k_tc_rows<EPI_CONV>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    GWE_CUDA_TRY(cudaFuncSetAttribute(k_tc_rows<EPI_RES>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    GWE_CUDA_TRY(cudaFuncSetAttribute(k_tc_rows<EPI_DZ>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    GWE_CUDA_TRY(cudaFuncSetAttribute(k_tc_rows<EPI_DGRAD>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    GWE_CUDA_TRY(cudaFuncSetAttribute(k_tc_rows<EPI_HEAD_U>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    GWE_CUDA_TRY(cudaFuncSetAttribute(k_tc_rows<EPI_HEAD_DH>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    GWE_CUDA_TRY(cudaFuncSetAttribute(k_tc_wgrad<48, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    GWE_CUDA_TRY(cudaFuncSetAttribute(k_tc_wgrad<80, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    GWE_CUDA_TRY(cudaFuncSetAttribute(k_tc_wgrad<144, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    GWE_CUDA_TRY(cudaFuncSetAttribute(k_tc_wgrad_tma<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTmaSmem));
    GWE_CUDA_TRY(cudaFuncSetAttribute(k_tc_wgrad_tma<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTmaSmem));
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

// cuTensorMapEncodeTiled from the driver through the runtime (no link-time dependency on libcuda)
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
    static const EncodeTiledFn fn = [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            f = nullptr;
        return reinterpret_cast<EncodeTiledFn>(f);
    }();
    return fn;
}

// 16-bit tensor of `rank` dimensions (dims[0] channels, contiguous), boxes of 64 channels x box_rows
// rows (x 1 in the higher dimensions), 128-byte swizzle, zero fill out of range
bool encode_bf16_map(CUtensorMap *map, const void *base, int rank, const uint64_t *dims, const uint64_t *strides,
                     int box_rows) {
    const EncodeTiledFn fn = encode_tiled();
    if (!fn || (reinterpret_cast<uintptr_t>(base) & 15)) return false;
    cuuint64_t gd[4], gs[3];
    cuuint32_t box[4], es[4];
    for (int i = 0; i < rank; ++i) {
        gd[i] = dims[i];
        box[i] = i == 0 ? 64 : (i == 1 ? box_rows : 1);
        es[i] = 1;
        if (i + 1 < rank) {
            gs[i] = strides[i];
            if (strides[i] % 16) return false;
        }
    }
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, (cuuint32_t)rank, const_cast<void *>(base), gd, gs, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The tensor-map form of a row GEMM's A tiles, where the shapes allow one: windows a multiple of 128
// rows (a tile lies in one window), segments of a multiple of 64 channels.  Otherwise (e.g. R = 32)
// the per-thread copies stage A in the chunk-column layout.
void make_rows_tma(RowGemm &p) {
    p.a_tma = 0;
    if (!g_tma_copies.load() || p.W % kRows || p.rows % p.W || p.rows >= (int64_t(1) << 31)) return;
    const int64_t nwin = p.rows / p.W;
    for (int si = 0; si < p.nseg; ++si) {
        const RowSeg &s = p.seg[si];
        if (s.C % 64 || s.C > s.ld) return;
        const uint64_t dims[4] = {(uint64_t)s.C, (uint64_t)p.W, (uint64_t)nwin, s.boff ? 2u : 1u};
        const uint64_t strides[3] = {(uint64_t)s.ld * 2, (uint64_t)p.W * s.ld * 2,
                                     (uint64_t)(s.boff ? s.boff : nwin * p.W * s.ld) * 2};
        if (!encode_bf16_map(&p.a_map[si], s.p, 4, dims, strides, kRows)) return;
        p.a_nb[si] = s.boff ? 2 : 1;
    }
    p.a_tma = 1;
}

template <int EPI>
gwe_status run_rows(RowGemm p, int sms, cudaStream_t st) {
    make_rows_tma(p);
    const int64_t tpb = (p.rows + kRows - 1) / kRows;
    p.n_tiles = tpb * p.nbranch;
    if (p.bn < p.N) p.bn = p.N;
    // at least 80 KB of shared memory per CTA, so that at most two CTAs (2 x <= 256 TMEM columns)
    // share an SM and no TMEM allocation has to wait; the conv, residual and dz epilogues stage
    // their stores per warp after the B image (dgrad, whose stages leave no room for it at two CTAs
    // per SM, stores directly: staged at 48-byte pitch it measured no faster)
    const size_t staging = EPI <= EPI_DZ ? (size_t)8 * kWarpStage : (EPI == EPI_DGRAD ? (size_t)8 * kWarpStageNarrow : 0);
    const size_t smem = std::max<size_t>((size_t)kRows * p.K * 2 + (size_t)p.bn * p.K * 2 + staging + 1024, 80 * 1024);
    const int grid = (int)std::min<int64_t>(p.n_tiles, (int64_t)sms * (smem <= 112 * 1024 ? 2 : 1));
    static const char *const kEpiName[6] = {"k_tc_rows:conv", "k_tc_rows:res",    "k_tc_rows:dz",
                                            "k_tc_rows:dgrad", "k_tc_rows:head_u", "k_tc_rows:head_dh"};
    ProfScope prof("k_tc_rows", st);
    ProfScope prof_epi(kEpiName[EPI], st);
    k_tc_rows<EPI><<<grid, 256, smem, st>>>(p);
    note_launch();
    GWE_CUDA_TRY(cudaGetLastError());
    return GWE_OK;
}

// The tensor-map form of a weight-gradient GEMM, when its shapes allow one: 64 or 128 channels of
// G and of every segment, windows a multiple of kTmaRows, 16-byte aligned rows of dW.  Returns
// false (and the caller takes the per-thread-copy kernel) otherwise.
bool make_wg_tma(const WgGemm &p, WgTma &t) {
    if (!g_tma_copies.load() || p.W % kTmaRows || p.rows % p.W || p.rows >= (int64_t(1) << 31) || (p.M != 64 && p.M != 128)) return false;
    if (p.nxs < 1 || p.nxs > 2 || p.N != p.nx + 16 || (p.nx != 64 && p.nx != 128)) return false;
    if ((reinterpret_cast<uintptr_t>(p.dW) & 15) || p.ldw % 4 || p.w_boff % 4) return false;
    std::memset(&t, 0, sizeof(t));
    const int64_t nwin = p.rows / p.W;
    {
        const uint64_t dims[3] = {(uint64_t)p.M, (uint64_t)p.rows, p.g_boff ? 2u : 1u};
        const uint64_t strides[2] = {(uint64_t)p.ldg * 2, (uint64_t)(p.g_boff ? p.g_boff : p.rows * p.ldg) * 2};
        if (!encode_bf16_map(&t.g_map, p.G, 3, dims, strides, kTmaRows)) return false;
    }
    int csum = 0;
    for (int si = 0; si < p.nxs; ++si) {
        const RowSeg &s = p.xs[si];
        if (s.C != 64 && s.C != 128) return false;
        const uint64_t dims[4] = {(uint64_t)s.C, (uint64_t)p.W, (uint64_t)nwin, s.boff ? 2u : 1u};
        const uint64_t strides[3] = {(uint64_t)s.ld * 2, (uint64_t)p.W * s.ld * 2,
                                     (uint64_t)(s.boff ? s.boff : nwin * p.W * s.ld) * 2};
        if (!encode_bf16_map(&t.x_map[si], s.p, 4, dims, strides, kTmaRows)) return false;
        t.x_blocks[si] = s.C / 64;
        t.x_shift[si] = s.shift;
        t.x_nb[si] = s.boff ? 2 : 1;
        csum += s.C;
    }
    if (csum != p.nx) return false;
    t.g_blocks = p.M / 64;
    t.g_nb = p.g_boff ? 2 : 1;
    t.nxs = p.nxs;
    t.W = p.W;
    t.tiles = p.rows / kTmaRows;
    t.M = p.M;
    t.nx = p.nx;
    t.ldw = p.ldw;
    t.dW = p.dW;
    t.w_boff = p.w_boff;
    t.db = p.db;
    t.db_nb = p.db_nb;
    t.err = p.err;
    return true;
}

gwe_status run_wgrad_tma(WgTma &t, int sms, cudaStream_t st) {
    const int NB = t.nx / 64 + 1;
    const size_t stage = (size_t)(2 + NB) * kTmaBlk;
    t.stages = (int)std::min<size_t>(kTmaMaxStages, (kTmaSmem - 1024) / stage);
    const size_t smem = t.stages * stage + 1024;
    // one CTA per SM (the stages fill its shared memory), one wave over both branches, contiguous
    // tile ranges
    const int64_t per_branch = std::max<int64_t>(1, sms / 2);
    t.tiles_per_cta = (int)std::max<int64_t>(1, (t.tiles + per_branch - 1) / per_branch);
    dim3 grid((unsigned)((t.tiles + t.tiles_per_cta - 1) / t.tiles_per_cta), 2);
    ProfScope prof("k_tc_wgrad", st);
    if (NB == 2)
        k_tc_wgrad_tma<2><<<grid, 128, smem, st>>>(t);
    else
        k_tc_wgrad_tma<3><<<grid, 128, smem, st>>>(t);
    note_launch();
    GWE_CUDA_TRY(cudaGetLastError());
    return GWE_OK;
}

gwe_status run_wgrad(WgGemm p, int sms, cudaStream_t st) {
    {
        WgTma t;
        if (make_wg_tma(p, t)) return run_wgrad_tma(t, sms, st);
    }
    p.tiles = (p.rows + kRows - 1) / kRows;
    // two stages of [G^T: 128 x 128 | X^T: N x 128] BF16; one CTA per SM when they exceed half of
    // the shared memory (this also keeps two 256-column TMEM allocations off one SM), else two.
    // (Three stages with one CTA per SM for N = 144 measured no faster.)
    const size_t smem = 2 * ((size_t)128 * 128 * 2 + (size_t)p.N * 128 * 2) + 128;
    const int per_sm = smem > 113 * 1024 ? 1 : 2;
    // one wave over both branches, contiguous tile ranges (fewer partial sums to add atomically)
    const int64_t per_branch = std::max<int64_t>(1, (int64_t)sms * per_sm / 2);
    p.tiles_per_cta = (int)std::max<int64_t>(1, (p.tiles + per_branch - 1) / per_branch);
    dim3 grid((unsigned)((p.tiles + p.tiles_per_cta - 1) / p.tiles_per_cta), 2);
    ProfScope prof("k_tc_wgrad", st);
    // N = nx + 16: the segments' columns, then the ones column for the bias gradient (nx = 32, 64, 128)
    if (p.N == 48)
        k_tc_wgrad<48, 2><<<grid, kWgThreads, smem, st>>>(p);
    else if (p.N == 80)
        k_tc_wgrad<80, 2><<<grid, kWgThreads, smem, st>>>(p);
    else if (p.N == 144)
        k_tc_wgrad<144, 2><<<grid, kWgThreads, smem, st>>>(p);
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
    // row-GEMM epilogues split the channels between two threads in groups of 16
    return d.k == 2 && d.R % 32 == 0 && d.S % 32 == 0 && 2 * d.R <= 128 && d.R + d.S <= 256 && d.S <= 128;
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
gwe_status fp32_head_w2_grad(gwe_model *m, const float *ru, int W, int C, const float *dlogit, float *gw,
                             cudaStream_t st);
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
    // B images from the current FP32 weights, gathered on the device on `st` (rebuilt when the
    // weights or the member change; no host round trip)
    const uint64_t stamp = m->wstamp;
    if (t->model != mi || t->stamp != stamp || t->layer_b == 0) {
        BwdGeo g;
        g.R = R;
        g.S = S;
        g.L = L;
        g.Pb = d.Pb;
        g.Pl = d.Pl;
        g.conv_b = t->conv_b = (size_t)2 * R * 2 * R * 2;
        g.rs_b = t->rs_b = (size_t)(R + S) * R * 2;
        g.dz_b = t->dz_b = (size_t)R * (R + S) * 2;
        g.dg_b = t->dg_b = (size_t)R * 4 * R * 2;
        g.layer_b = t->layer_b = t->conv_b + t->rs_b + t->dz_b + t->dg_b;
        GWE_CUDA_TRY(t->img.ensure(t->layer_b * 2 * L));
        const int64_t n = (int64_t)(t->layer_b / 2) * 2 * L;
        k_pack_bwd<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(blob, g, t->img.as<__nv_bfloat16>());
        note_launch();
        // the head's W_h1 as the B images of u and dh
        const int64_t nh = (int64_t)d.Hc * 2 * S;
        GWE_CUDA_TRY(t->head_img.ensure(2 * 2 * (size_t)nh));
        k_pack_head<<<(unsigned)((nh + 255) / 256), 256, 0, st>>>(blob + off_wh1(d), d.Hc, 2 * S,
                                                                  t->head_img.as<__half>(),
                                                                  t->head_img.as<__nv_bfloat16>() + nh);
        note_launch();
        GWE_CUDA_TRY(cudaGetLastError());
        t->model = mi;
        t->stamp = stamp;
    }
    const int C = std::min(batch, 128);                      // windows per chunk
    // BF16 handles: the fused forward kernel stores the stack inputs and skip sums; otherwise a
    // forward pass of row GEMMs computes them
    const bool fused_save = m->precision == GWE_BF16 && tc_save_supported(m, W);
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
    // the head on the tensor cores when its widths fit one MMA (N <= 256)
    const bool tc_head = d.Hc <= 256 && 2 * S <= 256 && d.Hc % 32 == 0;
    if (tc_head) {
        GWE_CUDA_TRY(t->hf16.ensure(2 * rows2 * S));
        GWE_CUDA_TRY(t->hb16.ensure(2 * rows2 * S));
        GWE_CUDA_TRY(t->hblo16.ensure(2 * rows2 * S));
        GWE_CUDA_TRY(t->dulo16.ensure(2 * rows * (size_t)d.Hc));
        GWE_CUDA_TRY(t->du16.ensure(2 * rows * (size_t)d.Hc));
        GWE_CUDA_TRY(t->ru32.ensure(sizeof(float) * rows * (size_t)d.Hc));
    }
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
        const int64_t xs_stride = 2 * rb * R;        // stack stride of xsave (this chunk)
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
        if (fused_save) {
            r = tc_forward_save(m, mi, sH, sL, Cc, W, t->dskip32.as<float>(), xsave, t->skip.as<float>(), st);
            if (r != GWE_OK) return r;
        } else {
            float *xa32 = x32, *xb32 = x32 + rows2 * R;
            __nv_bfloat16 *xa16 = x16, *xb16 = x16 + rows2 * R;
            r = fp32_input_proj(m, mi, sH, sL, rb, xa32, st);
            if (r != GWE_OK) return r;
            k_f32_to_bf16<<<1024, 256, 0, st>>>(xa32, xa16, 2 * rb * R);
            note_launch();
            for (int l = 0; l < L; ++l) {
                if (l % lps == 0)
                    GWE_CUDA_TRY(cudaMemcpyAsync(xsave + (size_t)(l / lps) * xs_stride, xa32, sizeof(float) * 2 * rb * R,
                                                 cudaMemcpyDeviceToDevice, st));
                r = layer_fwd(l, xa32, xa16, xb32, xb16, nullptr, z16, l == 0 ? 1 : 0);
                if (r != GWE_OK) return r;
                std::swap(xa32, xb32);
                std::swap(xa16, xb16);
            }
        }
        // ---- head: dskip and the head's gradients
        if (tc_head) {
            // h = ReLU(skip) in FP16 and BF16; u = [h_H | h_L] . W_h1^T (FP16 operands, as in the forward)
            // with du = (u + b_h1 > 0) dlogit w_h2 (BF16 hi and lo) and ReLU(u + b_h1) in its epilogue;
            // dh = du . W_h1 (BF16 operands) with dskip = (h > 0) dh (FP32 and BF16); dW_h1 = du^T h per
            // branch half of its columns from the BF16 splits; dw_h2, db_h2 in FP32
            const int Hc = d.Hc;
            const int64_t nhw = (int64_t)Hc * 2 * S;
            const float *dl = dlogit + (int64_t)c0 * W;
            __nv_bfloat16 *hb16 = t->hb16.as<__nv_bfloat16>(), *du16 = t->du16.as<__nv_bfloat16>();
            // FP16 bits through the row GEMM's BF16-typed staging (a copy of 16-bit words)
            const __nv_bfloat16 *hf16 = reinterpret_cast<const __nv_bfloat16 *>(t->hf16.as<__half>());
            float *ru32 = t->ru32.as<float>();
            __nv_bfloat16 *hblo16 = t->hblo16.as<__nv_bfloat16>(), *dulo16 = t->dulo16.as<__nv_bfloat16>();
            k_relu_h<<<1024, 256, 0, st>>>(t->skip.as<float>(), t->hf16.as<__half>(), hb16, hblo16, 2 * rb * S);
            note_launch();
            RowGemm pu{};
            pu.seg[0] = seg(hf16, 0, S, S, 0);
            pu.seg[1] = seg(hf16 + rb * S, 0, S, S, 0);
            pu.nseg = 2;
            pu.K = 2 * S;
            pu.N = Hc;
            pu.bimg = reinterpret_cast<const uint8_t *>(t->head_img.as<__nv_bfloat16>());
            pu.rows = rb;
            pu.W = W;
            pu.nbranch = 1;
            pu.err = err;
            pu.R = R;
            pu.bias = blob + off_bh1(d);
            pu.bias2 = blob + off_wh2(d);
            pu.aux = dl;
            pu.o16 = du16;
            pu.o16_lo = dulo16;
            pu.o32 = ru32;
            r = run_rows<EPI_HEAD_U>(pu, sms, st);
            if (r != GWE_OK) return r;
            RowGemm pd{};
            pd.seg[0] = seg(du16, 0, Hc, Hc, 0);
            pd.nseg = 1;
            pd.K = Hc;
            pd.N = 2 * S;
            pd.bimg = reinterpret_cast<const uint8_t *>(t->head_img.as<__nv_bfloat16>() + nhw);
            pd.rows = rb;
            pd.W = W;
            pd.nbranch = 1;
            pd.err = err;
            pd.R = R;
            pd.mask16 = hb16;
            pd.mask_boff = rb * S;
            pd.o32 = t->dskip32.as<float>();
            pd.o32_boff = rb * S;
            pd.o16 = t->dskip16.as<__nv_bfloat16>();
            pd.o16_boff = rb * S;
            r = run_rows<EPI_HEAD_DH>(pd, sms, st);
            if (r != GWE_OK) return r;
            // dW_h1 = du^T h from the BF16 splits du = du_hi + du_lo, h = h_hi + h_lo: the three products
            // hi.hi, hi.lo and lo.hi accumulate into the same gradient (the lo.lo term is dropped), so
            // that the sum over the batch keeps about 16 significant bits; db_h1 from the ones column
            // of the two passes with X = h_hi (du_hi + du_lo summed)
            const __nv_bfloat16 *Gs[3] = {du16, du16, dulo16}, *Xs[3] = {hb16, hblo16, hb16};
            for (int m0 = 0; m0 < Hc; m0 += 128) {
                for (int pass = 0; pass < 3; ++pass) {
                    WgGemm g{};
                    g.G = Gs[pass] + m0;
                    g.g_boff = 0;
                    g.ldg = Hc;
                    g.M = std::min(128, Hc - m0);
                    g.xs[0] = seg(Xs[pass], rb * S, S, S, 0);
                    g.nxs = 1;
                    g.nx = S;
                    g.N = S + 16;
                    g.db = pass == 1 ? nullptr : gw + off_bh1(d) + m0;
                    g.db_nb = 1;
                    g.rows = rb;
                    g.W = W;
                    g.dW = gw + off_wh1(d) + (int64_t)m0 * 2 * S;
                    g.ldw = 2 * S;
                    g.w_boff = S;
                    g.err = err;
                    r = run_wgrad(g, sms, st);
                    if (r != GWE_OK) return r;
                }
            }
            r = fp32_head_w2_grad(m, ru32, W, Cc, dl, gw, st);
            if (r != GWE_OK) return r;
        } else {
            r = fp32_head_backward(m, mi, t->skip.as<float>(), rb, W, Cc, dlogit + (int64_t)c0 * W,
                                   t->dskip32.as<float>(), gw, st);
            if (r != GWE_OK) return r;
            k_f32_to_bf16<<<1024, 256, 0, st>>>(t->dskip32.as<float>(), t->dskip16.as<__nv_bfloat16>(), 2 * rb * S);
            note_launch();
        }
        // ---- branches, stack by stack in reverse
        int hi = 0;   // dx buffers: [hi] = dL/dx_{l+1}
        GWE_CUDA_TRY(cudaMemsetAsync(t->dx32[hi].ptr, 0, sizeof(float) * 2 * rb * R, st));
        GWE_CUDA_TRY(cudaMemsetAsync(t->dx16[hi].ptr, 0, 2 * 2 * rb * R, st));
        for (int k = stacks - 1; k >= 0; --k) {
            GWE_CUDA_TRY(cudaMemcpyAsync(x32, xsave + (size_t)k * xs_stride, sizeof(float) * 2 * rb * R,
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
    // a device-side wait that gave up leaves its site in the error word (the fused forward's in its own)
    if (fused_save) {
        r = tc_check(m, st);
        if (r != GWE_OK) return r;
    }
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

extern "C" gwe_status gwe_set_tensor_map_copies(int on) {
    gwe::clear_error();
    GWE_ARG_CHECK(on == 0 || on == 1, "on must be 0 or 1");
    gwe::g_tma_copies.store(on);
    return GWE_OK;
}
