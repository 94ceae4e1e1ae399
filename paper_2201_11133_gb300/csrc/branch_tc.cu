// Fused tensor-core forward of the two-branch WaveNet detector ensemble
// (arXiv:2201.11133, section "Materials and Methods", paragraph "AI
// architecture", Fig. 1), 16-bit operands on tcgen05 with FP32 accumulation.
//
// One persistent CTA per SM walks a static list of jobs; a job is one
// (slide, model, window): both detector branches of one 1 s window, followed
// by the head.  A job runs as a stream of 128-sample time tiles in time order;
// every tile goes through all layers of both branches and then the head, so
// activations never leave the SM except the lagged rows of the dilated
// convolutions (below).
//
// Per layer l (dilation d), per branch, on a tile of 128 rows t0..t0+127:
//   conv   a = [x_l(t-d) | x_l(t)] . Wconv^T        tcgen05, BF16 x BF16 -> FP32 TMEM
//          (K = 2R: the lagged and the current rows are two descriptors into
//           one staging buffer whose first 128 rows hold the lag history)
//   gate   z = tanh(a_f + b_f) * sigmoid(a_g + b_g)   registers, FP16x2 tanh.approx
//          (the g half of Wconv and b_conv are pre-halved, so that
//           sigmoid(g) = 0.5 tanh(g/2) + 0.5 costs one tanh)
//   res    r = z . Wres^T  -> TMEM (reuses the conv columns), FP16 x FP16
//          x_{l+1} = x_l + r + b_res                   FP32, held in registers
//   skip   s += z . Wskip^T                            FP32, accumulated in TMEM
// Head, per tile, on h = ReLU([s_H + sum b_skip ; s_L + sum b_skip]) (FP16):
//   u = h . W_h1^T (TMEM), logit = b_h2 + w_h2 . ReLU(u + b_h1), p = sigmoid(logit) (FP32)
//
// Lag history: the rows x_l(t0-d .. ) needed by the next tiles are written to
// a per-CTA ring in global memory (d rows per layer, L2-resident) and brought
// back into the staging buffer with bulk async copies one layer ahead.
//
// Warp roles (384 threads): warp 0 weight producer (bulk copies of each
// layer's prepared weight image into a 4-entry ring), warp 1 TMEM owner and
// MMA issuer, warps 4-7 epilogue of branch H, warps 8-11 epilogue of branch L
// (thread = row).  Warps 2-3 are idle.  The two branches ping-pong on the
// tensor core: one branch's MMAs run while the other's gate runs.
//
// Every wait is bounded (wall clock); on timeout the kernel records the wait
// site in an error word, lets every role leave its loops and frees TMEM.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <atomic>
#include <map>
#include <mutex>
#include <tuple>
#include <string>
#include <vector>

#include "gwe_internal.h"
#include "tc_ptx.cuh"

namespace gwe {
namespace {

using namespace tc;

constexpr int kThreads = 640;
constexpr int kTile = 128;
constexpr uint64_t kWaitNs = 4000000000ull;   // 4 s per wait

constexpr uint32_t pow2ceil(uint32_t x) {
    uint32_t p = 32;
    while (p < x) p <<= 1;
    return p;
}
constexpr uint32_t cmax(uint32_t a, uint32_t b) { return a > b ? a : b; }

// F8 = false: conv operands BF16.  F8 = true: conv operands FP8 E4M3 (the residual stream's copy
// scaled per input channel, the weights per output channel); everything after the conv as for BF16.
template <int R, int S, int HC, bool F8 = false>
struct TcShape {
    static constexpr int XB = F8 ? 1 : 2;         // bytes per conv-operand element
    static constexpr int XROW = R * XB;           // bytes of one row of x (lag ring row)
    static constexpr int N1 = 2 * R;              // conv outputs: f then g
    static constexpr int RC = R * XB / 16;        // 16-byte chunks of one row of x
    static constexpr int KR = R / 16;             // K steps of the residual/skip MMAs (FP16 z)
    static constexpr int NH = HC <= 128 ? 1 : 2;  // head output pieces
    static constexpr int HP = HC / NH;
    static constexpr int HQ = S / 2;              // K width of one head weight piece
    static constexpr int NHP = 4 * NH;            // head weight pieces: (nh, K quarter)
    static constexpr uint32_t STAGE_ROWS = 256;
    static constexpr uint32_t STAGE_LBO = STAGE_ROWS * 16;
    static constexpr uint32_t STAGE_BYTES = cmax(STAGE_LBO * RC, 256 * S);   // x rows, or the head operand
    static constexpr uint32_t CONV_BYTES = N1 * 2 * R * XB;
    static constexpr uint32_t RES_BYTES = R * R * 2;
    static constexpr uint32_t SKIP_BYTES = S * R * 2;
    static constexpr uint32_t RS_BYTES = RES_BYTES + SKIP_BYTES;
    static constexpr uint32_t HEADP_BYTES = HP * HQ * 2;
    // per-layer bias slots: conv = FP32 b_conv [2R] (16-bit path) or FP32 {scale, bias} [2R] (FP8);
    // res = FP32 b_res [R] (+ FP8: the next layer's input quantisation factors [R])
    static constexpr uint32_t CB_BYTES = F8 ? 16 * R : 8 * R;
    static constexpr uint32_t RB_BYTES = F8 ? 8 * R : 4 * R;
    static constexpr uint32_t ECONV = cmax(CONV_BYTES, HEADP_BYTES);
    static constexpr uint32_t ERS = cmax(RS_BYTES, HEADP_BYTES);
    static constexpr uint32_t TMEM_BR = 2 * R + S;
    static constexpr uint32_t TMEM_COLS = pow2ceil(2 * TMEM_BR);
    static constexpr uint32_t TMEM_BSTRIDE = TMEM_COLS / 2;
    // shared memory map
    static constexpr uint32_t OFF_STAGE = 0;
    static constexpr uint32_t OFF_ENT = 2 * STAGE_BYTES;               // [branch]{conv entry, rs entry}
    static constexpr uint32_t ENT_BR = ECONV + ERS;
    static constexpr uint32_t OFF_BIAS = OFF_ENT + 2 * ENT_BR;         // [branch]{conv slots x2, res slots x2}
    static constexpr uint32_t BIAS_BR = 2 * CB_BYTES + 2 * RB_BYTES;
    static constexpr uint32_t OFF_PART = OFF_BIAS + 2 * BIAS_BR;
    static constexpr uint32_t OFF_BAR = OFF_PART + 4 * kTile * 4;
    static constexpr uint32_t N_BAR = 40;
    static constexpr uint32_t OFF_MISC = OFF_BAR + N_BAR * 8;
    static constexpr uint32_t SMEM = OFF_MISC + 64 + 128;    // + alignment slack
    // per-branch parameter block (bytes): w_in[R], b_in[R], bskip_sum[S] (FP32), FP8: the input
    // projection's quantisation factors [R]; then per layer the conv slot and the res slot
    static constexpr uint32_t HDR_BYTES = 8 * R + 4 * S + (F8 ? 4 * R : 0);
    static constexpr uint32_t PL_BYTES = CB_BYTES + RB_BYTES;
    static __host__ __device__ constexpr uint32_t pb_bytes(int L) { return HDR_BYTES + L * PL_BYTES; }
    static __host__ __device__ constexpr uint32_t ph_bytes() { return ((8 * HC + 4) + 15) & ~15u; }
    static __host__ __device__ constexpr uint32_t pm_bytes(int L) { return 2 * pb_bytes(L) + ph_bytes(); }
    // per-model weight image: per layer [conv H][conv L][rs H][rs L], then the head pieces
    static constexpr uint32_t LAYER_IMG = 2 * CONV_BYTES + 2 * RS_BYTES;
    static __host__ __device__ constexpr uint64_t img_bytes(int L) {
        return (uint64_t)L * LAYER_IMG + (uint64_t)NHP * HEADP_BYTES;
    }
    static_assert(R % 32 == 0 && S % 32 == 0 && HP % 16 == 0, "channel counts");
    static_assert(N1 <= 256 && S <= 256 && HP <= 256, "MMA N limit");
    static_assert(HP <= 2 * R, "head piece must fit the conv TMEM columns");
    static_assert(TMEM_COLS <= 512, "TMEM");
    static_assert(OFF_MISC + 64 + 128 <= 232448, "shared memory per block");
};

// barrier indices
enum {
    B_WFULL = 0,       // [2 branches][2 entries: conv, rs]
    B_WEMPTY = 4,      // [2][2]
    B_LAG = 8,         // [2]
    B_XREADY = 10,     // [2]
    B_CONV = 12,       // [2]
    B_ZREADY = 14,     // [2]
    B_RS = 16,         // [2]
    B_HREADY = 18,     // [2]
    B_HEAD = 20,
    B_WG = 21,         // [2]
    B_PAIR = 23,
    B_FIN = 24,        // [2]
    B_BIAS = 26,       // [2 branches][4 slots: b_conv x2, b_res x2]
    B_GO = 34,         // branch 1 may start its tile (branch 0's first gate is done)
    B_SKIP = 35        // [2] the skip MMAs of a layer completed
};

struct TcParams {
    const uint8_t *wimg;       // [n_models] weight images
    uint64_t wimg_stride;
    const uint8_t *pblob;      // [n_models] parameter blocks
    uint64_t pblob_stride;
    const float *sH, *sL;
    int64_t nw;                // windows of all segments
    int W, stride;
    // Segments (n_seg > 1): segment g holds windows [seg_w0[g], seg_w0[g + 1]) and starts at sample
    // seg_s0[g] of the strain arrays; its window w is samples seg_s0[g] + (w - seg_w0[g]) * stride.
    // n_seg == 1: one segment starting at sample 0 (tables unused).
    int n_seg;
    const int64_t *seg_w0;     // device [n_seg + 1]
    const int64_t *seg_s0;     // device [n_seg]
    int n_models;
    float *out;
    int logits;
    uint8_t *ring;             // per-CTA lag history
    uint64_t ring_cta_bytes;   // per-CTA stride
    uint64_t ring_pp;          // offset of the second ring of a CTA (cross-window reuse), 0: one ring
    const uint8_t *zeros;      // >= 2 KiB of zeros
    int L, lps;
    uint64_t ring_rows;        // lag-history rows per branch (sum of dilations)
    int *err;                  // error word: wait site of the first timeout
    int n16;                   // 16-bit path: layers l < n16 take FP16 conv operands, the others BF16
    // Allocation sizes of the ring (bytes, all CTAs) and of the projections (FP16 elements): every
    // computed lag-copy source, history-row store and projection store is checked against them; an
    // address outside records a site >= 40 in the error word and the access is not made.
    uint64_t ring_alloc;
    uint64_t proj_alloc;
    int model0;                // jobs cover models model0 .. model0 + n_models - 1
    // Projection mode (proj != NULL): instead of the head, store per branch the head's first
    // convolution restricted to that branch, P_H = W_h1[:, H] ReLU(s_H) + b_h1 and
    // P_L = W_h1[:, L] ReLU(s_L), FP16, laid out [branch][window][Hc/8][W][8] (relative to model
    // model0's block); time slides then only evaluate ReLU(P_H + P_L') . w_h2 + b_h2.
    uint16_t *proj;
    uint64_t wait_ns;          // limit of every device-side wait
    int dbg_drop;              // test hook: 1 = branch 0's producer issues nothing (its consumers' waits run out)
    // Cross-window reuse (0 = off).  Window w+1 of a segment starts stride samples after window w,
    // so its tile t is window w's tile t + reuse_shift.  Layer l's output at a position p that is at
    // least r_l - 1 samples from the window start (r_l the receptive field after layer l) does not
    // see the zero padding and equals window w's at p + stride.  For tile t, layers 0 .. lstar[t]
    // satisfy this on all 128 rows (lstar[t] = -1: none); their x_{lstar+1} and partial skip sum
    // are taken from window w's tile t + reuse_shift (exactly the values recomputation would give)
    // through a per-CTA carry buffer, and the tile starts at layer lstar[t] + 1.
    // With reuse the CTA keeps two rings and alternates them per job: a tile that computes every
    // layer may need lagged rows of a layer that an earlier (reusing) tile of the same window
    // skipped; those rows are the previous window's, at the same ring offsets (the shift is a
    // multiple of every dilation), and are read from the previous job's ring.
    int reuse_shift;
    // Training save mode (save_x != NULL, one model, no reuse): the input of every stack, x_l for
    // l % lps == 0, FP32 [stack][branch][window][W][R], and the skip sum with its biases before the
    // head's ReLU, FP32 [branch][window][W][S]: what the backward's per-stack recomputation starts
    // from.
    float *save_x;
    float *save_skip;
    float *carry;              // per CTA: [branch][tile < NT - reuse_shift][(RH + SH) / 4][256 threads] float4
    uint64_t carry_cta_floats;
    int8_t lstar[64];
};

// contiguous job range [j0, j1) of this CTA: consecutive windows of one model follow each other,
// which cross-window reuse needs
__device__ __forceinline__ void job_range(int64_t n_jobs, int64_t &j0, int64_t &j1) {
    const int64_t q = n_jobs / gridDim.x, rm = n_jobs % gridDim.x, c = blockIdx.x;
    j0 = c * q + (c < rm ? c : rm);
    j1 = j0 + q + (c < rm ? 1 : 0);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&h);
}
__device__ __forceinline__ uint32_t pack_h2(float a, float b) {
    __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&h);
}
// conv operand pair of the 16-bit path: FP16 (f16 = true) or BF16
__device__ __forceinline__ uint32_t pack_x2(float a, float b, bool f16) {
    return f16 ? pack_h2(a, b) : pack_bf16(a, b);
}
__device__ __forceinline__ float tanh_f32(float x) {
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ uint32_t tanh_h2(uint32_t x) {
    uint32_t y;
    asm("tanh.approx.f16x2 %0, %1;" : "=r"(y) : "r"(x));
    return y;
}
__device__ __forceinline__ uint32_t hadd2(uint32_t a, uint32_t b) {
    uint32_t y;
    asm("add.rn.f16x2 %0, %1, %2;" : "=r"(y) : "r"(a), "r"(b));
    return y;
}
__device__ __forceinline__ uint32_t hfma2(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t y;
    asm("fma.rn.f16x2 %0, %1, %2, %3;" : "=r"(y) : "r"(a), "r"(b), "r"(c));
    return y;
}
__device__ __forceinline__ uint32_t hmul2(uint32_t a, uint32_t b) {
    uint32_t y;
    asm("mul.rn.f16x2 %0, %1, %2;" : "=r"(y) : "r"(a), "r"(b));
    return y;
}
__device__ __forceinline__ void sts128(uint32_t addr, uint4 v) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
                 : "memory");
}
__device__ __forceinline__ uint4 lds128(uint32_t addr) {
    uint4 v;
    asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(addr)
                 : "memory");
    return v;
}

// segment of window w (the last g with seg_w0[g] <= w; empty segments are skipped over)
__device__ __forceinline__ int find_segment(const int64_t *w0, int n_seg, int64_t w) {
    int lo = 0, hi = n_seg - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (w0[mid] <= w)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// job j -> (model, window): windows of all segments, model-major
struct Job {
    int m;
    int64_t w;       // window index over all segments
    int64_t wloc;    // window index within its segment
    int64_t nws;     // windows of its segment
    int64_t s0;      // first sample of the window in the strain arrays
};
__device__ __forceinline__ Job decode_job(const TcParams &p, int64_t j) {
    Job q;
    q.w = j % p.nw;
    q.m = p.model0 + (int)(j / p.nw);
    if (p.n_seg > 1) {
        const int g = find_segment(p.seg_w0, p.n_seg, q.w);
        q.wloc = q.w - p.seg_w0[g];
        q.nws = p.seg_w0[g + 1] - p.seg_w0[g];
        q.s0 = p.seg_s0[g] + q.wloc * (int64_t)p.stride;
    } else {
        q.wloc = q.w;
        q.nws = p.nw;
        q.s0 = q.w * (int64_t)p.stride;
    }
    return q;
}

// SAVE: training save mode (stack inputs and skip sums stored; BF16 only), a separate instantiation
// so that the inference kernels carry none of its code
template <int R, int S, int HC, bool F8, bool SAVE = false>
__global__ void __launch_bounds__(kThreads, 1) k_branch_tc(const TcParams p) {
    using Sh = TcShape<R, S, HC, F8>;
    constexpr int RH = R / 2;          // channels per epilogue thread (half of a row)
    constexpr int SH = S / 2;
    constexpr int HPH = Sh::HP / 2;
    // TMEM column of the gate output z for K step ks (16 channels): the epilogue half that owns
    // channels [hf*RH, hf*RH + RH) packs them, two per column, at the start of its f columns
    auto zcol = [](int ks) -> uint32_t { return (uint32_t)((ks / (RH / 16)) * RH + 8 * (ks % (RH / 16))); };
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + Sh::OFF_BAR);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + Sh::OFF_MISC);
    int *abort_flag = reinterpret_cast<int *>(smem + Sh::OFF_MISC + 8);
    float *part = reinterpret_cast<float *>(smem + Sh::OFF_PART);
    const uint32_t s_base = smem_u32(smem);
    const uint32_t s_stage = s_base + Sh::OFF_STAGE;
    const uint32_t s_ent = s_base + Sh::OFF_ENT;
    const uint32_t s_bias = s_base + Sh::OFF_BIAS;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int NT = p.W / kTile;
    const int L = p.L, lps = p.lps;
    const int64_t n_jobs = (int64_t)p.n_models * p.nw;

    if (tid == 0) {
        for (int b = 0; b < 2; ++b) {
            for (int e = 0; e < 2; ++e) {
                mbar_init(&bar[B_WFULL + 2 * b + e], 1);
                mbar_init(&bar[B_WEMPTY + 2 * b + e], 1);
            }
            mbar_init(&bar[B_LAG + b], 1);
            mbar_init(&bar[B_XREADY + b], 8);
            mbar_init(&bar[B_CONV + b], 1);
            mbar_init(&bar[B_ZREADY + b], 8);
            mbar_init(&bar[B_RS + b], 1);
            mbar_init(&bar[B_SKIP + b], 1);
            mbar_init(&bar[B_HREADY + b], 8);
            mbar_init(&bar[B_WG + b], 8);
            mbar_init(&bar[B_FIN + b], 1);
            for (int k = 0; k < 4; ++k) mbar_init(&bar[B_BIAS + 4 * b + k], 1);
        }
        mbar_init(&bar[B_HEAD], 1);
        mbar_init(&bar[B_PAIR], 16);
        mbar_init(&bar[B_GO], 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 1) tmem_alloc(tmem_slot, Sh::TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp < 4) {
        const int b = warp >> 1;               // branch served by this warp
        if ((warp & 1) == 0) {
            // -------------------------------------------------------- producer of branch b
            // Per tile and layer: that layer's weights (+ biases) into the branch's conv and rs
            // entries, and the lagged rows of the layer into the staging buffer; branch 0 also
            // streams the head weight pieces through its two entries.
            if (lane == 0) {
                uint32_t it[2] = {0, 0};       // items issued per entry
                uint32_t lag_issued = 0, ph_h = 0, g = 0, g_conv = 0, g_res = 0;
                bool ok = true, first = true;
                uint8_t *ring_c = p.ring + (uint64_t)blockIdx.x * p.ring_cta_bytes + (uint64_t)b * p.ring_rows * Sh::XROW;
                auto take = [&](int e, int site) -> bool {
                    return mbar_wait(&bar[B_WEMPTY + 2 * b + e], ((it[e] & 1) ^ 1), abort_flag, p.err, site, p.wait_ns);
                };
                // lagged rows of layer l for the tile at t0 (ring par of this job, or the previous
                // job's ring when the source rows were taken over from the previous window)
                auto issue_lag = [&](int l, int t0, bool ru, uint32_t par) -> bool {
                    const int d = 1 << (l % lps);
                    const int n = d < kTile ? d : kTile;
                    const uint32_t bytes = (uint32_t)n * 16;
                    const uint64_t roff = (uint64_t)(l / lps) * ((1u << lps) - 1) + (uint64_t)(d - 1);
                    const int ts = t0 / kTile - (d < kTile ? 1 : d / kTile);   // tile holding the source rows
                    const bool prev = ru && ts >= 0 && ts < NT - p.reuse_shift && l <= p.lstar[ts];
                    const uint8_t *src = ring_c + (uint64_t)(par ^ (prev ? 1u : 0u)) * p.ring_pp + roff * Sh::XROW +
                                         (uint64_t)(t0 & (d - 1)) * 16;
                    if (t0 >= d && (uint64_t)(src - p.ring) + (uint64_t)(Sh::RC - 1) * d * 16 + bytes > p.ring_alloc) {
                        atomicCAS(p.err, 0, 41);   // a lag source outside the ring: copy nothing, stop
                        *abort_flag = 1;
                        return false;
                    }
                    mbar_arrive_expect_tx(&bar[B_LAG + b], bytes * Sh::RC);
                    uint8_t *dst0 = smem + Sh::OFF_STAGE + b * Sh::STAGE_BYTES + (kTile - n) * 16;
#pragma unroll
                    for (int c = 0; c < Sh::RC; ++c)
                        bulk_g2s(dst0 + c * Sh::STAGE_LBO, (t0 < d) ? p.zeros : src + (uint64_t)c * d * 16, bytes,
                                 &bar[B_LAG + b]);
                    ++lag_issued;
                    return true;
                };
                // test hook: branch 0's producer issues nothing, so the MMA warp's first wait runs out
                if (p.dbg_drop == 1 && b == 0) ok = false;
                int64_t j0, j1;
                job_range(n_jobs, j0, j1);
                for (int64_t j = j0; j < j1 && ok; ++j) {
                    const Job q = decode_job(p, j);
                    const bool ru = p.reuse_shift > 0 && j > j0 && q.wloc > 0;
                    const uint32_t par = (uint32_t)((j - j0) & 1);
                    const uint8_t *wm = p.wimg + (uint64_t)q.m * p.wimg_stride;
                    const uint8_t *play = p.pblob + (uint64_t)q.m * p.pblob_stride + b * Sh::pb_bytes(L) + Sh::HDR_BYTES;
                    for (int tt = 0; tt < NT && ok; ++tt) {
                        const int l0 = ru ? p.lstar[tt] + 1 : 0;
                        for (int l = l0; l < L; ++l, ++g) {
                            // conv entry: free once the previous conv (or head piece) MMA completed
                            if (!(ok = take(0, 1))) break;
                            mbar_arrive_expect_tx(&bar[B_WFULL + 2 * b + 0], Sh::CONV_BYTES);
                            bulk_g2s(smem + Sh::OFF_ENT + b * Sh::ENT_BR,
                                     wm + (uint64_t)l * Sh::LAYER_IMG + (uint64_t)b * Sh::CONV_BYTES, Sh::CONV_BYTES,
                                     &bar[B_WFULL + 2 * b + 0]);
                            // b_conv of this layer into slot g & 1 (its previous reader, the gate two
                            // layers back, finished before the conv that just freed the entry)
                            mbar_arrive_expect_tx(&bar[B_BIAS + 4 * b + (g & 1)], Sh::CB_BYTES);
                            bulk_g2s(smem + Sh::OFF_BIAS + b * Sh::BIAS_BR + (g & 1) * Sh::CB_BYTES,
                                     play + (uint64_t)l * Sh::PL_BYTES, Sh::CB_BYTES, &bar[B_BIAS + 4 * b + (g & 1)]);
                            g_conv = g + 1;
                            ++it[0];
                            // lagged rows: the staging buffer is free once the previous conv completed
                            // (first layer of a tile: once the previous tile's head has read it)
                            if (l > l0 || first) {
                                if (!(ok = issue_lag(l, tt * kTile, ru, par))) break;
                            } else {
                                ok = mbar_wait(&bar[B_HREADY + b], ph_h & 1, abort_flag, p.err, 3, p.wait_ns) &&
                                     mbar_wait(&bar[B_HEAD], ph_h & 1, abort_flag, p.err, 4, p.wait_ns);
                                if (!ok) break;
                                ++ph_h;
                                if (!(ok = issue_lag(l, tt * kTile, ru, par))) break;
                            }
                            first = false;
                            // rs entry
                            if (!(ok = take(1, 5))) break;
                            mbar_arrive_expect_tx(&bar[B_WFULL + 2 * b + 1], Sh::RS_BYTES);
                            bulk_g2s(smem + Sh::OFF_ENT + b * Sh::ENT_BR + Sh::ECONV,
                                     wm + (uint64_t)l * Sh::LAYER_IMG + 2ull * Sh::CONV_BYTES + (uint64_t)b * Sh::RS_BYTES,
                                     Sh::RS_BYTES, &bar[B_WFULL + 2 * b + 1]);
                            mbar_arrive_expect_tx(&bar[B_BIAS + 4 * b + 2 + (g & 1)], Sh::RB_BYTES);
                            bulk_g2s(smem + Sh::OFF_BIAS + b * Sh::BIAS_BR + 2 * Sh::CB_BYTES + (g & 1) * Sh::RB_BYTES,
                                     play + (uint64_t)l * Sh::PL_BYTES + Sh::CB_BYTES, Sh::RB_BYTES,
                                     &bar[B_BIAS + 4 * b + 2 + (g & 1)]);
                            g_res = g + 1;
                            ++it[1];
                        }
                        if (!ok || b != 0) continue;
                        for (int pc = 0; pc < Sh::NHP; ++pc) {
                            const int e = pc & 1;
                            if (!(ok = take(e, 6))) break;
                            mbar_arrive_expect_tx(&bar[B_WFULL + e], Sh::HEADP_BYTES);
                            bulk_g2s(smem + Sh::OFF_ENT + e * Sh::ECONV,
                                     wm + (uint64_t)L * Sh::LAYER_IMG + (uint64_t)pc * Sh::HEADP_BYTES, Sh::HEADP_BYTES,
                                     &bar[B_WFULL + e]);
                            ++it[e];
                        }
                    }
                }
                // never leave with copies in flight (the copies issued last on every barrier land)
                for (int e = 0; e < 2; ++e)
                    if (it[e] > 0)
                        mbar_wait_drain(&bar[B_WFULL + 2 * b + e], (it[e] - 1) & 1, p.err, 7, p.wait_ns);
                if (lag_issued > 0)
                    mbar_wait_drain(&bar[B_LAG + b], (lag_issued - 1) & 1, p.err, 8, p.wait_ns);
                for (uint32_t k = 0; k < 2 && k < g_conv; ++k) {  // last b_conv of both slots
                    const uint32_t gg = g_conv - 1 - k;
                    mbar_wait_drain(&bar[B_BIAS + 4 * b + (gg & 1)], (gg >> 1) & 1, p.err, 9, p.wait_ns);
                }
                for (uint32_t k = 0; k < 2 && k < g_res; ++k) {   // last b_res of both slots
                    const uint32_t gg = g_res - 1 - k;
                    mbar_wait_drain(&bar[B_BIAS + 4 * b + 2 + (gg & 1)], (gg >> 1) & 1, p.err, 9, p.wait_ns);
                }
            }
        } else {
            // -------------------------------------------------------- MMA issuer of branch b (+ head on branch 0)
            if (lane == 0) {
                constexpr uint32_t ID_CONV = F8 ? idesc_e4m3(128, Sh::N1) : idesc_f16(128, Sh::N1, 1);
                // layers l < n16 of the 16-bit path: both conv operands FP16 (same descriptor form as
                // the residual / skip MMAs); never one FP16 and one BF16 operand
                constexpr uint32_t ID_CONV16 = idesc_f16(128, Sh::N1, 0);
                constexpr uint32_t ID_RES = idesc_f16(128, R, 0);
                constexpr uint32_t ID_SKIP = idesc_f16(128, S, 0);
                constexpr uint32_t ID_HEAD = idesc_f16(128, Sh::HP, 0);
                uint32_t it[2] = {0, 0}, ph_x = 0, ph_lag = 0, ph_z = 0, ph_h = 0, ph_go = 0;
                bool ok = true;
                const uint32_t st = s_stage + b * Sh::STAGE_BYTES;
                const uint32_t dcol = tmem + b * Sh::TMEM_BSTRIDE;
                const uint32_t e_conv = s_ent + b * Sh::ENT_BR, e_rs = e_conv + Sh::ECONV;
                // descriptors of K step 0; a K step of 16 advances two chunk columns (descriptor
                // addresses count 16-byte units, and these sums never carry out of the address field)
                const uint64_t a_lag0 = sdesc(st, Sh::STAGE_LBO, 128);
                const uint64_t a_cur0 = sdesc(st + kTile * 16, Sh::STAGE_LBO, 128);
                const uint64_t b_conv0 = sdesc(e_conv, Sh::N1 * 16, 128);
                const uint64_t b_res0 = sdesc(e_rs, R * 16, 128);
                const uint64_t b_skip0 = sdesc(e_rs + Sh::RES_BYTES, S * 16, 128);
                constexpr uint64_t A_STEP = 2 * Sh::STAGE_LBO / 16;
                int64_t j0, j1;
                job_range(n_jobs, j0, j1);
                for (int64_t j = j0; j < j1 && ok; ++j) {
                    const bool ru = p.reuse_shift > 0 && j > j0 && decode_job(p, j).wloc > 0;
                    for (int tt = 0; tt < NT && ok; ++tt) {
                        const int l0 = ru ? p.lstar[tt] + 1 : 0;
                        // Ping-pong: branch 1 starts a tile once branch 0's first gate is done, so
                        // that one branch's MMAs overlap the other's gate for the rest of the tile.
                        if (b == 1) {
                            if (!(ok = mbar_wait(&bar[B_GO], ph_go & 1, abort_flag, p.err, 19, p.wait_ns))) break;
                            ++ph_go;
                        }
                        for (int l = l0; l < L; ++l) {
                            const int d = 1 << (l % lps);
                            const int n = d < kTile ? d : kTile;
                            // the lagged rows and the weights land while the epilogue is still in the
                            // residual of the previous layer: test them first, so that only the MMA
                            // issue follows the epilogue's hand-off
                            ok = mbar_wait(&bar[B_LAG + b], ph_lag & 1, abort_flag, p.err, 11, p.wait_ns) &&
                                 mbar_wait(&bar[B_WFULL + 2 * b], it[0] & 1, abort_flag, p.err, 12, p.wait_ns) &&
                                 mbar_wait(&bar[B_XREADY + b], ph_x & 1, abort_flag, p.err, 10, p.wait_ns);
                            if (!ok) break;
                            ++ph_x;
                            ++ph_lag;
                            tc_fence_after();
                            // K = 2R in steps of 16: the lagged rows (staging rows 128 - n ..), then the current ones
                            const uint64_t a_lag = a_lag0 + (uint64_t)(kTile - n);
                            const uint32_t id_conv = (!F8 && l < p.n16) ? ID_CONV16 : ID_CONV;
                            auto conv_mma = [&](uint64_t ad, uint64_t bd, uint32_t acc) {
                                if constexpr (F8)
                                    mma_f8(dcol, ad, bd, ID_CONV, acc);
                                else
                                    mma_f16(dcol, ad, bd, id_conv, acc);
                            };
                            conv_mma(a_lag, b_conv0, 0u);
#pragma unroll
                            for (int ks = 1; ks < Sh::RC / 2; ++ks)
                                conv_mma(a_lag + ks * A_STEP, b_conv0 + ks * (2 * Sh::N1), 1u);
#pragma unroll
                            for (int ks = Sh::RC / 2; ks < Sh::RC; ++ks)
                                conv_mma(a_cur0 + (ks - Sh::RC / 2) * A_STEP, b_conv0 + ks * (2 * Sh::N1), 1u);
                            mma_commit(&bar[B_CONV + b]);
                            mma_commit(&bar[B_WEMPTY + 2 * b]);
                            ++it[0];
                            ok = mbar_wait(&bar[B_WFULL + 2 * b + 1], it[1] & 1, abort_flag, p.err, 14, p.wait_ns) &&
                                 mbar_wait(&bar[B_ZREADY + b], ph_z & 1, abort_flag, p.err, 13, p.wait_ns);
                            if (!ok) break;
                            ++ph_z;
                            if (b == 0 && l == l0) mbar_arrive(&bar[B_GO]);
                            tc_fence_after();
                            // z (FP16, two per column) sits in the f columns: channels [16ks, 16ks+16)
                            // at column zcol(ks); r goes to the g columns, s accumulates after them
#pragma unroll
                            for (int ks = 0; ks < Sh::KR; ++ks)
                                mma_f16_ta(dcol + R, dcol + zcol(ks), b_res0 + ks * (2 * R), ID_RES, ks > 0 ? 1u : 0u);
                            // the residual needs r only: release it before the skip MMAs (they run
                            // while the epilogue updates x; this thread's MMAs execute in issue order,
                            // so the next conv cannot overwrite z before the skip MMAs have read it)
                            mma_commit(&bar[B_RS + b]);
                            mma_f16_ta(dcol + 2 * R, dcol + zcol(0), b_skip0, ID_SKIP, l > 0 ? 1u : 0u);
#pragma unroll
                            for (int ks = 1; ks < Sh::KR; ++ks)
                                mma_f16_ta(dcol + 2 * R, dcol + zcol(ks), b_skip0 + ks * (2 * S), ID_SKIP, 1u);
                            mma_commit(&bar[B_SKIP + b]);
                            mma_commit(&bar[B_WEMPTY + 2 * b + 1]);
                            ++it[1];
                        }
                        if (!ok || b != 0) continue;
                        // head (branch 0's MMA warp): u[nh] = sum over K quarters of h . W_h1[nh, quarter]^T
                        ok = mbar_wait(&bar[B_HREADY + 0], ph_h & 1, abort_flag, p.err, 15, p.wait_ns) &&
                             mbar_wait(&bar[B_HREADY + 1], ph_h & 1, abort_flag, p.err, 16, p.wait_ns);
                        if (!ok) break;
                        ++ph_h;
                        for (int pc = 0; pc < Sh::NHP && ok; ++pc) {
                            const int e = pc & 1, nh = pc >> 2, kq = pc & 3;
                            ok = mbar_wait(&bar[B_WFULL + e], it[e] & 1, abort_flag, p.err, 17, p.wait_ns);
                            if (!ok) break;
                            tc_fence_after();
                            const uint32_t ha = s_stage + (kq >> 1) * Sh::STAGE_BYTES + (kq & 1) * (Sh::HQ / 8) * (kTile * 16);
                            const uint32_t we = s_ent + e * Sh::ECONV;
#pragma unroll
                            for (int ks = 0; ks < Sh::HQ / 16; ++ks) {
                                const uint64_t ad = sdesc(ha + 2 * ks * (kTile * 16), kTile * 16, 128);
                                const uint64_t bd = sdesc(we + 2 * ks * (Sh::HP * 16), Sh::HP * 16, 128);
                                if (p.proj)   // P_H pieces in branch 0's columns, P_L pieces in branch 1's
                                    mma_f16(tmem + (kq >> 1) * Sh::TMEM_BSTRIDE + nh * Sh::HP, ad, bd, ID_HEAD,
                                            ((kq & 1) || ks > 0) ? 1u : 0u);
                                else
                                    mma_f16(tmem + nh * Sh::TMEM_BSTRIDE, ad, bd, ID_HEAD, (kq > 0 || ks > 0) ? 1u : 0u);
                            }
                            mma_commit(&bar[B_WEMPTY + e]);
                            ++it[e];
                        }
                        if (ok) mma_commit(&bar[B_HEAD]);
                    }
                }
                // all MMAs issued by this thread complete before TMEM is released
                mma_commit(&bar[B_FIN + b]);
                mbar_wait_drain(&bar[B_FIN + b], 0, p.err, 18, p.wait_ns);
            }
        }
    } else {
        // ------------------------------------------------------------ epilogue (thread = row, half the channels)
        const int eg = warp - 4;
        const int b = eg >> 3;                         // 0: Hanford branch, 1: Livingston branch
        const int hf = (eg >> 2) & 1;                  // channel half
        const int q = warp & 3;                        // TMEM lane quarter of this warp
        const int r = q * 32 + lane;                   // row within the tile
        const uint32_t t_lane = (uint32_t)(q * 32) << 16;
        const uint32_t t_conv = tmem + t_lane + b * Sh::TMEM_BSTRIDE;
        const uint32_t t_skip = t_conv + 2 * R;
        const uint32_t st = s_stage + b * Sh::STAGE_BYTES;
        const uint32_t sb = s_bias + b * Sh::BIAS_BR;
        const int c0 = hf * RH;                        // first channel of this thread
        uint8_t *ring_c = p.ring + (uint64_t)blockIdx.x * p.ring_cta_bytes + (uint64_t)b * p.ring_rows * Sh::XROW;
        uint32_t ph_conv = 0, ph_rs = 0, ph_head = 0, ph_wg = 0, ph_pair = 0;
        uint32_t g = 0;                                // computed layers so far: bias slot g & 1, use (g >> 1)
        const int ntr = NT - p.reuse_shift;            // tiles that can take layers from the previous window
        float4 *carry_t = reinterpret_cast<float4 *>(p.carry + (uint64_t)blockIdx.x * p.carry_cta_floats) +
                          (uint64_t)b * ntr * ((RH + SH) / 4) * 256 + (hf * kTile + r);
        bool ok = true;
        float x[RH];
        const uint32_t half2_half = 0x38003800u;     // (0.5, 0.5) in FP16x2

        auto warp_wait = [&](int idx, uint32_t parity, int site) -> bool {
            bool w = mbar_wait(&bar[idx], parity, abort_flag, p.err, site, p.wait_ns);
            return __all_sync(0xffffffffu, w);
        };
        auto warp_arrive = [&](int idx) {
            __syncwarp();
            if (lane == 0) mbar_arrive(&bar[idx]);
        };
        // x (FP32 registers) -> this thread's chunks of the staging row for the conv of layer lc:
        // FP16 (lc < n16) or BF16, or FP8 E4M3 after multiplying by layer lc's per-channel
        // quantisation factors `inv` (FP32)
        auto store_x = [&](const float *inv_g, uint32_t inv_s, int lc) {
            if constexpr (F8) {
#pragma unroll
                for (int c = 0; c < RH / 16; ++c) {
                    uint32_t wv[4];
#pragma unroll
                    for (int k4 = 0; k4 < 4; ++k4) {
                        float4 iv;
                        if (inv_g)
                            iv = __ldg(reinterpret_cast<const float4 *>(inv_g) + 4 * c + k4);
                        else {
                            const uint4 u = lds128(inv_s + (16 * c + 4 * k4) * 4);
                            iv = make_float4(__uint_as_float(u.x), __uint_as_float(u.y), __uint_as_float(u.z),
                                             __uint_as_float(u.w));
                        }
                        const int o = 16 * c + 4 * k4;
                        const uint32_t lo = __nv_cvt_float2_to_fp8x2(make_float2(x[o] * iv.x, x[o + 1] * iv.y),
                                                                     __NV_SATFINITE, __NV_E4M3);
                        const uint32_t hi = __nv_cvt_float2_to_fp8x2(make_float2(x[o + 2] * iv.z, x[o + 3] * iv.w),
                                                                     __NV_SATFINITE, __NV_E4M3);
                        wv[k4] = lo | (hi << 16);
                    }
                    sts128(st + (hf * (RH / 16) + c) * Sh::STAGE_LBO + (kTile + r) * 16,
                           make_uint4(wv[0], wv[1], wv[2], wv[3]));
                }
            } else {
                const bool f16 = lc < p.n16;
#pragma unroll
                for (int c = 0; c < RH / 8; ++c) {
                    uint4 v;
                    v.x = pack_x2(x[8 * c + 0], x[8 * c + 1], f16);
                    v.y = pack_x2(x[8 * c + 2], x[8 * c + 3], f16);
                    v.z = pack_x2(x[8 * c + 4], x[8 * c + 5], f16);
                    v.w = pack_x2(x[8 * c + 6], x[8 * c + 7], f16);
                    sts128(st + (hf * (RH / 8) + c) * Sh::STAGE_LBO + (kTile + r) * 16, v);
                }
            }
        };
        // z for 16 channels starting at ch from the f / g accumulator columns, in FP32:
        // f = acc_f + b_f, g/2 = acc_g + b_g/2 (the g half of the conv weights and biases is
        // pre-halved), z = tanh(f) * (0.5 tanh(g/2) + 0.5); z leaves as FP16 pairs (the operand of
        // the residual / skip MMAs).  FP8: acc is first multiplied by the output channel's weight
        // scale (FP32 {scale, bias} pairs).
        auto gate16 = [&](const uint32_t (&fr)[16], const uint32_t (&gr)[16], int ch, uint32_t bslot, uint32_t (&zz)[8]) {
#pragma unroll
            for (int jq = 0; jq < 4; ++jq) {          // four channels (two pairs) per step
                float f[4], gv[4];
                if constexpr (F8) {
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int jj = 2 * jq + h;
                        const uint4 sf = lds128(bslot + (ch + 2 * jj) * 8);          // {s, b} of f channels 2jj, 2jj+1
                        const uint4 sg4 = lds128(bslot + (R + ch + 2 * jj) * 8);     // same for g
                        f[2 * h] = fmaf(__uint_as_float(fr[2 * jj]), __uint_as_float(sf.x), __uint_as_float(sf.y));
                        f[2 * h + 1] = fmaf(__uint_as_float(fr[2 * jj + 1]), __uint_as_float(sf.z), __uint_as_float(sf.w));
                        gv[2 * h] = fmaf(__uint_as_float(gr[2 * jj]), __uint_as_float(sg4.x), __uint_as_float(sg4.y));
                        gv[2 * h + 1] = fmaf(__uint_as_float(gr[2 * jj + 1]), __uint_as_float(sg4.z), __uint_as_float(sg4.w));
                    }
                } else {
                    // FP32 biases of f channels ch + 4jq .. + 3 and of the matching g channels
                    const uint4 bf = lds128(bslot + (ch + 4 * jq) * 4);
                    const uint4 bg = lds128(bslot + (R + ch + 4 * jq) * 4);
                    f[0] = __uint_as_float(fr[4 * jq]) + __uint_as_float(bf.x);
                    f[1] = __uint_as_float(fr[4 * jq + 1]) + __uint_as_float(bf.y);
                    f[2] = __uint_as_float(fr[4 * jq + 2]) + __uint_as_float(bf.z);
                    f[3] = __uint_as_float(fr[4 * jq + 3]) + __uint_as_float(bf.w);
                    gv[0] = __uint_as_float(gr[4 * jq]) + __uint_as_float(bg.x);
                    gv[1] = __uint_as_float(gr[4 * jq + 1]) + __uint_as_float(bg.y);
                    gv[2] = __uint_as_float(gr[4 * jq + 2]) + __uint_as_float(bg.z);
                    gv[3] = __uint_as_float(gr[4 * jq + 3]) + __uint_as_float(bg.w);
                }
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const float s0 = fmaf(tanh_f32(gv[2 * h]), 0.5f, 0.5f), s1 = fmaf(tanh_f32(gv[2 * h + 1]), 0.5f, 0.5f);
                    zz[2 * jq + h] = pack_h2(tanh_f32(f[2 * h]) * s0, tanh_f32(f[2 * h + 1]) * s1);
                }
            }
        };

        int64_t j0, j1;
        job_range(n_jobs, j0, j1);
        for (int64_t j = j0; j < j1 && ok; ++j) {
            const Job jb = decode_job(p, j);
            const bool ru = p.reuse_shift > 0 && j > j0 && jb.wloc > 0;                 // take from the previous window
            const bool cw = p.reuse_shift > 0 && j + 1 < j1 && jb.wloc + 1 < jb.nws;    // give to the next one
            uint8_t *ring_b = ring_c + (uint64_t)((j - j0) & 1) * p.ring_pp;
            const uint8_t *pm = p.pblob + (uint64_t)jb.m * p.pblob_stride;
            const uint8_t *pbr = pm + b * Sh::pb_bytes(L);
            const float4 *w_in4 = reinterpret_cast<const float4 *>(pbr) + c0 / 4;
            const float4 *b_in4 = reinterpret_cast<const float4 *>(pbr) + R / 4 + c0 / 4;
            const float4 *bsk4 = reinterpret_cast<const float4 *>(pbr) + R / 2 + hf * (SH / 4);
            const float *phd = reinterpret_cast<const float *>(pm + 2 * Sh::pb_bytes(L));
            const float *b1 = phd, *w2 = phd + HC;
            const float b2 = __ldg(phd + 2 * HC);
            const float *sv = (b ? p.sL : p.sH) + jb.s0;
            float *outp = p.out + ((int64_t)(jb.m - p.model0) * p.nw + jb.w) * (int64_t)p.W;
            for (int tt = 0; tt < NT && ok; ++tt) {
                const int t0 = tt * kTile;
                const int l0 = ru ? p.lstar[tt] + 1 : 0;
                // carry slot written by this tile for the next window's tile tt - shift (-1: none)
                const int lgive = (cw && tt >= p.reuse_shift) ? p.lstar[tt - p.reuse_shift] : -1;
                if (l0 > 0) {
                    // x_{l0} and the skip sum of layers < l0 from the previous window (same thread wrote them)
                    const float4 *cs = carry_t + (uint64_t)tt * ((RH + SH) / 4) * 256;
#pragma unroll
                    for (int k4 = 0; k4 < RH / 4; ++k4) {
                        const float4 v = cs[(uint64_t)k4 * 256];
                        x[4 * k4 + 0] = v.x;
                        x[4 * k4 + 1] = v.y;
                        x[4 * k4 + 2] = v.z;
                        x[4 * k4 + 3] = v.w;
                    }
#pragma unroll
                    for (int k8 = 0; k8 < SH / 8; ++k8) {
                        const float4 u0 = cs[(uint64_t)(RH / 4 + 2 * k8) * 256];
                        const float4 u1 = cs[(uint64_t)(RH / 4 + 2 * k8 + 1) * 256];
                        const uint32_t sv8[8] = {__float_as_uint(u0.x), __float_as_uint(u0.y), __float_as_uint(u0.z),
                                                 __float_as_uint(u0.w), __float_as_uint(u1.x), __float_as_uint(u1.y),
                                                 __float_as_uint(u1.z), __float_as_uint(u1.w)};
                        tmem_st8(t_skip + hf * SH + 8 * k8, sv8);
                    }
                    tmem_st_wait();
                    // quantisation factors of layer l0 (FP8): the residual slot of layer l0 - 1
                    store_x(reinterpret_cast<const float *>(pbr + Sh::HDR_BYTES + (uint64_t)(l0 - 1) * Sh::PL_BYTES +
                                                            Sh::CB_BYTES) + R + c0, 0u, l0);
                    fence_proxy_async_smem();
                    tc_fence_before();
                    warp_arrive(B_XREADY + b);
                } else {
                    // input 1x1 convolution x_0 = w_in s + b_in (FP32), BF16 copy for the MMA
                    const float sval = __ldg(sv + t0 + r);
#pragma unroll
                    for (int c4 = 0; c4 < RH / 4; ++c4) {
                        const float4 wi = __ldg(w_in4 + c4), bi = __ldg(b_in4 + c4);
                        x[4 * c4 + 0] = fmaf(wi.x, sval, bi.x);
                        x[4 * c4 + 1] = fmaf(wi.y, sval, bi.y);
                        x[4 * c4 + 2] = fmaf(wi.z, sval, bi.z);
                        x[4 * c4 + 3] = fmaf(wi.w, sval, bi.w);
                    }
                    store_x(reinterpret_cast<const float *>(pbr + 8 * R + 4 * S) + c0, 0u, 0);
                    fence_proxy_async_smem();
                    tc_fence_before();
                    warp_arrive(B_XREADY + b);
                }
                for (int l = l0; l < L; ++l, ++g) {
                    const int d = 1 << (l % lps);
                    const int n = d < kTile ? d : kTile;
                    if (SAVE && l % lps == 0) {
                        // stack input x_l of this thread's row and channels
                        float4 *dx = reinterpret_cast<float4 *>(
                            p.save_x + ((((int64_t)(l / lps) * 2 + b) * p.nw + jb.w) * p.W + t0 + r) * R + c0);
#pragma unroll
                        for (int k4 = 0; k4 < RH / 4; ++k4)
                            dx[k4] = make_float4(x[4 * k4], x[4 * k4 + 1], x[4 * k4 + 2], x[4 * k4 + 3]);
                    }
                    // the bias slot lands long before the conv MMAs complete: test it first, so that
                    // only the conv barrier's test stands between the MMAs' completion and the gate
                    if (!warp_wait(B_BIAS + 4 * b + (g & 1), (g >> 1) & 1, 36) ||
                        !warp_wait(B_CONV + b, ph_conv & 1, 30)) { ok = false; break; }
                    ++ph_conv;
                    tc_fence_after();
                    // gate: z = tanh(f + b_f) * (0.5 tanh(g/2 + b_g/2) + 0.5), FP32
                    {
                        const uint32_t bslot = sb + (g & 1) * Sh::CB_BYTES;
                        uint32_t fa[16], ga[16];
                        tmem_ld16(t_conv + c0, fa);
                        tmem_ld16(t_conv + R + c0, ga);
                        tmem_ld_wait();
                        uint32_t z0[8];
                        if constexpr (RH == 32) {
                            uint32_t fb[16], gbv[16], z1[8];
                            tmem_ld16(t_conv + c0 + 16, fb);
                            tmem_ld16(t_conv + R + c0 + 16, gbv);
                            gate16(fa, ga, c0, bslot, z0);
                            tmem_ld_wait();
                            gate16(fb, gbv, c0 + 16, bslot, z1);
                            tmem_st8(t_conv + c0 + 8, z1);
                        } else {
                            gate16(fa, ga, c0, bslot, z0);
                        }
                        tmem_st8(t_conv + c0, z0);
                        tmem_st_wait();
                    }
                    tc_fence_before();
                    warp_arrive(B_ZREADY + b);
                    // lag history of layer l for the following tiles (and, when the next window takes
                    // over layers, for its full tiles): rows t0+r, r >= 128 - n.  Written after the
                    // gate's hand-off, while the res MMAs run (x still holds x_l, and the FP8 staging
                    // row is rewritten only by the residual below), so that the warps holding the
                    // last rows do not delay the gate.
                    const uint64_t roff_h = (uint64_t)(l / lps) * ((1u << lps) - 1) + (uint64_t)(d - 1);
                    uint8_t *dst = ring_b + roff_h * Sh::XROW + (uint64_t)((t0 + r) & (d - 1)) * 16;
                    // the last 16-byte chunk this thread stores (chunk columns of its half, d rows apart)
                    const bool in_ring = (uint64_t)(dst - p.ring) + (uint64_t)(hf * (Sh::RC / 2) + Sh::RC / 2 - 1) * d * 16 +
                                             16 <= p.ring_alloc;
                    if ((tt + 1 < NT || cw) && r >= kTile - n && !in_ring) atomicCAS(p.err, 0, 42);
                    if ((tt + 1 < NT || cw) && r >= kTile - n && in_ring) {
                        if constexpr (F8) {
                            // the quantised row is still in the staging buffer (rewritten after the rs MMA)
#pragma unroll
                            for (int c = 0; c < RH / 16; ++c) {
                                const int ck = hf * (RH / 16) + c;
                                *reinterpret_cast<uint4 *>(dst + (uint64_t)ck * d * 16) =
                                    lds128(st + ck * Sh::STAGE_LBO + (kTile + r) * 16);
                            }
                        } else {
                            // the format of layer l's conv operand
                            const bool f16 = l < p.n16;
#pragma unroll
                            for (int c = 0; c < RH / 8; ++c) {
                                uint4 v;
                                v.x = pack_x2(x[8 * c + 0], x[8 * c + 1], f16);
                                v.y = pack_x2(x[8 * c + 2], x[8 * c + 3], f16);
                                v.z = pack_x2(x[8 * c + 4], x[8 * c + 5], f16);
                                v.w = pack_x2(x[8 * c + 6], x[8 * c + 7], f16);
                                *reinterpret_cast<uint4 *>(dst + (uint64_t)(hf * (RH / 8) + c) * d * 16) = v;
                            }
                        }
                    }
                    // residual: x_{l+1} = (x_l + b_res) + W_res z  (FP32).  The bias is added while the
                    // residual MMAs run, so that only the TMEM load and one add follow their completion.
                    if (!warp_wait(B_BIAS + 4 * b + 2 + (g & 1), (g >> 1) & 1, 37)) { ok = false; break; }
                    const uint32_t rslot = sb + 2 * Sh::CB_BYTES + (g & 1) * Sh::RB_BYTES;
                    if (l + 1 < L) {
                        const uint32_t bres = rslot + c0 * 4;
#pragma unroll
                        for (int k4 = 0; k4 < RH / 4; ++k4) {
                            const uint4 bb = lds128(bres + 16 * k4);
                            x[4 * k4 + 0] += __uint_as_float(bb.x);
                            x[4 * k4 + 1] += __uint_as_float(bb.y);
                            x[4 * k4 + 2] += __uint_as_float(bb.z);
                            x[4 * k4 + 3] += __uint_as_float(bb.w);
                        }
                    }
                    if (!warp_wait(B_RS + b, ph_rs & 1, 31)) { ok = false; break; }
                    ++ph_rs;
                    tc_fence_after();
                    if (l + 1 < L) {
                        uint32_t rr[RH];
                        if constexpr (RH == 32) {
                            tmem_ld32(t_conv + R + c0, rr);
                        } else {
                            tmem_ld16(t_conv + R + c0, rr);
                        }
                        tmem_ld_wait();
#pragma unroll
                        for (int k = 0; k < RH; ++k) x[k] += __uint_as_float(rr[k]);
                        store_x(nullptr, rslot + (R + c0) * 4, l + 1);
                        fence_proxy_async_smem();
                        tc_fence_before();
                        warp_arrive(B_XREADY + b);
                        if (l == lgive) {
                            // x_{l+1} and the skip sum of layers <= l for the next window's tile tt - shift
                            // (the skip MMAs of layer l complete after r is released)
                            if (!warp_wait(B_SKIP + b, g & 1, 38)) { ok = false; break; }
                            tc_fence_after();
                            float4 *cd = carry_t + (uint64_t)(tt - p.reuse_shift) * ((RH + SH) / 4) * 256;
#pragma unroll
                            for (int k4 = 0; k4 < RH / 4; ++k4)
                                cd[(uint64_t)k4 * 256] = make_float4(x[4 * k4], x[4 * k4 + 1], x[4 * k4 + 2], x[4 * k4 + 3]);
#pragma unroll
                            for (int cc = 0; cc < SH / 16; ++cc) {
                                uint32_t sr[16];
                                tmem_ld16(t_skip + hf * SH + 16 * cc, sr);
                                tmem_ld_wait();
#pragma unroll
                                for (int k4 = 0; k4 < 4; ++k4)
                                    cd[(uint64_t)(RH / 4 + 4 * cc + k4) * 256] =
                                        make_float4(__uint_as_float(sr[4 * k4]), __uint_as_float(sr[4 * k4 + 1]),
                                                    __uint_as_float(sr[4 * k4 + 2]), __uint_as_float(sr[4 * k4 + 3]));
                            }
                        }
                    }
                }
                if (!ok) break;
                // the last layer's skip MMAs complete before the skip sum is read for the head
                if (!warp_wait(B_SKIP + b, (g - 1) & 1, 39)) { ok = false; break; }
                tc_fence_after();
                // history rows written with ordinary stores are read by bulk copies of later tiles
                fence_proxy_async_global();
                // every row's history copy has read the staging buffer before it becomes the head operand
                warp_arrive(B_WG + b);
                if (!warp_wait(B_WG + b, ph_wg & 1, 32)) { ok = false; break; }
                ++ph_wg;
                // head operand h = ReLU(skip + sum of skip biases), FP16, rows-128 layout in this branch's staging buffer
#pragma unroll
                for (int cc = 0; cc < SH / 16; ++cc) {
                    const int ch = hf * SH + 16 * cc;
                    uint32_t sr[16];
                    tmem_ld16(t_skip + ch, sr);
                    tmem_ld_wait();
                    float h[16];
#pragma unroll
                    for (int k4 = 0; k4 < 4; ++k4) {
                        const float4 bs = __ldg(bsk4 + 4 * cc + k4);
                        h[4 * k4 + 0] = __uint_as_float(sr[4 * k4 + 0]) + bs.x;
                        h[4 * k4 + 1] = __uint_as_float(sr[4 * k4 + 1]) + bs.y;
                        h[4 * k4 + 2] = __uint_as_float(sr[4 * k4 + 2]) + bs.z;
                        h[4 * k4 + 3] = __uint_as_float(sr[4 * k4 + 3]) + bs.w;
                    }
                    if constexpr (SAVE) {
                        float4 *ds = reinterpret_cast<float4 *>(
                            p.save_skip + (((int64_t)b * p.nw + jb.w) * p.W + t0 + r) * S + ch);
#pragma unroll
                        for (int k4 = 0; k4 < 4; ++k4)
                            ds[k4] = make_float4(h[4 * k4], h[4 * k4 + 1], h[4 * k4 + 2], h[4 * k4 + 3]);
                    }
#pragma unroll
                    for (int k = 0; k < 16; ++k) h[k] = fmaxf(h[k], 0.f);
                    sts128(st + (ch / 8) * (kTile * 16) + r * 16,
                           make_uint4(pack_h2(h[0], h[1]), pack_h2(h[2], h[3]), pack_h2(h[4], h[5]), pack_h2(h[6], h[7])));
                    sts128(st + (ch / 8 + 1) * (kTile * 16) + r * 16,
                           make_uint4(pack_h2(h[8], h[9]), pack_h2(h[10], h[11]), pack_h2(h[12], h[13]),
                                      pack_h2(h[14], h[15])));
                }
                fence_proxy_async_smem();
                tc_fence_before();
                warp_arrive(B_HREADY + b);
                if (!warp_wait(B_HEAD, ph_head & 1, 33)) { ok = false; break; }
                ++ph_head;
                tc_fence_after();
                if (p.proj) {
                    // P_b (+ b_h1 for the Hanford branch), FP16, 16-byte chunks of 8 channels, rows contiguous
                    uint16_t *pw = p.proj + ((uint64_t)b * p.nw + (uint64_t)jb.w) * (uint64_t)HC * p.W;
                    // the highest element this thread stores: chunk HC/8 - 1 of its row
                    const bool in_proj = (uint64_t)(pw - p.proj) + ((uint64_t)(HC / 8 - 1) * p.W + t0 + r) * 8 + 8 <=
                                         p.proj_alloc;
                    if (!in_proj) atomicCAS(p.err, 0, 43);
                    const uint32_t t_p = tmem + t_lane + b * Sh::TMEM_BSTRIDE;
                    constexpr int HH = HC / 2;       // channels per thread (half)
#pragma unroll
                    for (int cc = 0; cc < HH / 16; ++cc) {
                        const int ch = hf * HH + 16 * cc;
                        uint32_t ur[16];
                        tmem_ld16(t_p + ch, ur);
                        tmem_ld_wait();
                        float u[16];
#pragma unroll
                        for (int jj = 0; jj < 16; ++jj)
                            u[jj] = __uint_as_float(ur[jj]) + (b == 0 ? __ldg(b1 + ch + jj) : 0.f);
                        uint4 v0 = make_uint4(pack_h2(u[0], u[1]), pack_h2(u[2], u[3]), pack_h2(u[4], u[5]),
                                              pack_h2(u[6], u[7]));
                        uint4 v1 = make_uint4(pack_h2(u[8], u[9]), pack_h2(u[10], u[11]), pack_h2(u[12], u[13]),
                                              pack_h2(u[14], u[15]));
                        if (in_proj) {
                            *reinterpret_cast<uint4 *>(pw + ((uint64_t)(ch / 8) * p.W + t0 + r) * 8) = v0;
                            *reinterpret_cast<uint4 *>(pw + ((uint64_t)(ch / 8 + 1) * p.W + t0 + r) * 8) = v1;
                        }
                    }
                    // P overlaps the skip columns: no thread restores the next tile's carried skip sum
                    // (cross-window reuse) before every thread of both branches has read its P
                    tc_fence_before();
                    warp_arrive(B_PAIR);
                    if (!warp_wait(B_PAIR, ph_pair & 1, 34)) { ok = false; break; }
                    ++ph_pair;
                    continue;
                }
                float acc = 0.f;
                if (b < Sh::NH) {
                    const uint32_t t_u = tmem + t_lane + b * Sh::TMEM_BSTRIDE + hf * HPH;
#pragma unroll
                    for (int cc = 0; cc < HPH / 16; ++cc) {
                        uint32_t ur[16];
                        tmem_ld16(t_u + 16 * cc, ur);
                        tmem_ld_wait();
#pragma unroll
                        for (int jj = 0; jj < 16; ++jj) {
                            const int ch = b * Sh::HP + hf * HPH + 16 * cc + jj;
                            const float u = __uint_as_float(ur[jj]) + __ldg(b1 + ch);
                            acc = fmaf(__ldg(w2 + ch), fmaxf(u, 0.f), acc);
                        }
                    }
                }
                // single buffer: no warp can write the next tile's partials before this tile's
                // are read, since the next head needs this reader's rows of the next tile first
                float *pp = part;
                pp[(2 * b + hf) * kTile + r] = acc;
                tc_fence_before();
                warp_arrive(B_PAIR);
                if (!warp_wait(B_PAIR, ph_pair & 1, 34)) { ok = false; break; }
                ++ph_pair;
                if (b == 0 && hf == 0) {
                    const float lg = ((pp[r] + pp[kTile + r]) + (pp[2 * kTile + r] + pp[3 * kTile + r])) + b2;
                    outp[t0 + r] = p.logits ? lg : 1.f / (1.f + expf(-lg));
                }
            }
        }
    }
    __syncwarp();
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, Sh::TMEM_COLS);
    }
}

// Time slides on the branch projections: for each slide k, Hanford window w is paired with
// Livingston window (w + k) mod n_w (within w's segment), and
//   out[slide][w][t] = sigmoid(b_h2 + sum_j w_h2[j] ReLU(P_H[w][t][j] + P_L[w'][t][j]))
// (the head's first convolution is linear in [s_H ; s_L], so the branch pass runs once per window
// and a slide costs 3 Hc operations per sample).
//
// Arithmetic (identical for every launch shape, so that all shapes give the same bits): the Hc
// channels form Hc/16 pairs of 16-byte chunks; per pair, FP16x2 ReLU-adds and products accumulate
// in one FP16x2 word over its 16 channels, which is widened to FP32 and summed (x + y); the pair
// sums are added in a balanced binary tree in pair order; b_h2 is added last, then the sigmoid.
//
// Register blocking: the offsets are taken in pieces of up to B values in arithmetic progression
// k0, k0 + dw, ..., k0 + (nb - 1) dw (dw: the offset list's most common step), and a block pairs
// a piece with A Hanford windows of one segment spaced by the same step, w0 + a dw.  Pair (a, b)
// reads Livingston window (w0 + k0 + (a + b) dw) mod n_w, which depends on s = a + b only, so the
// block streams the A + B - 1 Livingston tiles through registers once each and every tile serves
// up to min(A, B) pairs: the L2 -> SM traffic per offset-sample is (A + B - 1) / (A B) of the tile
// bytes (7/16 at 4 x 4, 11/32 at 4 x 8).  Offsets outside a progression form pieces of one.
// Threads: one chunk pair per thread; a warp holds QL pairs of SPW samples (lane = pair-in-warp x
// SPW + sample, so every load request reads whole 128-byte lines), QH warps hold the other pairs.
// The pair sums are reduced by recursive halving across the warp's lanes (shuffles) and then
// across the warps through shared memory.
template <int HC>
struct SlideGeo {
    static constexpr int NP = HC / 16;             // chunk pairs (leaves of the summation tree)
    static constexpr int QL = NP < 4 ? NP : 4;     // pairs per warp
    static constexpr int QH = NP / QL;             // warps per block
    static constexpr int SPB = 32 / QL;            // samples per block
    static constexpr int THREADS = 32 * QH;
    static constexpr int MIN_BLOCKS = 512 / THREADS;   // at most 128 registers per thread
    static_assert(NP >= 1 && NP % QL == 0 && (QH & (QH - 1)) == 0, "pair layout");
};

template <int N>
__device__ __forceinline__ float tree_sum(const float *x) {
    if constexpr (N == 1) {
        return x[0];
    } else {
        return tree_sum<N / 2>(x) + tree_sum<N / 2>(x + N / 2);
    }
}

// one pair's sum for Hanford chunks h[0..1] and Livingston chunks l0, l1 with head weights wv
__device__ __forceinline__ float slide_pair(const uint4 (&h)[2], const uint4 &l0, const uint4 &l1,
                                            const uint32_t (&wv)[8]) {
    const uint32_t one2 = 0x3C003C00u;            // (1, 1) in FP16x2
    const uint32_t hv[8] = {h[0].x, h[0].y, h[0].z, h[0].w, h[1].x, h[1].y, h[1].z, h[1].w};
    const uint32_t lv[8] = {l0.x, l0.y, l0.z, l0.w, l1.x, l1.y, l1.z, l1.w};
    uint32_t acc = 0u;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        uint32_t r;
        asm("fma.rn.relu.f16x2 %0, %1, %2, %3;" : "=r"(r) : "r"(hv[j]), "r"(one2), "r"(lv[j]));
        acc = hfma2(r, wv[j], acc);
    }
    const float2 f = __half22float2(*reinterpret_cast<const __half2 *>(&acc));
    return f.x + f.y;
}

// Grid: x = run of A dw windows (taken as dw residues of A windows each, and split where a segment
// ends), y = 32-sample tile, z = group of `ppb` pieces.  pieces[i] = (first slide index, count).
template <int HC, int A, int B>
__global__ void __launch_bounds__(SlideGeo<HC>::THREADS, SlideGeo<HC>::MIN_BLOCKS) k_slide_head(
    const uint16_t *__restrict__ proj, int64_t nw, int W, const int32_t *__restrict__ koff,
    const int2 *__restrict__ pieces, int n_pieces, int ppb, int dw, int n_seg, const int64_t *__restrict__ seg_w0,
    const float *__restrict__ w2, const float *__restrict__ b2p, float *__restrict__ out, int64_t slide_stride,
    int logits) {
    using G = SlideGeo<HC>;
    constexpr int V = A * B;                       // pair values per thread and piece
    constexpr int NS = A + B - 1;                  // Livingston tiles per piece
    constexpr int PF = NS < 4 ? NS : 4;            // tiles in flight
    constexpr int VL = V / G::QL;                  // values a lane holds after the in-warp halving
    static_assert(V % G::QL == 0, "values per lane");
    __shared__ float part[G::QH > 1 ? G::QH * V * G::SPB : 1];
    const int lane = threadIdx.x & 31, qh = threadIdx.x >> 5;
    const int qlo = lane / G::SPB, ts = lane % G::SPB;
    const int q = qh * G::QL + qlo;                // this thread's chunk pair
    const int tb = blockIdx.y * G::SPB;
    const int pc0 = blockIdx.z * ppb;
    const int pc1 = min(n_pieces, pc0 + ppb);
    uint32_t wv[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) wv[j] = pack_h2(__ldg(w2 + 16 * q + 2 * j), __ldg(w2 + 16 * q + 2 * j + 1));
    const float b2 = __ldg(b2p);
    const uint64_t wst = (uint64_t)HC * W / 8;     // 16-byte chunks per window
    // this thread's first chunk in Hanford window 0 and in Livingston window 0 (the second chunk of
    // the pair is W chunks further)
    const uint4 *Hp = reinterpret_cast<const uint4 *>(proj) + (uint64_t)(2 * q) * W + tb + ts;
    const uint4 *Lp = Hp + (uint64_t)nw * wst;
    // offset of this lane's values after the halving: level l keeps the upper half on bit l of qlo
    int voff = 0;
#pragma unroll
    for (int l = 0; (1 << l) < G::QL; ++l) voff += ((qlo >> l) & 1) * (V >> (l + 1));
    const int64_t wrun = (int64_t)blockIdx.x * A * dw;
    const int64_t wend = min(nw, wrun + (int64_t)A * dw);
    for (int64_t wa = wrun, rho = 0; rho < dw; wa = wrun + ++rho) {
      while (wa < wend) {
        // windows wa + a dw, a < na, all in wa's segment
        int64_t sw0 = 0, snw = nw;
        if (n_seg > 1) {
            const int g = find_segment(seg_w0, n_seg, wa);
            sw0 = seg_w0[g];
            snw = seg_w0[g + 1] - sw0;
        }
        const int na = (int)((min(wend, sw0 + snw) - wa + dw - 1) / dw);
        uint4 h[A][2];
#pragma unroll
        for (int a = 0; a < A; ++a) {
            if (a < na) {
                const uint4 *hp = Hp + (uint64_t)(wa + (int64_t)a * dw) * wst;
                h[a][0] = __ldg(hp);
                h[a][1] = __ldg(hp + W);
            } else {
                h[a][0] = h[a][1] = make_uint4(0u, 0u, 0u, 0u);
            }
        }
        const uint4 *Ls = Lp + (uint64_t)sw0 * wst;    // Livingston window 0 of the segment
        const int sn = (int)snw;
        for (int pc = pc0; pc < pc1; ++pc) {
            const int2 pe = pieces[pc];
            const int nb = pe.y;
            const int ns = na + nb - 1;
            // Livingston row of step s: (r0 + s dw) mod n_w; the loads run through s = 0, 1, ... in
            // order, so the row advances by dw per load (no division in the loop)
            const int64_t t0 = (wa - sw0) + (int64_t)koff[pe.x];
            int rl;
            if (t0 >= 0 && t0 < snw) {
                rl = (int)t0;
            } else if (t0 >= snw && t0 < 2 * snw) {
                rl = (int)(t0 - snw);
            } else {
                const int64_t m = t0 % snw;
                rl = (int)(m < 0 ? m + snw : m);
            }
            auto next_row = [&]() -> const uint4 * {
                const uint4 *lp = Ls + (uint64_t)rl * wst;
                rl += dw;
                while (rl >= sn) rl -= sn;
                return lp;
            };
            uint4 lr[PF][2];
#pragma unroll
            for (int s = 0; s < PF; ++s) {
                if (s < ns) {
                    const uint4 *lp = next_row();
                    lr[s][0] = __ldg(lp);
                    lr[s][1] = __ldg(lp + W);
                }
            }
            float v[V];
#pragma unroll
            for (int i = 0; i < V; ++i) v[i] = 0.f;
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                if (s < ns) {
                    const uint4 l0 = lr[s % PF][0], l1 = lr[s % PF][1];
                    if (s + PF < ns) {
                        const uint4 *lp = next_row();
                        lr[s % PF][0] = __ldg(lp);
                        lr[s % PF][1] = __ldg(lp + W);
                    }
#pragma unroll
                    for (int a = 0; a < A; ++a) {
                        const int b = s - a;
                        if (b >= 0 && b < B) {
                            if (a < na && b < nb) v[a * B + b] = slide_pair(h[a], l0, l1, wv);
                        }
                    }
                }
            }
            // recursive halving over the warp's pairs: level l adds the pair groups that differ in
            // bit l of qlo (pair-sum order of the balanced tree); each lane keeps half the values
#pragma unroll
            for (int l = 0; (1 << l) < G::QL; ++l) {
                const int n = V >> l, hh = n >> 1;
                const bool up = (qlo >> l) & 1;
#pragma unroll
                for (int j = 0; j < hh; ++j) {
                    const float send = up ? v[j] : v[j + hh];
                    const float keep = up ? v[j + hh] : v[j];
                    v[j] = keep + __shfl_xor_sync(0xffffffffu, send, G::SPB << l);
                }
            }
            auto emit = [&](int vi, int tt, float sum) {
                const int a = vi / B, b = vi % B;
                if (a < na && b < nb) {
                    const float lg = sum + b2;
                    out[(uint64_t)(pe.x + b) * slide_stride + (uint64_t)(wa + (int64_t)a * dw) * W + tb + tt] =
                        logits ? lg : 1.f / (1.f + expf(-lg));
                }
            };
            if constexpr (G::QH == 1) {
#pragma unroll
                for (int j = 0; j < VL; ++j) emit(voff + j, ts, v[j]);
            } else {
                // then across the warps: one thread per (value, sample) adds the QH partial sums
#pragma unroll
                for (int j = 0; j < VL; ++j) part[(qh * V + voff + j) * G::SPB + ts] = v[j];
                __syncthreads();
                for (int i = threadIdx.x; i < V * G::SPB; i += G::THREADS) {
                    float x[G::QH];
#pragma unroll
                    for (int k = 0; k < G::QH; ++k) x[k] = part[k * V * G::SPB + i];
                    emit(i / G::SPB, i % G::SPB, tree_sum<G::QH>(x));
                }
                __syncthreads();
            }
        }
        wa += (int64_t)na * dw;
      }
    }
}

}  // namespace
}  // namespace gwe

// ============================================================================ host side
namespace gwe {
namespace {

// Test hooks (gwe_debug_config): limit of every device-side wait, and a dropped producer.
uint64_t g_wait_ns = kWaitNs;
int g_dbg_drop = 0;
uint64_t g_dbg_ring_margin = 0;   // test hook: the address checks see a ring this many bytes smaller
std::atomic<int> g_reuse{1};   // cross-window reuse on (gwe_set_cross_window_reuse)

// Cross-window reuse plan (fields of TcParams): for stride a multiple of the tile with
// W/2 <= stride < W, window w+1's tile t is window w's tile t + stride/128; layer l's output there
// is free of the window-start padding once 128 t >= r_l - 1, r_l = 1 + sum_{l' <= l} (k - 1) d_l'.
// The last layer is always computed (lstar <= L - 2).  stride < W/2 would make a tile both take
// and give, which the carry buffer does not support: no reuse then.
void plan_reuse(const Dims &d, int W, int stride, bool enable, TcParams &p) {
    p.reuse_shift = 0;
    p.carry = nullptr;
    p.carry_cta_floats = 0;
    std::memset(p.lstar, -1, sizeof(p.lstar));
    const int NT = W / kTile;
    if (!enable || stride % kTile != 0 || stride >= W || 2 * stride < W || NT > 64 || d.L < 2) return;
    const int shift = stride / kTile;
    std::vector<int64_t> rl(d.L);
    int64_t rf = 1;
    for (int l = 0; l < d.L; ++l) {
        rf += (int64_t)(d.k - 1) << (l % d.lps);
        rl[l] = rf;
    }
    bool any = false;
    for (int t = 0; t < NT - shift; ++t) {
        int ls = -1;
        for (int l = 0; l < d.L - 1 && l < 127; ++l) {
            if (rl[l] - 1 <= (int64_t)kTile * t)
                ls = l;
            else
                break;
        }
        p.lstar[t] = (int8_t)ls;
        any = any || ls >= 0;
    }
    if (any) p.reuse_shift = shift;
}

// Device buffers of one forward geometry besides the handle's weights: the lag rings and the carry
// buffer of the persistent kernel, the slide projections and the segment / offset tables.  The
// handle keeps one set for its own calls; a plan owns another, so that later calls on the handle
// can neither move nor overwrite what its captured graph points at.
struct TcWork {
    DevBuf ring, carry, proj, koff, segtab;
    void release() {
        ring.release();
        carry.release();
        proj.release();
        koff.release();
        segtab.release();
    }
};

// Launch shape of the slide heads: Hanford windows per block (A), consecutive offsets per piece
// (B: 4 or 8) and pieces per block (0: all pieces in one block).
struct SlideShape {
    int a = 4;
    int b = 8;
    int ppb = 0;
};

struct TcState {
    int variant = -1;            // 0: (R, S, Hc) = (32, 32, 32); 1: (64, 128, 256)
    bool f8 = false;             // FP8 E4M3 dilated convolutions (else 16-bit: FP16 / BF16)
    int n16 = 0;                 // 16-bit path: layers l < n16 take FP16 conv operands, the rest BF16
    std::vector<float> amax;     // FP8: calibrated max |x_l| per [model][branch][layer][channel]
    DevBuf img, pblob, zeros, err, slides;
    TcWork work;                 // buffers of the handle's own forward calls
    uint64_t img_stride = 0, pblob_stride = 0;
    int sms = 0;
};

int tc_variant(const Dims &d) {
    if (d.k != 2) return -1;
    if (d.R == 32 && d.S == 32 && d.Hc == 32) return 0;
    if (d.R == 64 && d.S == 128 && d.Hc == 256) return 1;
    return -1;
}

inline uint16_t to_bf16(float f) {
    __nv_bfloat16 h = __float2bfloat16_rn(f);
    uint16_t u;
    std::memcpy(&u, &h, 2);
    return u;
}
inline uint16_t to_f16(float f) {
    __half h = __float2half_rn(f);
    uint16_t u;
    std::memcpy(&u, &h, 2);
    return u;
}

// element (n, k) of a K-major operand with `rows` rows in the chunk-column layout
inline size_t chunk_off(int rows, int n, int k) { return (size_t)(k / 8) * rows * 16 + (size_t)n * 16 + (k % 8) * 2; }
inline size_t chunk_off8(int rows, int n, int k) { return (size_t)(k / 16) * rows * 16 + (size_t)n * 16 + (k % 16); }
inline void put16(std::vector<uint8_t> &v, size_t off, uint16_t x) { std::memcpy(v.data() + off, &x, 2); }

// FP8 scaling.  Activations: x_l[i] ~ s_l[i] * q with q E4M3 and s_l[i] = kF8Margin * amax_l[i] / 448,
// so that the calibrated maximum lands at 448 / kF8Margin and values up to kF8Margin times it stay
// in range (larger ones saturate).  Weights: the activation scales are folded into the input
// columns, then every output row o is scaled by its own w_o = max_k |W'[o][k]| / 448.
constexpr float kF8Margin = 16.f;
constexpr float kE4M3Max = 448.f;

inline float f8_act_scale(float amax) { return amax > 0.f ? kF8Margin * amax / kE4M3Max : 1.f; }
inline uint8_t to_e4m3(float f) { return (uint8_t)__nv_cvt_float_to_fp8(f, __NV_SATFINITE, __NV_E4M3); }

// n16 (16-bit path): layers l < n16 store their conv weights in FP16, the others in BF16
template <int R, int S, int HC, bool F8>
void build_images(const Dims &d, const float *hb, const float *amax, int n16, std::vector<uint8_t> &img,
                  std::vector<uint8_t> &pbl, uint64_t &img_stride, uint64_t &pb_stride) {
    using Sh = TcShape<R, S, HC, F8>;
    // amax (FP8 only): [model][branch][layer][channel]
    auto act_s = [&](int mi, int b, int l, int i) -> float {
        return f8_act_scale(amax[(((int64_t)mi * 2 + b) * d.L + l) * R + i]);
    };
    const int L = d.L;
    img_stride = (Sh::img_bytes(L) + 255) & ~uint64_t(255);
    pb_stride = ((uint64_t)Sh::pm_bytes(L) + 255) & ~uint64_t(255);
    img.assign(img_stride * d.n_models, 0);
    pbl.assign(pb_stride * d.n_models, 0);
    for (int mi = 0; mi < d.n_models; ++mi) {
        const float *src = hb + (int64_t)mi * d.P;
        uint8_t *im0 = img.data() + img_stride * mi;
        std::vector<uint8_t> tmp;
        std::vector<float> wscale(F8 ? (size_t)2 * L * 2 * R : 0);   // FP8: w_o per [branch][layer][o]
        for (int l = 0; l < L; ++l) {
            for (int b = 0; b < 2; ++b) {
                // conv item: rows n = output channel (g half pre-halved), k < R lag tap, k >= R current tap
                tmp.assign(Sh::CONV_BYTES, 0);
                const float *wc = src + off_wconv(d, b, l);
                if constexpr (F8) {
                    // E4M3 W'[o][k] / w_o with W' = W * s_l (per input channel); w_o goes to the conv slot
                    for (int o = 0; o < 2 * R; ++o) {
                        float mx = 0.f;
                        for (int k = 0; k < 2 * R; ++k)
                            mx = std::max(mx, std::fabs(wc[((int64_t)o * 2 + (k / R)) * R + k % R] * act_s(mi, b, l, k % R)));
                        const float wo = mx > 0.f ? mx / kE4M3Max : 1.f;
                        for (int k = 0; k < 2 * R; ++k) {
                            const float v = wc[((int64_t)o * 2 + (k / R)) * R + k % R] * act_s(mi, b, l, k % R);
                            tmp[chunk_off8(2 * R, o, k)] = to_e4m3(v / wo);
                        }
                        wscale[((int64_t)b * L + l) * 2 * R + o] = wo;
                    }
                } else {
                    const bool f16 = l < n16;
                    for (int o = 0; o < 2 * R; ++o)
                        for (int k = 0; k < 2 * R; ++k) {
                            const int tap = k < R ? 0 : 1, i = k % R;
                            float v = wc[((int64_t)o * 2 + tap) * R + i];
                            if (o >= R) v *= 0.5f;
                            put16(tmp, chunk_off(2 * R, o, k), f16 ? to_f16(v) : to_bf16(v));
                        }
                }
                std::memcpy(im0 + (uint64_t)l * Sh::LAYER_IMG + (uint64_t)b * Sh::CONV_BYTES, tmp.data(), tmp.size());
                // rs item: W_res [R x R] then W_skip [S x R], FP16
                tmp.assign(Sh::RS_BYTES, 0);
                const float *wr = src + off_wres(d, b, l), *ws = src + off_wskip(d, b, l);
                for (int o = 0; o < R; ++o)
                    for (int k = 0; k < R; ++k) put16(tmp, chunk_off(R, o, k), to_f16(wr[(int64_t)o * R + k]));
                for (int o = 0; o < S; ++o)
                    for (int k = 0; k < R; ++k)
                        put16(tmp, Sh::RES_BYTES + chunk_off(S, o, k), to_f16(ws[(int64_t)o * R + k]));
                std::memcpy(im0 + (uint64_t)l * Sh::LAYER_IMG + 2ull * Sh::CONV_BYTES + (uint64_t)b * Sh::RS_BYTES,
                            tmp.data(), tmp.size());
            }
        }
        // head pieces pc = (nh, kq): rows = u channels nh*HP + n; K = h channels kq*HQ .. of [h_H ; h_L]
        const float *w1 = src + off_wh1(d);
        for (int pc = 0; pc < Sh::NHP; ++pc) {
            const int nh = pc >> 2, kq = pc & 3;
            tmp.assign(Sh::HEADP_BYTES, 0);
            for (int n = 0; n < Sh::HP; ++n)
                for (int k = 0; k < Sh::HQ; ++k)
                    put16(tmp, chunk_off(Sh::HP, n, k),
                          to_f16(w1[(int64_t)(nh * Sh::HP + n) * 2 * S + kq * Sh::HQ + k]));
            std::memcpy(im0 + (uint64_t)L * Sh::LAYER_IMG + (uint64_t)pc * Sh::HEADP_BYTES, tmp.data(), tmp.size());
        }
        // parameter block
        uint8_t *pm = pbl.data() + pb_stride * mi;
        for (int b = 0; b < 2; ++b) {
            uint8_t *pb = pm + (uint64_t)b * Sh::pb_bytes(L);
            float *w_in = reinterpret_cast<float *>(pb), *b_in = w_in + R, *bsk = b_in + R;
            const float *bb = src + off_branch(d, b);
            for (int c = 0; c < R; ++c) {
                w_in[c] = bb[c];
                b_in[c] = bb[R + c];
            }
            for (int c = 0; c < S; ++c) {
                double acc = 0.0;
                for (int l = 0; l < L; ++l) acc += src[off_bskip(d, b, l) + c];
                bsk[c] = (float)acc;
            }
            if constexpr (F8) {   // quantisation factors 1 / s_0 of the input projection's output
                float *inv0 = bsk + S;
                for (int c = 0; c < R; ++c) inv0[c] = 1.f / act_s(mi, b, 0, c);
            }
            for (int l = 0; l < L; ++l) {
                uint8_t *pl = pb + Sh::HDR_BYTES + (uint64_t)l * Sh::PL_BYTES;
                const float *bc = src + off_bconv(d, b, l);
                if constexpr (F8) {
                    // {scale, bias} per output channel, g half pre-halved
                    float *sb = reinterpret_cast<float *>(pl);
                    for (int o = 0; o < 2 * R; ++o) {
                        const float hlf = o < R ? 1.f : 0.5f;
                        sb[2 * o] = hlf * wscale[((int64_t)b * L + l) * 2 * R + o];
                        sb[2 * o + 1] = hlf * bc[o];
                    }
                } else {
                    // FP32 b_conv, g half pre-halved
                    float *bcs = reinterpret_cast<float *>(pl);
                    for (int o = 0; o < 2 * R; ++o) bcs[o] = o < R ? bc[o] : 0.5f * bc[o];
                }
                float *br = reinterpret_cast<float *>(pl + Sh::CB_BYTES);
                for (int c = 0; c < R; ++c) br[c] = src[off_bres(d, b, l) + c];
                if constexpr (F8) {   // quantisation factors of the next layer's input
                    for (int c = 0; c < R; ++c) br[R + c] = l + 1 < L ? 1.f / act_s(mi, b, l + 1, c) : 1.f;
                }
            }
        }
        float *ph = reinterpret_cast<float *>(pm + 2ull * Sh::pb_bytes(L));
        for (int j = 0; j < HC; ++j) {
            ph[j] = src[off_bh1(d) + j];
            ph[HC + j] = src[off_wh2(d) + j];
        }
        ph[2 * HC] = src[off_bh2(d)];
    }
}

// The images of the 16-bit path built on the device from the FP32 blobs (one thread per blob
// element scatters it; the skip-bias sums by k_pack_bsk); the same bytes as build_images<.., false>.
__device__ __forceinline__ size_t chunk_off_d(int rows, int n, int k) {
    return (size_t)(k / 8) * rows * 16 + (size_t)n * 16 + (k % 8) * 2;
}

template <int R, int S, int HC>
__global__ void k_pack_tc16(const float *__restrict__ blob, int64_t P, int n_models, int L, int n16, int64_t Pb,
                            int64_t Pl, uint8_t *__restrict__ img, uint64_t img_stride, uint8_t *__restrict__ pbl,
                            uint64_t pb_stride) {
    using Sh = TcShape<R, S, HC, false>;
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= P * n_models) return;
    const int mi = (int)(gid / P);
    const int64_t e = gid % P;
    const float v = blob[gid];
    uint8_t *im = img + img_stride * mi;
    uint8_t *pm = pbl + pb_stride * mi;
    auto put_b16 = [&](size_t off, float x) {
        const __nv_bfloat16 h = __float2bfloat16_rn(x);
        *reinterpret_cast<__nv_bfloat16 *>(im + off) = h;
    };
    auto put_f16 = [&](size_t off, float x) { *reinterpret_cast<__half *>(im + off) = __float2half_rn(x); };
    if (e < 2 * Pb) {
        const int b = (int)(e / Pb);
        int64_t r = e % Pb;
        float *pf = reinterpret_cast<float *>(pm + (uint64_t)b * Sh::pb_bytes(L));
        if (r < 2 * R) {                       // w_in, b_in
            pf[r] = v;
            return;
        }
        r -= 2 * R;
        const int l = (int)(r / Pl);
        int64_t q = r % Pl;
        float *pl = reinterpret_cast<float *>(reinterpret_cast<uint8_t *>(pf) + Sh::HDR_BYTES + (uint64_t)l * Sh::PL_BYTES);
        const uint64_t lay = (uint64_t)l * Sh::LAYER_IMG;
        if (q < 4LL * R * R) {                 // conv (o, tap, i) -> row o, K = tap * R + i; g half halved
            const int o = (int)(q / (2 * R)), k = (int)(q % (2 * R));
            const float x = o < R ? v : 0.5f * v;
            const size_t off = lay + (uint64_t)b * Sh::CONV_BYTES + chunk_off_d(2 * R, o, k);
            if (l < n16) put_f16(off, x); else put_b16(off, x);
            return;
        }
        if ((q -= 4LL * R * R) < 2 * R) {      // b_conv (FP32, g half halved)
            pl[q] = q < R ? v : 0.5f * v;
            return;
        }
        if ((q -= 2 * R) < (int64_t)R * R) {   // w_res (o, k)
            put_f16(lay + 2ull * Sh::CONV_BYTES + (uint64_t)b * Sh::RS_BYTES + chunk_off_d(R, (int)(q / R), (int)(q % R)), v);
            return;
        }
        if ((q -= (int64_t)R * R) < R) {       // b_res
            reinterpret_cast<float *>(reinterpret_cast<uint8_t *>(pl) + Sh::CB_BYTES)[q] = v;
            return;
        }
        if ((q -= R) < (int64_t)S * R) {       // w_skip (o, k)
            put_f16(lay + 2ull * Sh::CONV_BYTES + (uint64_t)b * Sh::RS_BYTES + Sh::RES_BYTES +
                        chunk_off_d(S, (int)(q / R), (int)(q % R)),
                    v);
            return;
        }
        return;                                // b_skip: summed by k_pack_bsk
    }
    int64_t h = e - 2 * Pb;
    if (h < (int64_t)HC * 2 * S) {             // w_h1 (j, c) -> piece (j / HP, c / HQ), row j % HP, K c % HQ
        const int j = (int)(h / (2 * S)), c = (int)(h % (2 * S));
        const int pc = (j / Sh::HP) * 4 + c / Sh::HQ;
        put_f16((uint64_t)L * Sh::LAYER_IMG + (uint64_t)pc * Sh::HEADP_BYTES + chunk_off_d(Sh::HP, j % Sh::HP, c % Sh::HQ), v);
        return;
    }
    h -= (int64_t)HC * 2 * S;
    reinterpret_cast<float *>(pm + 2ull * Sh::pb_bytes(L))[h] = v;   // b_h1 [HC], w_h2 [HC], b_h2
}

// summed skip biases per (model, branch, channel), FP64 in layer order as the host builder
template <int R, int S, int HC>
__global__ void k_pack_bsk(const float *__restrict__ blob, int64_t P, int n_models, int L, int64_t Pb, int64_t Pl,
                           uint8_t *__restrict__ pbl, uint64_t pb_stride) {
    using Sh = TcShape<R, S, HC, false>;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_models * 2 * S) return;
    const int mi = i / (2 * S), b = (i / S) % 2, c = i % S;
    const float *src = blob + (int64_t)mi * P + (int64_t)b * Pb + 2 * R;
    const int64_t boff = (int64_t)2 * R * 2 * R + 2 * R + (int64_t)R * R + R + (int64_t)S * R;   // b_skip in a layer
    double acc = 0.0;
    for (int l = 0; l < L; ++l) acc += (double)src[(int64_t)l * Pl + boff + c];
    reinterpret_cast<float *>(pbl + pb_stride * mi + (uint64_t)b * Sh::pb_bytes(L))[2 * R + c] = (float)acc;
}

template <int R, int S, int HC, bool F8>
cudaError_t set_tc_attr() {
    cudaError_t e = cudaFuncSetAttribute(k_branch_tc<R, S, HC, F8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)TcShape<R, S, HC, F8>::SMEM);
    if (e != cudaSuccess) return e;
    if (!F8) {
        e = cudaFuncSetAttribute(k_branch_tc<R, S, HC, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)TcShape<R, S, HC, false>::SMEM);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Everything one forward needs on the device, prepared by setup_tc (buffers grown, tables
// uploaded) and launched by issue_tc, which only enqueues kernels (so that it can be captured
// into a CUDA graph).
struct TcLaunch {
    TcParams p;
    int grid_max = 0;            // CTAs of the zero-lag launch (all models)
    int grid_slide = 0;          // CTAs of the per-model projection launches
    int64_t nw = 0;
    int n_slides = 0;
    const int32_t *dsl = nullptr;
    const int2 *dpieces[2] = {nullptr, nullptr};   // offset pieces of at most 4 / 8 offsets in step dwin
    int n_pieces[2] = {0, 0};
    int dwin = 1;
    const int64_t *d_w0 = nullptr;
    float *out = nullptr;
    bool logits = false;
    uint16_t *proj = nullptr;
    SlideShape shape;
};

// the slide-head shape of launches that are not autotuned (gwe_forward, gwe_forward_segments and
// plans created without GWE_PLAN_AUTOTUNE)
std::mutex g_plan_shape_mu;
SlideShape g_plan_shape;

// Window step of the slide heads' register blocking: the most common positive difference of
// consecutive offsets (the smaller one on a tie), 1 when there is none or it is not below the
// window count.
int slide_step(const int32_t *k, int n, int64_t nw) {
    std::map<int64_t, int> cnt;
    for (int i = 1; i < n; ++i) {
        const int64_t d = (int64_t)k[i] - k[i - 1];
        if (d > 0 && d < nw && d <= (1 << 20)) ++cnt[d];
    }
    int64_t best = 1;
    int nb = 0;
    for (const auto &kv : cnt)
        if (kv.second > nb) best = kv.first, nb = kv.second;
    return (int)best;
}

template <int R, int S, int HC, bool F8>
gwe_status setup_tc(gwe_model *m, TcState &s, TcWork &wk, const float *sH, const float *sL, const Segments &sg,
                    int W, int stride, const int32_t *slides_host, int n_slides, float *out, bool logits,
                    cudaStream_t st, TcLaunch &L) {
    using Sh = TcShape<R, S, HC, F8>;
    const Dims &d = m->dims;
    const int64_t nw = sg.total_windows();
    L.nw = nw;
    if (nw <= 0) return GWE_OK;
    uint64_t ring_rows = 0;
    for (int l = 0; l < d.L; ++l) ring_rows += (uint64_t)1 << (l % d.lps);
    const uint64_t ring_cta = (2 * ring_rows * Sh::XROW + 255) & ~uint64_t(255);
    const int64_t max_jobs = (int64_t)d.n_models * nw;
    const int grid_max = (int)std::min<int64_t>(s.sms, max_jobs);
    TcParams &p = L.p;
    plan_reuse(d, W, stride, g_reuse.load() != 0, p);
    const uint64_t n_rings = p.reuse_shift > 0 ? 2 : 1;
    GWE_CUDA_TRY(wk.ring.ensure(n_rings * ring_cta * grid_max));
    // small host tables go up with cudaMemcpyAsync from pageable memory, which stages them before
    // returning; the slide offsets stay raw (they wrap within each window's segment on the device)
    // The slide heads take the offsets in pieces of values in arithmetic progression with the list's
    // most common positive step dwin (k, k + dwin, ...), at most 4 or 8 long: table [offsets, padded
    // to 8 bytes][pieces of <= 4][pieces of <= 8], (first index, count).
    const int32_t *dsl = nullptr;
    if (n_slides > 0) {
        L.dwin = slide_step(slides_host, n_slides, nw);
        const int64_t dwin = L.dwin;
        std::vector<int32_t> tab((size_t)n_slides + (n_slides & 1));
        std::copy(slides_host, slides_host + n_slides, tab.begin());
        const size_t pc_at = tab.size();
        for (int bi = 0; bi < 2; ++bi) {
            const int bmax = bi == 0 ? 4 : 8;
            int np = 0;
            for (int i = 0; i < n_slides;) {
                int j = i + 1;
                while (j < n_slides && j - i < bmax && (int64_t)slides_host[j] == (int64_t)slides_host[j - 1] + dwin) ++j;
                tab.push_back(i);
                tab.push_back(j - i);
                ++np;
                i = j;
            }
            L.n_pieces[bi] = np;
        }
        GWE_CUDA_TRY(wk.koff.ensure(sizeof(int32_t) * tab.size()));
        GWE_CUDA_TRY(cudaMemcpyAsync(wk.koff.ptr, tab.data(), sizeof(int32_t) * tab.size(), cudaMemcpyHostToDevice, st));
        dsl = wk.koff.as<int32_t>();
        L.dpieces[0] = reinterpret_cast<const int2 *>(dsl + pc_at);
        L.dpieces[1] = L.dpieces[0] + L.n_pieces[0];
    }
    const int n_seg = (int)sg.s0.size();
    const int64_t *d_w0 = nullptr, *d_s0 = nullptr;
    if (n_seg > 1) {
        std::vector<int64_t> tab(2 * (size_t)n_seg + 1);
        tab[0] = 0;
        for (int g = 0; g < n_seg; ++g) {
            tab[g + 1] = tab[g] + sg.nw[g];
            tab[n_seg + 1 + g] = sg.s0[g];
        }
        GWE_CUDA_TRY(wk.segtab.ensure(sizeof(int64_t) * tab.size()));
        GWE_CUDA_TRY(cudaMemcpyAsync(wk.segtab.ptr, tab.data(), sizeof(int64_t) * tab.size(), cudaMemcpyHostToDevice, st));
        d_w0 = wk.segtab.as<int64_t>();
        d_s0 = d_w0 + n_seg + 1;
    }
    p.wimg = s.img.as<uint8_t>();
    p.wimg_stride = s.img_stride;
    p.pblob = s.pblob.as<uint8_t>();
    p.pblob_stride = s.pblob_stride;
    p.nw = nw;
    p.W = W;
    p.stride = stride;
    p.n_seg = n_seg > 1 ? n_seg : 1;
    p.seg_w0 = d_w0;
    p.seg_s0 = d_s0;
    if (n_seg == 1) sH += sg.s0[0], sL += sg.s0[0];
    p.sH = sH;
    p.sL = sL;
    p.n_models = d.n_models;
    p.out = out;
    p.logits = logits ? 1 : 0;
    p.ring = wk.ring.as<uint8_t>();
    p.ring_alloc = n_rings * ring_cta * grid_max;
    p.ring_alloc = p.ring_alloc > g_dbg_ring_margin ? p.ring_alloc - g_dbg_ring_margin : 0;
    p.proj_alloc = 0;
    p.ring_cta_bytes = n_rings * ring_cta;
    p.ring_pp = n_rings > 1 ? ring_cta : 0;
    p.zeros = s.zeros.as<uint8_t>();
    p.L = d.L;
    p.lps = d.lps;
    p.ring_rows = ring_rows;
    p.err = s.err.as<int>();
    p.n16 = s.f8 ? 0 : s.n16;
    p.model0 = 0;
    p.proj = nullptr;
    p.save_x = nullptr;
    p.save_skip = nullptr;
    p.wait_ns = g_wait_ns;
    p.dbg_drop = g_dbg_drop;
    if (p.reuse_shift > 0) {
        const int ntr = W / kTile - p.reuse_shift;
        p.carry_cta_floats = (uint64_t)2 * ntr * (R / 2 + S / 2) * 256;
        GWE_CUDA_TRY(wk.carry.ensure(sizeof(float) * p.carry_cta_floats * grid_max));
        p.carry = wk.carry.as<float>();
    }
    L.grid_max = grid_max;
    L.grid_slide = (int)std::min<int64_t>(s.sms, nw);
    L.n_slides = n_slides;
    {
        std::lock_guard<std::mutex> lk(g_plan_shape_mu);
        L.shape = g_plan_shape;
    }
    L.dsl = dsl;
    L.d_w0 = d_w0;
    L.out = out;
    L.logits = logits;
    if (n_slides > 0) {
        // Time slides: per model, one branch pass storing the projections, then the slide heads.
        const uint64_t proj_elems = 2ull * (uint64_t)nw * HC * W;
        GWE_CUDA_TRY(wk.proj.ensure(proj_elems * sizeof(uint16_t)));
        L.proj = wk.proj.as<uint16_t>();
        p.proj_alloc = proj_elems;
    }
    return GWE_OK;
}

template <int HC, int A, int B>
void launch_slide_head(const TcLaunch &L, const float *w2, const float *b2, float *out, cudaStream_t st) {
    using G = SlideGeo<HC>;
    const int bi = B == 4 ? 0 : 1;
    const int np = L.n_pieces[bi];
    const int ppb = L.shape.ppb > 0 ? std::min(L.shape.ppb, np) : np;
    const int64_t run = (int64_t)A * L.dwin;
    dim3 g2((unsigned)((L.nw + run - 1) / run), (unsigned)(L.p.W / G::SPB), (unsigned)((np + ppb - 1) / ppb));
    k_slide_head<HC, A, B><<<g2, G::THREADS, 0, st>>>(L.proj, L.nw, L.p.W, L.dsl, L.dpieces[bi], np, ppb, L.dwin,
                                                       L.p.n_seg,
                                                       L.d_w0, w2, b2, out, (int64_t)L.p.n_models * L.nw * L.p.W,
                                                       L.logits ? 1 : 0);
}

// the slide heads of model mi (projections already in L.proj)
template <int HC>
gwe_status issue_slide_heads(gwe_model *m, TcState &s, const TcLaunch &L, int mi, cudaStream_t st) {
    const Dims &d = m->dims;
    // w_h2 and b_h2 are read from the handle's FP32 blob on the device, so that a recorded graph
    // picks up later weight changes
    const float *w2 = m->w32.as<float>() + (int64_t)mi * d.P + off_wh2(d);
    const float *b2 = m->w32.as<float>() + (int64_t)mi * d.P + off_bh2(d);
    float *out = L.out + (int64_t)mi * L.nw * L.p.W;
    ProfScope prof("k_slide_head", st);
    if (L.shape.b == 8) {
        if (L.shape.a == 2) launch_slide_head<HC, 2, 8>(L, w2, b2, out, st);
        else launch_slide_head<HC, 4, 8>(L, w2, b2, out, st);
    } else {
        if (L.shape.a == 2) launch_slide_head<HC, 2, 4>(L, w2, b2, out, st);
        else launch_slide_head<HC, 4, 4>(L, w2, b2, out, st);
    }
    note_launch();
    GWE_CUDA_TRY(cudaGetLastError());
    return GWE_OK;
}

template <int R, int S, int HC, bool F8>
gwe_status issue_tc(gwe_model *m, TcState &s, const TcLaunch &L, cudaStream_t st) {
    using Sh = TcShape<R, S, HC, F8>;
    if (L.nw <= 0) return GWE_OK;
    if (L.n_slides == 0) {
        ProfScope prof("k_branch_tc", st);
        k_branch_tc<R, S, HC, F8><<<L.grid_max, kThreads, Sh::SMEM, st>>>(L.p);
        note_launch();
        GWE_CUDA_TRY(cudaGetLastError());
        return GWE_OK;
    }
    for (int mi = 0; mi < m->dims.n_models; ++mi) {
        TcParams q = L.p;
        q.model0 = mi;
        q.n_models = 1;
        q.proj = L.proj;
        {
            ProfScope prof("k_branch_tc", st);
            k_branch_tc<R, S, HC, F8><<<L.grid_slide, kThreads, Sh::SMEM, st>>>(q);
            note_launch();
        }
        GWE_CUDA_TRY(cudaGetLastError());
        gwe_status r = issue_slide_heads<HC>(m, s, L, mi, st);
        if (r != GWE_OK) return r;
    }
    return GWE_OK;
}

template <int R, int S, int HC, bool F8>
gwe_status launch_tc(gwe_model *m, TcState &s, const float *sH, const float *sL, const Segments &sg, int W,
                     int stride, const int32_t *slides_host, int n_slides, float *out, bool logits, cudaStream_t st) {
    TcLaunch L;
    gwe_status r = setup_tc<R, S, HC, F8>(m, s, s.work, sH, sL, sg, W, stride, slides_host, n_slides, out, logits, st, L);
    if (r != GWE_OK) return r;
    return issue_tc<R, S, HC, F8>(m, s, L, st);
}

// compile-time shape of one instantiation of the tensor-core kernel
template <int R_, int S_, int HC_, bool F8_>
struct TcTag {
    static constexpr int R = R_, S = S_, HC = HC_;
    static constexpr bool F8 = F8_;
};

// fn(TcTag<...>{}) for the handle's shape and operand type
template <class Fn>
auto tc_dispatch(const TcState &s, Fn &&fn) {
    if (s.variant == 0) return s.f8 ? fn(TcTag<32, 32, 32, true>{}) : fn(TcTag<32, 32, 32, false>{});
    return s.f8 ? fn(TcTag<64, 128, 256, true>{}) : fn(TcTag<64, 128, 256, false>{});
}

// Unit-variance white Gaussian noise for the default FP8 calibration: sample i of stream `seed`
// is Box-Muller on two 24-bit uniforms drawn from splitmix64(seed * 2^32 + i).
__global__ void k_calib_noise(float *__restrict__ out, int64_t n, uint64_t seed) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t z = (seed << 32) + (uint64_t)i + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    const float u1 = ((float)(z >> 40) + 1.f) * (1.f / 16777216.f);      // (0, 1]
    const float u2 = (float)((z >> 16) & 0xffffffu) * (1.f / 16777216.f); // [0, 1)
    out[i] = sqrtf(-2.f * logf(u1)) * cospif(2.f * u2);
}

constexpr int kCalibWindows = 64;

// releases a temporary device buffer on every return path
struct TmpBuf {
    DevBuf b;
    ~TmpBuf() { b.release(); }
};

// FP32 activation maxima over the windows of (sH, sL) into s.amax
gwe_status measure_amax(gwe_model *m, TcState &s, const float *sH, const float *sL, int W, int stride, int64_t nw,
                        cudaStream_t st) {
    const Dims &d = m->dims;
    const size_t na = (size_t)d.n_models * 2 * d.L * d.R;
    TmpBuf tb;
    DevBuf &buf = tb.b;
    GWE_CUDA_TRY(buf.ensure(na * sizeof(float) + 64));
    float *amax = buf.as<float>();
    unsigned *keys = reinterpret_cast<unsigned *>(buf.as<uint8_t>() + na * sizeof(float));
    gwe_status r = fp32_act_amax(m, sH, sL, W, stride, nw, amax, keys, st);
    if (r == GWE_OK) {
        s.amax.assign(na, 0.f);
        cudaError_t e = cudaMemcpyAsync(s.amax.data(), amax, na * sizeof(float), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            set_error(std::string("FP8 calibration: ") + cudaGetErrorString(e));
            r = GWE_ERR_CUDA;
        }
    }
    return r;
}

// weight images of the handle's shape and operand type from the host blob, uploaded
gwe_status build_upload(gwe_model *m, TcState &s, const float *hb) {
    const Dims &d = m->dims;
    std::vector<uint8_t> img, pbl;
    tc_dispatch(s, [&](auto t) {
        using T = decltype(t);
        build_images<T::R, T::S, T::HC, T::F8>(d, hb, s.amax.data(), s.n16, img, pbl, s.img_stride, s.pblob_stride);
        return 0;
    });
    GWE_CUDA_TRY(s.img.ensure(img.size()));
    GWE_CUDA_TRY(cudaMemcpy(s.img.ptr, img.data(), img.size(), cudaMemcpyHostToDevice));
    GWE_CUDA_TRY(s.pblob.ensure(pbl.size()));
    GWE_CUDA_TRY(cudaMemcpy(s.pblob.ptr, pbl.data(), pbl.size(), cudaMemcpyHostToDevice));
    return GWE_OK;
}

// the images of a 16-bit handle from its device FP32 blobs (m->w32), on `st`
gwe_status build_device(gwe_model *m, TcState &s, cudaStream_t st) {
    const Dims &d = m->dims;
    return tc_dispatch(s, [&](auto t) -> gwe_status {
        using T = decltype(t);
        using Sh = TcShape<T::R, T::S, T::HC, false>;
        if constexpr (T::F8) {
            set_error("device weight packing covers the 16-bit path only");
            return GWE_ERR_UNSUPPORTED;
        } else {
            s.img_stride = (Sh::img_bytes(d.L) + 255) & ~uint64_t(255);
            s.pblob_stride = ((uint64_t)Sh::pm_bytes(d.L) + 255) & ~uint64_t(255);
            GWE_CUDA_TRY(s.img.ensure(s.img_stride * d.n_models));
            GWE_CUDA_TRY(s.pblob.ensure(s.pblob_stride * d.n_models));
            GWE_CUDA_TRY(cudaMemsetAsync(s.img.ptr, 0, s.img_stride * d.n_models, st));
            GWE_CUDA_TRY(cudaMemsetAsync(s.pblob.ptr, 0, s.pblob_stride * d.n_models, st));
            const int64_t n = d.P * d.n_models;
            k_pack_tc16<T::R, T::S, T::HC><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
                m->w32.as<float>(), d.P, d.n_models, d.L, s.n16, d.Pb, d.Pl, s.img.as<uint8_t>(), s.img_stride,
                s.pblob.as<uint8_t>(), s.pblob_stride);
            const int nb = d.n_models * 2 * T::S;
            k_pack_bsk<T::R, T::S, T::HC><<<(unsigned)((nb + 127) / 128), 128, 0, st>>>(
                m->w32.as<float>(), d.P, d.n_models, d.L, d.Pb, d.Pl, s.pblob.as<uint8_t>(), s.pblob_stride);
            note_launch(2);
            GWE_CUDA_TRY(cudaGetLastError());
            return GWE_OK;
        }
    });
}

}  // namespace

bool tc_supported(const Dims &d) { return tc_variant(d) >= 0 && d.lps <= 10; }

gwe_status tc_rebuild_from_device(gwe_model *m, cudaStream_t st) {
    TcState *s = reinterpret_cast<TcState *>(m->tc);
    if (!s || s->variant < 0) {
        set_error("tensor-core path not prepared");
        return GWE_ERR_UNSUPPORTED;
    }
    if (!s->f8) return build_device(m, *s, st);
    // FP8: the E4M3 images need the per-row maxima of the scaled weights; built on the host
    const Dims &d = m->dims;
    GWE_CUDA_TRY(cudaStreamSynchronize(st));
    std::vector<float> hb((size_t)d.P * d.n_models);
    GWE_CUDA_TRY(cudaMemcpy(hb.data(), m->w32.ptr, hb.size() * sizeof(float), cudaMemcpyDeviceToHost));
    return build_upload(m, *s, hb.data());
}

gwe_status tc_prepare(gwe_model *m, const float *hb, bool f8) {
    const Dims &d = m->dims;
    if (!tc_supported(d)) {
        set_error("tensor-core path supports (R, S, Hc) = (32, 32, 32) or (64, 128, 256), kernel 2, "
                  "layers_per_stack <= 10");
        return GWE_ERR_UNSUPPORTED;
    }
    TcState *s = reinterpret_cast<TcState *>(m->tc);
    if (!s) {
        s = new TcState();
        m->tc = s;
    }
    if (s->variant < 0) s->n16 = f8 ? 0 : d.L / 3;   // default: the first third of the layers in FP16
    s->variant = tc_variant(d);
    s->f8 = f8;
    if (f8 && s->amax.size() != (size_t)d.n_models * 2 * d.L * d.R) {
        // default activation scales: FP32 pass over synthetic whitened (unit-variance white) noise
        const int W = 4096, stride = 2048;
        const int64_t n = (int64_t)(kCalibWindows - 1) * stride + W;
        TmpBuf tn;
        DevBuf &noise = tn.b;
        GWE_CUDA_TRY(noise.ensure(2 * n * sizeof(float)));
        k_calib_noise<<<(unsigned)((n + 255) / 256), 256>>>(noise.as<float>(), n, 1);
        k_calib_noise<<<(unsigned)((n + 255) / 256), 256>>>(noise.as<float>() + n, n, 2);
        note_launch();
        note_launch();
        GWE_CUDA_TRY(cudaGetLastError());
        gwe_status r = measure_amax(m, *s, noise.as<float>(), noise.as<float>() + n, W, stride, kCalibWindows, 0);
        if (r != GWE_OK) return r;
    }
    gwe_status r = build_upload(m, *s, hb);
    if (r != GWE_OK) return r;
    GWE_CUDA_TRY(s->zeros.ensure(4096));
    GWE_CUDA_TRY(cudaMemset(s->zeros.ptr, 0, 4096));
    GWE_CUDA_TRY(s->err.ensure(256));
    GWE_CUDA_TRY(cudaMemset(s->err.ptr, 0, 256));
    GWE_CUDA_TRY(cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, m->device));
    GWE_CUDA_TRY(tc_dispatch(*s, [](auto t) {
        using T = decltype(t);
        return set_tc_attr<T::R, T::S, T::HC, T::F8>();
    }));
    return GWE_OK;
}

gwe_status tc_calibrate(gwe_model *m, const float *sH, const float *sL, int64_t n, int W, int stride,
                        cudaStream_t st) {
    TcState *s = reinterpret_cast<TcState *>(m->tc);
    if (!s || s->variant < 0 || !s->f8) {
        set_error("FP8 path not prepared");
        return GWE_ERR_UNSUPPORTED;
    }
    const Dims &d = m->dims;
    const int64_t nw = (n - W) / stride + 1;
    gwe_status r = measure_amax(m, *s, sH, sL, W, stride, nw, st);
    if (r != GWE_OK) return r;
    std::vector<float> hb((size_t)d.P * d.n_models);
    GWE_CUDA_TRY(cudaMemcpy(hb.data(), m->w32.ptr, hb.size() * sizeof(float), cudaMemcpyDeviceToHost));
    return build_upload(m, *s, hb.data());
}

gwe_status tc_set_amax(gwe_model *m, const float *amax) {
    TcState *s = reinterpret_cast<TcState *>(m->tc);
    if (!s || s->variant < 0 || !s->f8) {
        set_error("FP8 path not prepared");
        return GWE_ERR_UNSUPPORTED;
    }
    const Dims &d = m->dims;
    s->amax.assign(amax, amax + (size_t)d.n_models * 2 * d.L * d.R);
    std::vector<float> hb((size_t)d.P * d.n_models);
    GWE_CUDA_TRY(cudaMemcpy(hb.data(), m->w32.ptr, hb.size() * sizeof(float), cudaMemcpyDeviceToHost));
    return build_upload(m, *s, hb.data());
}

gwe_status tc_set_f16_layers(gwe_model *m, int n16) {
    TcState *s = reinterpret_cast<TcState *>(m->tc);
    if (!s || s->variant < 0 || s->f8) {
        set_error("gwe_model_set_f16_layers: needs a GWE_BF16 handle");
        return GWE_ERR_UNSUPPORTED;
    }
    if (n16 < 0 || n16 > m->dims.L) {
        set_error("gwe_model_set_f16_layers: n must lie in [0, layers]");
        return GWE_ERR_ARG;
    }
    if (n16 == s->n16) return GWE_OK;
    GWE_CUDA_TRY(cudaDeviceSynchronize());   // no launch may still read the old images
    s->n16 = n16;
    const Dims &d = m->dims;
    std::vector<float> hb((size_t)d.P * d.n_models);
    GWE_CUDA_TRY(cudaMemcpy(hb.data(), m->w32.ptr, hb.size() * sizeof(float), cudaMemcpyDeviceToHost));
    return build_upload(m, *s, hb.data());
}

int tc_f16_layers(gwe_model *m) {
    const TcState *s = reinterpret_cast<const TcState *>(m->tc);
    return (s && s->variant >= 0 && !s->f8) ? s->n16 : 0;
}

gwe_status tc_get_amax(gwe_model *m, float *amax) {
    TcState *s = reinterpret_cast<TcState *>(m->tc);
    if (!s || s->variant < 0 || !s->f8) {
        set_error("FP8 path not prepared");
        return GWE_ERR_UNSUPPORTED;
    }
    std::copy(s->amax.begin(), s->amax.end(), amax);
    return GWE_OK;
}

void tc_release(gwe_model *m) {
    TcState *s = reinterpret_cast<TcState *>(m->tc);
    if (!s) return;
    s->img.release();
    s->pblob.release();
    s->zeros.release();
    s->err.release();
    s->slides.release();
    s->work.release();
    delete s;
    m->tc = nullptr;
}

gwe_status tc_forward(gwe_model *m, const float *sH, const float *sL, const Segments &sg, int W, int stride,
                      const int32_t *slides, int n_slides, float *out, bool logits, cudaStream_t st) {
    TcState *s = reinterpret_cast<TcState *>(m->tc);
    if (!s || s->variant < 0) {
        set_error("tensor-core path not prepared");
        return GWE_ERR_UNSUPPORTED;
    }
    if (W % kTile != 0) {
        set_error("tensor-core path needs window to be a multiple of 128");
        return GWE_ERR_UNSUPPORTED;
    }
    return tc_dispatch(*s, [&](auto t) {
        using T = decltype(t);
        return launch_tc<T::R, T::S, T::HC, T::F8>(m, *s, sH, sL, sg, W, stride, slides, n_slides, out, logits, st);
    });
}

bool tc_save_supported(gwe_model *m, int W) {
    const TcState *s = reinterpret_cast<const TcState *>(m->tc);
    return s && s->variant >= 0 && !s->f8 && W % kTile == 0 && W >= kTile;
}

gwe_status tc_forward_save(gwe_model *m, int mi, const float *xH, const float *xL, int nwin, int W, float *logits,
                           float *save_x, float *save_skip, cudaStream_t st) {
    TcState *s = reinterpret_cast<TcState *>(m->tc);
    if (!s || s->variant < 0 || s->f8 || W % kTile != 0 || nwin <= 0 || mi < 0 || mi >= m->dims.n_models) {
        set_error("training save forward: needs a BF16 tensor-core handle and a window that is a multiple of 128");
        return GWE_ERR_UNSUPPORTED;
    }
    Segments sg;
    sg.s0.push_back(0);
    sg.nw.push_back(nwin);
    return tc_dispatch(*s, [&](auto t) -> gwe_status {
        using T = decltype(t);
        using Sh = TcShape<T::R, T::S, T::HC, false>;
        TcLaunch L;
        // windows back to back (stride = W): no cross-window reuse, every layer of every tile runs
        gwe_status r = setup_tc<T::R, T::S, T::HC, false>(m, *s, s->work, xH, xL, sg, W, W, nullptr, 0, logits, true,
                                                          st, L);
        if (r != GWE_OK) return r;
        if (L.p.reuse_shift != 0) {
            set_error("training save forward: cross-window reuse must be off");
            return GWE_ERR_UNSUPPORTED;
        }
        L.p.model0 = mi;
        L.p.n_models = 1;
        L.p.save_x = save_x;
        L.p.save_skip = save_skip;
        const int grid = (int)std::min<int64_t>(s->sms, nwin);
        ProfScope prof("k_branch_tc", st);
        k_branch_tc<T::R, T::S, T::HC, false, true><<<grid, kThreads, Sh::SMEM, st>>>(L.p);
        note_launch();
        GWE_CUDA_TRY(cudaGetLastError());
        return GWE_OK;
    });
}

void set_cross_window_reuse(int enable) { g_reuse.store(enable ? 1 : 0); }

gwe_status debug_config(int drop, double wait_seconds) {
    if (drop < 0 || drop > 1 || !(wait_seconds > 0.0) || wait_seconds > 60.0) {
        set_error("gwe_debug_config: drop must be 0 or 1 and wait_seconds in (0, 60]");
        return GWE_ERR_ARG;
    }
    g_dbg_drop = drop;
    g_wait_ns = (uint64_t)(wait_seconds * 1e9);
    return GWE_OK;
}

gwe_status debug_ring_margin(int64_t bytes) {
    if (bytes < 0) {
        set_error("gwe_debug_ring_margin: bytes must be >= 0");
        return GWE_ERR_ARG;
    }
    g_dbg_ring_margin = (uint64_t)bytes;
    return GWE_OK;
}

gwe_status tc_check(gwe_model *m, cudaStream_t st) {
    TcState *s = reinterpret_cast<TcState *>(m->tc);
    if (!s) return GWE_OK;
    GWE_CUDA_TRY(cudaStreamSynchronize(st));
    int e = 0;
    GWE_CUDA_TRY(cudaMemcpy(&e, s->err.ptr, sizeof(int), cudaMemcpyDeviceToHost));
    if (e != 0) {
        cudaMemset(s->err.ptr, 0, sizeof(int));
        if (e >= 40) {
            set_error("an address check of the tensor-core kernel failed (site " + std::to_string(e) +
                      "); the access was not made and the outputs are invalid");
            return GWE_ERR_CUDA;
        }
        set_error("a device-side wait of the tensor-core kernel timed out (site " + std::to_string(e) + ")");
        return GWE_ERR_TIMEOUT;
    }
    return GWE_OK;
}

}  // namespace gwe

// ============================================================================ allocation-free forward
// A variant of the tensor-core forward for callers that must not allocate device memory while
// they stream: its lag-history ring, zero rows and error word live in one fixed file-scope device
// array instead of buffers the handle grows on demand.  The array is part of the library image,
// so every GPU that loads the library holds it until the process exits.
namespace gwe {
namespace {

constexpr size_t kStaticScratchBytes = 24u << 20;     // 24 MiB
constexpr size_t kStaticZeroOff = 0;                  // 4 KiB of zero rows
constexpr size_t kStaticRingOff = 4096;               // per-CTA lag rings
constexpr int kMaxDevices = 64;

static __device__ __align__(256) uint8_t g_static_scratch[kStaticScratchBytes];

// Device address of the array, looked up once per device and CUDA context: the array's name in
// host code is only a stand-in for it.  The lookup is keyed on the context's unique id
// (cuCtxGetId, reached through the runtime's driver entry point) as well as the device ordinal,
// because cudaDeviceReset destroys the primary context and the module, and the next context may
// place the array at another address.
typedef CUresult (*PfnCtxGetCurrent)(CUcontext *);
typedef CUresult (*PfnCtxGetId)(CUcontext, unsigned long long *);

struct StaticSlot {
    unsigned long long ctx_id = 0;
    uint8_t *ptr = nullptr;
};
std::mutex g_static_mu;
StaticSlot g_static_slot[kMaxDevices];
PfnCtxGetCurrent g_ctx_get_current = nullptr;
PfnCtxGetId g_ctx_get_id = nullptr;

gwe_status static_scratch(uint8_t **out) {
    int dev = 0;
    GWE_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("gwe_forward_static: device ordinal out of range");
        return GWE_ERR_UNSUPPORTED;
    }
    GWE_CUDA_TRY(cudaSetDevice(dev));   // makes the device's primary context current (allocates nothing)
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_ctx_get_current || !g_ctx_get_id) {
        void *f1 = nullptr, *f2 = nullptr;
        cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = q1;
        GWE_CUDA_TRY(cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1));
        GWE_CUDA_TRY(cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2));
        if (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2) {
            set_error("gwe_forward_static: cuCtxGetCurrent / cuCtxGetId not available from the driver");
            return GWE_ERR_CUDA;
        }
        g_ctx_get_current = reinterpret_cast<PfnCtxGetCurrent>(f1);
        g_ctx_get_id = reinterpret_cast<PfnCtxGetId>(f2);
    }
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (g_ctx_get_current(&ctx) != CUDA_SUCCESS || ctx == nullptr || g_ctx_get_id(ctx, &id) != CUDA_SUCCESS) {
        set_error("gwe_forward_static: no current CUDA context");
        return GWE_ERR_CUDA;
    }
    StaticSlot &slot = g_static_slot[dev];
    if (slot.ptr == nullptr || slot.ctx_id != id) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || p == nullptr) {
            set_error(std::string("gwe_forward_static: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
            return GWE_ERR_CUDA;
        }
        slot.ptr = reinterpret_cast<uint8_t *>(p);
        slot.ctx_id = id;
    }
    *out = slot.ptr;
    return GWE_OK;
}

template <int R, int S, int HC, bool F8>
gwe_status launch_tc_static(gwe_model *m, TcState &s, uint8_t *scratch, const float *sH, const float *sL, int64_t nw,
                            int W, int stride, float *out, int *status, cudaStream_t st) {
    using Sh = TcShape<R, S, HC, F8>;
    const Dims &d = m->dims;
    const int64_t n_jobs = (int64_t)d.n_models * nw;
    uint64_t ring_rows = 0;
    for (int l = 0; l < d.L; ++l) ring_rows += (uint64_t)1 << (l % d.lps);
    const uint64_t ring_cta = (2 * ring_rows * Sh::XROW + 255) & ~uint64_t(255);
    const uint64_t cap = kStaticScratchBytes - kStaticRingOff;
    if (ring_cta > cap) {
        set_error("gwe_forward_static: one CTA's lag ring (" + std::to_string(ring_cta) +
                  " bytes) exceeds the fixed scratch (" + std::to_string(cap) + " bytes)");
        return GWE_ERR_ARG;
    }
    const int grid = (int)std::min<int64_t>(std::min<int64_t>(s.sms, n_jobs), (int64_t)(cap / ring_cta));
    // a timeout goes to the caller's status word, or without one to the handle's error word, which
    // gwe_sync reads (and clears) as for every other call on the handle
    int *err = status ? status : s.err.as<int>();
    // the zero rows must be zero; the ring needs no clearing (rows before a window's start are read
    // from the zero rows)
    GWE_CUDA_TRY(cudaMemsetAsync(scratch + kStaticZeroOff, 0, kStaticRingOff - kStaticZeroOff, st));
    if (status) GWE_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int), st));
    TcParams p;
    p.wimg = s.img.as<uint8_t>();
    p.wimg_stride = s.img_stride;
    p.pblob = s.pblob.as<uint8_t>();
    p.pblob_stride = s.pblob_stride;
    p.sH = sH;
    p.sL = sL;
    p.nw = nw;
    p.W = W;
    p.stride = stride;
    p.n_seg = 1;
    p.seg_w0 = nullptr;
    p.seg_s0 = nullptr;
    p.n_models = d.n_models;
    p.out = out;
    p.logits = 0;
    p.ring = scratch + kStaticRingOff;
    p.ring_alloc = (uint64_t)grid * ring_cta;
    p.proj_alloc = 0;
    p.ring_cta_bytes = ring_cta;
    p.ring_pp = 0;
    p.zeros = scratch + kStaticZeroOff;
    p.L = d.L;
    p.lps = d.lps;
    p.ring_rows = ring_rows;
    p.err = err;
    p.n16 = s.f8 ? 0 : s.n16;
    p.model0 = 0;
    p.proj = nullptr;
    p.save_x = nullptr;
    p.save_skip = nullptr;
    p.wait_ns = g_wait_ns;
    p.dbg_drop = g_dbg_drop;
    plan_reuse(d, W, stride, false, p);   // no carry buffer in the fixed scratch
    k_branch_tc<R, S, HC, F8><<<grid, kThreads, Sh::SMEM, st>>>(p);
    note_launch();
    GWE_CUDA_TRY(cudaGetLastError());
    return GWE_OK;
}

}  // namespace
}  // namespace gwe

using namespace gwe;

extern "C" gwe_status gwe_forward_static(gwe_model *m, const float *strain_H, const float *strain_L, int64_t n,
                                         int window, int stride, float *out_prob, int *status, void *stream) {
    clear_error();
    GWE_ARG_CHECK(m != nullptr, "model is NULL");
    GWE_ARG_CHECK(strain_H != nullptr && strain_L != nullptr && out_prob != nullptr, "NULL buffer");
    GWE_ARG_CHECK(window > 0 && stride > 0 && stride <= window, "bad window/stride");
    GWE_ARG_CHECK(n >= window, "n_samples < window");
    if (m->precision != GWE_BF16 && m->precision != GWE_FP8) {
        set_error("gwe_forward_static: the handle must use a tensor-core precision (GWE_BF16 or GWE_FP8)");
        return GWE_ERR_UNSUPPORTED;
    }
    TcState *s = reinterpret_cast<TcState *>(m->tc);
    if (!s || s->variant < 0) {
        set_error("gwe_forward_static: tensor-core path not prepared");
        return GWE_ERR_UNSUPPORTED;
    }
    if (window % kTile != 0) {
        set_error("gwe_forward_static: window must be a multiple of 128");
        return GWE_ERR_UNSUPPORTED;
    }
    const int64_t nw = (n - window) / stride + 1;
    uint8_t *scratch = nullptr;
    gwe_status st = static_scratch(&scratch);
    if (st != GWE_OK) return st;
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    return tc_dispatch(*s, [&](auto t) {
        using T = decltype(t);
        return launch_tc_static<T::R, T::S, T::HC, T::F8>(m, *s, scratch, strain_H, strain_L, nw, window, stride,
                                                          out_prob, status, cs);
    });
}

// ============================================================================ forward plans
// A plan fixes one batched forward (science segments x time slides on given device buffers),
// optionally autotunes the launch shape of the slide heads on those buffers, and captures every
// launch of the forward into one CUDA graph; an execution is one graph launch.
namespace gwe {
namespace {

struct PlanImpl {
    gwe_model *model = nullptr;
    TcWork work;                  // the plan's own rings, carry, projections and tables
    TcLaunch L;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int n_kernels = 0;            // kernels in the graph
    double tuned_ms = 0.0, default_ms = 0.0;
    ~PlanImpl() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        work.release();
    }
};

// autotuned slide-head shapes per geometry, shared by the plans of a process
struct ShapeKey {
    int hc, W, n_slides, n_seg;
    int64_t nw;
    bool operator<(const ShapeKey &o) const {
        return std::tie(hc, W, n_slides, n_seg, nw) < std::tie(o.hc, o.W, o.n_slides, o.n_seg, o.nw);
    }
};
struct ShapeVal {
    SlideShape shape;
    double tuned_ms, default_ms;
};
std::mutex g_shape_mu;
std::map<ShapeKey, ShapeVal> g_shapes;

// Times every candidate shape of model 0's slide heads (projections computed first) with CUDA
// events on `st` and keeps the fastest: samples per block 64 / 128 / 256 (those dividing the
// window) x all offsets per block or a quarter of them per block (more, smaller blocks).
template <int R, int S, int HC, bool F8>
gwe_status autotune_slides(gwe_model *m, TcState &s, PlanImpl &P, cudaStream_t st) {
    using Sh = TcShape<R, S, HC, F8>;
    TcLaunch &L = P.L;
    const ShapeKey key{HC, L.p.W, L.n_slides, L.p.n_seg, L.nw};
    {
        std::lock_guard<std::mutex> lk(g_shape_mu);
        auto it = g_shapes.find(key);
        if (it != g_shapes.end()) {
            L.shape = it->second.shape;
            P.tuned_ms = it->second.tuned_ms;
            P.default_ms = it->second.default_ms;
            return GWE_OK;
        }
    }
    ProfSuspend quiet;
    TcParams q = L.p;
    q.model0 = 0;
    q.n_models = 1;
    q.proj = L.proj;
    k_branch_tc<R, S, HC, F8><<<L.grid_slide, kThreads, Sh::SMEM, st>>>(q);
    GWE_CUDA_TRY(cudaGetLastError());
    std::vector<SlideShape> cands;
    for (int a : {2, 4}) {
        for (int b : {4, 8}) {
            cands.push_back(SlideShape{a, b, 0});
            const int np = L.n_pieces[b == 4 ? 0 : 1];
            const int quarter = std::max(1, (np + 3) / 4);
            if (quarter < np) cands.push_back(SlideShape{a, b, quarter});
        }
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    GWE_CUDA_TRY(cudaEventCreate(&e0));
    cudaError_t ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) {
        cudaEventDestroy(e0);
        GWE_CUDA_TRY(ce);
    }
    double best = 1e300, dflt = 0.0;
    SlideShape best_shape;
    gwe_status r = GWE_OK;
    for (const SlideShape &c : cands) {
        L.shape = c;
        double t_min = 1e300;
        for (int rep = 0; rep < 3 && r == GWE_OK; ++rep) {
            ce = cudaEventRecord(e0, st);
            if (ce == cudaSuccess) r = issue_slide_heads<HC>(m, s, L, 0, st);
            if (ce == cudaSuccess && r == GWE_OK) ce = cudaEventRecord(e1, st);
            if (ce == cudaSuccess && r == GWE_OK) ce = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (ce == cudaSuccess && r == GWE_OK) ce = cudaEventElapsedTime(&ms, e0, e1);
            if (ce != cudaSuccess) {
                set_error(std::string("slide-head autotuning: ") + cudaGetErrorString(ce));
                r = GWE_ERR_CUDA;
            }
            if (rep > 0) t_min = std::min(t_min, (double)ms);   // the first run warms up
        }
        if (r != GWE_OK) break;
        if (c.a == 4 && c.b == 8 && c.ppb == 0) dflt = t_min;
        if (t_min < best) {
            best = t_min;
            best_shape = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (r != GWE_OK) return r;
    L.shape = best_shape;
    P.tuned_ms = best;
    P.default_ms = dflt;
    std::lock_guard<std::mutex> lk(g_shape_mu);
    g_shapes[key] = ShapeVal{best_shape, best, dflt};
    return GWE_OK;
}

template <int R, int S, int HC, bool F8>
gwe_status plan_build(gwe_model *m, TcState &s, PlanImpl &P, const float *sH, const float *sL, const Segments &sg,
                      int W, int stride, const int32_t *slides, int n_slides, float *out, int flags, cudaStream_t st) {
    gwe_status r = setup_tc<R, S, HC, F8>(m, s, P.work, sH, sL, sg, W, stride, slides, n_slides, out, false, st, P.L);
    if (r != GWE_OK) return r;
    if ((flags & GWE_PLAN_AUTOTUNE) && n_slides > 0 && P.L.nw > 0) {
        r = autotune_slides<R, S, HC, F8>(m, s, P, st);
        if (r != GWE_OK) return r;
    }
    // the tables went up from pageable memory and the tuning ran on `st`: finish both first
    GWE_CUDA_TRY(cudaStreamSynchronize(st));
    cudaStream_t cs = nullptr;
    GWE_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    const int64_t before = gwe_launch_count();
    cudaGraph_t g = nullptr;
    cudaError_t ce;
    {
        ProfSuspend quiet;
        ce = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (ce == cudaSuccess) {
            r = issue_tc<R, S, HC, F8>(m, s, P.L, cs);
            const cudaError_t ee = cudaStreamEndCapture(cs, &g);
            if (ce == cudaSuccess) ce = ee;
        }
    }
    P.n_kernels = (int)(gwe_launch_count() - before);
    note_launch(-P.n_kernels);     // captured, not launched
    cudaStreamDestroy(cs);
    if (r != GWE_OK) {
        if (g) cudaGraphDestroy(g);
        return r;
    }
    if (ce != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        set_error(std::string("gwe_plan_create: stream capture failed: ") + cudaGetErrorString(ce));
        return GWE_ERR_CUDA;
    }
    P.graph = g;
    GWE_CUDA_TRY(cudaGraphInstantiate(&P.exec, P.graph, 0));
    return GWE_OK;
}

}  // namespace
}  // namespace gwe

struct gwe_plan {
    gwe::PlanImpl *impl;
};

extern "C" gwe_status gwe_plan_create(gwe_model *m, const float *strain_H, const float *strain_L,
                                      const int64_t *seg_start, const int64_t *seg_len, int n_segments, int window,
                                      int stride, const int32_t *slides, int n_slides, float *out_prob, int flags,
                                      void *stream, gwe_plan **out) {
    clear_error();
    GWE_ARG_CHECK(out != nullptr, "out is NULL");
    *out = nullptr;
    GWE_ARG_CHECK(m != nullptr, "model is NULL");
    GWE_ARG_CHECK(strain_H != nullptr && strain_L != nullptr && out_prob != nullptr, "NULL buffer");
    GWE_ARG_CHECK(seg_start != nullptr && seg_len != nullptr && n_segments > 0, "no segments");
    GWE_ARG_CHECK(window > 0 && stride > 0 && stride <= window, "bad window/stride");
    GWE_ARG_CHECK(n_slides >= 0 && (n_slides == 0 || slides != nullptr), "slides is NULL with n_slides > 0");
    GWE_ARG_CHECK((flags & ~GWE_PLAN_AUTOTUNE) == 0, "unknown flags");
    Segments sg;
    for (int g = 0; g < n_segments; ++g) {
        GWE_ARG_CHECK(seg_start[g] >= 0 && seg_len[g] >= 0, "negative segment start or length");
        sg.s0.push_back(seg_start[g]);
        sg.nw.push_back(seg_len[g] >= window ? (seg_len[g] - window) / stride + 1 : 0);
    }
    GWE_ARG_CHECK(sg.total_windows() > 0, "the segments hold no window");
    if (m->precision != GWE_BF16 && m->precision != GWE_FP8) {
        set_error("gwe_plan_create: plans use the tensor-core path (GWE_BF16 or GWE_FP8 handles)");
        return GWE_ERR_UNSUPPORTED;
    }
    TcState *s = reinterpret_cast<TcState *>(m->tc);
    if (!s || s->variant < 0) {
        set_error("gwe_plan_create: tensor-core path not prepared");
        return GWE_ERR_UNSUPPORTED;
    }
    if (window % kTile != 0) {
        set_error("gwe_plan_create: window must be a multiple of 128");
        return GWE_ERR_UNSUPPORTED;
    }
    gwe::PlanImpl *P = new gwe::PlanImpl();
    P->model = m;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    gwe_status r = tc_dispatch(*s, [&](auto t) {
        using T = decltype(t);
        return gwe::plan_build<T::R, T::S, T::HC, T::F8>(m, *s, *P, strain_H, strain_L, sg, window, stride, slides,
                                                         n_slides, out_prob, flags, st);
    });
    if (r != GWE_OK) {
        delete P;
        return r;
    }
    *out = new gwe_plan{P};
    return GWE_OK;
}

extern "C" gwe_status gwe_plan_execute(gwe_plan *plan, void *stream) {
    clear_error();
    GWE_ARG_CHECK(plan != nullptr && plan->impl != nullptr, "plan is NULL");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    ProfScope prof("gwe_plan", st);
    GWE_CUDA_TRY(cudaGraphLaunch(plan->impl->exec, st));
    note_launch(plan->impl->n_kernels);
    return GWE_OK;
}

extern "C" gwe_status gwe_plan_shape(const gwe_plan *plan, int *window_tile, int *offset_tile, int *pieces_per_block,
                                     int *n_kernels, double *tuned_ms, double *default_ms) {
    clear_error();
    GWE_ARG_CHECK(plan != nullptr && plan->impl != nullptr, "plan is NULL");
    const gwe::PlanImpl &P = *plan->impl;
    const int np = P.L.n_pieces[P.L.shape.b == 4 ? 0 : 1];
    if (window_tile) *window_tile = P.L.shape.a;
    if (offset_tile) *offset_tile = P.L.shape.b;
    if (pieces_per_block) *pieces_per_block = P.L.shape.ppb > 0 ? std::min(P.L.shape.ppb, np) : np;
    if (n_kernels) *n_kernels = P.n_kernels;
    if (tuned_ms) *tuned_ms = P.tuned_ms;
    if (default_ms) *default_ms = P.default_ms;
    return GWE_OK;
}

extern "C" gwe_status gwe_set_slide_shape(int window_tile, int offset_tile, int pieces_per_block) {
    clear_error();
    GWE_ARG_CHECK(window_tile == 2 || window_tile == 4, "window_tile must be 2 or 4");
    GWE_ARG_CHECK(offset_tile == 4 || offset_tile == 8, "offset_tile must be 4 or 8");
    GWE_ARG_CHECK(pieces_per_block >= 0, "pieces_per_block must be >= 0");
    std::lock_guard<std::mutex> lk(gwe::g_plan_shape_mu);
    gwe::g_plan_shape = gwe::SlideShape{window_tile, offset_tile, pieces_per_block};
    return GWE_OK;
}

extern "C" void gwe_plan_destroy(gwe_plan *plan) {
    if (!plan) return;
    delete plan->impl;
    delete plan;
}
