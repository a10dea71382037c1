// Neural collaborative filtering, the paper's CF model (Sec. "Collaborative
// Filtering Model"): the application index i and the power-cap-pair index j
// select rows of two embedding tables (d = 32 each), the two rows are
// concatenated and passed through an MLP 64 -> 128 -> 64 -> 1 with SELU
// hidden units; the output is the predicted entry P_ij.
//
// Training (mini-batches of observed entries, mean squared error, Adam) is in
// ncf_train.cu.
//
// Completion (every application x every setting) factors the first layer
// over the concatenation, x W1 = Ea_i W1[0:32] + Es_j W1[32:64], so it costs
// one small FP32 product per application and per setting (A_i = Ea_i W1a + b1,
// S_j = Es_j W1s) instead of one per pair.  The pair work is then
//   h1 = SELU(A_i + S_j)   (128 values, in packed FP16 pairs: one add, two
//                           min/max, one exponential (ex2.approx.f16x2) and two
//                           fused multiply-adds per pair of values, written
//                           straight into an FP16 UMMA operand image in shared
//                           memory),
//   z2 = h1 W2             (tcgen05.mma kind::f16, FP16 operands, M = 128
//                           settings, N = 64, K = 128, FP32 accumulation in TMEM),
//   y  = SELU(z2 + b2) . w3 + b3   (epilogue from tcgen05.ld, the dot in FP32),
// in a persistent kernel: a CTA keeps one block of 128 settings' S rows in
// registers and walks its applications, with two operand images and two TMEM
// accumulators in flight, so the tensor core works on tile t while the SMs
// build tile t + 1 and finish tile t - 1.
#include <cuda_fp16.h>

#include "common.cuh"
#include "kernels.h"
#include "tc_util.cuh"

namespace ocf {

namespace {

using namespace tc;

constexpr float SELU_L = 1.0507009873554804934193349852946f;
constexpr float SELU_A = 1.6732632423543772848170429916717f;

__device__ __forceinline__ uint32_t h2u(__half2 h) { return *reinterpret_cast<uint32_t *>(&h); }
__device__ __forceinline__ __half2 u2h(uint32_t u) { return *reinterpret_cast<__half2 *>(&u); }

// SELU of two FP16 values without a branch:
//   lambda max(z, 0) + lambda alpha (2^(log2(e) min(z, 0)) - 1).
__device__ __forceinline__ uint32_t selu_h2(__half2 z) {
    const __half2 zero = __float2half2_rn(0.f);
    const __half2 t = __hmul2(__hmin2(z, zero), __float2half2_rn(1.4426950408889634f));
    uint32_t e;
    asm("ex2.approx.f16x2 %0, %1;" : "=r"(e) : "r"(h2u(t)));
    const __half2 la = __float2half2_rn(SELU_L * SELU_A);
    const __half2 neg = __hfma2(u2h(e), la, __hneg2(la));
    return h2u(__hfma2(__hmax2(z, zero), __float2half2_rn(SELU_L), neg));
}
__device__ __forceinline__ uint32_t pack_h2(float lo, float hi) {
    return h2u(__floats2half2_rn(lo, hi));
}

// ---------------------------------------------------------------- completion
// out[r][c] = bias[c] + sum_t E[r][t] W[t][c]  (W: 32 rows of the first layer,
// row stride 128), FP32.  W stays in shared memory; two rows per pass of a
// 256-thread CTA.
__global__ void __launch_bounds__(256) k_ncf_first_layer(int64_t rows, const float *__restrict__ E,
                                                         const float *__restrict__ W,
                                                         const float *__restrict__ bias,
                                                         float *__restrict__ out) {
    __shared__ float Ws[NCF_D * NCF_H1];
    for (int e = threadIdx.x; e < NCF_D * NCF_H1; e += blockDim.x) Ws[e] = W[e];
    __syncthreads();
    const int c = threadIdx.x & (NCF_H1 - 1);
    const float b = bias ? bias[c] : 0.f;
    for (int64_t r = blockIdx.x * 2 + (threadIdx.x >> 7); r < rows; r += (int64_t)gridDim.x * 2) {
        const float *e = E + r * NCF_D;
        float s = b;
#pragma unroll 8
        for (int t = 0; t < NCF_D; ++t) s = fmaf(__ldg(e + t), Ws[t * NCF_H1 + c], s);
        out[r * NCF_H1 + c] = s;
    }
}

// W2 [128 in][64 out] FP32 -> the FP16 UMMA B operand (N = 64 outputs x
// K = 128 inputs, K-major, no swizzle): element (o, t) at byte
// (o / 8) * 2048 + (t / 8) * 128 + (o % 8) * 16 + (t % 8) * 2.
__global__ void k_ncf_w2_image(const float *__restrict__ W2, __half *__restrict__ img) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < NCF_H1 * NCF_H2;
         e += gridDim.x * blockDim.x) {
        const int t = e / NCF_H2, o = e % NCF_H2;
        const int byte = (o >> 3) * (NCF_H1 * 16) + (t >> 3) * 128 + (o & 7) * 16 + (t & 7) * 2;
        img[byte / 2] = __float2half_rn(W2[e]);
    }
}

constexpr int NP_THREADS = 256;
constexpr int NP_TM = 128;                         // settings per tile (UMMA M)
constexpr uint32_t NP_IMG = NP_TM * NCF_H1 * 2;    // 32 KB operand image of h1
constexpr uint32_t NP_OFF_W2 = 0, NP_OFF_H = 16384, NP_OFF_PAR = NP_OFF_H + 2 * NP_IMG;
constexpr uint32_t NP_OFF_A = NP_OFF_PAR + 2 * NCF_H2 * 4;          // A rows (FP16) of two tiles
constexpr uint32_t NP_OFF_Y = NP_OFF_A + 2 * NCF_H1 * 4;            // [2][128] partial y
constexpr uint32_t NP_OFF_BAR = NP_OFF_Y + 2 * NP_TM * 4;
constexpr uint32_t NP_SMEM = NP_OFF_BAR + 64;
constexpr uint32_t NP_TMEM_COLS = 2 * NCF_H2;      // two accumulators of 64 columns

// Work of CTA c of G: with G >= the number of setting blocks nsb, one block
// sb = c mod nsb and the applications r, r + R, ... (r = c div nsb, R = the
// number of CTAs on sb); otherwise blocks c, c + G, ... with every
// application.  Tile k of the CTA is (application, setting block).
struct Work {
    int64_t nsb, sb0, sb_step, i0, i_step, napps, nblocks;
    __device__ __forceinline__ void init(int64_t m, int64_t n, int64_t c, int64_t G) {
        nsb = (n + NP_TM - 1) / NP_TM;
        if (G >= nsb) {
            sb0 = c % nsb; sb_step = nsb; nblocks = 1;
            const int64_t R = G / nsb + (sb0 < G % nsb ? 1 : 0);
            i0 = c / nsb; i_step = R;
            napps = i0 < m ? (m - 1 - i0) / R + 1 : 0;
        } else {
            sb0 = c; sb_step = G; nblocks = (nsb - 1 - c) / G + 1;
            i0 = 0; i_step = 1; napps = m;
        }
    }
    __device__ __forceinline__ int64_t tiles() const { return napps * nblocks; }
    __device__ __forceinline__ void tile(int64_t k, int64_t &i, int64_t &sb) const {
        const int64_t b = k / napps;
        i = i0 + (k - b * napps) * i_step;
        sb = sb0 + b * sb_step;
    }
};

// This thread's share of the block's S rows, as FP16 pairs kept in registers
// while the CTA walks its applications: rows 8 rb + r8 for rb in {w, w + 8}
// (warp w, lane = 8 cs + r8), 8-column chunks c8 = cs, cs + 4, cs + 8, cs + 12.
__device__ __forceinline__ void load_s(const NcfPredArgs &a, int64_t sb, int warp, int lane,
                                       uint4 (&sv)[2][4]) {
    const int r8 = lane & 7, cs = lane >> 3;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int64_t j = sb * NP_TM + 8 * (warp + 8 * h) + r8;
        const bool ok = j < a.n;
        const float4 *S4 = reinterpret_cast<const float4 *>(a.S + (ok ? j : 0) * NCF_H1);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            float4 y0 = make_float4(0.f, 0.f, 0.f, 0.f), y1 = y0;
            if (ok) {
                y0 = __ldg(S4 + 2 * (cs + 4 * kk));
                y1 = __ldg(S4 + 2 * (cs + 4 * kk) + 1);
            }
            sv[h][kk] = make_uint4(pack_h2(y0.x, y0.y), pack_h2(y0.z, y0.w),
                                   pack_h2(y1.x, y1.y), pack_h2(y1.z, y1.w));
        }
    }
}

// h1 = SELU(A_i + S_j) for the thread's rows and chunks into the operand image
// (a quarter-warp stores one contiguous 128-byte run: conflict-free); A_i is
// read from shared memory (four distinct 16-byte words per instruction).
__device__ __forceinline__ void build_h1(const uint4 *A_s, const uint4 (&sv)[2][4],
                                         const bool (&ok)[2], unsigned char *img, int warp,
                                         int lane) {
    const int r8 = lane & 7, cs = lane >> 3;
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        const int c8 = cs + 4 * kk;
        const uint4 x = A_s[c8];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const uint4 y = sv[h][kk];
            uint4 pk = make_uint4(0, 0, 0, 0);
            if (ok[h])
                pk = make_uint4(selu_h2(__hadd2(u2h(x.x), u2h(y.x))),
                                selu_h2(__hadd2(u2h(x.y), u2h(y.y))),
                                selu_h2(__hadd2(u2h(x.z), u2h(y.z))),
                                selu_h2(__hadd2(u2h(x.w), u2h(y.w))));
            *reinterpret_cast<uint4 *>(img + (warp + 8 * h) * (NCF_H1 * 16) + c8 * 128 + r8 * 16) = pk;
        }
    }
}

__global__ void __launch_bounds__(NP_THREADS, 2) k_ncf_predict_tc(NcfPredArgs a) {
    extern __shared__ __align__(1024) unsigned char sm[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t s0 = smem_u32(sm);
    const uint32_t bar_w2 = s0 + NP_OFF_BAR, bar_mma0 = bar_w2 + 8;   // bar_mma[b] = bar_mma0 + 8 b
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(sm + NP_OFF_BAR + 24);
    float *b2_s = reinterpret_cast<float *>(sm + NP_OFF_PAR);
    float *w3_s = b2_s + NCF_H2;
    uint4 *A_s = reinterpret_cast<uint4 *>(sm + NP_OFF_A);     // [2][16] (8 FP16 each)
    float *ypart = reinterpret_cast<float *>(sm + NP_OFF_Y);   // [2][128]
    Work w;
    w.init(a.m, a.n, blockIdx.x, gridDim.x);
    const int64_t K = w.tiles();

    if (tid == 0) {
        mbar_init(bar_w2, 1);
        mbar_init(bar_mma0, 1);
        mbar_init(bar_mma0 + 8, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    for (int c = tid; c < NCF_H2; c += NP_THREADS) {
        b2_s[c] = a.b2[c];
        w3_s[c] = a.w3[c];
    }
    const float b3 = a.b3[0];
    if (warp == 0) tc_alloc(smem_u32(tmem_slot), NP_TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    bool w2_pending = false;
    if (tid == 0 && K > 0) {
        mbar_expect_tx(bar_w2, NCF_H1 * NCF_H2 * 2);
        bulk_g2s(s0 + NP_OFF_W2, a.w2img, NCF_H1 * NCF_H2 * 2, bar_w2);
        w2_pending = true;
    }
    const uint32_t idesc = idesc_f16(NP_TM, NCF_H2);
    uint4 sv[2][4];
    int64_t cur_sb = -1;
    bool row_ok[2] = {false, false};
    bool bad = false;
    int64_t k = 0, issued = 0;   // issued: MMA chains committed (thread 0)
    for (; k <= K && !bad; ++k) {
        if (k < K) {   // build tile k, then hand it to the tensor core
            int64_t i, sb;
            w.tile(k, i, sb);
            if (sb != cur_sb) {
                load_s(a, sb, warp, lane, sv);
                row_ok[0] = sb * NP_TM + 8 * warp + (lane & 7) < a.n;
                row_ok[1] = sb * NP_TM + 8 * (warp + 8) + (lane & 7) < a.n;
                cur_sb = sb;
            }
            uint4 *Ak = A_s + (k & 1) * (NCF_H1 / 8);   // the other buffer belongs to tile k - 1
            if (tid < NCF_H1 / 8) {
                const float4 *src = reinterpret_cast<const float4 *>(a.A + i * NCF_H1) + 2 * tid;
                const float4 x0 = __ldg(src), x1 = __ldg(src + 1);
                Ak[tid] = make_uint4(pack_h2(x0.x, x0.y), pack_h2(x0.z, x0.w), pack_h2(x1.x, x1.y),
                                     pack_h2(x1.z, x1.w));
            }
            __syncthreads();
            build_h1(Ak, sv, row_ok, sm + NP_OFF_H + (uint32_t)(k & 1) * NP_IMG, warp, lane);
            fence_async_smem();
            tc_fence_before();
            bool ok = true;
            if (tid == 0) {
                tc_fence_after();
                if (k == 0) {
                    ok = mbar_wait(bar_w2, 0, a.wait_limit);
                    w2_pending = !ok;
                }
            }
            bad = __syncthreads_or(!ok);
            if (bad) break;
            if (tid == 0) {
                tc_fence_after();
                const uint32_t hb = s0 + NP_OFF_H + (uint32_t)(k & 1) * NP_IMG;
#pragma unroll
                for (int s = 0; s < NCF_H1 / 16; ++s)
                    tc_mma(tmem + (uint32_t)(k & 1) * NCF_H2, sdesc(hb + s * 256, 128, NCF_H1 * 16),
                           sdesc(s0 + NP_OFF_W2 + s * 256, 128, NCF_H1 * 16), idesc, s > 0);
                tc_commit(bar_mma0 + 8 * (uint32_t)(k & 1));
                issued = k + 1;
            }
        }
        if (k > 0) {   // finish tile k - 1 from its accumulator
            const int64_t kp = k - 1;
            int64_t i, sb;
            w.tile(kp, i, sb);
            const int64_t j0 = sb * NP_TM;
            const bool ok = mbar_wait(bar_mma0 + 8 * (uint32_t)(kp & 1), (uint32_t)((kp >> 1) & 1),
                                     a.wait_limit);
            tc_fence_after();
            const int q = warp & 3, cq = warp >> 2;   // TMEM lane quarter, column half
            uint32_t v[32];
            tc_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(kp & 1) * NCF_H2 +
                        (uint32_t)(32 * cq), v);
            tc_wait_ld();
            float p = 0.f;
#pragma unroll
            for (int c = 0; c < 32; c += 2) {
                const int cc = 32 * cq + c;
                const __half2 z = __floats2half2_rn(__uint_as_float(v[c]) + b2_s[cc],
                                                    __uint_as_float(v[c + 1]) + b2_s[cc + 1]);
                const float2 h = __half22float2(u2h(selu_h2(z)));
                p = fmaf(w3_s[cc], h.x, p);
                p = fmaf(w3_s[cc + 1], h.y, p);
            }
            ypart[cq * NP_TM + 32 * q + lane] = p;
            tc_fence_before();
            bad = __syncthreads_or(!ok);
            if (bad) break;
            if (tid < NP_TM) {
                const int64_t j = j0 + tid;
                if (j < a.n)
                    a.T[i * a.n + j] = (ypart[tid] + ypart[NP_TM + tid]) + b3;
            }
        }
    }
    if (bad) {
        // tiles from k - 1 on were not (or not surely) written: NaN, and the flag
        const float nan = __int_as_float(0x7fc00000);
        for (int64_t kk = (k > 0 ? k - 1 : 0); kk < K; ++kk) {
            int64_t i, sb;
            w.tile(kk, i, sb);
            const int64_t j = sb * NP_TM + tid;
            if (tid < NP_TM && j < a.n) a.T[i * a.n + j] = nan;
        }
        if (tid == 0) {
            atomicExch(a.err, 1);
            if (w2_pending) mbar_wait(bar_w2, 0);   // drain the weight copy (bounded)
            // let the (at most two) chains still in flight finish before the
            // accumulator is freed (bounded waits)
            for (int64_t x = issued >= 2 ? issued - 2 : 0; x < issued; ++x)
                mbar_wait(bar_mma0 + 8 * (uint32_t)(x & 1), (uint32_t)((x >> 1) & 1));
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tc_dealloc(tmem, NP_TMEM_COLS);
    }
}

}  // namespace

cudaError_t launch_ncf_first_layer(int64_t rows, const float *E, const float *W, const float *bias,
                                   float *out, cudaStream_t st) {
    if (rows <= 0) return cudaSuccess;
    int64_t blocks = (rows + 1) / 2;
    if (blocks > NUM_SMS_HINT * 8) blocks = NUM_SMS_HINT * 8;
    k_ncf_first_layer<<<(unsigned)blocks, 256, 0, st>>>(rows, E, W, bias, out);
    return cudaGetLastError();
}

cudaError_t launch_ncf_w2_image(const float *W2, void *img, cudaStream_t st) {
    k_ncf_w2_image<<<32, 256, 0, st>>>(W2, reinterpret_cast<__half *>(img));
    return cudaGetLastError();
}

cudaError_t prepare_ncf_predict_tc() {
    return cudaFuncSetAttribute(k_ncf_predict_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)NP_SMEM);
}

cudaError_t launch_ncf_predict_tc(const NcfPredArgs &a, int num_sms, cudaStream_t st) {
    if (a.m <= 0 || a.n <= 0) return cudaSuccess;
    // two CTAs per SM (one computes while the other waits at a barrier); when
    // the setting blocks fit, a multiple of their number so that every block
    // gets the same share of the applications
    const int64_t nsb = (a.n + NP_TM - 1) / NP_TM, tiles = a.m * nsb;
    int64_t g = 2 * (int64_t)num_sms;
    if (nsb <= g && g / nsb * nsb >= (g * 15) / 16) g = g / nsb * nsb;
    const int grid = (int)(tiles < g ? tiles : g);
    k_ncf_predict_tc<<<grid, NP_THREADS, NP_SMEM, st>>>(a);
    return cudaGetLastError();
}

}  // namespace ocf
