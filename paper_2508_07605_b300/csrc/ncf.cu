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
//   h1 = SELU(A_i + S_j)   (128 values, built straight into a BF16 UMMA operand
//                           image in shared memory),
//   z2 = h1 W2             (tcgen05.mma, M = 128 pairs, N = 64, K = 128, FP32
//                           accumulation in TMEM),
//   y  = SELU(z2 + b2) . w3 + b3   (epilogue from tcgen05.ld),
// in a persistent kernel with two operand images and two TMEM accumulators in
// flight, so the tensor core works on tile t while the SMs build tile t + 1
// and finish tile t - 1.
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"
#include "tc_util.cuh"

namespace ocf {

namespace {

using namespace tc;
typedef __nv_bfloat16 bf16;

constexpr float SELU_L = 1.0507009873554804934193349852946f;
constexpr float SELU_A = 1.6732632423543772848170429916717f;

__device__ __forceinline__ float selu_f(float z) {
    const float e = __expf(fminf(z, 0.f)) - 1.f;
    return z > 0.f ? SELU_L * z : (SELU_L * SELU_A) * e;
}
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&h);
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

// W2 [128 in][64 out] FP32 -> the UMMA B operand (N = 64 outputs x K = 128
// inputs, K-major, no swizzle): element (o, t) at byte
// (o / 8) * 2048 + (t / 8) * 128 + (o % 8) * 16 + (t % 8) * 2.
__global__ void k_ncf_w2_image(const float *__restrict__ W2, bf16 *__restrict__ img) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < NCF_H1 * NCF_H2;
         e += gridDim.x * blockDim.x) {
        const int t = e / NCF_H2, o = e % NCF_H2;
        const int byte = (o >> 3) * (NCF_H1 * 16) + (t >> 3) * 128 + (o & 7) * 16 + (t & 7) * 2;
        img[byte / 2] = __float2bfloat16_rn(W2[e]);
    }
}

constexpr int NP_THREADS = 256;
constexpr int NP_TM = 128;                         // pairs per tile (UMMA M)
constexpr uint32_t NP_IMG = NP_TM * NCF_H1 * 2;    // 32 KB operand image of h1
constexpr uint32_t NP_OFF_W2 = 0, NP_OFF_H = 16384, NP_OFF_PAR = NP_OFF_H + 2 * NP_IMG;
constexpr uint32_t NP_OFF_Y = NP_OFF_PAR + 2 * NCF_H2 * 4, NP_OFF_BAR = NP_OFF_Y + 2 * NP_TM * 4;
constexpr uint32_t NP_SMEM = NP_OFF_BAR + 64;
constexpr uint32_t NP_TMEM_COLS = 2 * NCF_H2;      // two accumulators of 64 columns

// h1 tile of application i, settings j0 .. j0 + 127, into the operand image:
// thread (warp w, lane = 8 cs + r8) builds rows 8 rb + r8 for rb in {w, w + 8},
// 8-column chunks c8 in {cs, cs + 4, cs + 8, cs + 12}; a quarter-warp stores
// one contiguous 128-byte run (conflict-free).
__device__ __forceinline__ void build_h1(const NcfPredArgs &a, int64_t i, int64_t j0,
                                         unsigned char *img, int warp, int lane) {
    const int r8 = lane & 7, cs = lane >> 3;
    float4 av[4][2];
    const float4 *A4 = reinterpret_cast<const float4 *>(a.A + i * NCF_H1);
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        av[kk][0] = __ldg(A4 + 2 * (cs + 4 * kk));
        av[kk][1] = __ldg(A4 + 2 * (cs + 4 * kk) + 1);
    }
#pragma unroll
    for (int rbi = 0; rbi < 2; ++rbi) {
        const int rb = warp + 8 * rbi, r = 8 * rb + r8;
        const int64_t j = j0 + r;
        const bool ok = j < a.n;
        const float4 *S4 = reinterpret_cast<const float4 *>(a.S + (ok ? j : 0) * NCF_H1);
        float4 sv[4][2];
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            sv[kk][0] = ok ? __ldg(S4 + 2 * (cs + 4 * kk)) : make_float4(0.f, 0.f, 0.f, 0.f);
            sv[kk][1] = ok ? __ldg(S4 + 2 * (cs + 4 * kk) + 1) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            const int c8 = cs + 4 * kk;
            uint4 pk = make_uint4(0, 0, 0, 0);
            if (ok) {
                const float4 x0 = av[kk][0], x1 = av[kk][1], y0 = sv[kk][0], y1 = sv[kk][1];
                pk = make_uint4(pack_bf16(selu_f(x0.x + y0.x), selu_f(x0.y + y0.y)),
                                pack_bf16(selu_f(x0.z + y0.z), selu_f(x0.w + y0.w)),
                                pack_bf16(selu_f(x1.x + y1.x), selu_f(x1.y + y1.y)),
                                pack_bf16(selu_f(x1.z + y1.z), selu_f(x1.w + y1.w)));
            }
            *reinterpret_cast<uint4 *>(img + rb * (NCF_H1 * 16) + c8 * 128 + r8 * 16) = pk;
        }
    }
}

__global__ void __launch_bounds__(NP_THREADS) k_ncf_predict_tc(NcfPredArgs a) {
    extern __shared__ __align__(1024) unsigned char sm[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t s0 = smem_u32(sm);
    const uint32_t bar_w2 = s0 + NP_OFF_BAR, bar_mma0 = bar_w2 + 8;   // bar_mma[b] = bar_mma0 + 8 b
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(sm + NP_OFF_BAR + 24);
    float *b2_s = reinterpret_cast<float *>(sm + NP_OFF_PAR);
    float *w3_s = b2_s + NCF_H2;
    float *ypart = reinterpret_cast<float *>(sm + NP_OFF_Y);   // [2][128]
    const int64_t tpa = (a.n + NP_TM - 1) / NP_TM;            // tiles per application
    const int64_t tiles = a.m * tpa;
    const int64_t K = (int64_t)blockIdx.x < tiles
                          ? (tiles - 1 - (int64_t)blockIdx.x) / gridDim.x + 1 : 0;

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
    const uint32_t idesc = idesc_bf16(NP_TM, NCF_H2);
    bool bad = false;
    int64_t k = 0, issued = 0;   // issued: MMA chains committed (thread 0)
    for (; k <= K && !bad; ++k) {
        if (k < K) {   // build tile k, then hand it to the tensor core
            const int64_t t = (int64_t)blockIdx.x + k * gridDim.x;
            const int64_t i = t / tpa, j0 = (t - i * tpa) * NP_TM;
            build_h1(a, i, j0, sm + NP_OFF_H + (uint32_t)(k & 1) * NP_IMG, warp, lane);
            fence_async_smem();
            tc_fence_before();
            bool ok = true;
            if (tid == 0) {
                tc_fence_after();
                if (k == 0) {
                    ok = mbar_wait(bar_w2, 0);
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
            const int64_t t = (int64_t)blockIdx.x + kp * gridDim.x;
            const int64_t i = t / tpa, j0 = (t - i * tpa) * NP_TM;
            const bool ok = mbar_wait(bar_mma0 + 8 * (uint32_t)(kp & 1), (uint32_t)((kp >> 1) & 1));
            tc_fence_after();
            const int q = warp & 3, half = warp >> 2;
            uint32_t v[32];
            tc_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(kp & 1) * NCF_H2 +
                        (uint32_t)(32 * half), v);
            tc_wait_ld();
            float p = 0.f;
#pragma unroll
            for (int c = 0; c < 32; ++c) {
                const int cc = 32 * half + c;
                p = fmaf(w3_s[cc], selu_f(__uint_as_float(v[c]) + b2_s[cc]), p);
            }
            ypart[half * NP_TM + 32 * q + lane] = p;
            tc_fence_before();
            bad = __syncthreads_or(!ok);
            if (bad) break;
            if (tid < NP_TM) {
                const int64_t j = j0 + tid;
                if (j < a.n) a.T[i * a.n + j] = ypart[tid] + ypart[NP_TM + tid] + b3;
            }
        }
    }
    if (bad) {
        // tiles from k - 1 on were not (or not surely) written: NaN, and the flag
        const float nan = __int_as_float(0x7fc00000);
        for (int64_t kk = (k > 0 ? k - 1 : 0); kk < K; ++kk) {
            const int64_t t = (int64_t)blockIdx.x + kk * gridDim.x;
            const int64_t i = t / tpa, j0 = (t - i * tpa) * NP_TM;
            if (tid < NP_TM && j0 + tid < a.n) a.T[i * a.n + j0 + tid] = nan;
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
    k_ncf_w2_image<<<32, 256, 0, st>>>(W2, reinterpret_cast<bf16 *>(img));
    return cudaGetLastError();
}

cudaError_t prepare_ncf_predict_tc() {
    return cudaFuncSetAttribute(k_ncf_predict_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)NP_SMEM);
}

cudaError_t launch_ncf_predict_tc(const NcfPredArgs &a, int num_sms, cudaStream_t st) {
    if (a.m <= 0 || a.n <= 0) return cudaSuccess;
    const int64_t tiles = a.m * ((a.n + NP_TM - 1) / NP_TM);
    const int64_t cap = 2 * (int64_t)num_sms;   // two CTAs per SM (84 KB shared, 128 TMEM columns)
    const int grid = (int)(tiles < cap ? tiles : cap);
    k_ncf_predict_tc<<<grid, NP_THREADS, NP_SMEM, st>>>(a);
    return cudaGetLastError();
}

}  // namespace ocf
