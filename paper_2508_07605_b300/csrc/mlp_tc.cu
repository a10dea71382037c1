// Fused forward pass of the learned warm start on the 5th-generation tensor
// cores: features -> W1 -> SELU -> W2 -> SELU -> W3 for 128-row tiles in one
// persistent kernel (one CTA per SM).
//
// Per tile, everything stays on the SM:
//   * the 128 rows' features (16 observations x (c_norm, g_norm, runtime),
//     padded to 64) are built from the CSR by one thread per row and stored
//     as a BF16 operand image in shared memory;
//   * each layer is a chain of tcgen05.mma (kind::f16, M = 128, K = 16 per
//     instruction, BF16 operands, FP32 accumulation in TMEM) issued by one
//     thread; tcgen05.commit signals an mbarrier when the chain is done;
//   * 16 warps read the accumulator back with tcgen05.ld (warp w owns TMEM
//     lanes 32 (w mod 4) .. +31 and a quarter of the columns), add the bias,
//     apply SELU and write the BF16 activation image for the next layer into
//     the same shared buffer;
//   * the last epilogue writes u, then four threads per row evaluate the
//     row's observed-entry RMSE under u V^T (the judge of the learned factor)
//     and append the rows above the threshold to the fallback list;
//   * W2 (128 KB) stays resident for the CTA's lifetime; W1 and W3 take
//     turns in a 32 KB stage buffer, fetched by bulk asynchronous copies
//     (cp.async.bulk + mbarrier transaction counts) while the epilogues run.
//
// Operand images: see mlp_tc.cuh.  The engine keeps the weights' BF16 copies
// in exactly that form (W2 as four 256 x 64 chunks along its inputs), so they
// reach shared memory by plain bulk copies.
//
// Every wait is bounded.  A CTA whose wait runs out records the event in
// *err, writes NaN rows for its remaining tiles (their observed-entry
// residual is then not finite, so the engine re-solves them by ALS), drains
// its outstanding copies with another bounded wait and frees its TMEM.
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"
#include "tc_util.cuh"
#include "mlp_tc.cuh"

namespace ocf {

namespace {

using namespace tc;
using namespace mlp;
typedef __nv_bfloat16 bf16;

constexpr int NTHREADS = 512;
constexpr uint32_t OFF_W2 = 0, OFF_STAGE = 131072, OFF_ACT = 163840, OFF_BAR = 229376;
constexpr uint32_t OFF_BIAS = OFF_BAR + 64;   // b1 | b2 | b3 (FP32)
constexpr uint32_t SMEM_BYTES = OFF_BIAS + 4 * (2 * 256 + 32);
constexpr uint32_t BYTES_W2 = 131072, BYTES_W1 = 32768, BYTES_W3 = 16384;
constexpr uint32_t TMEM_COLS = 512;   // layer-1 / layer-3 accumulator at 0, layer-2 at 256

// Observed-entry RMSE of the tile's 128 rows under u (shared memory, rows of
// U_STRIDE floats), one group of four lanes per row: per observation the
// four lanes read one 128-byte row of V (32 bytes each, coalesced), multiply
// by their eight components of u and add across the group.  The first 16
// observations come from the registers the feature phase filled (lane g holds
// slots g, g + 4, ...); a row with more observations reads the rest four at a
// time.  Lane 0 of the group writes the RMSE and the status and, when the row
// is above the threshold (or its residual is not finite), appends it to the
// fallback list.
constexpr int U_STRIDE = 36;   // 16-byte aligned rows, conflict-free float4 access

__device__ __forceinline__ float dot8(const float4 &ua, const float4 &ub, const float4 &x0,
                                      const float4 &x1) {
    float d = ua.x * x0.x;
    d = fmaf(ua.y, x0.y, d);
    d = fmaf(ua.z, x0.z, d);
    d = fmaf(ua.w, x0.w, d);
    d = fmaf(ub.x, x1.x, d);
    d = fmaf(ub.y, x1.y, d);
    d = fmaf(ub.z, x1.z, d);
    return fmaf(ub.w, x1.w, d);
}

__device__ __forceinline__ void residual_quad(const MlpTcArgs &a, int64_t i, const float *u_s,
                                              int rr, int g, const RowObs &o) {
    const unsigned gmask = 0xFu << ((threadIdx.x & 31) & ~3);
    const float4 ua = *reinterpret_cast<const float4 *>(u_s + rr * U_STRIDE + 8 * g);
    const float4 ub = *reinterpret_cast<const float4 *>(u_s + rr * U_STRIDE + 8 * g + 4);
    const float4 *V4 = reinterpret_cast<const float4 *>(a.V);
    float sse = 0.f;
    // two slots (eight observations) per round: 16 rows of V in flight per lane
#pragma unroll
    for (int bp = 0; bp < 4; bp += 2) {
        int32_t jq[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) jq[k] = __shfl_sync(gmask, o.j[bp + (k >> 2)], k & 3, 4);
        float4 x0[8], x1[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            x0[k] = make_float4(0.f, 0.f, 0.f, 0.f);
            x1[k] = x0[k];
            if (jq[k] >= 0) {
                x0[k] = __ldg(V4 + (int64_t)jq[k] * (MLP_K_OUT / 4) + 2 * g);
                x1[k] = __ldg(V4 + (int64_t)jq[k] * (MLP_K_OUT / 4) + 2 * g + 1);
            }
        }
#pragma unroll
        for (int b2 = 0; b2 < 2; ++b2) {
            float mine = 0.f;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float d = dot8(ua, ub, x0[4 * b2 + q], x1[4 * b2 + q]);
                d += __shfl_xor_sync(gmask, d, 2, 4);
                d += __shfl_xor_sync(gmask, d, 1, 4);
                if (q == g) mine = d;
            }
            if (o.j[bp + b2] >= 0) {
                const float e = o.v[bp + b2] - mine;
                sse = fmaf(e, e, sse);
            }
        }
    }
    for (int64_t t0 = o.beg + 16; t0 < o.end; t0 += 4) {   // group-uniform
        const int64_t t = t0 + g;
        int32_t j = -1;
        float r = 0.f;
        if (t < o.end) {
            j = __ldg(a.idx + t);
            r = __ldg(a.val + t);
            if (j < 0 || (int64_t)j >= a.n) j = -1;
        }
        float mine = 0.f;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int32_t jo = __shfl_sync(gmask, j, q, 4);
            float4 x0 = make_float4(0.f, 0.f, 0.f, 0.f), x1 = x0;
            if (jo >= 0) {
                x0 = __ldg(V4 + (int64_t)jo * (MLP_K_OUT / 4) + 2 * g);
                x1 = __ldg(V4 + (int64_t)jo * (MLP_K_OUT / 4) + 2 * g + 1);
            }
            float d = dot8(ua, ub, x0, x1);
            d += __shfl_xor_sync(gmask, d, 2, 4);
            d += __shfl_xor_sync(gmask, d, 1, 4);
            if (q == g) mine = d;
        }
        if (j >= 0) {
            const float e = r - mine;
            sse = fmaf(e, e, sse);
        }
    }
    sse += __shfl_xor_sync(gmask, sse, 2, 4);
    sse += __shfl_xor_sync(gmask, sse, 1, 4);
    if (g == 0 && i < a.m) {
        const int64_t s = o.end - o.beg;
        const float rmse = (o.ok && s > 0) ? sqrtf(sse / (float)s) : 0.0f;
        if (a.row_rmse) a.row_rmse[i] = rmse;
        const bool fb = !(rmse <= a.threshold);
        if (a.status) a.status[i] = fb ? ST_FALLBACK : ST_OK;
        if (fb)
            a.list[atomicAdd(reinterpret_cast<unsigned long long *>(a.count), 1ull)] = (int32_t)i;
    }
}

__device__ __forceinline__ void prefetch_l2(const void *p) {
    asm volatile("prefetch.global.L2 [%0];\n" ::"l"(p));
}

// One warp, while layer 2 runs: pull the next tile's row pointers, column
// indices and values into L2 so that its feature phase does not wait on DRAM.
__device__ __forceinline__ void prefetch_tile(const MlpTcArgs &a, int64_t nr0, int lane) {
    const int64_t nr1 = nr0 + TM < a.m ? nr0 + TM : a.m;
    for (int64_t e = nr0 + 16 * lane; e <= nr1; e += 16 * 32) prefetch_l2(a.ptr + e);
    const int64_t p0 = __ldg(a.ptr + nr0), p1 = __ldg(a.ptr + nr1);
    if (p0 < 0 || p1 < p0 || p1 > a.nnz) return;
    for (int64_t t = p0 + 32 * lane; t < p1; t += 32 * 32) {
        prefetch_l2(a.idx + t);
        prefetch_l2(a.val + t);
    }
}

__global__ void __launch_bounds__(NTHREADS, 1) k_mlp_forward_tc(MlpTcArgs a) {
    extern __shared__ __align__(1024) unsigned char sm[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q = warp & 3, cq = warp >> 2;   // TMEM lane quarter, column quarter
    const uint32_t s0 = smem_u32(sm);
    const uint32_t bar_w2 = s0 + OFF_BAR, bar_st = bar_w2 + 8, bar_mma = bar_w2 + 16;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(sm + OFF_BAR + 24);
    float *bias_s = reinterpret_cast<float *>(sm + OFF_BIAS);   // b1 [0,256) b2 [256,512) b3
    const int64_t tiles = (a.m + TM - 1) / TM;
    const unsigned char *img = reinterpret_cast<const unsigned char *>(a.img);

    if (tid == 0) {
        mbar_init(bar_w2, 1);
        mbar_init(bar_st, 1);
        mbar_init(bar_mma, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    for (int c = tid; c < 2 * MLP_H + MLP_K_OUT; c += NTHREADS)
        bias_s[c] = c < MLP_H ? a.b1[c] : (c < 2 * MLP_H ? a.b2[c - MLP_H] : a.b3[c - 2 * MLP_H]);
    if (warp == 0) tc_alloc(smem_u32(tmem_slot), TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    // bar_st completes alternately for W1 (parity 0) and W3 (parity 1); the
    // copies not yet waited for are drained if a wait runs out
    bool st_pending = false, w2_pending = false;
    uint32_t st_par = 0;   // parity of the pending bar_st phase
    if (tid == 0 && (int64_t)blockIdx.x < tiles) {
        mbar_expect_tx(bar_w2, BYTES_W2);
        for (uint32_t c = 0; c < BYTES_W2; c += 32768)
            bulk_g2s(s0 + OFF_W2 + c, img + 2 * MLP_IMG_W2F + c, 32768, bar_w2);
        mbar_expect_tx(bar_st, BYTES_W1);
        bulk_g2s(s0 + OFF_STAGE, img + 2 * MLP_IMG_W1, BYTES_W1, bar_st);
        st_pending = w2_pending = true;
    }
    const uint32_t id256 = idesc_bf16(TM, 256), id32 = idesc_bf16(TM, MLP_K_OUT);
    uint32_t mma_count = 0;   // completions of bar_mma so far (parity = count & 1)
    bool first = true, bad = false;
    RowObs obs;   // this lane's share of its row, from the feature phase to the residual

    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int64_t row0 = tile * TM;
        const bool has_next = tile + (int64_t)gridDim.x < tiles;
        if (!bad) {
            // ---- features -> ACT (K = 64), four lanes per row
            features_quad(a, row0 + (tid >> 2), tid >> 2, tid & 3, sm + OFF_ACT, obs);
            fence_async_smem();
            __syncthreads();
            // ---- layer 1: ACT (128 x 64) x W1 (256 x 64)^T -> TMEM [0, 256)
            bool okw = true;
            if (tid == 0) {
                if (first) {
                    okw = mbar_wait(bar_w2, 0, a.wait_limit);
                    w2_pending = !okw;
                }
                okw = okw && mbar_wait(bar_st, 0, a.wait_limit);
                st_pending = !okw;
                tc_fence_after();
                if (okw)
                    for (int s = 0; s < MLP_INP / 16; ++s)
                        tc_mma(tmem, sdesc(s0 + OFF_ACT + s * 256, 128, MLP_INP * 16),
                               sdesc(s0 + OFF_STAGE + s * 256, 128, MLP_INP * 16), id256, s > 0);
                tc_commit(bar_mma);
            }
            first = false;
            bool okm = mbar_wait(bar_mma, mma_count & 1, a.wait_limit);
            ++mma_count;
            bad = __syncthreads_or(!okm || !okw);
        }
        if (!bad) {
            tc_fence_after();
            if (tid == 0) {   // W1 is free: fetch W3 while the epilogue runs
                mbar_expect_tx(bar_st, BYTES_W3);
                bulk_g2s(s0 + OFF_STAGE, img + 2 * MLP_IMG_W3F, BYTES_W3, bar_st);
                st_pending = true;
                st_par = 1;
            }
            epi_hidden(tmem, 0, q, lane, 64 * cq, bias_s, sm + OFF_ACT);
            fence_async_smem();
            tc_fence_before();
            __syncthreads();
            // ---- layer 2: ACT (128 x 256) x W2 (256 x 256)^T -> TMEM [256, 512)
            if (tid == 0) {
                tc_fence_after();
                for (int s = 0; s < MLP_H / 16; ++s)   // W2: four 256 x 64 chunks
                    tc_mma(tmem + 256, sdesc(s0 + OFF_ACT + s * 256, 128, MLP_H * 16),
                           sdesc(s0 + OFF_W2 + (s >> 2) * 32768 + (s & 3) * 256, 128, 64 * 16),
                           id256, s > 0);
                tc_commit(bar_mma);
            }
            if (warp == 1 && has_next) prefetch_tile(a, row0 + (int64_t)gridDim.x * TM, lane);
            const bool okm = mbar_wait(bar_mma, mma_count & 1, a.wait_limit);
            ++mma_count;
            bad = __syncthreads_or(!okm);
        }
        if (!bad) {
            tc_fence_after();
            epi_hidden(tmem, 256, q, lane, 64 * cq, bias_s + MLP_H, sm + OFF_ACT);
            fence_async_smem();
            tc_fence_before();
            __syncthreads();
            // ---- layer 3: ACT (128 x 256) x W3 (32 x 256)^T -> TMEM [0, 32)
            bool okw = true;
            if (tid == 0) {
                okw = mbar_wait(bar_st, 1, a.wait_limit);
                st_pending = !okw;
                tc_fence_after();
                if (okw)
                    for (int s = 0; s < MLP_H / 16; ++s)
                        tc_mma(tmem, sdesc(s0 + OFF_ACT + s * 256, 128, MLP_H * 16),
                               sdesc(s0 + OFF_STAGE + s * 256, 128, MLP_H * 16), id32, s > 0);
                tc_commit(bar_mma);
            }
            const bool okm = mbar_wait(bar_mma, mma_count & 1, a.wait_limit);
            ++mma_count;
            bad = __syncthreads_or(!okm || !okw);
        }
        if (!bad) {
            tc_fence_after();
            if (tid == 0 && has_next) {   // W3 is free: fetch the next tile's W1
                mbar_expect_tx(bar_st, BYTES_W1);
                bulk_g2s(s0 + OFF_STAGE, img + 2 * MLP_IMG_W1, BYTES_W1, bar_st);
                st_pending = true;
                st_par = 0;
            }
            // u = acc + b3: columns [8 cq, 8 cq + 8) of this warp's rows -> Y and
            // shared memory (ACT is free: layer 3 is done)
            float *u_s = reinterpret_cast<float *>(sm + OFF_ACT);
            uint32_t v[8];
            tc_ld8(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(8 * cq), v);
            tc_wait_ld();
            const int r = 32 * q + lane;
            const int64_t i = row0 + r;
            float y[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) y[e] = __uint_as_float(v[e]) + bias_s[2 * MLP_H + 8 * cq + e];
            const float4 y0 = make_float4(y[0], y[1], y[2], y[3]);
            const float4 y1 = make_float4(y[4], y[5], y[6], y[7]);
            float4 *us = reinterpret_cast<float4 *>(u_s + r * U_STRIDE + 8 * cq);
            us[0] = y0;
            us[1] = y1;
            if (i < a.m) {
                float4 *dst = reinterpret_cast<float4 *>(a.Y + i * MLP_K_OUT + 8 * cq);
                dst[0] = y0;
                dst[1] = y1;
            }
            tc_fence_before();
            __syncthreads();   // TMEM [0, 32) read; u rows complete
            residual_quad(a, row0 + (tid >> 2), u_s, tid >> 2, tid & 3, obs);
            __syncthreads();   // ACT free before the next tile's features
        }
        if (bad && tid < TM) {   // rows of a tile that could not be computed: NaN, fallback
            const int64_t i = row0 + tid;
            if (i < a.m) {
                float4 *dst = reinterpret_cast<float4 *>(a.Y + i * MLP_K_OUT);
                const float nan = __int_as_float(0x7fc00000);
                for (int e = 0; e < MLP_K_OUT / 4; ++e) dst[e] = make_float4(nan, nan, nan, nan);
                if (a.row_rmse) a.row_rmse[i] = nan;
                if (a.status) a.status[i] = ST_FALLBACK;
                a.list[atomicAdd(reinterpret_cast<unsigned long long *>(a.count), 1ull)] =
                    (int32_t)i;
            }
        }
    }
    if (bad && tid == 0) {
        atomicExch(a.err, 1);
        // drain (bounded): the weight copies not yet waited for, and the products
        // of the last commit (which covers every earlier one; its phase is the
        // barrier's latest, as each earlier one was waited for)
        if (w2_pending) mbar_wait(bar_w2, 0);
        if (st_pending) mbar_wait(bar_st, st_par);
        if (mma_count > 0) mbar_wait(bar_mma, (mma_count - 1) & 1);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tc_dealloc(tmem, TMEM_COLS);
    }
}

}  // namespace

size_t mlp_forward_tc_smem() { return SMEM_BYTES; }

cudaError_t prepare_mlp_forward_tc() {
    return cudaFuncSetAttribute(k_mlp_forward_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)SMEM_BYTES);
}

cudaError_t launch_mlp_forward_tc(const MlpTcArgs &a, int num_sms, cudaStream_t st) {
    if (a.m <= 0) return cudaSuccess;
    const int64_t tiles = (a.m + TM - 1) / TM;
    const int grid = (int)(tiles < num_sms ? tiles : num_sms);
    k_mlp_forward_tc<<<grid, NTHREADS, SMEM_BYTES, st>>>(a);
    return cudaGetLastError();
}

}  // namespace ocf
