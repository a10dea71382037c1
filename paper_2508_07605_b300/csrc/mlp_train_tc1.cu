// One training step of the learned warm start on the 5th-generation tensor
// cores, one CTA per 128-row tile: the variant for large batches (more tiles
// than half the SMs), where every SM already has a tile of its own and the
// cluster-pair kernel of mlp_train_tc.cu would only add exchange work.  A
// CTA loops over tiles when there are more tiles than SMs.  The network,
// the loss and the order of the products are those of mlp_train_tc.cu; here
// one CTA computes all units of every layer:
//   F1  Z1 = X W1                    -> TMEM [0, 256)   epilogue: A1 = H1 = SELU(Z1 + b1)
//   F2  Z2 = H1 W2  (4 chunks of W2) -> TMEM [256, 512) epilogue: A2 = H2 = SELU(Z2 + b2)
//   F3  Y  = H2 W3                   -> TMEM [0, 32)    epilogue: d = Y + b3 - t,
//       dY = (2/B) G d (FP32, then the BF16 image), loss d^T G d, db3 = column sums
//   W3  dW3 = H2^T dY                -> TMEM [0, 64)    drained to the CTA's partial sums
//   B1  dH2 = dY W3^T                -> TMEM [0, 256)   epilogue: A2 = dZ2 = dH2 * SELU'(Z2 + b2)
//       (Z2 still in TMEM [256, 512)), db2 = column sums
//   W2  dW2^T = dZ2^T H1             -> TMEM [0, 512)   drained
//   B2  dH1 = dZ2 W2^T (4 chunks)    -> TMEM [256, 512), and Z1 = X W1 again -> TMEM [0, 256)
//       epilogue: A1 = dZ1 = dH1 * SELU'(Z1 + b1), db1 = column sums
//   W1  dW1^T = dZ1^T X              -> TMEM [0, 128)   drained
// Shared memory holds the feature image X, two 64 KB activation images A1,
// A2, the 8 KB image of dY and a two-slot ring of 32 KB weight chunks
// fetched by bulk asynchronous copies.
//
// Each CTA owns a slot of partial sums (the layout of the cluster slots of
// mlp_train_tc.cu; loss entries 16 .. 31 stay zero): its first tile stores,
// later tiles add, in a fixed order, so a step is bit-reproducible.  One
// thread (tid 0) issues the bulk copies and the MMAs; 16 warps run the
// epilogues.  Every wait is bounded: a CTA whose wait runs out sets err[1],
// stops, waits (bounded) for its copies in flight and frees its TMEM; the
// reduction then leaves the parameters untouched and reports NaN.
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"
#include "mlp_tc.cuh"
#include "tc_util.cuh"

namespace ocf {

namespace {

using namespace tc;
using namespace mlp;

constexpr int NTHREADS = 512;
constexpr uint32_t OFF_X = 0;                       // 128 x 64 features (16 KB)
constexpr uint32_t OFF_A1 = 16384;                  // H1, later dZ1 (128 x 256)
constexpr uint32_t OFF_A2 = OFF_A1 + 65536;         // H2, later dZ2 (128 x 256)
constexpr uint32_t OFF_DY = OFF_A2 + 65536;         // dY (128 x 32)
constexpr uint32_t OFF_RING = OFF_DY + 8192;        // two weight slots of 32 KB
constexpr uint32_t SLOT = 32768;
constexpr uint32_t OFF_G = OFF_RING + 2 * SLOT;     // G, 32 x 32 FP32
constexpr uint32_t OFF_BIAS = OFF_G + 4096;         // b1 | b2 | b3 (FP32)
constexpr uint32_t OFF_BAR = OFF_BIAS + 4 * (2 * MLP_H + MLP_K_OUT);
constexpr uint32_t SMEM_BYTES = OFF_BAR + 64;
static_assert(SMEM_BYTES <= 232448, "shared memory of one CTA");
static_assert(OFF_RING % 1024 == 0 && OFF_DY % 1024 == 0, "operand alignment");

// Offsets inside one CTA's slot of partial sums (floats).
constexpr int64_t PW2 = MLP_PART_W2, PW1 = MLP_PART_W1, PW3 = MLP_PART_W3, PB1 = MLP_PART_B1,
                  PB2 = MLP_PART_B2, PB3 = MLP_PART_B3, PL = MLP_PART_LOSS;
static_assert(PL + 32 <= MLP_PART_STRIDE && MLP_PART_STRIDE % 32 == 0, "partial slot");

// The weight chunks one tile streams through the ring, in order.
constexpr int CHUNKS = 12;
__device__ __forceinline__ void chunk_src(int c, int64_t &elem, uint32_t &bytes) {
    if (c == 0 || c == 11) { elem = MLP_IMG_W1; bytes = 32768; }
    else if (c <= 4) { elem = MLP_IMG_W2F + (int64_t)(c - 1) * (MLP_H * 64); bytes = 32768; }
    else if (c == 5) { elem = MLP_IMG_W3F; bytes = 16384; }
    else if (c == 6) { elem = MLP_IMG_W3B; bytes = 16384; }
    else { elem = MLP_IMG_W2B + (int64_t)(c - 7) * (MLP_H * 64); bytes = 32768; }
}

constexpr uint32_t MN_A = 1u << 15, MN_B = 1u << 16;   // operand read MN-major

// Column sums over the warp's 32 rows: v[e] is this lane's value of column
// e; on return lane l holds the sum over the 32 lanes of column l (in v[0]).
// 31 exchanges: at each halving step a lane keeps one half of its columns
// and receives the partner's values of that half.
__device__ __forceinline__ float warp_colsum32(float (&v)[32], int lane) {
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
        const bool upper = (lane & s) != 0;
#pragma unroll
        for (int e = 0; e < s; ++e) {
            const float send = upper ? v[e] : v[e + s];
            const float keep = upper ? v[e + s] : v[e];
            v[e] = keep + __shfl_xor_sync(FULL, send, s);
        }
    }
    return v[0];
}

// dZ = dH * SELU'(Z + b) for this warp's 32 rows and columns [c0, c0 + 32):
// dH at TMEM column tdh, the pre-activation accumulator at tz; the BF16
// result goes to the image act (K = 256); the column sums (the bias
// gradient) to pb[c0 + lane].
__device__ __forceinline__ void epi_dz(uint32_t tq, uint32_t tdh, uint32_t tz, int c0, int r,
                                       int lane, const float *bias_s, unsigned char *act,
                                       float *pb, bool first) {
    uint32_t vh[32], vz[32];
    tc_ld32(tq + tdh + (uint32_t)c0, vh);
    tc_ld32(tq + tz + (uint32_t)c0, vz);
    tc_wait_ld();
    float dz[32];
#pragma unroll
    for (int e = 0; e < 32; ++e)
        dz[e] = __uint_as_float(vh[e]) * dselu_f(__uint_as_float(vz[e]) + bias_s[c0 + e]);
    unsigned char *row = act + (r >> 3) * (MLP_H * 16) + (r & 7) * 16;
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        uint32_t pk[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) pk[e] = pack_bf16(dz[8 * g + 2 * e], dz[8 * g + 2 * e + 1]);
        *reinterpret_cast<uint4 *>(row + (c0 / 8 + g) * 128) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    }
    const float s = warp_colsum32(dz, lane);
    acc_store(pb + c0 + lane, s, first);
}

__global__ void __launch_bounds__(NTHREADS, 1) k_mlp_train_tc1(MlpTrainArgs a) {
    extern __shared__ __align__(1024) unsigned char sm[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q = warp & 3, cq = warp >> 2;   // TMEM lane quarter, column quarter
    const uint32_t s0 = smem_u32(sm);
    const uint32_t bar_full = s0 + OFF_BAR, bar_free = bar_full + 16, bar_mma = bar_full + 32;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(sm + OFF_BAR + 40);
    float *G_s = reinterpret_cast<float *>(sm + OFF_G);
    float *bias_s = reinterpret_cast<float *>(sm + OFF_BIAS);   // b1 [0,256) b2 [256,512) b3
    const int64_t tiles = (a.m + TM - 1) / TM;
    const unsigned char *img = reinterpret_cast<const unsigned char *>(a.img);
    float *part = a.part + (int64_t)blockIdx.x * MLP_PART_STRIDE;

    if (tid == 0) {
        mbar_init(bar_full, 1);
        mbar_init(bar_full + 8, 1);
        mbar_init(bar_free, 1);
        mbar_init(bar_free + 8, 1);
        mbar_init(bar_mma, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        if (blockIdx.x == 0 && a.adam) a.adam->t += 1;   // the reduction runs step t + 1
    }
    for (int c = tid; c < 2 * MLP_H + MLP_K_OUT; c += NTHREADS)
        bias_s[c] = c < MLP_H ? a.b1[c] : (c < 2 * MLP_H ? a.b2[c - MLP_H] : a.b3[c - 2 * MLP_H]);
    for (int e = tid; e < MLP_K_OUT * MLP_K_OUT; e += NTHREADS) G_s[e] = a.G[e];   // complete at launch
    pdl_trigger();
    if (warp == 0) tc_alloc(smem_u32(tmem_slot), 512);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t tq = tmem + ((uint32_t)(32 * q) << 16);   // this warp's TMEM lanes

    // ---- issuing thread: chunk g of the stream (tile-local index g % 12) goes
    // to slot g % 2; "full" and "free" complete once per chunk of their slot.
    uint32_t issued = 0, arrived = 0;
    auto issue = [&](uint32_t g) -> bool {   // after the chunk two before it left the slot
        const uint32_t s = g & 1;
        if (g >= 2 && !mbar_wait(bar_free + 8 * s, ((g - 2) >> 1) & 1, a.wait_limit)) return false;
        int64_t elem;
        uint32_t bytes;
        chunk_src((int)(g % CHUNKS), elem, bytes);
        mbar_expect_tx(bar_full + 8 * s, bytes);
        bulk_g2s(s0 + OFF_RING + s * SLOT, img + 2 * elem, bytes, bar_full + 8 * s);
        issued = g + 1;
        return true;
    };
    auto ready = [&](uint32_t g) -> bool {
        const bool ok = mbar_wait(bar_full + 8 * (g & 1), (g >> 1) & 1, a.wait_limit);
        if (ok) arrived = g + 1;
        tc_fence_after();
        return ok;
    };
    auto slot = [&](uint32_t g) -> uint32_t { return s0 + OFF_RING + (g & 1) * SLOT; };
    auto release = [&](uint32_t g) { tc_commit(bar_free + 8 * (g & 1)); };
    const uint32_t id256 = idesc_bf16(TM, 256), id32 = idesc_bf16(TM, MLP_K_OUT);
    // X W1 (or its recomputation) from the chunk in slot(g) -> TMEM [0, 256)
    auto mma_l1 = [&](uint32_t g) {
        for (int s = 0; s < MLP_INP / 16; ++s)
            tc_mma(tmem, sdesc(s0 + OFF_X + s * 256, 128, MLP_INP * 16),
                   sdesc(slot(g) + s * 256, 128, 64 * 16), id256, s > 0);
    };
    // A (K = 256, image at off) times four streamed 256 x 64 chunks g0 .. g0 + 3
    // -> TMEM column dcol; issues chunk g + 1 after consuming chunk g >= g0 + 1
    auto mma_streamed = [&](uint32_t off, uint32_t g0, uint32_t dcol) -> bool {
        for (uint32_t kc = 0; kc < 4; ++kc) {
            const uint32_t g = g0 + kc;
            if (!ready(g)) return false;
            for (int s = 0; s < 4; ++s)
                tc_mma(tmem + dcol, sdesc(s0 + off + (4 * kc + s) * 256, 128, MLP_H * 16),
                       sdesc(slot(g) + s * 256, 128, 64 * 16), id256, (kc | s) != 0);
            release(g);
            if (kc >= 1 && !issue(g + 1)) return false;
        }
        return true;
    };

    uint32_t mma_count = 0;   // completions of bar_mma so far
    bool bad = false;
    // One MMA phase: tid 0 runs `body` (waits, MMAs, copies), commits, and
    // everyone waits for the products; false (CTA-uniform) when a wait ran out.
    auto phase = [&](auto &&body) -> bool {
        bool ok = true;
        if (tid == 0) {
            tc_fence_after();
            ok = body();
            tc_commit(bar_mma);
        }
        const bool okm = mbar_wait(bar_mma, mma_count & 1, a.wait_limit);
        ++mma_count;
        const bool fail = __syncthreads_or(!(ok && okm)) != 0;
        tc_fence_after();
        return !fail;
    };
    auto sync_images = [&]() {   // epilogue writes -> visible to the tensor cores
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
    };

    const float *b1_s = bias_s, *b2_s = bias_s + MLP_H, *b3_s = bias_s + 2 * MLP_H;
    int it = 0;
    for (int64_t tile = blockIdx.x; tile < tiles && !bad; tile += gridDim.x, ++it) {
        const int64_t row0 = tile * TM;
        const bool first = it == 0, has_next = tile + (int64_t)gridDim.x < tiles;
        const uint32_t G0 = (uint32_t)it * CHUNKS;
        const int r = 32 * q + lane;   // this thread's row in the epilogues
        const int64_t i = row0 + r;
        bool okc = true;
        if (tid == 0 && first) okc = issue(G0) && issue(G0 + 1);
        if (tid < TM && row0 + tid < a.m)   // the tile's targets into L2 for the loss epilogue
            asm volatile("prefetch.global.L2 [%0];\n" ::"l"(a.T + (row0 + tid) * MLP_K_OUT));
        {
            RowObs obs;
            features_quad(a, row0 + (tid >> 2), tid >> 2, tid & 3, sm + OFF_X, obs);
        }
        sync_images();

        // ---- F1 -> TMEM [0, 256); epilogue H1
        if (!phase([&] {
                if (!okc || !ready(G0)) return false;
                mma_l1(G0);
                release(G0);
                return issue(G0 + 2);
            })) { bad = true; break; }
        epi_hidden(tmem, 0, q, lane, 64 * cq, b1_s, sm + OFF_A1);
        sync_images();

        // ---- F2 -> TMEM [256, 512); epilogue H2 (Z2 stays in TMEM)
        if (!phase([&] { return mma_streamed(OFF_A1, G0 + 1, 256); })) { bad = true; break; }
        epi_hidden(tmem, 256, q, lane, 64 * cq, b2_s, sm + OFF_A2);
        sync_images();

        // ---- F3 -> TMEM [0, 32); epilogue: loss, dY, db3.  The row's targets
        // are loaded before the wait, in the rotated order of the epilogue:
        // register chunk k holds components 8 ((k + cq) mod 4) .. + 7, so this
        // warp's outputs j = 8 cq + jj come first.
        const bool live = i < a.m;
        float4 tp[8];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int c = 8 * ((k + cq) & 3);
            tp[2 * k] = tp[2 * k + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (live) {
                tp[2 * k] = __ldg(reinterpret_cast<const float4 *>(a.T + i * MLP_K_OUT + c));
                tp[2 * k + 1] = __ldg(reinterpret_cast<const float4 *>(a.T + i * MLP_K_OUT + c + 4));
            }
        }
        if (!phase([&] {
                if (!ready(G0 + 5)) return false;
                for (int s = 0; s < MLP_H / 16; ++s)
                    tc_mma(tmem, sdesc(s0 + OFF_A2 + s * 256, 128, MLP_H * 16),
                           sdesc(slot(G0 + 5) + s * 256, 128, MLP_H * 16), id32, s > 0);
                release(G0 + 5);
                return issue(G0 + 6);
            })) { bad = true; break; }
        {
            uint32_t v[4][8];
#pragma unroll
            for (int k = 0; k < 4; ++k) tc_ld8(tq + 8 * ((k + cq) & 3), v[k]);
            tc_wait_ld();
            float d[32];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int c = 8 * ((k + cq) & 3);
                const float t[8] = {tp[2 * k].x, tp[2 * k].y, tp[2 * k].z, tp[2 * k].w,
                                    tp[2 * k + 1].x, tp[2 * k + 1].y, tp[2 * k + 1].z, tp[2 * k + 1].w};
#pragma unroll
                for (int e = 0; e < 8; ++e)
                    d[8 * k + e] = live ? __uint_as_float(v[k][e]) + b3_s[c + e] - t[e] : 0.f;
            }
            float g[8], l = 0.f;
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) {
                const float *Gr = G_s + (8 * cq + jj) * MLP_K_OUT;
                float s = 0.f;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float4 *Gk = reinterpret_cast<const float4 *>(Gr + 8 * ((k + cq) & 3));
                    const float4 ga = Gk[0], gb = Gk[1];
                    s = fmaf(ga.x, d[8 * k], s);
                    s = fmaf(ga.y, d[8 * k + 1], s);
                    s = fmaf(ga.z, d[8 * k + 2], s);
                    s = fmaf(ga.w, d[8 * k + 3], s);
                    s = fmaf(gb.x, d[8 * k + 4], s);
                    s = fmaf(gb.y, d[8 * k + 5], s);
                    s = fmaf(gb.z, d[8 * k + 6], s);
                    s = fmaf(gb.w, d[8 * k + 7], s);
                }
                l = fmaf(d[jj], s, l);
                g[jj] = s * a.scale;
            }
            *reinterpret_cast<uint4 *>(sm + OFF_DY + (r >> 3) * (MLP_K_OUT * 16) + cq * 128 +
                                       (r & 7) * 16) =
                make_uint4(pack_bf16(g[0], g[1]), pack_bf16(g[2], g[3]), pack_bf16(g[4], g[5]),
                           pack_bf16(g[6], g[7]));
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) {
                const float s = warp_sum(g[jj]);
                if (lane == 0) acc_store(part + PB3 + q * MLP_K_OUT + 8 * cq + jj, s, first);
            }
            l = warp_sum(l);
            if (lane == 0) {
                acc_store(part + PL + warp, l, first);
                if (first) part[PL + 16 + warp] = 0.f;   // the slot layout has 32 loss entries
            }
        }
        sync_images();

        // ---- dW3 = H2^T dY -> TMEM [32 h, 32 h + 32) for inputs [128 h, 128 h + 128)
        if (!phase([&] {
                for (int h = 0; h < 2; ++h)
                    for (int s = 0; s < TM / 16; ++s)
                        tc_mma(tmem + 32 * h,
                               sdesc(s0 + OFF_A2 + s * 2 * (MLP_H * 16) + h * 16 * 128,
                                     MLP_H * 16, 128),
                               sdesc(s0 + OFF_DY + s * 2 * (MLP_K_OUT * 16), MLP_K_OUT * 16, 128),
                               id32 | MN_A | MN_B, s > 0);
                return issue(G0 + 7);
            })) { bad = true; break; }
        if (cq < 2) {   // input c = 128 cq + r: dW3[c][0 .. 32)
            uint32_t v[32];
            tc_ld32(tq + 32 * cq, v);
            tc_wait_ld();
            float4 *dst = reinterpret_cast<float4 *>(part + PW3 + (int64_t)(128 * cq + r) * MLP_K_OUT);
#pragma unroll
            for (int e4 = 0; e4 < 8; ++e4) {
                float4 x = make_float4(__uint_as_float(v[4 * e4]), __uint_as_float(v[4 * e4 + 1]),
                                       __uint_as_float(v[4 * e4 + 2]), __uint_as_float(v[4 * e4 + 3]));
                if (!first) {
                    const float4 o = dst[e4];
                    x.x += o.x; x.y += o.y; x.z += o.z; x.w += o.w;
                }
                dst[e4] = x;
            }
        }
        tc_fence_before();
        __syncthreads();

        // ---- B1: dH2 = dY W3^T -> TMEM [0, 256); epilogue dZ2 (over H2), db2
        if (!phase([&] {
                if (!ready(G0 + 6)) return false;
                for (int s = 0; s < MLP_K_OUT / 16; ++s)
                    tc_mma(tmem, sdesc(s0 + OFF_DY + s * 256, 128, MLP_K_OUT * 16),
                           sdesc(slot(G0 + 6) + s * 256, 128, MLP_K_OUT * 16), id256, s > 0);
                release(G0 + 6);
                return issue(G0 + 8);
            })) { bad = true; break; }
#pragma unroll 1
        for (int hh = 0; hh < 2; ++hh)
            epi_dz(tq, 0, 256, 64 * cq + 32 * hh, r, lane, b2_s, sm + OFF_A2, part + PB2 + q * MLP_H,
                   first);
        sync_images();

        // ---- dW2^T = dZ2^T H1 -> TMEM [256 h, 256 h + 256) for outputs [128 h, + 128)
        if (!phase([&] {
                for (int h = 0; h < 2; ++h)
                    for (int s = 0; s < TM / 16; ++s)
                        tc_mma(tmem + 256 * h,
                               sdesc(s0 + OFF_A2 + s * 2 * (MLP_H * 16) + h * 16 * 128,
                                     MLP_H * 16, 128),
                               sdesc(s0 + OFF_A1 + s * 2 * (MLP_H * 16), MLP_H * 16, 128),
                               id256 | MN_A | MN_B, s > 0);
                return true;
            })) { bad = true; break; }
        {   // output o = 128 (cq / 2) + r, inputs [128 (cq % 2), + 128): dW2[in][o]
            const int h = cq >> 1, o = 128 * h + r, in0 = 128 * (cq & 1);
#pragma unroll 1
            for (int b = 0; b < 4; b += 2) {
                uint32_t v0[32], v1[32];
                tc_ld32(tq + 256 * h + in0 + 32 * b, v0);
                tc_ld32(tq + 256 * h + in0 + 32 * b + 32, v1);
                tc_wait_ld();
                float *dst = part + PW2 + (int64_t)(in0 + 32 * b) * MLP_H + o;
#pragma unroll
                for (int e = 0; e < 32; ++e) acc_store(dst + e * MLP_H, __uint_as_float(v0[e]), first);
#pragma unroll
                for (int e = 0; e < 32; ++e)
                    acc_store(dst + (32 + e) * MLP_H, __uint_as_float(v1[e]), first);
            }
        }
        tc_fence_before();
        __syncthreads();

        // ---- B2: dH1 = dZ2 W2^T -> TMEM [256, 512); Z1 again -> TMEM [0, 256);
        // epilogue dZ1 (over H1), db1
        if (!phase([&] {
                if (!mma_streamed(OFF_A2, G0 + 7, 256)) return false;
                if (!ready(G0 + 11)) return false;
                mma_l1(G0 + 11);
                release(G0 + 11);
                return !has_next || issue(G0 + 12);
            })) { bad = true; break; }
#pragma unroll 1
        for (int hh = 0; hh < 2; ++hh)
            epi_dz(tq, 256, 0, 64 * cq + 32 * hh, r, lane, b1_s, sm + OFF_A1, part + PB1 + q * MLP_H,
                   first);
        sync_images();

        // ---- dW1^T = dZ1^T X -> TMEM [64 h, 64 h + 64) for outputs [128 h, + 128)
        if (!phase([&] {
                for (int h = 0; h < 2; ++h)
                    for (int s = 0; s < TM / 16; ++s)
                        tc_mma(tmem + 64 * h,
                               sdesc(s0 + OFF_A1 + s * 2 * (MLP_H * 16) + h * 16 * 128,
                                     MLP_H * 16, 128),
                               sdesc(s0 + OFF_X + s * 2 * (MLP_INP * 16), MLP_INP * 16, 128),
                               idesc_bf16(TM, MLP_INP) | MN_A | MN_B, s > 0);
                return !has_next || issue(G0 + 13);
            })) { bad = true; break; }
        {   // output o = 128 (cq / 2) + r, inputs [32 (cq % 2), + 32): dW1[in][o]
            const int h = cq >> 1, o = 128 * h + r, in0 = 32 * (cq & 1);
            uint32_t v[32];
            tc_ld32(tq + 64 * h + in0, v);
            tc_wait_ld();
            float *dst = part + PW1 + (int64_t)in0 * MLP_H + o;
#pragma unroll
            for (int e = 0; e < 32; ++e) acc_store(dst + e * MLP_H, __uint_as_float(v[e]), first);
        }
        tc_fence_before();
        __syncthreads();   // TMEM and the images are reused by the next tile
    }
    if (bad && tid == 0) {
        atomicExch(a.err + 1, 1);
        for (uint32_t g = arrived; g < issued; ++g)   // copies still in flight (bounded)
            mbar_wait(bar_full + 8 * (g & 1), (g >> 1) & 1);
        mbar_wait(bar_mma, (mma_count - 1) & 1);       // products of the phase that gave up
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tc_dealloc(tmem, 512);
    }
}

}  // namespace

cudaError_t prepare_mlp_train_tc1() {
    return cudaFuncSetAttribute(k_mlp_train_tc1, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)SMEM_BYTES);
}

// grid: one CTA per tile, at most one per SM (the slots of partial sums)
cudaError_t launch_mlp_train_tc1(const MlpTrainArgs &a, int grid, bool pdl, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(NTHREADS);
    cfg.dynamicSmemBytes = SMEM_BYTES;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k_mlp_train_tc1, a);
}

}  // namespace ocf
