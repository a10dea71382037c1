// One training step of the learned warm start on the 5th-generation tensor
// cores: features -> forward -> loss -> backward -> weight gradients for
// 128-row tiles, fused in one kernel.  The network is the one of mlp_tc.cu
// (48 -> 256 -> 256 -> 32, SELU); the loss of a batch of B rows with targets
// t_r is (1/B) sum_r (y_r - t_r)^T G (y_r - t_r), G = V^T V, i.e. the mean
// squared error of the row's predicted runtimes y_r V^T.
//
// For batches of at most one tile per two SMs (mlp_train_tc1.cu takes larger
// ones): a tile is shared by the two CTAs of a cluster (rank c = 0, 1), each
// on its own SM, one tile per cluster.  Both CTAs hold all 128 rows (M = 128 in every product) and CTA c computes
// the half c of every layer's units (N = 128), so that each SM does half the
// products, half the epilogues and fetches half the weights.  The hidden
// activations, dY and dZ2, whose full width the next product reads, are
// written by each CTA into its own and its partner's shared memory
// (distributed shared memory), followed by a cluster barrier.  Per tile
// (TMEM columns of CTA c; "h" = this CTA's half of the units):
//   F1  Z1h = X W1h                   -> [0, 128)    E1: H1h = SELU(Z1h + b1h) -> A1 (both CTAs)
//   F2  Z2h = H1 W2h (4 chunks)       -> [128, 256)  E2: H2h = SELU(Z2h + b2h) -> A2 (both CTAs)
//       (Z2h stays in TMEM until E5)
//   F3  Y = H2 W3 (both CTAs)         -> [0, 32)     E3: d = Y + b3 - t; outputs j in 16c .. 16c+15:
//       dY_j = (2/B) (G d)_j -> dY image (both CTAs), loss d_j (G d)_j, db3_j
//   W3  dW3[in h] = H2[:, h]^T dY     -> [32, 64)    E4: drained to the partial sums
//   B1  dH2h = dY W3h^T               -> [256, 384)  E5: dZ2h = dH2h * SELU'(Z2h + b2h) -> A2 (both), db2h
//   W2  dW2^T[out h] = dZ2h^T H1      -> [256, 512)  E6: drained
//   B2  dH1h = dZ2 W2h^T (4 chunks)   -> [0, 128),  Z1h = X W1h again -> [128, 256)
//       E7: dZ1h = dH1h * SELU'(Z1h + b1h) -> A1 (own half only), db1h
//   W1  dW1^T[out h] = dZ1h^T X       -> [256, 320)  E8: drained
// G (32 x 32) must be complete when the kernel starts (the engine computes it
// once per V).  W3 and B1, and W2 and B2, are issued back to back: the drains run while
// the next products do.  The weight-gradient products read the activation
// images MN-major (the same bytes the forward products read K-major; see
// mlp_tc.cuh), so nothing is transposed in shared memory.  All products are
// kind::f16 (BF16 operands, FP32 accumulation); SELU' uses the FP32
// pre-activations from TMEM.
//
// Each cluster owns a slot of partial sums (weight and bias gradients, loss)
// in global memory, its two CTAs writing disjoint halves; k_mlp_reduce_adam
// adds the slots in cluster order and applies Adam, so a step is bit-
// reproducible.  Rows at or beyond B get zero features and a zero dY and
// contribute nothing.
//
// Warps 0 .. 15 run the epilogues (warp w owns TMEM lanes 32 (w mod 4) ..
// + 31, i.e. 32 rows, and a quarter of the columns); lane 0 of warp 16
// issues the bulk copies of 16 KB weight chunks into a four-slot ring and
// the MMAs.  Every mbarrier wait is bounded: a CTA whose wait runs out sets
// err[1] and skips the remaining work, but keeps taking part in every
// barrier of the cluster, so its partner never waits for it; at the end it
// waits (bounded) for its copies and products in flight and frees its TMEM.
// The reduction then leaves the parameters untouched and reports NaN.
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"
#include "mlp_tc.cuh"
#include "tc_util.cuh"

namespace ocf {

namespace {

using namespace tc;
using namespace mlp;

constexpr int EPI_THREADS = 512, NTHREADS = EPI_THREADS + 32;   // + the issuing warp
constexpr int HALF = MLP_H / 2;                     // units of a layer per CTA
constexpr uint32_t OFF_X = 0;                       // 128 x 64 features (16 KB)
constexpr uint32_t OFF_A1 = 16384;                  // H1, later dZ1 (128 x 256)
constexpr uint32_t OFF_A2 = OFF_A1 + 65536;         // H2, later dZ2 (128 x 256)
constexpr uint32_t OFF_DY = OFF_A2 + 65536;         // dY (128 x 32)
constexpr uint32_t OFF_RING = OFF_DY + 8192;        // four weight slots of 16 KB
constexpr uint32_t SLOT = 16384;
constexpr int NSLOT = 4;
constexpr uint32_t OFF_G = OFF_RING + NSLOT * SLOT; // G, 32 x 32 FP32
constexpr uint32_t OFF_BIAS = OFF_G + 4096;         // b1 | b2 | b3 (FP32)
constexpr uint32_t OFF_BAR = OFF_BIAS + 4 * (2 * MLP_H + MLP_K_OUT);
constexpr uint32_t SMEM_BYTES = OFF_BAR + 128;
static_assert(SMEM_BYTES <= 232448, "shared memory of one CTA");
static_assert(OFF_RING % 1024 == 0 && OFF_DY % 1024 == 0 && OFF_BAR % 8 == 0, "alignment");
static_assert(MLP_GRAM_PARTS % 8 == 0, "G slices are added eight at a time");

// Offsets inside a cluster's slot of partial sums (floats).
constexpr int64_t PW2 = MLP_PART_W2, PW1 = MLP_PART_W1, PW3 = MLP_PART_W3, PB1 = MLP_PART_B1,
                  PB2 = MLP_PART_B2, PB3 = MLP_PART_B3, PL = MLP_PART_LOSS;
static_assert(PL + 32 <= MLP_PART_STRIDE && MLP_PART_STRIDE % 32 == 0, "partial slot");

// The weight chunks CTA c streams through the ring for one tile, in order:
// 0 W1h (F1), 1-4 W2h forward chunks (F2), 5 W3 (F3, whole), 6 W3h backward
// (B1), 7-10 W2h backward chunks (B2), 11 W1h (Z1 again).  "h": the rows of
// the image that belong to this CTA's half of the units (a contiguous range).
constexpr int CHUNKS = 12;
__device__ __forceinline__ void chunk_src(int k, int c, int64_t &elem, uint32_t &bytes) {
    bytes = 16384;
    if (k == 0 || k == 11) elem = MLP_IMG_W1 + (int64_t)c * HALF * MLP_INP;
    else if (k <= 4) elem = MLP_IMG_W2F + (int64_t)(k - 1) * (MLP_H * 64) + (int64_t)c * HALF * 64;
    else if (k == 5) elem = MLP_IMG_W3F;
    else if (k == 6) { elem = MLP_IMG_W3B + (int64_t)c * HALF * MLP_K_OUT; bytes = 8192; }
    else elem = MLP_IMG_W2B + (int64_t)(k - 7) * (MLP_H * 64) + (int64_t)c * HALF * 64;
}

constexpr uint32_t MN_A = 1u << 15, MN_B = 1u << 16;   // operand read MN-major

// ---- cluster helpers
__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;\n" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t peer_addr(uint32_t local, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(r) : "r"(local), "r"(rank));
    return r;
}
__device__ __forceinline__ void st_peer16(uint32_t addr, uint4 v) {
    asm volatile("st.shared::cluster.v4.b32 [%0], {%1,%2,%3,%4};\n" ::"r"(addr), "r"(v.x), "r"(v.y),
                 "r"(v.z), "r"(v.w)
                 : "memory");
}
__device__ __forceinline__ void st_peer8(uint32_t addr, uint32_t a, uint32_t b) {
    asm volatile("st.shared::cluster.v2.b32 [%0], {%1,%2};\n" ::"r"(addr), "r"(a), "r"(b) : "memory");
}
// Every thread of both CTAs: writes before it (own and partner's shared
// memory, generic proxy) are visible after it, also to the tensor cores.
__device__ __forceinline__ void cluster_barrier() {
    __syncwarp();   // the .aligned forms want converged warps (the issuing warp diverges)
    asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;\n" ::
                     : "memory");
}
__device__ __forceinline__ void cluster_sync_images() {
    asm volatile("fence.proxy.async;\n" ::: "memory");
    tc_fence_before();
    cluster_barrier();
    tc_fence_after();
}

__device__ __forceinline__ void tc_ld4(uint32_t taddr, uint32_t (&v)[4]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3])
                 : "r"(taddr));
}

// 32 BF16 values of row r, columns [col, col + 32) of a K = 256 image at
// image offset `off`: to this CTA's shared memory and, if remote, to the
// partner's (peer = the partner's address of this CTA's shared memory base).
__device__ __forceinline__ void put_row32(unsigned char *sm, uint32_t peer, bool remote,
                                          uint32_t off, int r, int col, const float (&x)[32]) {
    const uint32_t row = off + (r >> 3) * (MLP_H * 16) + (r & 7) * 16;
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        uint4 pk;
        pk.x = pack_bf16(x[8 * g], x[8 * g + 1]);
        pk.y = pack_bf16(x[8 * g + 2], x[8 * g + 3]);
        pk.z = pack_bf16(x[8 * g + 4], x[8 * g + 5]);
        pk.w = pack_bf16(x[8 * g + 6], x[8 * g + 7]);
        const uint32_t o = row + (col / 8 + g) * 128;
        *reinterpret_cast<uint4 *>(sm + o) = pk;
        if (remote) st_peer16(peer + o, pk);
    }
}

// dZ = dH * SELU'(Z + b) for this warp's 32 rows and the 32 columns [col,
// col + 32) of the layer (TMEM: dH at tdh, the pre-activation accumulator at
// tz, both for this CTA's half), 16 columns at a time: the BF16 result goes
// to the image at `off` (and the partner's, if remote); the column sums (the
// bias gradient) to pb[col + lane].
__device__ __forceinline__ void epi_dz(unsigned char *sm, uint32_t peer, bool remote, uint32_t off,
                                       uint32_t tdh, uint32_t tz, int col, int r, int lane,
                                       const float *bias_s, float *pb, bool first) {
    const uint32_t row = off + (r >> 3) * (MLP_H * 16) + (r & 7) * 16;
    float colsum = 0.f;
#pragma unroll 1
    for (int hh = 0; hh < 2; ++hh) {
        uint32_t vh[16], vz[16];
        tc_ld16(tdh + 16 * hh, vh);
        tc_ld16(tz + 16 * hh, vz);
        tc_wait_ld();
        float dz[16];
#pragma unroll
        for (int e = 0; e < 16; ++e)
            dz[e] = __uint_as_float(vh[e]) * dselu_f(__uint_as_float(vz[e]) + bias_s[col + 16 * hh + e]);
#pragma unroll
        for (int g = 0; g < 2; ++g) {
            uint4 pk;
            pk.x = pack_bf16(dz[8 * g], dz[8 * g + 1]);
            pk.y = pack_bf16(dz[8 * g + 2], dz[8 * g + 3]);
            pk.z = pack_bf16(dz[8 * g + 4], dz[8 * g + 5]);
            pk.w = pack_bf16(dz[8 * g + 6], dz[8 * g + 7]);
            const uint32_t o = row + ((col + 16 * hh) / 8 + g) * 128;
            *reinterpret_cast<uint4 *>(sm + o) = pk;
            if (remote) st_peer16(peer + o, pk);
        }
        // column sums of the 16 columns: lane l ends with column l mod 16
        // summed over its half-warp, then the two halves are added
#pragma unroll
        for (int s = 8; s >= 1; s >>= 1) {
            const bool upper = (lane & s) != 0;
#pragma unroll
            for (int e = 0; e < s; ++e) {
                const float send = upper ? dz[e] : dz[e + s];
                const float keep = upper ? dz[e + s] : dz[e];
                dz[e] = keep + __shfl_xor_sync(FULL, send, s);
            }
        }
        const float t = dz[0] + __shfl_xor_sync(FULL, dz[0], 16);
        if ((lane >> 4) == hh) colsum = t;   // lane l keeps column l: half l / 16
    }
    acc_store(pb + col + lane, colsum, first);
}

__global__ void __launch_bounds__(NTHREADS, 1) k_mlp_train_tc(MlpTrainArgs a) {
    extern __shared__ __align__(1024) unsigned char sm[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool issuer = tid == EPI_THREADS;                 // lane 0 of warp 16
    const int q = warp & 3, cq = (warp >> 2) & 3;           // TMEM lane quarter, column quarter
    const uint32_t s0 = smem_u32(sm);
    const int c = (int)cluster_rank();
    const uint32_t peer = peer_addr(s0, (uint32_t)(c ^ 1));
    const int64_t cluster = blockIdx.x >> 1;
    const uint32_t bar_full = s0 + OFF_BAR, bar_free = bar_full + 8 * NSLOT;
    const uint32_t bar_a = bar_free + 8 * NSLOT, bar_b = bar_a + 8;
    const uint32_t bar_drain = bar_b + 16;   // after the TMEM slot
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(sm + OFF_BAR + 8 * (2 * NSLOT + 2));
    float *G_s = reinterpret_cast<float *>(sm + OFF_G);
    float *bias_s = reinterpret_cast<float *>(sm + OFF_BIAS);   // b1 [0,256) b2 [256,512) b3
    const unsigned char *img = reinterpret_cast<const unsigned char *>(a.img);
    float *part = a.part + cluster * MLP_PART_STRIDE;

    if (tid == 0) {
        for (int s = 0; s < NSLOT; ++s) {
            mbar_init(bar_full + 8 * s, 1);
            mbar_init(bar_free + 8 * s, 1);
        }
        mbar_init(bar_a, 1);
        mbar_init(bar_b, 1);
        mbar_init(bar_drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        if (blockIdx.x == 0 && a.adam) a.adam->t += 1;   // the reduction runs step t + 1
    }
    for (int e = tid; e < 2 * MLP_H + MLP_K_OUT; e += NTHREADS)
        bias_s[e] = e < MLP_H ? a.b1[e] : (e < 2 * MLP_H ? a.b2[e - MLP_H] : a.b3[e - 2 * MLP_H]);
    for (int e = tid; e < MLP_K_OUT * MLP_K_OUT; e += NTHREADS) G_s[e] = a.G[e];
    if (warp == 0) tc_alloc(smem_u32(tmem_slot), 512);
    pdl_trigger();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t tq = tmem + ((uint32_t)(32 * q) << 16);   // this warp's TMEM lanes

    // ---- issuing thread.  Chunk g of the stream (tile-local index g % 12)
    // goes to slot g % 4; "full" and "free" complete once per chunk of their slot.
    uint32_t issued = 0, arrived = 0, released = 0, commits_b = 0;
    auto issue = [&](uint32_t g) -> bool {   // after the chunk four before it left the slot
        const uint32_t s = g % NSLOT;
        if (g >= NSLOT && !mbar_wait(bar_free + 8 * s, ((g - NSLOT) / NSLOT) & 1, a.wait_limit))
            return false;
        int64_t elem;
        uint32_t bytes;
        chunk_src((int)(g % CHUNKS), c, elem, bytes);
        mbar_expect_tx(bar_full + 8 * s, bytes);
        bulk_g2s(s0 + OFF_RING + s * SLOT, img + 2 * elem, bytes, bar_full + 8 * s);
        issued = g + 1;
        return true;
    };
    auto top_up = [&](uint32_t limit) -> bool {   // keep the ring full, up to chunk `limit`
        while (issued < limit && issued < released + NSLOT)
            if (!issue(issued)) return false;
        return true;
    };
    auto ready = [&](uint32_t g) -> bool {
        const bool ok = mbar_wait(bar_full + 8 * (g % NSLOT), (g / NSLOT) & 1, a.wait_limit);
        if (ok) arrived = g + 1;
        tc_fence_after();
        return ok;
    };
    auto slot = [&](uint32_t g) -> uint32_t { return s0 + OFF_RING + (g % NSLOT) * SLOT; };
    auto release = [&](uint32_t g) {
        tc_commit(bar_free + 8 * (g % NSLOT));
        released = g + 1;
    };
    const uint32_t id128 = idesc_bf16(TM, HALF), id32 = idesc_bf16(TM, MLP_K_OUT);
    // X W1h from the chunk in slot(g) -> TMEM column dcol
    auto mma_l1 = [&](uint32_t g, uint32_t dcol) {
        for (int s = 0; s < MLP_INP / 16; ++s)
            tc_mma(tmem + dcol, sdesc(s0 + OFF_X + s * 256, 128, MLP_INP * 16),
                   sdesc(slot(g) + s * 256, 128, 64 * 16), id128, s > 0);
    };
    // A (K = 256, image at off) times four streamed 128 x 64 chunks g0 .. g0 + 3
    auto mma_streamed = [&](uint32_t off, uint32_t g0, uint32_t dcol) -> bool {
        for (uint32_t kc = 0; kc < 4; ++kc) {
            const uint32_t g = g0 + kc;
            if (!ready(g)) return false;
            for (int s = 0; s < 4; ++s)
                tc_mma(tmem + dcol, sdesc(s0 + off + (4 * kc + s) * 256, 128, MLP_H * 16),
                       sdesc(slot(g) + s * 256, 128, 64 * 16), id128, (kc | s) != 0);
            release(g);
        }
        return true;
    };
    // weight-gradient product: A = rows of this CTA's half of an image read
    // MN-major (K = 256 image at aoff), B = an image read MN-major (K = bk,
    // N = bn) -> TMEM column dcol
    auto mma_wgrad = [&](uint32_t aoff, uint32_t boff, int bk, uint32_t idesc, uint32_t dcol) {
        for (int s = 0; s < TM / 16; ++s)
            tc_mma(tmem + dcol,
                   sdesc(s0 + aoff + s * 2 * (MLP_H * 16) + c * (HALF / 8) * 128, MLP_H * 16, 128),
                   sdesc(s0 + boff + s * 2 * (bk * 16), bk * 16, 128), idesc | MN_A | MN_B, s > 0);
    };

    uint32_t na = 0, nb = 0;   // completions of bar_a / bar_b waited for by the epilogue warps
    bool bad = false;
    auto wait_a = [&]() -> bool {
        const bool ok = mbar_wait(bar_a, na & 1, a.wait_limit);
        ++na;
        tc_fence_after();
        return ok;
    };
    auto wait_b = [&]() -> bool {
        const bool ok = mbar_wait(bar_b, nb & 1, a.wait_limit);
        ++nb;
        tc_fence_after();
        return ok;
    };

    const float *b1_s = bias_s, *b2_s = bias_s + MLP_H, *b3_s = bias_s + 2 * MLP_H;
    {   // one tile per cluster
        const int64_t row0 = cluster * TM;
        const bool first = true;
        const uint32_t G0 = 0;
        const int r = 32 * q + lane;   // this thread's row in the epilogues
        const int64_t i = row0 + r;
        bool ok = true;   // this thread's view of the current phase
        if (!bad) {
            if (issuer) ok = top_up(G0 + 4);
            if (tid < TM && row0 + tid < a.m)   // the tile's targets into L2 for the loss epilogue
                asm volatile("prefetch.global.L2 [%0];\n" ::"l"(a.T + (row0 + tid) * MLP_K_OUT));
            if (tid < EPI_THREADS) {
                RowObs obs;
                features_quad(a, row0 + (tid >> 2), tid >> 2, tid & 3, sm + OFF_X, obs);
            }
        }
        fence_async_smem();
        tc_fence_before();
        bad = __syncthreads_or(bad || !ok) != 0;

        // ---- F1 -> [0, 128); E1: H1h -> A1 of both CTAs
        if (!bad) {
            if (issuer) {
                tc_fence_after();
                ok = ready(G0);
                if (ok) mma_l1(G0, 0);
                release(G0);
                tc_commit(bar_a);
                ok = ok && top_up(G0 + CHUNKS);
            } else if (tid < EPI_THREADS) {
                ok = wait_a();
                uint32_t v[32];
                tc_ld32(tq + 32 * cq, v);
                tc_wait_ld();
                const int col = HALF * c + 32 * cq;
                float x[32];
#pragma unroll
                for (int e = 0; e < 32; ++e) x[e] = selu_f(__uint_as_float(v[e]) + b1_s[col + e]);
                put_row32(sm, peer, true, OFF_A1, r, col, x);
            }
        }
        bad = __syncthreads_or(bad || !ok) != 0;
        cluster_sync_images();

        // ---- F2 -> [128, 256); E2: H2h -> A2 of both CTAs (Z2h stays in TMEM)
        if (!bad) {
            if (issuer) {
                tc_fence_after();
                ok = mma_streamed(OFF_A1, G0 + 1, HALF);
                tc_commit(bar_a);
                ok = ok && top_up(G0 + CHUNKS);
            } else if (tid < EPI_THREADS) {
                ok = wait_a();
                uint32_t v[32];
                tc_ld32(tq + HALF + 32 * cq, v);
                tc_wait_ld();
                const int col = HALF * c + 32 * cq;
                float x[32];
#pragma unroll
                for (int e = 0; e < 32; ++e) x[e] = selu_f(__uint_as_float(v[e]) + b2_s[col + e]);
                put_row32(sm, peer, true, OFF_A2, r, col, x);
            }
        }
        bad = __syncthreads_or(bad || !ok) != 0;
        cluster_sync_images();

        // ---- F3 (whole Y in both CTAs) -> [0, 32); E3 for the outputs
        // j = 16 c + 4 cq + jj: dY_j -> dY image of both CTAs, loss, db3_j.
        // Register chunk k holds components 4 ((k + k4) mod 8) .. + 3, so this
        // warp's outputs come first; the targets are loaded before the wait.
        const int k4 = 4 * c + cq;
        const bool live = i < a.m;
        float4 tp[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            tp[k] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (!bad && live && tid < EPI_THREADS)
                tp[k] = __ldg(reinterpret_cast<const float4 *>(a.T + i * MLP_K_OUT + 4 * ((k + k4) & 7)));
        }
        if (!bad) {
            if (issuer) {
                tc_fence_after();
                ok = ready(G0 + 5);
                if (ok)
                    for (int s = 0; s < MLP_H / 16; ++s)
                        tc_mma(tmem, sdesc(s0 + OFF_A2 + s * 256, 128, MLP_H * 16),
                               sdesc(slot(G0 + 5) + s * 256, 128, MLP_H * 16), id32, s > 0);
                release(G0 + 5);
                tc_commit(bar_a);
                ok = ok && top_up(G0 + CHUNKS);
            } else if (tid < EPI_THREADS) {
                ok = wait_a();
                uint32_t v[8][4];
#pragma unroll
                for (int k = 0; k < 8; ++k) tc_ld4(tq + 4 * ((k + k4) & 7), v[k]);
                tc_wait_ld();
                float d[32];
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int cc = 4 * ((k + k4) & 7);
                    const float4 t = tp[k];
                    d[4 * k] = live ? __uint_as_float(v[k][0]) + b3_s[cc] - t.x : 0.f;
                    d[4 * k + 1] = live ? __uint_as_float(v[k][1]) + b3_s[cc + 1] - t.y : 0.f;
                    d[4 * k + 2] = live ? __uint_as_float(v[k][2]) + b3_s[cc + 2] - t.z : 0.f;
                    d[4 * k + 3] = live ? __uint_as_float(v[k][3]) + b3_s[cc + 3] - t.w : 0.f;
                }
                float g[4], l = 0.f;
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) {
                    const float *Gr = G_s + (4 * k4 + jj) * MLP_K_OUT;
                    float s = 0.f;
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        const float4 gk = *reinterpret_cast<const float4 *>(Gr + 4 * ((k + k4) & 7));
                        s = fmaf(gk.x, d[4 * k], s);
                        s = fmaf(gk.y, d[4 * k + 1], s);
                        s = fmaf(gk.z, d[4 * k + 2], s);
                        s = fmaf(gk.w, d[4 * k + 3], s);
                    }
                    l = fmaf(d[jj], s, l);
                    g[jj] = s * a.scale;
                }
                const uint32_t o = OFF_DY + (r >> 3) * (MLP_K_OUT * 16) + (k4 >> 1) * 128 +
                                   (r & 7) * 16 + (k4 & 1) * 8;
                const uint32_t w0 = pack_bf16(g[0], g[1]), w1 = pack_bf16(g[2], g[3]);
                *reinterpret_cast<uint2 *>(sm + o) = make_uint2(w0, w1);
                st_peer8(peer + o, w0, w1);
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) {
                    const float s = warp_sum(g[jj]);
                    if (lane == 0) acc_store(part + PB3 + q * MLP_K_OUT + 4 * k4 + jj, s, first);
                }
                l = warp_sum(l);
                if (lane == 0) acc_store(part + PL + 16 * c + warp, l, first);
            }
        }
        bad = __syncthreads_or(bad || !ok) != 0;
        cluster_sync_images();

        // ---- W3: dW3[in in half c] -> [32, 64), and B1: dH2h -> [256, 384).
        // E4 drains dW3 while B1 runs; E5: dZ2h -> A2 of both CTAs, db2h.
        if (!bad) {
            if (issuer) {
                tc_fence_after();
                mma_wgrad(OFF_A2, OFF_DY, MLP_K_OUT, id32, 32);
                tc_commit(bar_a);
                ok = ready(G0 + 6);
                if (ok)
                    for (int s = 0; s < MLP_K_OUT / 16; ++s)
                        tc_mma(tmem + 256, sdesc(s0 + OFF_DY + s * 256, 128, MLP_K_OUT * 16),
                               sdesc(slot(G0 + 6) + s * 256, 128, MLP_K_OUT * 16), id128, s > 0);
                release(G0 + 6);
                tc_commit(bar_b);
                ++commits_b;
                ok = ok && top_up(G0 + CHUNKS);
            } else if (tid < EPI_THREADS) {
                ok = wait_a();
                if (cq == 0) {   // input HALF c + r: dW3[in][0 .. 32)
                    uint32_t v[32];
                    tc_ld32(tq + 32, v);
                    tc_wait_ld();
                    float4 *dst = reinterpret_cast<float4 *>(part + PW3 + (int64_t)(HALF * c + r) * MLP_K_OUT);
#pragma unroll
                    for (int e4 = 0; e4 < 8; ++e4) {
                        float4 x = make_float4(__uint_as_float(v[4 * e4]), __uint_as_float(v[4 * e4 + 1]),
                                               __uint_as_float(v[4 * e4 + 2]), __uint_as_float(v[4 * e4 + 3]));
                        if (!first) {
                            const float4 p = dst[e4];
                            x.x += p.x; x.y += p.y; x.z += p.z; x.w += p.w;
                        }
                        dst[e4] = x;
                    }
                }
                ok = wait_b() && ok;
                epi_dz(sm, peer, true, OFF_A2, tq + 256 + 32 * cq, tq + HALF + 32 * cq,
                       HALF * c + 32 * cq, r, lane, b2_s, part + PB2 + q * MLP_H, first);
            }
        }
        bad = __syncthreads_or(bad || !ok) != 0;
        cluster_sync_images();

        // ---- W2: dW2^T[out in half c] -> [256, 512), and B2: dH1h -> [0, 128)
        // with Z1h again -> [128, 256).  E6 drains dW2 while B2 runs; E7: dZ1h
        // -> A1 (this CTA only: only its own dW1 half reads it), db1h.
        if (!bad) {
            if (issuer) {
                tc_fence_after();
                mma_wgrad(OFF_A2, OFF_A1, MLP_H, idesc_bf16(TM, MLP_H), 256);
                tc_commit(bar_a);
                ok = mma_streamed(OFF_A2, G0 + 7, 0);
                ok = ok && top_up(G0 + CHUNKS) && ready(G0 + 11);
                if (ok) mma_l1(G0 + 11, HALF);
                release(G0 + 11);
                tc_commit(bar_b);
                ++commits_b;
            } else if (tid < EPI_THREADS) {
                ok = wait_a();
                {   // output o = HALF c + r, inputs [64 cq, + 64): dW2[in][o]
                    const int o = HALF * c + r;
#pragma unroll 1
                    for (int hh = 0; hh < 2; ++hh) {
                        uint32_t v[32];
                        tc_ld32(tq + 256 + 64 * cq + 32 * hh, v);
                        tc_wait_ld();
                        float *dst = part + PW2 + (int64_t)(64 * cq + 32 * hh) * MLP_H + o;
#pragma unroll
                        for (int e = 0; e < 32; ++e) acc_store(dst + e * MLP_H, __uint_as_float(v[e]), first);
                    }
                }
                ok = wait_b() && ok;
                epi_dz(sm, peer, false, OFF_A1, tq + 32 * cq, tq + HALF + 32 * cq, HALF * c + 32 * cq,
                       r, lane, b1_s, part + PB1 + q * MLP_H, first);
            }
        }
        fence_async_smem();
        tc_fence_before();
        bad = __syncthreads_or(bad || !ok) != 0;

        // ---- W1: dW1^T[out in half c] -> [256, 320); E8 drains it
        if (!bad) {
            if (issuer) {
                tc_fence_after();
                mma_wgrad(OFF_A1, OFF_X, MLP_INP, idesc_bf16(TM, MLP_INP), 256);
                tc_commit(bar_a);
            } else if (tid < EPI_THREADS) {
                ok = wait_a();
                const int o = HALF * c + r;   // inputs [16 cq, + 16): dW1[in][o]
                uint32_t v[16];
                tc_ld16(tq + 256 + 16 * cq, v);
                tc_wait_ld();
                float *dst = part + PW1 + (int64_t)(16 * cq) * MLP_H + o;
#pragma unroll
                for (int e = 0; e < 16; ++e) acc_store(dst + e * MLP_H, __uint_as_float(v[e]), first);
            }
        }
        tc_fence_before();
        bad = __syncthreads_or(bad || !ok) != 0;
    }
    if (bad && issuer) {
        atomicExch(a.err + 1, 1);
        for (uint32_t g = arrived; g < issued; ++g)   // copies still in flight (bounded)
            mbar_wait(bar_full + 8 * (g % NSLOT), (g / NSLOT) & 1);
        // every product issued so far: a commit to a barrier of its own, whose
        // first phase no earlier wait can alias (bounded)
        tc_commit(bar_drain);
        mbar_wait(bar_drain, 0);
    }
    // neither CTA leaves while its partner may still write into its shared memory
    cluster_barrier();
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tc_dealloc(tmem, 512);
    }
}

// G = V^T V over the first 32 components of V's rows (stride KP).  CTA b
// stages its contiguous slice of rows in shared memory and sums it into
// Gpart[b] (thread t: G[t / 8][4 (t % 8) .. + 3]); the last CTA to finish
// (a ticket taken after the partial is visible) adds the MLP_GRAM_PARTS
// partials in b order into G and resets the ticket, so G does not depend on
// the order in which the CTAs ran.
constexpr int GRAM_ROWS = 64;   // rows staged per round
__global__ void __launch_bounds__(256) k_mlp_gram(int64_t n, int KP, const float *__restrict__ V,
                                                  float *__restrict__ Gpart, float *__restrict__ G,
                                                  unsigned int *__restrict__ ticket) {
    __shared__ __align__(16) float Vs[GRAM_ROWS][MLP_K_OUT];
    __shared__ bool last;
    const int t = threadIdx.x, p = t >> 3, q0 = 4 * (t & 7);
    const int64_t per = (n + MLP_GRAM_PARTS - 1) / MLP_GRAM_PARTS;
    const int64_t j0 = blockIdx.x * per, j1 = j0 + per < n ? j0 + per : n;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int64_t r0 = j0; r0 < j1; r0 += GRAM_ROWS) {
        const int rows = (int)(j1 - r0 < GRAM_ROWS ? j1 - r0 : GRAM_ROWS);
        for (int e = t; e < GRAM_ROWS * MLP_K_OUT / 4; e += 256) {
            const int rr = e / (MLP_K_OUT / 4), c4 = e % (MLP_K_OUT / 4);
            float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
            if (rr < rows) {
                const float *src = V + (r0 + rr) * KP + 4 * c4;
                x = make_float4(src[0], src[1], src[2], src[3]);
            }
            reinterpret_cast<float4 *>(&Vs[rr][0])[c4] = x;
        }
        __syncthreads();
#pragma unroll 8
        for (int rr = 0; rr < GRAM_ROWS; ++rr) {
            const float a = Vs[rr][p];
            const float4 b = *reinterpret_cast<const float4 *>(&Vs[rr][q0]);
            acc.x = fmaf(a, b.x, acc.x);
            acc.y = fmaf(a, b.y, acc.y);
            acc.z = fmaf(a, b.z, acc.z);
            acc.w = fmaf(a, b.w, acc.w);
        }
        __syncthreads();
    }
    reinterpret_cast<float4 *>(Gpart + (int64_t)blockIdx.x * MLP_K_OUT * MLP_K_OUT)[t] = acc;
    __threadfence();
    __syncthreads();
    if (t == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 *src = reinterpret_cast<const float4 *>(Gpart) + t;
#pragma unroll
    for (int b0 = 0; b0 < MLP_GRAM_PARTS; b0 += 8) {   // eight loads in flight, added in b order
        float4 x[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) x[u] = __ldcg(src + (b0 + u) * (MLP_K_OUT * MLP_K_OUT / 4));
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            g.x += x[u].x; g.y += x[u].y; g.z += x[u].z; g.w += x[u].w;
        }
    }
    reinterpret_cast<float4 *>(G)[t] = g;
    if (t == 0) *ticket = 0u;
}

}  // namespace

int mlp_train_tc_slots(int64_t B, int num_sms) {
    const int64_t tiles = (B + TM - 1) / TM;
    if (tiles <= num_sms / 2) return (int)tiles;   // one cluster pair per tile
    return (int)(tiles < num_sms ? tiles : num_sms);
}

cudaError_t prepare_mlp_train_tc() {
    cudaError_t e = cudaFuncSetAttribute(k_mlp_train_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)SMEM_BYTES);
    if (e != cudaSuccess) return e;
    return prepare_mlp_train_tc1();
}

cudaError_t launch_mlp_train_tc(const MlpTrainArgs &a, int num_sms, bool pdl, cudaStream_t st) {
    if (a.m <= 0) return cudaErrorInvalidValue;
    const int64_t tiles = (a.m + TM - 1) / TM;
    const int slots = mlp_train_tc_slots(a.m, num_sms);
    if (tiles > num_sms / 2) return launch_mlp_train_tc1(a, slots, pdl, st);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(2 * slots));
    cfg.blockDim = dim3(NTHREADS);
    cfg.dynamicSmemBytes = SMEM_BYTES;
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;   // the two CTAs of a tile
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 2 : 1;
    return cudaLaunchKernelEx(&cfg, k_mlp_train_tc, a);
}

cudaError_t launch_mlp_gram(int64_t n, int KP, const float *V, float *Gpart, float *G,
                            unsigned int *ticket, cudaStream_t st) {
    k_mlp_gram<<<MLP_GRAM_PARTS, 256, 0, st>>>(n, KP, V, Gpart, G, ticket);
    return cudaGetLastError();
}

}  // namespace ocf
