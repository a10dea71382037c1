// Reconstruction T = U V^T on the 5th-generation tensor cores, fused with
// Algorithm 2 (Sec. "Optimal Power setting Selection"), for the BF16-Gram
// precision mode at k = 32.
//
// The contraction is the split-BF16 form of the Gram path: every factor value
// x is carried as hi = bf16(x), lo = bf16(x - hi), and T ~ Uh Vh^T + Uh Vl^T +
// Ul Vh^T with FP32 accumulation (the dropped Ul Vl^T is ~2^-18 relative).
// The selection is then exact in FP32 on the T the kernel produces (the
// value it writes when the dense matrix is requested).
//
// One persistent CTA per SM, 18 warps with fixed roles:
//   * warp 16 streams the settings in chunks of 256 (hi and lo operand images
//     of V, 32 KB) into a two-stage shared ring with cp.async.bulk;
//   * warp 17 owns the tensor memory (512 columns: two 256-column
//     accumulators) and issues, per chunk, six tcgen05.mma (M = 128 rows of
//     U, N = 256 settings, K = 16) into the free accumulator, then commits
//     to the chunk's "stage free" and "accumulator full" mbarriers;
//   * warps 0..15 read an accumulator (warp w: TMEM lanes 32 (w mod 4) ..,
//     64 of the 256 columns, 16 at a time), release it, and run the screened
//     Algorithm 2 on their settings of their row, one thread per row; the
//     chunk holding the baseline setting goes first so that t_b is known; the
//     four column quarters of a row are merged at the end of the tile.
// Accumulator j of chunk g is reused by chunk g + 2, so the tensor cores fill
// one accumulator while the epilogue drains the other.
//
// Every mbarrier wait is bounded (a.wait_limit polls); a wait that runs out
// sets *err, the thread stops waiting and the producer and MMA warps stop
// issuing (the CTA's results are then unspecified; *err says so).  Before the
// CTA frees its TMEM and exits, the producer waits for its last copy into each
// buffer and the MMA warp for its last commit, again with a bound, so that no
// copy or product is still in flight.
#include "alg2.cuh"
#include "common.cuh"
#include "kernels.h"
#include "tc_util.cuh"

namespace ocf {

namespace {

using namespace tc;

constexpr int TM = 128, CN = 256, KPT = 32;
constexpr int NEPI = 16;                       // epilogue warps
constexpr int GS = 32;                         // settings per TMEM load and screening group
constexpr int NCQ = NEPI / 4;                  // column groups (warps per TMEM lane quarter)
constexpr int CPW = CN / NCQ;                  // settings per epilogue warp and chunk
constexpr int PRODUCER = NEPI, ISSUER = NEPI + 1;
constexpr int NTHREADS = (NEPI + 2) * 32;
constexpr uint32_t HALF_BYTES = CN * KPT * 2;  // one BF16 image of a chunk
constexpr uint32_t CHUNK_BYTES = 2 * HALF_BYTES;
constexpr uint32_t OFF_VB = 0;                             // 2 stages x (hi | lo)
constexpr uint32_t OFF_UH = 2 * CHUNK_BYTES;               // U hi image, 128 x 32
constexpr uint32_t OFF_UL = OFF_UH + TM * KPT * 2;         // U lo image
constexpr uint32_t OFF_TB = OFF_UL + TM * KPT * 2;         // t_b per row
constexpr uint32_t OFF_CAND = OFF_TB + TM * 4;             // [TM][4] candidates
constexpr uint32_t OFF_BAR = OFF_CAND + TM * 4 * sizeof(Cand);
constexpr int STASH_LD = GS + 4;                           // floats per lane: 144 B, conflict-free rows
constexpr uint32_t OFF_STASH = OFF_BAR + 128;              // per lane: the group's runtimes
constexpr uint32_t OFF_THR = OFF_STASH + NEPI * 32 * STASH_LD * 4;  // [TM][4] screening thresholds
constexpr uint32_t OFF_CG = OFF_THR + TM * 4 * 4;                   // c + g table (when it fits)
constexpr uint32_t TMEM_COLS = 512;
constexpr int BAR_TILE = 1, BAR_EPI = 2;                    // named barriers

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
    __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&h);
}

// Per group of GS settings of a row (one TMEM load, indices compile-time after
// unrolling, so the values stay in registers): the dense output if requested,
// then a branch-free screen (validity and the smallest energy estimate, three
// instructions per element) and, only when the group's smallest estimate can
// still win or tie, the exact evaluation of the elements within the bound.
// The lanes of a warp hold different rows, so an exact evaluation taken by one
// lane is paid by all; once a row has a best, few groups pass its threshold.
__device__ __forceinline__ void store_group(const uint32_t (&v)[GS], float *trow, int64_t j0,
                                            int64_t n, bool vec) {
    if (vec && j0 + GS <= n) {
#pragma unroll
        for (int e = 0; e < GS; e += 4)
            *reinterpret_cast<float4 *>(trow + j0 + e) =
                make_float4(__uint_as_float(v[e]), __uint_as_float(v[e + 1]),
                            __uint_as_float(v[e + 2]), __uint_as_float(v[e + 3]));
    } else {
#pragma unroll
        for (int e = 0; e < GS; ++e)
            if (j0 + e < n) trow[j0 + e] = __uint_as_float(v[e]);
    }
}

// chunk processed at position s of a tile: the baseline's chunk first
__device__ __forceinline__ int chunk_at(int s, int cb) { return s == 0 ? cb : (s <= cb ? s - 1 : s); }

__global__ void __launch_bounds__(NTHREADS, 1) k_predict_select_tc(PredictTcArgs a) {
    extern __shared__ __align__(1024) unsigned char sm[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t s0 = smem_u32(sm);
    const uint32_t bar = s0 + OFF_BAR;
    // full[2] @0, empty[2] @16, afull[2] @32, aempty[2] @48, TMEM slot @64, drain @72
    auto full = [&](int b) { return bar + 8 * b; };
    auto empty = [&](int b) { return bar + 16 + 8 * b; };
    auto afull = [&](int b) { return bar + 32 + 8 * b; };
    auto aempty = [&](int b) { return bar + 48 + 8 * b; };
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(sm + OFF_BAR + 64);
    const int64_t tiles = (a.m + TM - 1) / TM;
    const int nch = (int)((a.n + CN - 1) / CN);
    const int cb = (int)(a.base / CN);
    const bool cg_smem = a.n <= PREDICT_TC_CG_MAX;
    float *cg_s = reinterpret_cast<float *>(sm + OFF_CG);

    if (tid == 0) {
        for (int b = 0; b < 2; ++b) {
            mbar_init(full(b), 1);
            mbar_init(empty(b), 1);
            mbar_init(afull(b), 1);
            mbar_init(aempty(b), NEPI);
        }
        mbar_init(bar + 72, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (cg_smem && a.select)   // padded with +inf to whole chunks
        for (int64_t j = tid; j < (int64_t)nch * CN; j += NTHREADS)
            cg_s[j] = j < a.n ? a.cg[j] : __int_as_float(0x7f800000);
    if (warp == ISSUER) tc_alloc(smem_u32(tmem_slot), TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    bool bad = false;

    if (warp == PRODUCER) {
        if (lane == 0) {
            const unsigned char *img = reinterpret_cast<const unsigned char *>(a.Vimg);
            int64_t g = 0;   // copies issued
            for (int64_t tile = blockIdx.x; tile < tiles && !bad; tile += gridDim.x)
                for (int s = 0; s < nch; ++s, ++g) {
                    const int vb = (int)(g & 1);
                    const uint32_t ph = (uint32_t)((g >> 1) & 1);
                    if (!mbar_wait(empty(vb), ph ^ 1u, a.wait_limit)) {
                        bad = true;
                        break;
                    }
                    mbar_expect_tx(full(vb), CHUNK_BYTES);
                    bulk_g2s(s0 + OFF_VB + vb * CHUNK_BYTES,
                             img + (int64_t)chunk_at(s, cb) * CHUNK_BYTES, CHUNK_BYTES, full(vb));
                }
            // drain: no copy may land after the CTA has gone; the last two copies
            // (one per buffer) are the only ones that can be in flight (a no-op when
            // the MMA warp consumed them all)
            for (int64_t x = g >= 2 ? g - 2 : 0; x < g; ++x)
                mbar_wait(full((int)(x & 1)), (uint32_t)((x >> 1) & 1));
        }
    } else if (warp == ISSUER) {
        const uint32_t idesc = idesc_bf16(TM, CN);
        int64_t g = 0, last = -1;   // the last chunk whose products were committed
        for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
            named_sync(BAR_TILE, (NEPI + 1) * 32);   // this tile's U images are written
            for (int s = 0; s < nch; ++s, ++g) {
                const int vb = (int)(g & 1), ab = (int)(g & 1);
                const uint32_t ph = (uint32_t)((g >> 1) & 1);
                if (lane == 0) {
                    // once a wait gave up, nothing more is issued (the loops still run
                    // for the tile barrier the epilogue warps take part in)
                    if (!bad && !mbar_wait(full(vb), ph, a.wait_limit)) bad = true;
                    if (!bad && !mbar_wait(aempty(ab), ph ^ 1u, a.wait_limit)) bad = true;
                    if (!bad) {
                        tc_fence_after();
                        const uint32_t d = tmem + (uint32_t)(ab * CN);
                        const uint32_t vh = s0 + OFF_VB + vb * CHUNK_BYTES, vl = vh + HALF_BYTES;
#pragma unroll
                        for (int ks = 0; ks < KPT / 16; ++ks) {
                            const uint64_t ah = sdesc(s0 + OFF_UH + ks * 256, 128, KPT * 16);
                            const uint64_t al = sdesc(s0 + OFF_UL + ks * 256, 128, KPT * 16);
                            const uint64_t bh = sdesc(vh + ks * 256, 128, KPT * 16);
                            const uint64_t bl = sdesc(vl + ks * 256, 128, KPT * 16);
                            tc_mma(d, ah, bh, idesc, ks > 0);
                            tc_mma(d, ah, bl, idesc, 1);
                            tc_mma(d, al, bh, idesc, 1);
                        }
                        tc_commit(empty(vb));
                        tc_commit(afull(ab));
                        last = g;
                    }
                }
                __syncwarp();
            }
        }
        // drain: every product issued finishes before TMEM is freed (a commit to
        // a barrier of its own, whose first phase no earlier wait can alias)
        if (lane == 0 && last >= 0) {
            tc_commit(bar + 72);
            mbar_wait(bar + 72, 0);
        }
    } else {
        // ---------------- epilogue warps
        const int q = warp & 3, cq = warp >> 2;
        const int r = 32 * q + lane;            // row of the tile (TMEM lane)
        float *tb_s = reinterpret_cast<float *>(sm + OFF_TB);
        Cand *cand_s = reinterpret_cast<Cand *>(sm + OFF_CAND);
        const int col_b = (int)(a.base - (int64_t)cb * CN);
        float *stash_s = reinterpret_cast<float *>(sm + OFF_STASH);
        volatile float *thr_s = reinterpret_cast<volatile float *>(sm + OFF_THR);
        const float inf = __int_as_float(0x7f800000);
        auto cg_of = [&](int64_t j) { return cg_smem ? cg_s[j] : a.cg_pad[j]; };
        int64_t g = 0;
        for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
            const int64_t row0 = tile * TM;
            // U tile -> split BF16 operand images (row ur, components 8 ug .. 8 ug + 7)
            for (int it = tid; it < TM * 4; it += NEPI * 32) {
                const int ur = it >> 2, ug = it & 3;
                const int64_t iu = row0 + ur;
                float x[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const int p = 8 * ug + e;
                    x[e] = (iu < a.m && p < a.k) ? a.U[iu * a.ldu + p] : 0.0f;
                }
                uint32_t hw[4], lw[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const float h0 = __bfloat162float(__float2bfloat16_rn(x[2 * e]));
                    const float h1 = __bfloat162float(__float2bfloat16_rn(x[2 * e + 1]));
                    hw[e] = pack2(h0, h1);
                    lw[e] = pack2(x[2 * e] - h0, x[2 * e + 1] - h1);
                }
                const uint32_t off = (ur >> 3) * (KPT * 16) + ug * 128 + (ur & 7) * 16;
                *reinterpret_cast<uint4 *>(sm + OFF_UH + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                *reinterpret_cast<uint4 *>(sm + OFF_UL + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
            }
            // this row's screening threshold, shared by its four column quarters
            thr_s[r * 4 + cq] = inf;
            fence_async_smem();
            named_sync(BAR_TILE, (NEPI + 1) * 32);

            const int64_t i = row0 + r;
            RowCtx rc{0.0f, -1.0f, 0.0f};
            uint32_t tsb = 0u;   // bit pattern of t*: valid runtimes are <= it
            Cand best{0.0f, 0.0f, -1, 0.0f};
            for (int s = 0; s < nch; ++s, ++g) {
                const int ab = (int)(g & 1);
                const uint32_t ph = (uint32_t)((g >> 1) & 1);
                if (!bad && !mbar_wait(afull(ab), ph, a.wait_limit)) bad = true;
                tc_fence_after();
                const uint32_t ta = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(ab * CN + CPW * cq);
                const int chunk = chunk_at(s, cb);
                if (s == 0) {   // the baseline's chunk: t_b of every row first
                    if (col_b >= CPW * cq && col_b < CPW * cq + CPW) {   // warp-uniform
                        const uint32_t tb = tc_ld1(ta + (uint32_t)(col_b - CPW * cq));
                        tc_wait_ld();
                        tb_s[r] = __uint_as_float(tb);
                    }
                    named_sync(BAR_EPI, NEPI * 32);
                    if (a.select) {
                        rc = alg2_row(tb_s[r], a.gamma);
                        tsb = rc.tstar > 0.0f ? __float_as_uint(rc.tstar) : 0u;
                    }
                }
                // groups of GS settings: one TMEM load in registers at a time
#pragma unroll 1
                for (int hh = 0; hh < CPW / GS; ++hh) {
                    uint32_t v[GS];
                    tc_ld32(ta + (uint32_t)(GS * hh), v);
                    tc_wait_ld();
                    if (hh == CPW / GS - 1) {   // all read: the accumulator is free
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(aempty(ab));
                    }
                    const int64_t j0 = (int64_t)chunk * CN + CPW * cq + GS * hh;
                    if (a.T && i < a.m) store_group(v, a.T + i * a.n, j0, a.n, a.t_vec);
                    if (a.select) {
                        // Screen, branch-free: w_e = (c + g) t of each element with
                        // t <= t* (one unsigned compare on the bit patterns: positive
                        // floats order like their bits; negatives and NaN fall outside;
                        // tsb = 0 for a row without a valid baseline), +inf otherwise
                        // (c + g is +inf past n), and the group's smallest w.  A zero t
                        // passes the compare; the exact evaluation rejects it.  The
                        // energy estimate is w / t_b = fl(w (1 / t_b)), monotone in w,
                        // so the group's smallest estimate is fl(min w (1 / t_b)).
                        const float4 *cg4 = reinterpret_cast<const float4 *>(
                            cg_smem ? (const float *)cg_s + j0 : a.cg_pad + j0);
                        float w[GS];
                        float wmin = inf;
#pragma unroll
                        for (int e4 = 0; e4 < GS / 4; ++e4) {
                            const float4 c = cg4[e4];
                            const float2 p0 = __fmul2_rn(make_float2(c.x, c.y),
                                                         make_float2(__uint_as_float(v[4 * e4]),
                                                                     __uint_as_float(v[4 * e4 + 1])));
                            const float2 p1 = __fmul2_rn(make_float2(c.z, c.w),
                                                         make_float2(__uint_as_float(v[4 * e4 + 2]),
                                                                     __uint_as_float(v[4 * e4 + 3])));
                            const float pw[4] = {p0.x, p0.y, p1.x, p1.y};
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                w[4 * e4 + e] = v[4 * e4 + e] <= tsb ? pw[e] : inf;
                                wmin = fminf(wmin, w[4 * e4 + e]);
                            }
                        }
                        // Exact evaluation only where the screen cannot exclude: the
                        // group's smallest estimate is at most the best's threshold
                        // (or no best yet); then every element within the bound of that
                        // minimum (usually the minimum alone) is evaluated exactly, in
                        // a per-row loop over the candidates' bit mask, with the group's
                        // runtimes stashed in shared memory for indexed access.
                        // The threshold is the smallest of the four quarters' (each
                        // derived from an exactly evaluated candidate of this row, so an
                        // element above it can neither win nor tie the row's final best;
                        // a quarter's value read before its latest update is only looser).
                        const float me = __fmul_rn(wmin, rc.rtb);
                        float4 tq;
                        asm volatile("ld.volatile.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                                     : "=f"(tq.x), "=f"(tq.y), "=f"(tq.z), "=f"(tq.w)
                                     : "r"(s0 + OFF_THR + (uint32_t)(16 * r)));
                        const float thr = fminf(fminf(fminf(tq.x, tq.y), fminf(tq.z, tq.w)),
                                                best.j >= 0 ? best.Ethr : inf);
                        const bool trig = wmin < inf && me <= thr;
                        if (__any_sync(FULL, trig)) {
                            float *stash = stash_s + (warp * 32 + lane) * STASH_LD;
#pragma unroll
                            for (int e = 0; e < GS; e += 4)
                                *reinterpret_cast<uint4 *>(stash + e) =
                                    make_uint4(v[e], v[e + 1], v[e + 2], v[e + 3]);
                            if (trig) {
                                float bound = fminf(alg2_bound(me, a.Ebase), thr);
                                // candidates by w alone: fl(w (1 / t_b)) <= bound implies
                                // w <= bound t_b (1 + 2^-22), so bw below keeps a superset
                                // (invalid elements carry w = inf); each is re-checked
                                // exactly below
                                const float bw = __fmul_rn(__fmul_rn(bound, rc.tb), 1.00000095367431640625f);
                                uint32_t mask = 0u;
#pragma unroll
                                for (int e = 0; e < GS; ++e) mask |= (w[e] <= bw ? 1u : 0u) << e;
                                while (mask) {
                                    const int e = __ffs(mask) - 1;
                                    mask &= mask - 1u;
                                    const float t = stash[e];
                                    if (t > 0.0f && __float_as_uint(t) <= tsb &&
                                        __fmul_rn(__fmul_rn(cg_of(j0 + e), t), rc.rtb) <= bound) {
                                        alg2_exact(best, rc, t, cg_of(j0 + e), a.Ebase, (int32_t)(j0 + e));
                                        bound = fminf(bound, best.Ethr);
                                    }
                                }
                                if (best.j >= 0) thr_s[r * 4 + cq] = best.Ethr;
                            }
                        }
                    }
                }
            }
            // merge the four column-quarters of each row
            if (a.select) {
                cand_s[r * 4 + cq] = best;
                named_sync(BAR_EPI, NEPI * 32);
                if (cq == 0 && i < a.m) {
#pragma unroll
                    for (int w = 1; w < NCQ; ++w)
                        if (better(cand_s[r * 4 + w], best)) best = cand_s[r * 4 + w];
                    if (a.best) a.best[i] = best.j;
                    if (a.saving) a.saving[i] = best.j >= 0 ? best.sv : 0.0f;
                }
            }
        }
    }
    if (bad) atomicExch(a.err, 1);
    tc_fence_before();
    __syncthreads();
    if (warp == ISSUER) {
        tc_fence_after();
        tc_dealloc(tmem, TMEM_COLS);
    }
}

// V (n x 32 FP32, rows of KP = 32) -> per chunk of 256 settings: hi image,
// then lo image (K-major core-matrix layout); settings beyond n are zero.
__global__ void k_v_image(const float *__restrict__ V, int64_t n, int nch,
                          unsigned char *__restrict__ img) {
    const int64_t total = (int64_t)nch * CN * (KPT / 8);   // one 8-component group per item
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = e / (KPT / 8);
        const int kc = (int)(e % (KPT / 8));
        const int c = (int)(j / CN), nn = (int)(j % CN);
        float x[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) x[t] = j < n ? V[j * KPT + 8 * kc + t] : 0.0f;
        uint32_t hw[4], lw[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const float h0 = __bfloat162float(__float2bfloat16_rn(x[2 * t]));
            const float h1 = __bfloat162float(__float2bfloat16_rn(x[2 * t + 1]));
            hw[t] = pack2(h0, h1);
            lw[t] = pack2(x[2 * t] - h0, x[2 * t + 1] - h1);
        }
        unsigned char *base = img + (int64_t)c * CHUNK_BYTES + (nn >> 3) * (KPT * 16) + kc * 128 +
                              (nn & 7) * 16;
        *reinterpret_cast<uint4 *>(base) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
        *reinterpret_cast<uint4 *>(base + HALF_BYTES) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
    }
}

}  // namespace

size_t predict_tc_image_bytes(int64_t n) { return (size_t)((n + CN - 1) / CN) * CHUNK_BYTES; }

cudaError_t prepare_predict_tc() {
    return cudaFuncSetAttribute(k_predict_select_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(OFF_CG + 4 * PREDICT_TC_CG_MAX));
}

cudaError_t launch_v_image(const float *V, int64_t n, void *img, cudaStream_t st) {
    const int nch = (int)((n + CN - 1) / CN);
    const int64_t items = (int64_t)nch * CN * (KPT / 8);
    int64_t blocks = (items + 255) / 256;
    if (blocks > NUM_SMS_HINT * 8) blocks = NUM_SMS_HINT * 8;
    k_v_image<<<(unsigned)blocks, 256, 0, st>>>(V, n, nch, reinterpret_cast<unsigned char *>(img));
    return cudaGetLastError();
}

cudaError_t launch_predict_select_tc(const PredictTcArgs &a, int num_sms, cudaStream_t st) {
    if (a.m <= 0 || a.n <= 0) return cudaSuccess;
    if (a.k > KPT || a.base < 0 || a.base >= a.n) return cudaErrorInvalidValue;
    if (a.select && a.n > PREDICT_TC_CG_MAX && !a.cg_pad) return cudaErrorInvalidValue;
    const int64_t tiles = (a.m + TM - 1) / TM;
    const int grid = (int)(tiles < num_sms ? tiles : num_sms);
    const int64_t npad = (a.n + CN - 1) / CN * CN;
    const size_t smem = OFF_CG + 4 * (a.n <= PREDICT_TC_CG_MAX ? npad : 0);
    k_predict_select_tc<<<grid, NTHREADS, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace ocf
