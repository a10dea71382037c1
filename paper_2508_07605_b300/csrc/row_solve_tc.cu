// Tensor-core masked Gram + Cholesky row solve (one ALS half-step), FP32 path.
//
// Same computation as k_row_solve (row_solve.cu): for every row i of a CSR
// matrix with F the fixed other factor,
//     A_i = sum_{j in Omega_i} f_j f_j^T + lambda I,   b_i = sum_{j in Omega_i} R_ij f_j,
// then A_i = L L^T, L y = b_i, L^T x_i = y  (the per-row ridge solve of ALS;
// Sec. "Collaborative Filtering Model" and "Online Performance Prediction").
//
// The Gram and the right-hand side are small dense contractions over the
// row's observations: with the staged factor rows S (obs x KP),
// A_i = S^T S and b_i = S^T r.  They run on the tensor cores with
// mma.sync.m16n8k8 TF32 in the 3-pass split form (x = hi + lo, both TF32;
// S^T S ~ hi^T hi + hi^T lo + lo^T hi, FP32 accumulation), which keeps FP32
// accuracy (the dropped lo^T lo term is ~2^-22 relative).  The A and B
// fragments of S^T S come from the same staged tile, so each 8-observation
// step costs 4 (KP=16) or 8 (KP=32) shared loads plus 9 or 24 MMAs; only
// the lower-triangle 16x8 blocks are formed.
//
// Mapping: KP in {16, 32}.  With WPS = 1 a warp forms the Grams of SPW =
// 32/KP systems one after another with all 32 lanes, then factorises them in
// parallel, one KP-lane segment per system (lane q owns row q of A).  With
// WPS = 4 a CTA of 4 warps splits one long row's observations, sums the
// partial Grams in a fixed order through shared memory, and warp 0 solves.
// Staging: lane t loads observation t's factor row (16-byte loads) into a
// padded tile (stride KP+8 floats: the fragment loads are conflict-free).
//
// FP64 factorisation at KP = 32 (packed): the B300's FP64 pipe spends the
// same time on a warp instruction whatever the number of active lanes, so
// the cost is the count of FP64 warp instructions, and lane-per-row spends
// two thirds of its update FMAs on the upper triangle.  There a warp forms
// two systems' Grams and factorises both at once, 16 lanes per system, lane i
// holding rows i and 31 - i of the lower triangle in 33 slots (slot e <= i:
// row i, column e; slot e > i: row 31 - i, column 32 - e), so column p of
// either row sits in a slot that does not depend on the lane (p and 32 - p).
// Step p then costs 31 - p FMA instructions for the two systems instead of
// 31 - p for one.  The forward substitution rides along with the
// factorisation (y_p is formed on the pivot step and broadcast with column
// p); the operations and their order are those of the lane-per-row path, so
// both give the same bits.
#include <cuda_bf16.h>
#include <stdint.h>

#include "common.cuh"
#include "kernels.h"
#include "mma_sync.cuh"

namespace ocf {

using namespace sm;

// Per-warp shared memory.  The staging buffers (NST stages of 32 factor
// rows) are dead once the warp's Gram is in registers, so the Gram / factor
// area of the solve phase overlays them: a warp needs max(staging, solve),
// not the sum, which keeps 16 warps per SM resident for KP = 32.
template <int KP, typename TC, bool BF, int NST, int SPW> struct alignas(16) TcSmem {
    // Staged rows padded to KP+8 elements (conflict-free fragment loads,
    // 16-byte aligned rows).  FP32: one tile of 32 rows per buffer.  BF16: the
    // hi and lo halves of each split row go to two tiles of 32 BF16 rows.
    static constexpr int ROWB = (BF ? 2 : 4) * (KP + 8);
    struct alignas(16) Stage {
        alignas(16) unsigned char stage[NST][BF ? 2 : 1][32][ROWB];
        float sr[NST][32];
    };
    struct alignas(16) Seg {
        union {
            float G[KP][KP + 1];   // Gram (lower triangle), then
            TC L[KP][KP + 1];      // the Cholesky factor of the same system
        };
        float b[KP];
        TC col[2][KP + 4];   // column p of L (double-buffered); [KP]: y_p (packed path)
        TC dinv[KP];         // inverse pivots (packed path)
    };
    union {
        Stage ld;
        Seg seg[SPW];
    };
};

// Pipeline depth (items in flight).  Measured on the 4096 x 1024 fit: 3 or 4
// stages do not shorten the U-half (its items wait on the tensor-core chain,
// not on the copies) and cost occupancy, so every configuration uses 2.
template <int KP, int WPS> constexpr int tc_stages() { return 2; }

// The packed FP64 layout (two systems per warp) and systems per warp.
template <int KP, typename TC, int WPS, bool SUMS> constexpr bool tc_pack() {
    return KP == 32 && sizeof(TC) == 8 && WPS == 1 && !SUMS;
}
template <int KP, typename TC, int WPS, bool SUMS> constexpr int tc_spw() {
    return WPS == 1 ? (tc_pack<KP, TC, WPS, SUMS>() ? 2 : 32 / KP) : 1;
}

template <int KP> struct Blocks {
    static constexpr int MB = KP / 16;
    // lower-triangle 16x8 blocks (mb, nb): nb <= 2*mb + 1
    static constexpr int NBLK = (KP == 16) ? 2 : 6;
    __device__ static constexpr int mb_of(int t) { return KP == 16 ? 0 : (t < 2 ? 0 : 1); }
    __device__ static constexpr int nb_of(int t) { return KP == 16 ? t : (t < 2 ? t : t - 2); }
};

// SUMS: this build adds the streaming refit's stored sums (kept out of the
// other builds, where the extra registers cost occupancy).
template <int KP, typename TC, int WPS, bool BF, bool SUMS = false>
__global__ void __launch_bounds__(WPS == 1 ? (sizeof(TC) == 8 && KP == 32 ? 128 : 256) : 32 * WPS)
k_row_solve_tc(SolveArgs<float> a) {
    constexpr int WARPS = (WPS == 1) ? ((sizeof(TC) == 8 && KP == 32) ? 4 : 8) : WPS;
    constexpr bool PACK = tc_pack<KP, TC, WPS, SUMS>();
    constexpr int SPW = tc_spw<KP, TC, WPS, SUMS>();   // systems per warp
    constexpr int MB = Blocks<KP>::MB;
    constexpr int NBLK = Blocks<KP>::NBLK;
    constexpr int NST = tc_stages<KP, WPS>();
    using WS = TcSmem<KP, TC, BF, NST, SPW>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    WS *smem = reinterpret_cast<WS *>(smem_raw);

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int gid = lane >> 2, tid4 = lane & 3;
    const int g = lane / KP, q = lane % KP;
    WS &W = smem[warp];
    const int64_t sys0 = (WPS == 1) ? ((int64_t)blockIdx.x * WARPS + warp) * SPW
                                    : (int64_t)blockIdx.x;
    const int64_t sys_stride = (WPS == 1) ? (int64_t)gridDim.x * WARPS * SPW
                                          : (int64_t)gridDim.x;
    pdl_trigger();
    if (a.m_dev || a.row_map) pdl_wait();         // the list comes from the preceding kernel
    const int64_t M = a.m_dev ? *a.m_dev : a.m;   // systems (a device count for compacted lists)

    for (int64_t base = sys0; base < M; base += sys_stride) {
        // ---------------- Gram phase -------------------------------------
        // The warp's work is a list of 32-observation items: the chunks of
        // its SPW systems in order (WPS = 1), or this warp's slice of the
        // chunks of one long system (WPS > 1).  Items are software-pipelined:
        // item w+1's factor rows stream into the other stage buffer with
        // cp.async (zero-filled past the row end) while item w is on the
        // tensor cores, and column indices are fetched two items ahead.
        int64_t beg_s[SPW], s_s[SPW];
        bool bad_s[SPW];
        int nch[SPW];
        int nitems = 0;
#pragma unroll
        for (int si = 0; si < SPW; ++si) {
            const int64_t i = base + si;
            int64_t beg = 0, end = 0;
            bad_s[si] = false;
            if (i < M) bad_s[si] = !row_bounds(a.ptr, a.row_map ? a.row_map[i] : i, a.nnz, beg, end);
            beg_s[si] = beg;
            s_s[si] = end - beg;
            if (WPS == 1) {
                nch[si] = (int)((s_s[si] + 31) / 32);
            } else {
                const int64_t all = (s_s[si] + 31) / 32;   // chunks of the system
                nch[si] = (int)((all > warp) ? (all - warp + WPS - 1) / WPS : 0);
            }
            nitems += nch[si];
        }
        // item w -> (system, first observation)
        auto item = [&](int w, int &si, int64_t &c0) {
            si = 0;
            if (SPW == 2 && w >= nch[0]) {
                w -= nch[0];
                si = 1;
            }
            c0 = (WPS == 1) ? (int64_t)w * 32 : ((int64_t)w * WPS + warp) * 32;
        };
        bool badf[SPW];
#pragma unroll
        for (int si = 0; si < SPW; ++si) badf[si] = false;
        auto load_idx = [&](int w) -> int32_t {
            int si; int64_t c0;
            item(w, si, c0);
            int64_t bg = 0, ss = 0;
#pragma unroll
            for (int t = 0; t < SPW; ++t) if (t == si) { bg = beg_s[t]; ss = s_s[t]; }
            const int64_t tt = c0 + lane;
            int32_t j = 0;
            if (tt < ss) {
                j = __ldg(a.idx + bg + tt);
                if (j < 0 || (int64_t)j >= a.n_other) {
#pragma unroll
                    for (int t = 0; t < SPW; ++t) if (t == si) badf[t] = true;
                    j = 0;
                }
            }
            return j;
        };
        auto issue = [&](int w, int32_t j, int buf) {
            int si; int64_t c0;
            item(w, si, c0);
            int64_t bg = 0, ss = 0;
#pragma unroll
            for (int t = 0; t < SPW; ++t) if (t == si) { bg = beg_s[t]; ss = s_s[t]; }
            const int64_t tt = c0 + lane;
            const bool v = tt < ss;
            if constexpr (BF) {
                // split row [hi (KP bf16) | lo (KP bf16)] -> hi tile, lo tile
                const unsigned char *src =
                    reinterpret_cast<const unsigned char *>(a.Fb) + (int64_t)j * KP * 4;
                constexpr int NCP = 2 * KP / 16;
#pragma unroll
                for (int e = 0; e < NCP; ++e) {
                    cp_async16(&W.ld.stage[buf][0][lane][16 * e], src + 16 * e, v ? 16 : 0);
                    cp_async16(&W.ld.stage[buf][1][lane][16 * e], src + 2 * KP + 16 * e, v ? 16 : 0);
                }
            } else {
                const unsigned char *src =
                    reinterpret_cast<const unsigned char *>(a.F + (int64_t)j * KP);
                constexpr int NCP = 4 * KP / 16;
#pragma unroll
                for (int e = 0; e < NCP; ++e)
                    cp_async16(&W.ld.stage[buf][0][lane][16 * e], src + 16 * e, v ? 16 : 0);
            }
            cp_async4(&W.ld.sr[buf][lane], v ? (const void *)(a.val + bg + tt) : (const void *)a.val,
                      v ? 4 : 0);
        };

        float d[SPW][NBLK][4], dr[SPW][MB][4];
#pragma unroll
        for (int si = 0; si < SPW; ++si) {
#pragma unroll
            for (int t = 0; t < NBLK; ++t)
#pragma unroll
                for (int e = 0; e < 4; ++e) d[si][t][e] = 0.0f;
#pragma unroll
            for (int mb = 0; mb < MB; ++mb)
#pragma unroll
                for (int e = 0; e < 4; ++e) dr[si][mb][e] = 0.0f;
        }
        pdl_wait();   // from here on the other factor is read
        if (nitems > 0) {
            // NST - 1 items in flight ahead of the one on the tensor cores; the
            // column indices of the next NST - 1 items wait in registers (jr).
            int32_t jr[NST - 1];
            issue(0, load_idx(0), 0);
            cp_async_commit();
#pragma unroll
            for (int t = 0; t < NST - 1; ++t) jr[t] = (1 + t < nitems) ? load_idx(1 + t) : 0;
#pragma unroll
            for (int p = 1; p < NST - 1; ++p) {
                if (p < nitems) issue(p, jr[0], p);
                cp_async_commit();
#pragma unroll
                for (int t = 0; t < NST - 2; ++t) jr[t] = jr[t + 1];
                jr[NST - 2] = (p + NST - 1 < nitems) ? load_idx(p + NST - 1) : 0;
            }
            for (int w = 0; w < nitems; ++w) {
                const int wn = w + NST - 1;
                if (wn < nitems) issue(wn, jr[0], wn % NST);
                cp_async_commit();
#pragma unroll
                for (int t = 0; t < NST - 2; ++t) jr[t] = jr[t + 1];
                jr[NST - 2] = (wn + NST - 1 < nitems) ? load_idx(wn + NST - 1) : 0;
                cp_async_wait<NST - 1>();
                __syncwarp();
                int si; int64_t c0;
                item(w, si, c0);
                int64_t ss = 0;
#pragma unroll
                for (int t = 0; t < SPW; ++t) if (t == si) ss = s_s[t];
                const int buf = w % NST;
                const int cnt = (int)min((int64_t)32, ss - c0);
                if constexpr (BF) {
                    // 16 observations per MMA step; fragments of the hi (H) and lo (L)
                    // tiles from ldmatrix.trans.  S^T S ~ H^T H + H^T L + L^T H and
                    // S^T r ~ H^T r_h + H^T r_l + L^T r_h: ~16-bit operands.
                    const int nks = (cnt + 15) / 16;
                    const __nv_bfloat16 *sH =
                        reinterpret_cast<const __nv_bfloat16 *>(&W.ld.stage[buf][0][0][0]);
                    const __nv_bfloat16 *sL =
                        reinterpret_cast<const __nv_bfloat16 *>(&W.ld.stage[buf][1][0][0]);
                    constexpr int LDE = WS::ROWB / 2;
                    const int mi = lane >> 3, rr = lane & 7;
                    for (int ks = 0; ks < nks; ++ks) {
                        const int k0 = ks * 16;
                        uint32_t aH[MB][4], aL[MB][4];
#pragma unroll
                        for (int mb = 0; mb < MB; ++mb) {
                            const int off = (k0 + (mi >> 1) * 8 + rr) * LDE + mb * 16 + (mi & 1) * 8;
                            ldsm_x4_trans(aH[mb], sH + off);
                            ldsm_x4_trans(aL[mb], sL + off);
                        }
                        float r0 = 0.f, r1 = 0.f, r2 = 0.f, r3 = 0.f;
                        if (gid == 0) {
                            r0 = W.ld.sr[buf][k0 + 2 * tid4];
                            r1 = W.ld.sr[buf][k0 + 2 * tid4 + 1];
                            r2 = W.ld.sr[buf][k0 + 2 * tid4 + 8];
                            r3 = W.ld.sr[buf][k0 + 2 * tid4 + 9];
                        }
                        const float h0 = __bfloat162float(__float2bfloat16_rn(r0));
                        const float h1 = __bfloat162float(__float2bfloat16_rn(r1));
                        const float h2 = __bfloat162float(__float2bfloat16_rn(r2));
                        const float h3 = __bfloat162float(__float2bfloat16_rn(r3));
                        const uint32_t rh0 = pack_bf16(h0, h1), rh1 = pack_bf16(h2, h3);
                        const uint32_t rl0 = pack_bf16(r0 - h0, r1 - h1);
                        const uint32_t rl1 = pack_bf16(r2 - h2, r3 - h3);
#pragma unroll
                        for (int sx = 0; sx < SPW; ++sx) {
                            if (sx != si) continue;
#pragma unroll
                            for (int ps = 0; ps < 3; ++ps) {   // pass-major, as above
#pragma unroll
                                for (int tb = 0; tb < NBLK; ++tb) {
                                    const int mb = Blocks<KP>::mb_of(tb), nb = Blocks<KP>::nb_of(tb);
                                    const int sm = nb >> 1, h = nb & 1;
                                    const uint32_t *bsrc = (ps == 1) ? aL[sm] : aH[sm];
                                    mma_bf16(d[sx][tb], ps == 0 ? aL[mb] : aH[mb], bsrc[h],
                                             bsrc[2 + h]);
                                }
#pragma unroll
                                for (int mb = 0; mb < MB; ++mb)
                                    mma_bf16(dr[sx][mb], ps == 0 ? aL[mb] : aH[mb],
                                             ps == 1 ? rl0 : rh0, ps == 1 ? rl1 : rh1);
                            }
                        }
                    }
                } else {
                const int nks = (cnt + 7) / 8;
                const float *stf = reinterpret_cast<const float *>(&W.ld.stage[buf][0][0][0]);
                constexpr int LDF = WS::ROWB / 4;
                for (int ks = 0; ks < nks; ++ks) {
                    const int k0 = ks * 8;
                    uint32_t ah[MB][4], al[MB][4];
#pragma unroll
                    for (int mb = 0; mb < MB; ++mb) {
                        split_tf32(stf[(k0 + tid4) * LDF + mb * 16 + gid], ah[mb][0], al[mb][0]);
                        split_tf32(stf[(k0 + tid4) * LDF + mb * 16 + gid + 8], ah[mb][1],
                                   al[mb][1]);
                        split_tf32(stf[(k0 + tid4 + 4) * LDF + mb * 16 + gid], ah[mb][2],
                                   al[mb][2]);
                        split_tf32(stf[(k0 + tid4 + 4) * LDF + mb * 16 + gid + 8], ah[mb][3],
                                   al[mb][3]);
                    }
                    uint32_t rh0, rl0, rh1, rl1;
                    split_tf32(gid == 0 ? W.ld.sr[buf][k0 + tid4] : 0.0f, rh0, rl0);
                    split_tf32(gid == 0 ? W.ld.sr[buf][k0 + tid4 + 4] : 0.0f, rh1, rl1);
#pragma unroll
                    for (int sx = 0; sx < SPW; ++sx) {
                        if (sx != si) continue;   // warp-uniform: accumulators stay in registers
                        // pass-major order: consecutive MMAs go to different
                        // accumulators, so the three passes of one block do not
                        // wait on each other back to back
#pragma unroll
                        for (int ps = 0; ps < 3; ++ps) {
#pragma unroll
                            for (int tb = 0; tb < NBLK; ++tb) {
                                const int mb = Blocks<KP>::mb_of(tb), nb = Blocks<KP>::nb_of(tb);
                                const int src_mb = nb >> 1, h = nb & 1;
                                const uint32_t *bsrc = (ps == 1) ? al[src_mb] : ah[src_mb];
                                mma_tf32(d[sx][tb], ps == 0 ? al[mb] : ah[mb], bsrc[h], bsrc[2 + h]);
                            }
#pragma unroll
                            for (int mb = 0; mb < MB; ++mb)
                                mma_tf32(dr[sx][mb], ps == 0 ? al[mb] : ah[mb],
                                         ps == 1 ? rl0 : rh0, ps == 1 ? rl1 : rh1);
                        }
                    }
                }
                }
                __syncwarp();   // this buffer is refilled NST items later
            }
        }
        cp_async_wait<0>();   // nothing in flight before the solve area overlays the stages
        __syncwarp();
        // fragments -> shared Gram (lower-triangle blocks) and RHS
#pragma unroll
        for (int si = 0; si < SPW; ++si) {
            float (*G)[KP + 1] = W.seg[si].G;
#pragma unroll
            for (int tb = 0; tb < NBLK; ++tb) {
                const int mb = Blocks<KP>::mb_of(tb), nb = Blocks<KP>::nb_of(tb);
                const int r0 = mb * 16 + gid, c = nb * 8 + 2 * tid4;
                G[r0][c] = d[si][tb][0];
                G[r0][c + 1] = d[si][tb][1];
                G[r0 + 8][c] = d[si][tb][2];
                G[r0 + 8][c + 1] = d[si][tb][3];
            }
            if (tid4 == 0) {
#pragma unroll
                for (int mb = 0; mb < MB; ++mb) {
                    W.seg[si].b[mb * 16 + gid] = dr[si][mb][0];
                    W.seg[si].b[mb * 16 + gid + 8] = dr[si][mb][2];
                }
            }
        }
        // an out-of-range column flags only the system it was read for
#pragma unroll
        for (int si = 0; si < SPW; ++si) bad_s[si] = bad_s[si] || (__any_sync(FULL, badf[si]) != 0);
        if constexpr (WPS > 1) {
            bad_s[0] = __syncthreads_or(bad_s[0]) != 0;
        } else {
            __syncwarp();
        }

        if constexpr (PACK) {
            // ------------- solve phase, packed: 16 lanes per system ------------
            const int sp = lane >> 4;   // system of this half-warp
            const int i = lane & 15;    // its rows i and 31 - i
            const int r2 = 31 - i;
            auto &S = W.seg[sp];
            bool bad = false;
            int64_t s = 0;
#pragma unroll
            for (int si = 0; si < SPW; ++si)
                if (si == sp) {
                    bad = bad_s[si];
                    s = s_s[si];
                }
            const double lam = double(a.lambda) * (a.wr ? double(s) : 1.0);   // weighted: lambda s_i
            const double d1 = double(S.G[i][i]) + lam, d2 = double(S.G[r2][r2]) + lam;
            double A[33];
#pragma unroll
            for (int e = 0; e < 33; ++e) {
                const bool first = e <= i;
                const double g = double(S.G[first ? i : r2][first ? e : 32 - e]);
                A[e] = (e == i) ? d1 : (e == i + 1) ? d2 : g;   // the two diagonals
            }
            double y1 = double(S.b[i]), y2 = double(S.b[r2]);
            __syncwarp();   // every lane has read G before L overwrites it
#pragma unroll
            for (int p = 0; p < 32; ++p) {
                // pivot: row p, on lane p (first row) or lane 31 - p (second row)
                const double piv = __shfl_sync(FULL, p <= 15 ? A[p] : A[32 - p], p <= 15 ? p : 31 - p, 16);
                const double inv = rsq(piv);
                const bool on1 = p <= 15 && i >= p;   // row i reaches column p
                const bool on2 = i <= 31 - p;         // row 31 - i reaches column p
                if (on1) A[p] = A[p] * inv;
                if (on2) A[32 - p] = A[32 - p] * inv;
                double *cb = S.col[p & 1];
                if (on1) cb[i] = A[p];
                if (on2) cb[r2] = A[32 - p];
                if (p <= 15) {
                    if (i == p) { y1 = y1 * inv; cb[32] = y1; }
                } else {
                    if (i == 31 - p) { y2 = y2 * inv; cb[32] = y2; }
                }
                if (i == 0) S.dinv[p] = inv;
                __syncwarp();
                const double f1 = p <= 15 ? A[p] : 0.0, f2 = A[32 - p];
                const double yp = cb[32];
                if (p <= 15 && i > p) y1 = fma(-f1, yp, y1);
                if (r2 > p) y2 = fma(-f2, yp, y2);
#pragma unroll
                for (int e = 1; e < 33; ++e) {
                    const bool up1 = e > p;        // first-row slot e: column e
                    const bool up2 = e < 32 - p;   // second-row slot e: column 32 - e
                    if (up1 && up2) {
                        const bool first = e <= i;
                        A[e] = fma(-(first ? f1 : f2), cb[first ? e : 32 - e], A[e]);
                    } else if (up2) {
                        if (e > i) A[e] = fma(-f2, cb[32 - e], A[e]);
                    } else if (up1) {
                        if (e <= i) A[e] = fma(-f1, cb[e], A[e]);
                    }
                }
            }
            // L to shared memory (row-major) for the back substitution
#pragma unroll
            for (int e = 0; e < 33; ++e) {
                const bool first = e <= i;
                S.L[first ? i : r2][first ? e : 32 - e] = A[e];
            }
            __syncwarp();
            // back substitution L^T x = y
            double x1 = y1, x2 = y2;
#pragma unroll
            for (int p = 31; p >= 0; --p) {
                const double xp = __shfl_sync(FULL, p <= 15 ? x1 : x2, p <= 15 ? p : 31 - p, 16) *
                                  S.dinv[p];
                if (i < p) x1 = fma(-S.L[p][i], xp, x1);
                if (r2 < p) x2 = fma(-S.L[p][r2], xp, x2);
            }
            x1 = x1 * S.dinv[i];
            x2 = x2 * S.dinv[r2];
            bool fail = !isfinite(x1) || !isfinite(x2);
#pragma unroll
            for (int off = 1; off < 16; off <<= 1)
                fail |= __shfl_xor_sync(FULL, (int)fail, off) != 0;
            const int64_t is = base + sp;
            if (is < M) {
                const int64_t io = a.row_map ? a.row_map[is] : is;
                int32_t st = ST_OK;
                if (bad) st = ST_BAD;
                else if (s == 0) st = ST_EMPTY;
                else if (fail) st = ST_NOT_SPD;
                if (st != ST_OK) x1 = x2 = 0.0;
                if (i < a.kout) a.out[io * a.ldo + i] = (float)x1;
                if (r2 < a.kout) a.out[io * a.ldo + r2] = (float)x2;
                if (a.outb) {   // split BF16 copy [hi | lo] of the output row
                    __nv_bfloat16 *ob = reinterpret_cast<__nv_bfloat16 *>(a.outb) + io * 2 * KP;
                    const float xf1 = (float)x1, xf2 = (float)x2;
                    const __nv_bfloat16 h1 = __float2bfloat16_rn(xf1), h2 = __float2bfloat16_rn(xf2);
                    ob[i] = h1;
                    ob[KP + i] = __float2bfloat16_rn(xf1 - __bfloat162float(h1));
                    ob[r2] = h2;
                    ob[KP + r2] = __float2bfloat16_rn(xf2 - __bfloat162float(h2));
                }
                if (a.status && i == 0) a.status[io] = st;
            }
            __syncwarp();
            continue;
        }

        // ---------------- solve phase: one KP-lane segment per system --------
        const int slot = (WPS == 1) ? g : 0;
        bool bad = false;
        int64_t s = 0;
#pragma unroll
        for (int si = 0; si < SPW; ++si)
            if (si == slot) {
                bad = bad_s[si];
                s = s_s[si];
            }
        if (WPS == 1 || warp == 0) {
            auto &S = W.seg[slot];
            const bool writer = (WPS == 1) || g == 0;
            TC A[KP];
            TC bt;
            if constexpr (WPS > 1) {
#pragma unroll
                for (int e = 0; e < KP; ++e) A[e] = TC(smem[0].seg[0].G[q][e]);
                bt = TC(smem[0].seg[0].b[q]);
                for (int w = 1; w < WPS; ++w) {
#pragma unroll
                    for (int e = 0; e < KP; ++e) A[e] += TC(smem[w].seg[0].G[q][e]);
                    bt += TC(smem[w].seg[0].b[q]);
                }
            } else {
#pragma unroll
                for (int e = 0; e < KP; ++e) A[e] = TC(S.G[q][e]);
                bt = TC(S.b[q]);
            }
            if (SUMS && !bad && base + slot < M) {   // streaming: stored sums of earlier rows
                const int64_t i = a.row_map ? a.row_map[base + slot] : base + slot;
                float *gq = a.gram + (i * KP + q) * KP;
#pragma unroll
                for (int e = 0; e < KP; ++e) A[e] += TC(gq[e]);
                bt += TC(a.gram_b[i * KP + q]);
                s += a.gram_n[i];
                if (a.gram_keep && writer) {
#pragma unroll
                    for (int e = 0; e < KP; ++e) gq[e] = (float)A[e];
                    a.gram_b[i * KP + q] = (float)bt;
                    if (q == 0) a.gram_n[i] = s;
                }
            }
            const TC lam = TC(a.lambda) * (a.wr ? TC(s) : TC(1));   // weighted: lambda s_i
#pragma unroll
            for (int e = 0; e < KP; ++e)
                if (e == q) A[e] += lam;
            __syncwarp();   // every lane has read G before L overwrites it

            // Right-looking Cholesky, lane q owning row q.  l = A[q][p] / sqrt(piv)
            // for every lane (the pivot lane gets sqrt(piv) itself); a pivot that
            // is not > 0 turns the solution non-finite, which flags the row.
            TC dv[KP];
            TC myinv = TC(0);
#pragma unroll
            for (int p = 0; p < KP; ++p) {
                const TC piv = __shfl_sync(FULL, A[p], p, KP);
                const TC inv = rsq(piv);
                dv[p] = inv;
                if (q == p) myinv = inv;
                const TC l = A[p] * inv;
                A[p] = l;
                TC *cb = S.col[p & 1];
                if (writer) cb[q] = l;
                __syncwarp();
                constexpr int VN = 16 / (int)sizeof(TC);
#pragma unroll
                for (int r4 = ((p + 1) / VN) * VN; r4 < KP; r4 += VN) {
                    if constexpr (VN == 4) {
                        const float4 x = *reinterpret_cast<const float4 *>(cb + r4);
                        const TC xs[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
                        for (int e = 0; e < 4; ++e)
                            if (r4 + e > p) A[r4 + e] = my_fma(-l, xs[e], A[r4 + e]);
                    } else {
                        const double2 x = *reinterpret_cast<const double2 *>(cb + r4);
                        const TC xs[2] = {(TC)x.x, (TC)x.y};
#pragma unroll
                        for (int e = 0; e < 2; ++e)
                            if (r4 + e > p) A[r4 + e] = my_fma(-l, xs[e], A[r4 + e]);
                    }
                }
            }
            // forward substitution L y = b: after step q, y on lane q is final
            TC y = bt;
#pragma unroll
            for (int p = 0; p < KP; ++p) {
                const TC yp = __shfl_sync(FULL, y, p, KP) * dv[p];
                if (q > p) y = my_fma(-A[p], yp, y);
            }
            const TC yq = y * myinv;
            if (writer) {
#pragma unroll
                for (int e = 0; e < KP; ++e) S.L[q][e] = A[e];
            }
            __syncwarp();
            // back substitution L^T x = y
            TC x = yq;
#pragma unroll
            for (int p = KP - 1; p >= 0; --p) {
                const TC xp = __shfl_sync(FULL, x, p, KP) * dv[p];
                if (q < p) x = my_fma(-S.L[p][q], xp, x);
            }
            TC xq = x * myinv;
            bool fail = !isfinite(xq);
#pragma unroll
            for (int off = 1; off < KP; off <<= 1)
                fail |= __shfl_xor_sync(FULL, (int)fail, off) != 0;
            const int64_t is = base + slot;
            if (writer && is < M) {
                const int64_t i = a.row_map ? a.row_map[is] : is;
                int32_t st = ST_OK;
                if (bad) st = ST_BAD;
                else if (s == 0) st = ST_EMPTY;
                else if (fail) st = ST_NOT_SPD;
                if (st != ST_OK) xq = TC(0);
                if (q < a.kout) a.out[i * a.ldo + q] = (float)xq;
                if (a.outb) {   // split BF16 copy [hi | lo] of the output row
                    const float xf = (float)xq;
                    const __nv_bfloat16 hi = __float2bfloat16_rn(xf);
                    __nv_bfloat16 *ob = reinterpret_cast<__nv_bfloat16 *>(a.outb) + i * 2 * KP;
                    ob[q] = hi;
                    ob[KP + q] = __float2bfloat16_rn(xf - __bfloat162float(hi));
                }
                if (a.status && q == 0) a.status[i] = st;
            }
            __syncwarp();
        }
        if constexpr (WPS > 1) __syncthreads();
    }
}

template <int KP, typename TC, int WPS, bool BF, bool SUMS> static size_t tc_smem_bytes() {
    constexpr int WARPS = (WPS == 1) ? ((sizeof(TC) == 8 && KP == 32) ? 4 : 8) : WPS;
    return sizeof(TcSmem<KP, TC, BF, tc_stages<KP, WPS>(), tc_spw<KP, TC, WPS, SUMS>()>) * WARPS;
}

template <int KP, typename TC, int WPS, bool BF> static cudaError_t tc_attr() {
    cudaError_t e = cudaFuncSetAttribute(k_row_solve_tc<KP, TC, WPS, BF, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)tc_smem_bytes<KP, TC, WPS, BF, false>());
    if (e != cudaSuccess || BF) return e;
    return cudaFuncSetAttribute(k_row_solve_tc<KP, TC, WPS, false, true>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)tc_smem_bytes<KP, TC, WPS, BF, true>());
}

template <bool BF> static cudaError_t tc_attrs() {
    cudaError_t e;
    if ((e = tc_attr<16, float, 1, BF>()) != cudaSuccess) return e;
    if ((e = tc_attr<32, float, 1, BF>()) != cudaSuccess) return e;
    if ((e = tc_attr<16, float, 4, BF>()) != cudaSuccess) return e;
    if ((e = tc_attr<32, float, 4, BF>()) != cudaSuccess) return e;
    if ((e = tc_attr<16, double, 1, BF>()) != cudaSuccess) return e;
    if ((e = tc_attr<32, double, 1, BF>()) != cudaSuccess) return e;
    if ((e = tc_attr<16, double, 4, BF>()) != cudaSuccess) return e;
    return tc_attr<32, double, 4, BF>();
}

cudaError_t prepare_row_solve_tc() {
    cudaError_t e = tc_attrs<false>();
    if (e != cudaSuccess) return e;
    return tc_attrs<true>();
}

constexpr int64_t LONG_ROW_TC = 96;   // mean observations per row that warrant 4 warps

template <typename K>
static cudaError_t launch_pdl(K kernel, unsigned grid, unsigned block, size_t smem,
                              cudaStream_t st, const SolveArgs<float> &a) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, a);
}

template <int KP, typename TC, bool BF, bool SUMS>
static cudaError_t launch_tc_kp(const SolveArgs<float> &a, cudaStream_t st) {
    if (a.nnz >= LONG_ROW_TC * a.m) {
        int64_t blocks = a.m;
        if (blocks > NUM_SMS_HINT * 64) blocks = NUM_SMS_HINT * 64;
        return launch_pdl(k_row_solve_tc<KP, TC, 4, BF, SUMS>, (unsigned)blocks, 128,
                          tc_smem_bytes<KP, TC, 4, BF, SUMS>(), st, a);
    }
    // one system per warp at rank 32 with an FP32 factorisation: the packed
    // FP32x2 solver of solve32_tc.cu
    if constexpr (KP == 32 && sizeof(TC) == 4 && !SUMS) return launch_solve32_tc(a, BF, st);
    constexpr int WARPS = (sizeof(TC) == 8 && KP == 32) ? 4 : 8;
    const int64_t per = (int64_t)WARPS * tc_spw<KP, TC, 1, SUMS>();
    int64_t blocks = (a.m + per - 1) / per;
    if (blocks > NUM_SMS_HINT * 32) blocks = NUM_SMS_HINT * 32;
    return launch_pdl(k_row_solve_tc<KP, TC, 1, BF, SUMS>, (unsigned)blocks, WARPS * 32,
                      tc_smem_bytes<KP, TC, 1, BF, SUMS>(), st, a);
}

template <bool BF, bool SUMS>
static cudaError_t launch_tc_bf(const SolveArgs<float> &a, int KP, bool chol_fp64,
                                cudaStream_t st) {
    if (KP == 16)
        return chol_fp64 ? launch_tc_kp<16, double, BF, SUMS>(a, st)
                         : launch_tc_kp<16, float, BF, SUMS>(a, st);
    if (KP == 32)
        return chol_fp64 ? launch_tc_kp<32, double, BF, SUMS>(a, st)
                         : launch_tc_kp<32, float, BF, SUMS>(a, st);
    return cudaErrorInvalidValue;
}

cudaError_t launch_row_solve_tc(const SolveArgs<float> &a, int KP, bool chol_fp64, bool bf16,
                                cudaStream_t st) {
    if (a.m <= 0) return cudaSuccess;
    if (bf16 && !a.Fb) return cudaErrorInvalidValue;
    if (bf16 && a.gram) return cudaErrorInvalidValue;   // the streaming refit is FP32 / FP64 only
    if (a.resid || a.refine || a.u_given) {   // residual / refinement: rank-32 FP32 solver only
        if (KP != 32 || chol_fp64) return cudaErrorInvalidValue;
        return launch_solve32_tc(a, bf16, st);
    }
    if (bf16) return launch_tc_bf<true, false>(a, KP, chol_fp64, st);
    return a.gram ? launch_tc_bf<false, true>(a, KP, chol_fp64, st)
                  : launch_tc_bf<false, false>(a, KP, chol_fp64, st);
}

}  // namespace ocf
