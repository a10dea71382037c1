// Batched ALS: thousands of independent completion problems of uneven size
// (each its own applications x settings matrix, rank and observations) fitted
// in one persistent launch.
//
// Each problem is the ALS fit of Sec. "Collaborative Filtering Model" /
// "Online Performance Prediction" (see row_solve.cu): sweeps of a U-half and a
// V-half of ridge row solves.  Problems are independent, so they are spread
// over the GPU as whole units:
//   * the host sorts problems by estimated cost (largest first, LPT) and cuts
//     them into classes ("large", "small");
//   * a CTA of 8 warps is split into groups of W warps (W per class, chosen by
//     the autotuner); a group takes the next problem of the class from an
//     atomic queue and runs every sweep of it, synchronising its warps with a
//     named barrier; no CTA ever waits on another CTA;
//   * per problem, the group first builds the problem's CSC copy (stable
//     counting sort with per-column row bitmasks, as in transpose.cu) in
//     workspace memory, then alternates U- and V-half-steps, one system per
//     warp with the shared warp-level solve (solve_warp.cuh).
#include "common.cuh"
#include "kernels.h"
#include "packed_tri.cuh"
#include "solve_warp.cuh"

namespace ocf {

constexpr int BW = 8;   // warps per CTA

__device__ __forceinline__ void group_sync(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(nthreads) : "memory");
}

// Largest per-warp solve workspace (KP = 32), reused for smaller KP and for
// the CSC build (2 * n_max words per group fit in one warp's area).
using WS32 = WarpSmem<float, float, 32>;
static_assert(sizeof(WS32) >= 2 * 1024 * 4, "CSC scratch must fit one warp's area");

// Rank-32 systems two per warp (the fold-in solver's layout): half h of the
// warp solves system i0 + h, lane i accumulating rows i and i + 16 of its
// Gram directly in registers (16 + 32 values: row i never needs a column >= 16)
// from staged factor rows, 16 observations per half and round; lambda joins
// the diagonal when the pivot is broadcast; right-looking Cholesky with the
// column of L through shared memory (packed by columns), packed FP32x2 trailing
// updates, forward substitution on the pivot steps, back substitution from
// columns i and i + 16 in registers.
struct alignas(16) PairSmem32 {
    static constexpr int SROW = 36, SHALF = 16 * SROW + 16;   // half 1 starts 16 banks on
    static constexpr int LS = pk::NCOLP + 16, XS = 48;
    float stage[2 * SHALF];
    float sr[32];
    float L[2 * LS];
    float inv[2 * XS];
};
static_assert(sizeof(PairSmem32) <= sizeof(WarpSmem<float, float, 32>), "pair area fits a warp's area");

__device__ __forceinline__ void solve_pair32(const SolveArgs<float> &a, int64_t i0,
                                             PairSmem32 &W, int lane, int co_i, int co_i16) {
    using namespace pk;
    const int h = lane >> 4, i = lane & 15;
    const int64_t is = i0 + h;
    int64_t beg = 0, end = 0;
    bool bad = false;
    if (is < a.m) bad = !row_bounds(a.ptr, is, a.nnz, beg, end);
    const int64_t s = end - beg;
    const int64_t smax = max(s, (int64_t)__shfl_xor_sync(FULL, (long long)s, 16));
    float a0[16], a1[KP], b0 = 0.f, b1 = 0.f;
#pragma unroll
    for (int e = 0; e < 16; ++e) a0[e] = 0.f;
#pragma unroll
    for (int e = 0; e < KP; ++e) a1[e] = 0.f;
    float *st = W.stage + h * PairSmem32::SHALF;
    // ---- Gram + right-hand side, 16 observations of each system per round
    for (int64_t c0 = 0; c0 < smax; c0 += 16) {
        const int64_t t = c0 + i;
        float4 *dst = reinterpret_cast<float4 *>(st + i * PairSmem32::SROW);
        float r = 0.f;
        if (t < s) {
            int32_t j = __ldg(a.idx + beg + t);
            r = __ldg(a.val + beg + t);
            if (j < 0 || (int64_t)j >= a.n_other) {
                bad = true;
                j = 0;
                r = 0.f;
            }
            const float4 *src = reinterpret_cast<const float4 *>(a.F + (int64_t)j * KP);
#pragma unroll
            for (int e4 = 0; e4 < KP / 4; ++e4) dst[e4] = __ldg(src + e4);
        } else {
#pragma unroll
            for (int e4 = 0; e4 < KP / 4; ++e4) dst[e4] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        W.sr[lane] = r;
        __syncwarp();
        const int cnt = (int)min((int64_t)16, smax - c0);
        for (int tt = 0; tt < cnt; ++tt) {
            const float *x = st + tt * PairSmem32::SROW;
            const float fi = x[i], fi16 = x[i + 16], rr = W.sr[16 * h + tt];
            const float4 *x4 = reinterpret_cast<const float4 *>(x);
#pragma unroll
            for (int e4 = 0; e4 < KP / 4; ++e4) {
                const float4 v = x4[e4];
                if (e4 < 4) {
                    fma_pair(a0[4 * e4], a0[4 * e4 + 1], fi, v.x, v.y);
                    fma_pair(a0[4 * e4 + 2], a0[4 * e4 + 3], fi, v.z, v.w);
                }
                fma_pair(a1[4 * e4], a1[4 * e4 + 1], fi16, v.x, v.y);
                fma_pair(a1[4 * e4 + 2], a1[4 * e4 + 3], fi16, v.z, v.w);
            }
            b0 = fmaf(rr, fi, b0);
            b1 = fmaf(rr, fi16, b1);
        }
        __syncwarp();   // the stage is rewritten next round
    }
    bad = (__ballot_sync(FULL, bad) >> (16 * h)) & 0xffffu;
    // ---- Cholesky with the forward substitution (lambda added to each pivot)
    const float lam = a.wr ? (float)a.lambda * (float)(int)s : (float)a.lambda;   // weighted: lambda s_i
    float *SL = W.L + h * PairSmem32::LS;
    float y0 = b0, y1 = b1;
#pragma unroll
    for (int p = 0; p < KP; ++p) {
        const float piv = (p < 16 ? __shfl_sync(FULL, a0[p & 15], p, 16)
                                  : __shfl_sync(FULL, a1[p], p - 16, 16)) + lam;
        const float inv = rsqrtf(piv);
        float *Lc = SL + coloff(p) - colbase(p);   // Lc[r] = L[r][p]
        float l0 = 0.f;
        if (p < 16) {
            l0 = a0[p & 15] * inv;
            a0[p & 15] = l0;
            if (i >= colbase(p)) Lc[i] = l0;
        }
        const float l1 = a1[p] * inv;
        a1[p] = l1;
        if (colbase(p) <= 16 || i + 16 >= colbase(p)) Lc[i + 16] = l1;
        if (i == 0) W.inv[h * PairSmem32::XS + p] = inv;
        const float yp = (p < 16 ? __shfl_sync(FULL, y0, p, 16)
                                 : __shfl_sync(FULL, y1, p - 16, 16)) * inv;
        if (p < 16) {
            if (i > p) y0 = fmaf(-l0, yp, y0);
            y1 = fmaf(-l1, yp, y1);
        } else {
            if (i + 16 > p) y1 = fmaf(-l1, yp, y1);
        }
        __syncwarp();
#pragma unroll
        for (int r4 = ((p + 1) / 4) * 4; r4 < KP; r4 += 4) {
            const float4 c4 = *reinterpret_cast<const float4 *>(Lc + r4);
            const float cv[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
            for (int e = 0; e < 4; e += 2) {
                const int r = r4 + e;
                if (r > p) {
                    fma2_sub(a1[r], a1[r + 1], l1, cv[e], cv[e + 1]);
                    if (p < 16 && r < 16) fma2_sub(a0[r & 15], a0[(r + 1) & 15], l0, cv[e], cv[e + 1]);
                } else if (r + 1 > p) {
                    a1[r + 1] = fmaf(-l1, cv[e + 1], a1[r + 1]);
                    if (p < 16 && r + 1 < 16) a0[(r + 1) & 15] = fmaf(-l0, cv[e + 1], a0[(r + 1) & 15]);
                }
            }
        }
    }
    const float inv0 = W.inv[h * PairSmem32::XS + i], inv1 = W.inv[h * PairSmem32::XS + i + 16];
    // ---- back substitution L^T x = y
    const float2 xx = back_subst(SL, i, co_i, co_i16, y0 * inv0, y1 * inv1, inv0, inv1);
    float x0 = xx.x, x1 = xx.y;
    const unsigned fb = __ballot_sync(FULL, !isfinite(x0) || !isfinite(x1));
    const bool fail = ((fb >> (16 * h)) & 0xffffu) != 0u;
    if (is < a.m) {
        int32_t stc = ST_OK;
        if (bad) stc = ST_BAD;
        else if (s == 0) stc = ST_EMPTY;
        else if (fail) stc = ST_NOT_SPD;
        if (stc != ST_OK) x0 = x1 = 0.f;
        if (i < a.kout) a.out[is * a.ldo + i] = x0;
        if (i + 16 < a.kout) a.out[is * a.ldo + i + 16] = x1;
        if (a.status && i == 0) a.status[is] = stc;
    }
    __syncwarp();   // the pair area is reused by the next pair
}

template <int KP>
__device__ void solve_range(const SolveArgs<float> &a, int wig, int W, unsigned char *wsbase,
                            int warp, int lane) {
    using WS = WarpSmem<float, float, KP>;
    // each warp's area starts at warp * sizeof(WS32); solve_system indexes smem[warp]
    WS *mine = reinterpret_cast<WS *>(wsbase + (size_t)warp * sizeof(WS32));
    for (int64_t i = wig; i < a.m; i += W) solve_system<float, float, KP, 1, false>(a, i, mine, 0, lane);
}

__device__ void run_half(const SolveArgs<float> &a, int KP, int wig, int W, unsigned char *wsbase,
                         int warp, int lane, int co_i, int co_i16) {
    if (KP == 8) solve_range<8>(a, wig, W, wsbase, warp, lane);
    else if (KP == 16) solve_range<16>(a, wig, W, wsbase, warp, lane);
    else {   // rank 32: two systems per warp
        PairSmem32 *mine = reinterpret_cast<PairSmem32 *>(wsbase + (size_t)warp * sizeof(WS32));
        for (int64_t i0 = 2 * (int64_t)wig; i0 < a.m; i0 += 2 * (int64_t)W)
            solve_pair32(a, i0, *mine, lane, co_i, co_i16);
    }
}

__global__ void __launch_bounds__(BW * 32, 2) k_batched_als(BatchArgs b) {   // two CTAs per SM
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int32_t qslot[BW];
    __shared__ int32_t s_col[32];   // column offsets of the packed rank-32 factor, less their first row
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int t = 0; t < 32; ++t) s_col[t] = pk::coloff(t) - pk::colbase(t);
    }
    __syncthreads();
    const int co_i = s_col[lane & 15], co_i16 = s_col[(lane & 15) + 16];

    for (int c = 0; c < b.n_classes; ++c) {
        const int W = b.class_W[c];
        const int grp = warp / W, wig = warp % W;
        const int gthreads = 32 * W, gtid = threadIdx.x - grp * gthreads;
        const int bar = 1 + grp;
        const int32_t q_lo = c == 0 ? 0 : b.class_end[c - 1], q_hi = b.class_end[c];
        unsigned char *gbase = smem_raw + (size_t)grp * W * sizeof(WS32);
        for (;;) {
            if (gtid == 0) qslot[grp] = q_lo + atomicAdd(b.counter + c, 1);
            group_sync(bar, gthreads);
            const int32_t qi = qslot[grp];
            group_sync(bar, gthreads);   // qslot is rewritten by the next grab
            if (qi >= q_hi) break;
            const int32_t p = b.order[qi];
            const int64_t m = b.m[p], n = b.n[p];
            const int KP = padded_k(b.k[p]);
            const int64_t r0 = b.row_off[p], c0 = b.col_off[p];
            const int64_t e0 = b.row_ptr[r0], e1 = b.row_ptr[r0 + m];

            // ---- CSC of this problem: stable counting sort in shared memory
            uint32_t *mask = reinterpret_cast<uint32_t *>(gbase);   // [n]
            int32_t *run = reinterpret_cast<int32_t *>(gbase) + n;  // [n]
            for (int64_t j = gtid; j < n; j += gthreads) run[j] = 0;
            group_sync(bar, gthreads);
            for (int64_t t = e0 + gtid; t < e1; t += gthreads) {
                const int32_t j = b.col[t];
                if (j >= 0 && j < n) atomicAdd(&run[j], 1);
            }
            group_sync(bar, gthreads);
            if (wig == 0) {   // exclusive scan of the column counts by the group's first warp
                const int64_t per = (n + 31) / 32;
                const int64_t j0 = lane * per, j1 = min(n, j0 + per);
                int64_t local = 0;
                for (int64_t j = j0; j < j1; ++j) local += run[j];
                long long incl = local;
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const long long t = __shfl_up_sync(FULL, incl, off);
                    if (lane >= off) incl += t;
                }
                int64_t acc = e0 + incl - local;
                for (int64_t j = j0; j < j1; ++j) {
                    const int32_t t = run[j];
                    b.cptr[c0 + j + p] = acc;
                    run[j] = (int32_t)(acc - e0);
                    acc += t;
                }
                if (lane == 31) b.cptr[c0 + n + p] = e0 + incl;
            }
            group_sync(bar, gthreads);
            for (int64_t rs = 0; rs < m; rs += 32) {
                const int64_t re = min(m, rs + 32);
                for (int64_t j = gtid; j < n; j += gthreads) mask[j] = 0u;
                group_sync(bar, gthreads);
                for (int64_t r = rs + gtid / 32; r < re; r += W) {
                    const int64_t rb = b.row_ptr[r0 + r], rend = b.row_ptr[r0 + r + 1];
                    for (int64_t t = rb + lane; t < rend; t += 32) {
                        const int32_t j = b.col[t];
                        if (j >= 0 && j < n) atomicOr(&mask[j], 1u << (unsigned)(r - rs));
                    }
                }
                group_sync(bar, gthreads);
                for (int64_t r = rs + gtid / 32; r < re; r += W) {
                    const int64_t rb = b.row_ptr[r0 + r], rend = b.row_ptr[r0 + r + 1];
                    const uint32_t below = (1u << (unsigned)(r - rs)) - 1u;
                    for (int64_t t = rb + lane; t < rend; t += 32) {
                        const int32_t j = b.col[t];
                        if (j >= 0 && j < n) {
                            const int64_t pos = e0 + run[j] + __popc(mask[j] & below);
                            b.cidx[pos] = (int32_t)r;
                            b.cval[pos] = b.val[t];
                        }
                    }
                }
                group_sync(bar, gthreads);
                for (int64_t j = gtid; j < n; j += gthreads) run[j] += __popc(mask[j]);
                group_sync(bar, gthreads);
            }

            // ---- sweeps: U-half (rows vs V), V-half (columns vs U)
            float *U = b.Uw + b.fu_off[p];
            float *V = b.Vw + b.fv_off[p];
            SolveArgs<float> ua{m, b.nnz, b.row_ptr + r0, b.col, b.val, V, n, U, KP, KP,
                                nullptr, b.lambda};
            SolveArgs<float> va{n, b.nnz, b.cptr + c0 + p, b.cidx, b.cval, U, m, V, KP, KP,
                                nullptr, b.lambda};
            ua.wr = va.wr = b.wr;
            for (int s = 0; s < b.sweeps; ++s) {
                run_half(ua, KP, wig, W, gbase, wig, lane, co_i, co_i16);
                group_sync(bar, gthreads);
                run_half(va, KP, wig, W, gbase, wig, lane, co_i, co_i16);
                group_sync(bar, gthreads);
            }
        }
        __syncthreads();   // regroup for the next class
    }
}

// Padded factor layout: problem p's rows of KP_p floats start at f_off[p].
__global__ void k_batched_pack(int64_t P, const int64_t *__restrict__ rows,
                               const int32_t *__restrict__ k, const int64_t *__restrict__ t_off,
                               const int64_t *__restrict__ f_off, const float *__restrict__ src,
                               float *__restrict__ dst, int to_padded) {
    for (int64_t p = blockIdx.x; p < P; p += gridDim.x) {
        const int kp = k[p], KP = padded_k(kp);
        const int64_t r = rows[p];
        for (int64_t e = threadIdx.x; e < r * KP; e += blockDim.x) {
            const int64_t i = e / KP;
            const int q = (int)(e % KP);
            if (to_padded)
                dst[f_off[p] + e] = q < kp ? src[t_off[p] + i * kp + q] : 0.0f;
            else if (q < kp)
                dst[t_off[p] + i * kp + q] = src[f_off[p] + e];
        }
    }
}

size_t batched_smem_bytes() { return sizeof(WS32) * BW; }

cudaError_t prepare_batched() {
    return cudaFuncSetAttribute(k_batched_als, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)batched_smem_bytes());
}

cudaError_t launch_batched(const BatchArgs &b, int grid, cudaStream_t st) {
    k_batched_als<<<grid, BW * 32, batched_smem_bytes(), st>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_batched_pack(int64_t P, const int64_t *rows, const int32_t *k,
                                const int64_t *t_off, const int64_t *f_off, const float *src,
                                float *dst, bool to_padded, cudaStream_t st) {
    if (P <= 0) return cudaSuccess;
    const int64_t grid = P < NUM_SMS_HINT * 8 ? P : NUM_SMS_HINT * 8;
    k_batched_pack<<<(unsigned)grid, 256, 0, st>>>(P, rows, k, t_off, f_off, src, dst,
                                                   to_padded ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace ocf
