// Warp-level fused Gram + Cholesky solve of one system (one ALS row solve),
// shared by the per-half-step kernel (row_solve.cu) and the batched
// persistent kernel (batched.cu).  See row_solve.cu for the method.
#pragma once

#include "common.cuh"
#include "kernels.h"

namespace ocf {

template <typename TV, typename TC, int KP> struct alignas(16) WarpSmem {
    static constexpr int LD = KP + 16 / (int)sizeof(TV);   // padded staged row
    TV stage[32][LD];
    TV sr[32];
    TC col[2][KP];
    TC dinv[KP];
    TC L[KP][KP + 1];
    TC red[KP][KP + 1];   // partial Gram of this warp (WPS > 1)
    TC redb[KP];
};

__device__ __forceinline__ float my_rsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double my_rsqrt(double x) { return rsqrt(x); }

// a0 += f * x0, a1 += f * x1: in FP32 one packed fma.rn.f32x2 (each element
// rounds exactly like fmaf, so the results are those of two scalar FMAs).
__device__ __forceinline__ void fma_pair(float &a0, float &a1, float f, float x0, float x1) {
    const float2 r = __ffma2_rn(make_float2(f, f), make_float2(x0, x1), make_float2(a0, a1));
    a0 = r.x;
    a1 = r.y;
}
__device__ __forceinline__ void fma_pair(double &a0, double &a1, double f, double x0, double x1) {
    a0 = fma(f, x0, a0);
    a1 = fma(f, x1, a1);
}

// Solve system i.  WPS = 1: the calling warp alone (lanes in G = 32/KP groups);
// WPS > 1: the WPS warps of the CTA together (every warp of the CTA calls it).
// SUMS: the build supports the stored sums of the streaming refit (the
// batched kernel, which never uses them, leaves them out to save registers).
template <typename TV, typename TC, int KP, int WPS, bool SUMS = true>
__device__ __forceinline__ void solve_system(const SolveArgs<TV> &a, int64_t i,
                                             WarpSmem<TV, TC, KP> *smem, int warp, int lane) {
    constexpr int G = 32 / KP;
    using VT = typename Vec4<TV>::type;
    constexpr int VN = Vec4<TV>::N;
    const int g = lane / KP;
    const int q = lane % KP;
    WarpSmem<TV, TC, KP> &W = smem[warp];
    const int wsub = (WPS == 1) ? 0 : warp;   // this warp's slice of the observations
    {
        int64_t beg = 0, end = 0;
        bool bad = !row_bounds(a.ptr, i, a.nnz, beg, end);
        int64_t s = end - beg;

        // ---- staged masked Gram + RHS ---------------------------------------
        TV acc[KP];
#pragma unroll
        for (int e = 0; e < KP; ++e) acc[e] = TV(0);
        TV bq = TV(0);
        for (int64_t c0 = (int64_t)wsub * 32; c0 < s; c0 += 32 * WPS) {
            const int64_t t = c0 + lane;
            if (t < s) {
                int32_t j = __ldg(a.idx + beg + t);
                TV r = __ldg(a.val + beg + t);
                if (j < 0 || (int64_t)j >= a.n_other) {
                    bad = true;
                    j = 0;
                    r = TV(0);
                }
                const VT *src = reinterpret_cast<const VT *>(a.F + (int64_t)j * KP);
                VT *dst = reinterpret_cast<VT *>(&W.stage[lane][0]);
#pragma unroll
                for (int e4 = 0; e4 < KP / VN; ++e4) dst[e4] = __ldg(src + e4);
                W.sr[lane] = r;
            }
            __syncwarp();
            const int cnt = (int)min((int64_t)32, s - c0);
#pragma unroll 4
            for (int tt = g; tt < cnt; tt += G) {
                const TV *row = W.stage[tt];
                const TV fq = row[q];
                const TV r = W.sr[tt];
                const VT *rv = reinterpret_cast<const VT *>(row);
#pragma unroll
                for (int e4 = 0; e4 < KP / VN; ++e4) {
                    const VT x = rv[e4];
#pragma unroll
                    for (int e = 0; e < VN; e += 2)
                        fma_pair(acc[e4 * VN + e], acc[e4 * VN + e + 1], fq, vget(x, e),
                                 vget(x, e + 1));
                }
                bq = my_fma(r, fq, bq);
            }
            __syncwarp();
        }
        // sum the G groups (every group ends with the warp's total)
#pragma unroll
        for (int off = KP; off < 32; off <<= 1) {
#pragma unroll
            for (int e = 0; e < KP; ++e) acc[e] += __shfl_xor_sync(FULL, acc[e], off);
            bq += __shfl_xor_sync(FULL, bq, off);
        }
        TC A[KP];
        TC bt;
        if constexpr (WPS > 1) {
            // fixed-order sum of the WPS warps' partial Grams through shared memory
            bad = __syncthreads_or(bad) != 0;
            if (g == 0) {
#pragma unroll
                for (int e = 0; e < KP; ++e) W.red[q][e] = TC(acc[e]);
                W.redb[q] = TC(bq);
            }
            __syncthreads();
#pragma unroll
            for (int e = 0; e < KP; ++e) A[e] = smem[0].red[q][e];
            bt = smem[0].redb[q];
            for (int w = 1; w < WPS; ++w) {
#pragma unroll
                for (int e = 0; e < KP; ++e) A[e] += smem[w].red[q][e];
                bt += smem[w].redb[q];
            }
        } else {
            bad = __any_sync(FULL, bad) != 0;
#pragma unroll
            for (int e = 0; e < KP; ++e) A[e] = TC(acc[e]);
            bt = TC(bq);
        }
        if (SUMS && a.gram && !bad && (WPS == 1 || warp == 0)) {   // streaming: stored sums
            TV *gq = a.gram + (i * KP + q) * KP;
#pragma unroll
            for (int e = 0; e < KP; ++e) A[e] += TC(gq[e]);
            bt += TC(a.gram_b[i * KP + q]);
            s += a.gram_n[i];
            if (a.gram_keep && g == 0) {
#pragma unroll
                for (int e = 0; e < KP; ++e) gq[e] = TV(A[e]);
                a.gram_b[i * KP + q] = TV(bt);
                if (q == 0) a.gram_n[i] = s;
            }
        }
        const TC lam = TC(a.lambda) * (a.wr ? TC(s) : TC(1));   // weighted: lambda s_i
#pragma unroll
        for (int e = 0; e < KP; ++e)
            if (e == q) A[e] += lam;

        // With WPS > 1 every warp holds the summed system; warp 0 solves it.
        if (WPS == 1 || warp == 0) {

        // ---- Cholesky A = L L^T in TC (every group computes it; group 0 writes)
        bool fail = false;
#pragma unroll
        for (int p = 0; p < KP; ++p) {
            TC piv = __shfl_sync(FULL, A[p], p, KP);
            if (!(piv > TC(0))) {
                fail = true;
                piv = TC(1);
            }
            const TC inv = my_rsqrt(piv);
            const TC l = (q == p) ? piv * inv : A[p] * inv;
            A[p] = l;
            TC *cb = W.col[p & 1];
            if (g == 0) cb[q] = l;
            if (lane == 0) W.dinv[p] = inv;
            __syncwarp();
            // trailing update A[r] -= l L[r][p], r > p, two elements per instruction
            if (p + 1 < KP && ((p + 1) & 1)) A[p + 1] = my_fma(-l, cb[p + 1], A[p + 1]);
#pragma unroll
            for (int r = ((p + 1) & 1) ? p + 2 : p + 1; r + 1 < KP; r += 2)
                fma_pair(A[r], A[r + 1], -l, cb[r], cb[r + 1]);
        }

        // ---- forward substitution L y = b ---------------------------------
        TC y = bt, yq = TC(0);
#pragma unroll
        for (int p = 0; p < KP; ++p) {
            const TC yp = __shfl_sync(FULL, y, p, KP) * W.dinv[p];
            if (q == p) yq = yp;
            if (q > p) y = my_fma(-A[p], yp, y);
        }

        // ---- back substitution L^T x = y ----------------------------------
        if (g == 0) {
#pragma unroll
            for (int e = 0; e < KP; ++e) W.L[q][e] = A[e];
        }
        __syncwarp();
        TC x = yq, xq = TC(0);
#pragma unroll
        for (int p = KP - 1; p >= 0; --p) {
            const TC xp = __shfl_sync(FULL, x, p, KP) * W.dinv[p];
            if (q == p) xq = xp;
            if (q < p) x = my_fma(-W.L[p][q], xp, x);
        }
        __syncwarp();  // W is rewritten by the next system of this warp

        if (g == 0) {
            int32_t st = ST_OK;
            if (bad) st = ST_BAD;
            else if (s == 0) st = ST_EMPTY;
            else if (fail) st = ST_NOT_SPD;
            if (st != ST_OK) xq = TC(0);
            if (q < a.kout) a.out[i * a.ldo + q] = TV(xq);
            if (a.status && q == 0) a.status[i] = st;
        }
        }  // solver warp
        if constexpr (WPS > 1) __syncthreads();   // red[] and stage[] are reused next
    }
}

}  // namespace ocf
