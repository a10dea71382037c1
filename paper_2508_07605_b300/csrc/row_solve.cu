// Fused masked-Gram + Cholesky row solve (one ALS half-step).
//
// For every row i of a CSR matrix (a new application, an offline application,
// or -- on the CSC copy -- a setting), with F the fixed other factor:
//     A_i = sum_{j in Omega_i} f_j f_j^T + lambda I,   b_i = sum_{j in Omega_i} R_ij f_j,
//     A_i = L L^T,  L y = b_i,  L^T x_i = y.
// This is the per-row ridge solve of alternating least squares (the matrix
// factorisation model of collaborative filtering the paper builds on, Sec.
// "Collaborative Filtering Model"; the online fold-in of new rows of Sec.
// "Online Performance Prediction").
//
// Mapping: a "segment" of KP lanes owns one system; lane q of the segment
// owns row q of A (KP registers).  KP = 8/16/32 gives 4/2/1 systems per warp.
//   * Gram: the segment reads each observation's factor row f_j (KP contiguous
//     elements, L1/L2 resident) with broadcast 16-byte loads and lane q adds
//     f_j[q] * f_j into its row: KP FMAs per lane per observation, no shuffles
//     except the two that broadcast (j, R_ij) from a coalesced chunk load.
//   * Cholesky: right-looking, fully unrolled over the pivot p; column p of L
//     is exchanged through a double-buffered shared-memory vector (one store
//     per lane, broadcast loads), the rank-1 update stays in registers.
//   * Solves: forward substitution by shuffles; back substitution reads L^T
//     from a shared-memory copy of L (conflict-free, stride KP+1).
// A never touches HBM: per row the kernel reads the CSR row and s factor rows
// and writes one factor row.
#include "common.cuh"
#include "kernels.h"

namespace ocf {

template <typename TC, int KP> struct SegSmem {
    TC col[2][KP];
    TC dinv[KP];
    TC L[KP][KP + 1];
};

template <typename TV, typename TC, int KP, int WARPS>
__global__ void __launch_bounds__(WARPS * 32)
k_row_solve(SolveArgs<TV> a) {
    constexpr int SPW = 32 / KP;
    using VT = typename Vec4<TV>::type;
    constexpr int VN = Vec4<TV>::N;
    __shared__ SegSmem<TC, KP> smem[WARPS][SPW];

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int seg = lane / KP;
    const int q = lane % KP;
    SegSmem<TC, KP> &S = smem[warp][seg];
    const int64_t stride = (int64_t)gridDim.x * WARPS * SPW;

    for (int64_t base = ((int64_t)blockIdx.x * WARPS + warp) * SPW; base < a.m; base += stride) {
        const int64_t i = base + seg;
        const bool valid = i < a.m;
        int64_t beg = 0, end = 0;
        bool bad = false;
        if (valid) bad = !row_bounds(a.ptr, i, a.nnz, beg, end);
        const int64_t s = end - beg;

        // ---- masked Gram + RHS ------------------------------------------
        TV acc[KP];
#pragma unroll
        for (int e = 0; e < KP; ++e) acc[e] = TV(0);
        TV bq = TV(0);
        long long smax = s;
#pragma unroll
        for (int off = KP; off < 32; off <<= 1) smax = max(smax, __shfl_xor_sync(FULL, smax, off));
        for (int64_t c0 = 0; c0 < smax; c0 += KP) {
            const int64_t tme = c0 + q;
            int32_t jl = 0;
            TV rl = TV(0);
            if (tme < s) {
                jl = __ldg(a.idx + beg + tme);
                rl = __ldg(a.val + beg + tme);
                if (jl < 0 || (int64_t)jl >= a.n_other) {
                    bad = true;
                    jl = 0;
                }
            }
            const int cnt = (int)min((int64_t)KP, (int64_t)smax - c0);
#pragma unroll 4
            for (int t = 0; t < cnt; ++t) {
                const int32_t j = __shfl_sync(FULL, jl, t, KP);
                const TV r = __shfl_sync(FULL, rl, t, KP);
                if (c0 + t < s) {
                    const TV *fj = a.F + (int64_t)j * KP;
                    const VT *fv = reinterpret_cast<const VT *>(fj);
                    const TV fq = __ldg(fj + q);
#pragma unroll
                    for (int e4 = 0; e4 < KP / VN; ++e4) {
                        const VT x = __ldg(fv + e4);
#pragma unroll
                        for (int e = 0; e < VN; ++e)
                            acc[e4 * VN + e] = my_fma(fq, vget(x, e), acc[e4 * VN + e]);
                    }
                    bq = my_fma(r, fq, bq);
                }
            }
        }
#pragma unroll
        for (int off = 1; off < KP; off <<= 1) bad |= __shfl_xor_sync(FULL, (int)bad, off) != 0;

        // ---- Cholesky A = L L^T in TC ------------------------------------
        TC A[KP];
#pragma unroll
        for (int e = 0; e < KP; ++e) A[e] = TC(acc[e]) + ((e == q) ? TC(a.lambda) : TC(0));
        bool fail = false;
#pragma unroll
        for (int p = 0; p < KP; ++p) {
            TC piv = __shfl_sync(FULL, A[p], p, KP);
            if (!(piv > TC(0))) {
                fail = true;
                piv = TC(1);
            }
            const TC sq = my_sqrt(piv);
            const TC inv = TC(1) / sq;
            const TC l = (q == p) ? sq : A[p] * inv;
            A[p] = l;
            TC *cb = S.col[p & 1];
            cb[q] = l;
            if (q == 0) S.dinv[p] = inv;
            __syncwarp();
#pragma unroll
            for (int r = p + 1; r < KP; ++r) A[r] = my_fma(-l, cb[r], A[r]);
        }

        // ---- forward substitution L y = b ---------------------------------
        TC y = TC(bq), yq = TC(0);
#pragma unroll
        for (int p = 0; p < KP; ++p) {
            const TC yp = __shfl_sync(FULL, y, p, KP) * S.dinv[p];
            if (q == p) yq = yp;
            if (q > p) y = my_fma(-A[p], yp, y);
        }

        // ---- back substitution L^T x = y ----------------------------------
#pragma unroll
        for (int e = 0; e < KP; ++e) S.L[q][e] = A[e];
        __syncwarp();
        TC x = yq, xq = TC(0);
#pragma unroll
        for (int p = KP - 1; p >= 0; --p) {
            const TC xp = __shfl_sync(FULL, x, p, KP) * S.dinv[p];
            if (q == p) xq = xp;
            if (q < p) x = my_fma(-S.L[p][q], xp, x);
        }
        __syncwarp();  // S is rewritten by the next row of this segment

        if (valid) {
            int32_t st = ST_OK;
            if (bad) st = ST_BAD;
            else if (s == 0) st = ST_EMPTY;
            else if (fail) st = ST_NOT_SPD;
            if (st != ST_OK) xq = TC(0);
            if (q < a.kout) a.out[i * a.ldo + q] = TV(xq);
            if (a.status && q == 0) a.status[i] = st;
        }
    }
}

template <typename TV, typename TC, int KP>
static cudaError_t launch_kp(const SolveArgs<TV> &a, cudaStream_t st) {
    constexpr int WARPS = (sizeof(TC) == 8) ? 4 : 8;
    constexpr int SPW = 32 / KP;
    const int64_t per_cta = WARPS * SPW;
    int64_t blocks = (a.m + per_cta - 1) / per_cta;
    if (blocks > NUM_SMS_HINT * 64) blocks = NUM_SMS_HINT * 64;
    if (blocks < 1) return cudaSuccess;
    k_row_solve<TV, TC, KP, WARPS><<<(unsigned)blocks, WARPS * 32, 0, st>>>(a);
    return cudaGetLastError();
}

template <typename TV, typename TC>
cudaError_t launch_row_solve(const SolveArgs<TV> &a, int KP, cudaStream_t st) {
    if (a.m <= 0) return cudaSuccess;
    switch (KP) {
        case 8: return launch_kp<TV, TC, 8>(a, st);
        case 16: return launch_kp<TV, TC, 16>(a, st);
        case 32: return launch_kp<TV, TC, 32>(a, st);
        default: return cudaErrorInvalidValue;
    }
}

template cudaError_t launch_row_solve<float, float>(const SolveArgs<float> &, int, cudaStream_t);
template cudaError_t launch_row_solve<float, double>(const SolveArgs<float> &, int, cudaStream_t);
template cudaError_t launch_row_solve<double, double>(const SolveArgs<double> &, int,
                                                      cudaStream_t);

}  // namespace ocf
