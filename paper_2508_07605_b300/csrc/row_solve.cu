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
// Mapping (WPS warps per system; WPS = 1 for short rows, 4 for long rows):
//   * Staging: each warp takes 32 observations at a time; lane t loads
//     (j_t, R_t) and the whole factor row f_{j_t} (KP elements, 16-byte loads)
//     into a padded, bank-conflict-free shared-memory tile.  All 32 rows are
//     in flight at once, so global latency is paid once per 32 observations.
//   * Gram: the warp is G = 32/KP groups of KP lanes; group g takes the staged
//     observations t = g, g+G, ...; lane q of a group owns row q of A (KP
//     registers) and adds f_t[q] * f_t from 16-byte broadcast shared loads.
//     Groups (and, for WPS = 4, warps through shared memory in a fixed order)
//     are summed at the end.
//   * Cholesky: right-looking, fully unrolled over the pivot p; column p of L
//     is exchanged through a double-buffered shared vector, the rank-1 update
//     stays in registers.  Forward substitution by shuffles, back substitution
//     from a shared copy of L (stride KP+1, conflict-free).
// A never touches HBM: per row the kernel reads the CSR row and s factor rows
// and writes one factor row.
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

template <typename TV, typename TC, int KP, int WPS>
__global__ void __launch_bounds__(WPS == 1 ? 256 : 32 * WPS)
k_row_solve(SolveArgs<TV> a) {
    constexpr int WARPS = (WPS == 1) ? 8 : WPS;
    constexpr int G = 32 / KP;
    using VT = typename Vec4<TV>::type;
    constexpr int VN = Vec4<TV>::N;
    using WS = WarpSmem<TV, TC, KP>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    WS *smem = reinterpret_cast<WS *>(smem_raw);

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int g = lane / KP;
    const int q = lane % KP;
    WS &W = smem[warp];
    // WPS == 1: one system per warp; WPS > 1: one system per CTA.
    const int64_t sys0 = (WPS == 1) ? (int64_t)blockIdx.x * WARPS + warp : (int64_t)blockIdx.x;
    const int64_t sys_stride = (WPS == 1) ? (int64_t)gridDim.x * WARPS : (int64_t)gridDim.x;
    const int wsub = (WPS == 1) ? 0 : warp;   // this warp's slice of the observations

    for (int64_t i = sys0; i < a.m; i += sys_stride) {
        int64_t beg = 0, end = 0;
        bool bad = !row_bounds(a.ptr, i, a.nnz, beg, end);
        const int64_t s = end - beg;

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
                    for (int e = 0; e < VN; ++e)
                        acc[e4 * VN + e] = my_fma(fq, vget(x, e), acc[e4 * VN + e]);
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
#pragma unroll
        for (int e = 0; e < KP; ++e)
            if (e == q) A[e] += TC(a.lambda);

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
#pragma unroll
            for (int r = p + 1; r < KP; ++r) A[r] = my_fma(-l, cb[r], A[r]);
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

template <typename TV, typename TC, int KP, int WPS>
static size_t smem_bytes() {
    constexpr int WARPS = (WPS == 1) ? 8 : WPS;
    return sizeof(WarpSmem<TV, TC, KP>) * WARPS;
}

template <typename TV, typename TC, int KP, int WPS>
static cudaError_t set_attr() {
    return cudaFuncSetAttribute(k_row_solve<TV, TC, KP, WPS>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem_bytes<TV, TC, KP, WPS>());
}

template <typename TV, typename TC>
static cudaError_t set_attrs_tv() {
    cudaError_t e;
    if ((e = set_attr<TV, TC, 8, 1>()) != cudaSuccess) return e;
    if ((e = set_attr<TV, TC, 16, 1>()) != cudaSuccess) return e;
    if ((e = set_attr<TV, TC, 32, 1>()) != cudaSuccess) return e;
    if ((e = set_attr<TV, TC, 8, 4>()) != cudaSuccess) return e;
    if ((e = set_attr<TV, TC, 16, 4>()) != cudaSuccess) return e;
    return set_attr<TV, TC, 32, 4>();
}

cudaError_t prepare_row_solve() {
    cudaError_t e;
    if ((e = set_attrs_tv<float, float>()) != cudaSuccess) return e;
    if ((e = set_attrs_tv<float, double>()) != cudaSuccess) return e;
    return set_attrs_tv<double, double>();
}

// Observations per system above which a system gets a CTA of 4 warps.
constexpr int64_t LONG_ROW = 96;

template <typename TV, typename TC, int KP>
static cudaError_t launch_kp(const SolveArgs<TV> &a, cudaStream_t st) {
    const bool long_rows = a.nnz >= LONG_ROW * a.m;
    if (long_rows) {
        int64_t blocks = a.m;
        if (blocks > NUM_SMS_HINT * 64) blocks = NUM_SMS_HINT * 64;
        k_row_solve<TV, TC, KP, 4>
            <<<(unsigned)blocks, 128, smem_bytes<TV, TC, KP, 4>(), st>>>(a);
    } else {
        int64_t blocks = (a.m + 7) / 8;
        if (blocks > NUM_SMS_HINT * 32) blocks = NUM_SMS_HINT * 32;
        k_row_solve<TV, TC, KP, 1>
            <<<(unsigned)blocks, 256, smem_bytes<TV, TC, KP, 1>(), st>>>(a);
    }
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
