// Reconstruction T = U V^T fused with Algorithm 2 (energy-efficient power-cap
// selection, Sec. "Optimal Power setting Selection").
//
// Per application row i, with t_j the predicted normalised runtime of setting
// j and t_b that of the baseline (C_b, G_b):
//     p_j = t_b / t_j                    (predicted performance vs baseline)
//     valid iff t_j > 0 and 1 - p_j <= gamma
//     E_j = (c_j + g_j) / p_j,   saving_j = (E_base - E_j) / E_base,  E_base = C_b + G_b
// and the selected setting maximises saving_j (ties: smaller c_j + g_j, then
// smaller j).  The decision is taken in FP32 with correctly rounded
// operations in exactly this order, so it is reproducible bit for bit.
//
// The dense prediction is an m x n x k contraction with tiny k (8..32); the
// kernel keeps it in registers and feeds it straight into the selection, so
// T only reaches HBM when the caller asks for it.  Tile: 64 rows x 64
// settings per step, 256 threads, each thread a 4 x 4 register micro-tile
// from 16-byte shared-memory loads of the transposed U and V tiles.
#include "alg2.cuh"
#include "common.cuh"
#include "kernels.h"

namespace ocf {

template <int LANES> __device__ __forceinline__ float group_min(float v) {
#pragma unroll
    for (int off = 1; off < LANES; off <<= 1) v = fminf(v, __shfl_xor_sync(FULL, v, off));
    return v;
}

__device__ __forceinline__ Cand shfl_cand(const Cand &c, int off) {
    Cand o;
    o.sv = __shfl_xor_sync(FULL, c.sv, off);
    o.cg = __shfl_xor_sync(FULL, c.cg, off);
    o.j = __shfl_xor_sync(FULL, c.j, off);
    o.Ethr = __shfl_xor_sync(FULL, c.Ethr, off);
    return o;
}

constexpr int PT = 256;

// T[i][j] = sum_p U[i][p] V[j][p] as one FMA chain in p order (in TV), then
// the selection on float(T).  The baseline runtime uses the identical chain so
// that t_b equals T[i][base] bit for bit and the baseline's loss is exactly 0.
//
// Tile: BM rows x BN settings per step, 256 threads as TY x TX (TY = BM/4),
// each thread 4 rows (ty*4 + r) x 4 settings (tx + TX*c, strided so that a
// warp reads distinct V rows without bank conflicts).  U and V tiles are kept
// row-major in shared memory (rows padded by 16 bytes) and filled with 16-byte
// copies; the inner loop reads 4 consecutive p at a time (16-byte loads).
// BM = 16 keeps enough CTAs busy when rows are few, BM = 64 reuses each V
// tile over more rows when they are many.
template <typename TV, int KP, int BM>
__global__ void __launch_bounds__(PT) k_predict_select(PredictArgs<TV> a) {
    constexpr int TY = BM / 4, TX = PT / TY, BN = 4 * TX;
    constexpr int WPR = TX > 32 ? TX / 32 : 1;       // warps sharing one row group
    constexpr int VN = 16 / (int)sizeof(TV);          // elements per 16 bytes
    constexpr int LD = KP + VN;                       // padded row
    using VT = typename Vec4<TV>::type;
    __shared__ __align__(16) TV Us[BM][LD];
    __shared__ __align__(16) TV Vs[BN][LD];
    __shared__ float cgs[BN];
    __shared__ RowCtx rcs[BM];
    __shared__ Cand xw[TY][WPR][4];
    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    const bool sel = a.cg != nullptr;
    const int64_t row_tiles = (a.m + BM - 1) / BM;
    const bool u_vec = (a.ldu % VN) == 0 && a.k == KP &&
                       (reinterpret_cast<uintptr_t>(a.U) & 15) == 0;

    for (int64_t rt = blockIdx.x; rt < row_tiles; rt += gridDim.x) {
        const int64_t r0 = rt * BM;
        __syncthreads();
        if (u_vec) {
            for (int e = tid; e < BM * (KP / VN); e += PT) {
                const int ii = e / (KP / VN), p4 = e % (KP / VN);
                const int64_t r = r0 + ii;
                VT x;
                if (r < a.m) x = *reinterpret_cast<const VT *>(a.U + r * a.ldu + p4 * VN);
                else x = VT{};
                *reinterpret_cast<VT *>(&Us[ii][p4 * VN]) = x;
            }
        } else {
            for (int e = tid; e < BM * KP; e += PT) {
                const int ii = e / KP, p = e % KP;
                const int64_t r = r0 + ii;
                Us[ii][p] = (r < a.m && p < a.k) ? a.U[r * a.ldu + p] : TV(0);
            }
        }
        __syncthreads();
        if (sel && tid < BM) {
            const TV *vb = a.V + a.base * KP;
            TV acc = TV(0);
#pragma unroll
            for (int p = 0; p < KP; ++p) acc = my_fma(Us[tid][p], vb[p], acc);
            rcs[tid] = alg2_row((float)acc, a.gamma);
        }
        Cand best[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) best[r] = Cand{0.0f, 0.0f, -1, 0.0f};

        for (int64_t c0 = 0; c0 < a.n; c0 += BN) {
            __syncthreads();
            for (int e = tid; e < BN * (KP / VN); e += PT) {
                const int jj = e / (KP / VN), p4 = e % (KP / VN);
                const int64_t j = c0 + jj;
                VT x;
                if (j < a.n) x = __ldg(reinterpret_cast<const VT *>(a.V + j * KP) + p4);
                else x = VT{};
                *reinterpret_cast<VT *>(&Vs[jj][p4 * VN]) = x;
            }
            if (sel)
                for (int e = tid; e < BN; e += PT) cgs[e] = (c0 + e < a.n) ? a.cg[c0 + e] : 0.0f;
            __syncthreads();
            TV acc[4][4];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] = TV(0);
#pragma unroll
            for (int p4 = 0; p4 < KP; p4 += VN) {
                TV u[4][VN], v[4][VN];
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const VT x = *reinterpret_cast<const VT *>(&Us[ty * 4 + r][p4]);
#pragma unroll
                    for (int e = 0; e < VN; ++e) u[r][e] = vget(x, e);
                }
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const VT x = *reinterpret_cast<const VT *>(&Vs[tx + TX * c][p4]);
#pragma unroll
                    for (int e = 0; e < VN; ++e) v[c][e] = vget(x, e);
                }
#pragma unroll
                for (int e = 0; e < VN; ++e)
#pragma unroll
                    for (int r = 0; r < 4; ++r)
#pragma unroll
                        for (int c = 0; c < 4; ++c) acc[r][c] = my_fma(u[r][e], v[c][e], acc[r][c]);
            }
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int64_t i = r0 + ty * 4 + r;
                if (a.T && i < a.m) {
                    TV *trow = a.T + i * a.n;
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const int64_t j = c0 + tx + TX * c;
                        if (j < a.n) trow[j] = acc[r][c];
                    }
                }
            }
            if (sel) {
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const RowCtx rc = rcs[ty * 4 + r];
                    float est[4];
                    float emin = __int_as_float(0x7fffffff);
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const int64_t j = c0 + tx + TX * c;
                        est[c] = (j < a.n) ? alg2_estimate(rc, (float)acc[r][c], cgs[tx + TX * c])
                                           : __int_as_float(0x7fffffff);
                        emin = fminf(emin, est[c]);
                    }
                    // 16-row tiles (a warp per row): the lanes of a row agree on the
                    // row's smallest estimate.  64-row tiles (16 lanes per row): each
                    // thread screens with its own, which saves a cross-lane minimum per
                    // tile.  Sound: a thread's minimum is at least the row's, and
                    // alg2_bound increases with its argument, so the bound only gets
                    // looser and no setting that could win or tie is screened out.
                    if constexpr (TX >= 32) emin = group_min<32>(emin);
                    float bound = alg2_bound(emin, a.Ebase);
                    if (best[r].j >= 0) bound = fminf(bound, best[r].Ethr);
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        if (est[c] <= bound)
                            alg2_exact(best[r], rc, (float)acc[r][c], cgs[tx + TX * c], a.Ebase,
                                       (int32_t)(c0 + tx + TX * c));
                }
            }
        }
        if (sel) {
            constexpr int LANES = TX < 32 ? TX : 32;
#pragma unroll
            for (int r = 0; r < 4; ++r) {
#pragma unroll
                for (int off = 1; off < LANES; off <<= 1) {
                    const Cand o = shfl_cand(best[r], off);
                    if (better(o, best[r])) best[r] = o;
                }
            }
            if constexpr (WPR > 1) {
                const int wr = (tid % TX) / 32;
                if ((tid & 31) == 0)
#pragma unroll
                    for (int r = 0; r < 4; ++r) xw[ty][wr][r] = best[r];
                __syncthreads();
                if (tx == 0)
#pragma unroll
                    for (int r = 0; r < 4; ++r)
                        for (int w = 1; w < WPR; ++w)
                            if (better(xw[ty][w][r], best[r])) best[r] = xw[ty][w][r];
            }
            if (tx == 0) {
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const int64_t i = r0 + ty * 4 + r;
                    if (i < a.m) {
                        if (a.best) a.best[i] = best[r].j;
                        if (a.saving) a.saving[i] = best[r].j >= 0 ? best[r].sv : 0.0f;
                    }
                }
            }
        }
    }
}

template <typename TV, int BM>
static cudaError_t launch_bm(const PredictArgs<TV> &a, cudaStream_t st) {
    int64_t blocks = (a.m + BM - 1) / BM;
    if (blocks > NUM_SMS_HINT * 16) blocks = NUM_SMS_HINT * 16;
    switch (a.KP) {
        case 8: k_predict_select<TV, 8, BM><<<(unsigned)blocks, PT, 0, st>>>(a); break;
        case 16: k_predict_select<TV, 16, BM><<<(unsigned)blocks, PT, 0, st>>>(a); break;
        case 32: k_predict_select<TV, 32, BM><<<(unsigned)blocks, PT, 0, st>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename TV> cudaError_t launch_predict_select(const PredictArgs<TV> &a, cudaStream_t st) {
    if (a.m <= 0 || a.n <= 0) return cudaSuccess;
    if constexpr (sizeof(TV) == 4) {
        if ((a.m + 63) / 64 < 2 * NUM_SMS_HINT) return launch_bm<TV, 16>(a, st);
    }
    return launch_bm<TV, 64>(a, st);
}

template cudaError_t launch_predict_select<float>(const PredictArgs<float> &, cudaStream_t);
template cudaError_t launch_predict_select<double>(const PredictArgs<double> &, cudaStream_t);

// Algorithm 2 on a given dense FP32 matrix: one warp per row.
__global__ void __launch_bounds__(256)
k_select(int64_t m, int64_t n, const float *__restrict__ T, int64_t ld,
         const float *__restrict__ cg, int64_t base, float Eb, float gamma,
         int32_t *__restrict__ best, float *__restrict__ saving) {
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = w; i < m; i += nw) {
        const float *t = T + i * ld;
        const RowCtx rc = alg2_row(__ldg(t + base), gamma);
        Cand b{0.0f, 0.0f, -1, 0.0f};
        constexpr int U8 = 8;   // 8 steps of 32 settings in flight per load batch
        for (int64_t j0 = 0; j0 < n; j0 += 32 * U8) {
            float tj[U8], cj[U8];
#pragma unroll
            for (int u = 0; u < U8; ++u) {
                const int64_t j = j0 + 32 * u + lane;
                tj[u] = (j < n) ? __ldg(t + j) : 0.0f;
                cj[u] = (j < n) ? __ldg(cg + j) : 0.0f;
            }
#pragma unroll
            for (int u = 0; u < U8; ++u) {
                const int64_t j = j0 + 32 * u + lane;
                const float est =
                    (j < n) ? alg2_estimate(rc, tj[u], cj[u]) : __int_as_float(0x7fffffff);
                float bound = alg2_bound(group_min<32>(est), Eb);
                if (b.j >= 0) bound = fminf(bound, b.Ethr);
                if (est <= bound) alg2_exact(b, rc, tj[u], cj[u], Eb, (int32_t)j);
            }
        }
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const Cand o = shfl_cand(b, off);
            if (better(o, b)) b = o;
        }
        if (lane == 0) {
            if (best) best[i] = b.j;
            if (saving) saving[i] = b.j >= 0 ? b.sv : 0.0f;
        }
    }
}

cudaError_t launch_select(int64_t m, int64_t n, const float *T, int64_t ld, const float *cg,
                          int64_t base, float Ebase, float gamma, int32_t *best, float *saving,
                          cudaStream_t st) {
    if (m <= 0) return cudaSuccess;
    int64_t blocks = (m + 7) / 8;
    if (blocks > NUM_SMS_HINT * 16) blocks = NUM_SMS_HINT * 16;
    k_select<<<(unsigned)blocks, 256, 0, st>>>(m, n, T, ld, cg, base, Ebase, gamma, best, saving);
    return cudaGetLastError();
}

}  // namespace ocf
