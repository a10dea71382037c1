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
#include "common.cuh"
#include "kernels.h"

namespace ocf {

struct Cand {
    float sv;
    float cg;
    int32_t j;
};

// a better than b?  (saving desc, c+g asc, index asc; j < 0 means none)
__device__ __forceinline__ bool better(const Cand &a, const Cand &b) {
    if (a.j < 0) return false;
    if (b.j < 0) return true;
    if (a.sv != b.sv) return a.sv > b.sv;
    if (a.cg != b.cg) return a.cg < b.cg;
    return a.j < b.j;
}

__device__ __forceinline__ void alg2_consider(Cand &best, float tb, float t, float cg, float Eb,
                                              float gamma, int32_t j) {
    if (!(tb > 0.0f) || !(t > 0.0f)) return;
    const float p = __fdiv_rn(tb, t);
    const float loss = __fsub_rn(1.0f, p);
    if (!(loss <= gamma)) return;
    const float E = __fdiv_rn(cg, p);
    const float sv = __fdiv_rn(__fsub_rn(Eb, E), Eb);
    Cand c{sv, cg, j};
    if (better(c, best)) best = c;
}

__device__ __forceinline__ Cand shfl_cand(const Cand &c, int off) {
    Cand o;
    o.sv = __shfl_xor_sync(FULL, c.sv, off);
    o.cg = __shfl_xor_sync(FULL, c.cg, off);
    o.j = __shfl_xor_sync(FULL, c.j, off);
    return o;
}

constexpr int PT = 256;

template <typename TV>
__device__ __forceinline__ void load4(const TV *p, TV (&x)[4]) {
    if constexpr (sizeof(TV) == 4) {
        const float4 v = *reinterpret_cast<const float4 *>(p);
        x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
    } else {
        const double2 v0 = *reinterpret_cast<const double2 *>(p);
        const double2 v1 = *reinterpret_cast<const double2 *>(p + 2);
        x[0] = v0.x; x[1] = v0.y; x[2] = v1.x; x[3] = v1.y;
    }
}

// T[i][j] = sum_p U[i][p] V[j][p] as one FMA chain in p order (in TV), then
// the selection on float(T).  The baseline runtime uses the identical chain so
// that t_b equals T[i][base] bit for bit and the baseline's loss is exactly 0.
// Tile: BM rows x BN settings per step, 256 threads as TY x TX with TY = BM/4
// (each thread a 4 x 4 micro-tile); BM = 16 keeps enough CTAs in flight when
// there are few rows, BM = 64 reuses each V tile over more rows when there
// are many.
template <typename TV, int KP, int BM>
__global__ void __launch_bounds__(PT) k_predict_select(PredictArgs<TV> a) {
    constexpr int TY = BM / 4, TX = PT / TY, BN = 4 * TX;
    constexpr int WPR = TX > 32 ? TX / 32 : 1;       // warps sharing one row group
    __shared__ __align__(16) TV Us[KP][BM];
    __shared__ __align__(16) TV Vs[KP][BN + 4];
    __shared__ float cgs[BN];
    __shared__ float tbs[BM];
    __shared__ Cand xw[TY][WPR][4];
    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    const bool sel = a.cg != nullptr;
    const int64_t row_tiles = (a.m + BM - 1) / BM;
    const bool vec_store = sizeof(TV) == 4 && (a.n & 3) == 0 &&
                           ((reinterpret_cast<uintptr_t>(a.T) & 15) == 0);

    for (int64_t rt = blockIdx.x; rt < row_tiles; rt += gridDim.x) {
        const int64_t r0 = rt * BM;
        __syncthreads();
        for (int e = tid; e < KP * BM; e += PT) {
            const int ii = e / KP, p = e % KP;
            const int64_t r = r0 + ii;
            TV u = TV(0);
            if (r < a.m && p < a.k) u = a.U[r * a.ldu + p];
            Us[p][ii] = u;
        }
        __syncthreads();
        if (sel && tid < BM) {
            const TV *vb = a.V + a.base * KP;
            TV acc = TV(0);
#pragma unroll
            for (int p = 0; p < KP; ++p) acc = my_fma(Us[p][tid], vb[p], acc);
            tbs[tid] = (float)acc;
        }
        Cand best[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) best[r] = Cand{0.0f, 0.0f, -1};

        for (int64_t c0 = 0; c0 < a.n; c0 += BN) {
            __syncthreads();
            for (int e = tid; e < KP * BN; e += PT) {
                const int jj = e / KP, p = e % KP;
                const int64_t j = c0 + jj;
                Vs[p][jj] = (j < a.n) ? a.V[j * KP + p] : TV(0);
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
            for (int p = 0; p < KP; ++p) {
                TV u[4], v[4];
                load4<TV>(&Us[p][ty * 4], u);
                load4<TV>(&Vs[p][tx * 4], v);
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[r][c] = my_fma(u[r], v[c], acc[r][c]);
            }
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int64_t i = r0 + ty * 4 + r;
                if (i >= a.m) continue;
                const int64_t j0 = c0 + tx * 4;
                if (a.T) {
                    TV *trow = a.T + i * a.n;
                    if (vec_store && j0 + 3 < a.n) {
                        *reinterpret_cast<float4 *>(trow + j0) =
                            make_float4((float)acc[r][0], (float)acc[r][1], (float)acc[r][2],
                                        (float)acc[r][3]);
                    } else {
#pragma unroll
                        for (int c = 0; c < 4; ++c)
                            if (j0 + c < a.n) trow[j0 + c] = acc[r][c];
                    }
                }
                if (sel) {
                    const float tb = tbs[ty * 4 + r];
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        if (j0 + c < a.n)
                            alg2_consider(best[r], tb, (float)acc[r][c], cgs[tx * 4 + c],
                                          a.Ebase, a.gamma, (int32_t)(j0 + c));
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
    if (sizeof(TV) == 4 && (a.m + 63) / 64 < 2 * NUM_SMS_HINT) return launch_bm<TV, 16>(a, st);
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
        const float tb = __ldg(t + base);
        Cand b{0.0f, 0.0f, -1};
        for (int64_t j = lane; j < n; j += 32)
            alg2_consider(b, tb, __ldg(t + j), __ldg(cg + j), Eb, gamma, (int32_t)j);
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
