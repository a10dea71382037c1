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

template <int KP>
__device__ void solve_range(const SolveArgs<float> &a, int wig, int W, unsigned char *wsbase,
                            int warp, int lane) {
    using WS = WarpSmem<float, float, KP>;
    // each warp's area starts at warp * sizeof(WS32); solve_system indexes smem[warp]
    WS *mine = reinterpret_cast<WS *>(wsbase + (size_t)warp * sizeof(WS32));
    for (int64_t i = wig; i < a.m; i += W) solve_system<float, float, KP, 1, false>(a, i, mine, 0, lane);
}

__device__ void run_half(const SolveArgs<float> &a, int KP, int wig, int W, unsigned char *wsbase,
                         int warp, int lane) {
    if (KP == 8) solve_range<8>(a, wig, W, wsbase, warp, lane);
    else if (KP == 16) solve_range<16>(a, wig, W, wsbase, warp, lane);
    else solve_range<32>(a, wig, W, wsbase, warp, lane);
}

__global__ void __launch_bounds__(BW * 32, 2) k_batched_als(BatchArgs b) {   // two CTAs per SM
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int32_t qslot[BW];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

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
                run_half(ua, KP, wig, W, gbase, wig, lane);
                group_sync(bar, gthreads);
                run_half(va, KP, wig, W, gbase, wig, lane);
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
