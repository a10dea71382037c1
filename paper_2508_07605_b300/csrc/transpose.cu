// CSR -> CSC transpose by a stable counting sort on the column index.
//
// The V-half of an ALS sweep solves one system per setting (column) and needs
// the observations grouped by column (the sparse matrix of Sec. "Online
// Performance Prediction", seen column-wise).  Entries of one column keep
// increasing row order, so the V-half sums in a fixed order and a fit is
// bit-reproducible.
//
// Rows are cut into nb contiguous blocks of RB = 32 * S rows.  Pass 1 counts,
// per block, how many entries fall in each column (cnt[b][c], shared-memory
// atomics); pass 2 turns the counts into per-block exclusive offsets within
// each column and column totals; pass 3 scans the totals into col_ptr; pass 4
// places every entry at once: a block walks its rows in S sub-blocks of 32;
// for each sub-block it ORs, per column, a bit for every row that holds the
// column, so the stable rank of entry (r, c) inside its column is
// popc(mask[c] & bits below r) plus the column's entries from earlier
// sub-blocks and blocks.  A row holds each column at most once.
#include "common.cuh"
#include "kernels.h"

namespace ocf {

CscPlan csc_plan(int64_t m, int64_t n, int64_t nnz, int64_t nb_cap) {
    int64_t target = nnz / (n > 0 ? n : 1);   // counters ~ entries
    if (target < 148) target = 148;
    if (target > 4096) target = 4096;
    if (nb_cap > 0 && target > nb_cap) target = nb_cap;
    if (target < 1) target = 1;
    const int64_t mm = m > 0 ? m : 1;
    int64_t rb = (mm + target - 1) / target;
    rb = ((rb + 31) / 32) * 32;
    int64_t nb = (mm + rb - 1) / rb;
    while (nb_cap > 0 && nb > nb_cap) {   // rounding can overshoot a hard cap
        rb += 32;
        nb = (mm + rb - 1) / rb;
    }
    return CscPlan{rb, nb};
}

__global__ void k_csc_count(int64_t m, int64_t n, int64_t nnz, const int64_t *__restrict__ ptr,
                            const int32_t *__restrict__ idx, int32_t *__restrict__ cnt,
                            int64_t RB) {
    extern __shared__ int32_t sc[];
    const int64_t b = blockIdx.x;
    for (int64_t c = threadIdx.x; c < n; c += blockDim.x) sc[c] = 0;
    __syncthreads();
    const int64_t r0 = b * RB, r1 = min(m, r0 + RB);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int64_t r = r0 + warp; r < r1; r += nw) {
        int64_t beg, end;
        if (!row_bounds(ptr, r, nnz, beg, end)) continue;
        for (int64_t e = beg + lane; e < end; e += 32) {
            const int32_t c = __ldg(idx + e);
            if (c >= 0 && (int64_t)c < n) atomicAdd(&sc[c], 1);
        }
    }
    __syncthreads();
    for (int64_t c = threadIdx.x; c < n; c += blockDim.x) cnt[b * n + c] = sc[c];
}

// One CTA of 32 warps per 32 columns; warp w scans blocks [w*B, (w+1)*B).
__global__ void __launch_bounds__(1024)
k_csc_scan_blocks(int64_t n, int64_t nb, int32_t *__restrict__ cnt, int64_t *__restrict__ tot) {
    __shared__ int64_t part[32][33];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t c = (int64_t)blockIdx.x * 32 + lane;
    const int64_t B = (nb + 31) / 32;
    const int64_t b0 = w * B, b1 = min(nb, b0 + B);
    int64_t s = 0;
    if (c < n)
        for (int64_t b = b0; b < b1; ++b) s += cnt[b * n + c];
    part[w][lane] = s;
    __syncthreads();
    if (w == 0) {
        int64_t run = 0;
        for (int v = 0; v < 32; ++v) {
            const int64_t t = part[v][lane];
            part[v][lane] = run;
            run += t;
        }
        if (c < n) tot[c] = run;
    }
    __syncthreads();
    if (c < n) {
        int64_t run = part[w][lane];
        for (int64_t b = b0; b < b1; ++b) {
            const int32_t t = cnt[b * n + c];
            cnt[b * n + c] = (int32_t)run;
            run += t;
        }
    }
}

// Exclusive scan of tot[0..n) into cptr[0..n]; one CTA of 1024 threads.
__global__ void __launch_bounds__(1024)
k_csc_colptr(int64_t n, const int64_t *__restrict__ tot, int64_t *__restrict__ cptr) {
    __shared__ int64_t ws[32];
    const int64_t per = (n + blockDim.x - 1) / blockDim.x;
    const int64_t c0 = threadIdx.x * per, c1 = min(n, c0 + per);
    int64_t s = 0;
    for (int64_t c = c0; c < c1; ++c) s += tot[c];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    long long inc = s;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const long long t = __shfl_up_sync(FULL, inc, off);
        if (lane >= off) inc += t;
    }
    if (lane == 31) ws[w] = inc;
    __syncthreads();
    if (w == 0) {
        long long v = ws[lane];
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const long long t = __shfl_up_sync(FULL, v, off);
            if (lane >= off) v += t;
        }
        ws[lane] = v;
    }
    __syncthreads();
    int64_t run = inc - s + (w > 0 ? ws[w - 1] : 0);
    for (int64_t c = c0; c < c1; ++c) {
        cptr[c] = run;
        run += tot[c];
    }
    if (threadIdx.x == blockDim.x - 1) cptr[n] = run;
}

template <typename TV>
__global__ void __launch_bounds__(256)
k_csc_scatter(int64_t m, int64_t n, int64_t nnz, const int64_t *__restrict__ ptr,
              const int32_t *__restrict__ idx, const TV *__restrict__ val,
              const int32_t *__restrict__ cnt, const int64_t *__restrict__ cptr,
              int32_t *__restrict__ ridx, TV *__restrict__ cval, int64_t RB) {
    extern __shared__ uint32_t sm32[];
    uint32_t *mask = sm32;                              // [n] rows of the sub-block holding c
    int32_t *run = reinterpret_cast<int32_t *>(sm32 + n);   // [n] placed so far in column c
    const int64_t b = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int64_t c = threadIdx.x; c < n; c += blockDim.x) run[c] = cnt[b * n + c];
    const int64_t r0 = b * RB, r1 = min(m, r0 + RB);
    for (int64_t rs = r0; rs < r1; rs += 32) {
        const int64_t re = min(r1, rs + 32);
        for (int64_t c = threadIdx.x; c < n; c += blockDim.x) mask[c] = 0u;
        __syncthreads();
        for (int64_t r = rs + warp; r < re; r += nw) {
            int64_t beg, end;
            if (!row_bounds(ptr, r, nnz, beg, end)) continue;
            const uint32_t bit = 1u << (unsigned)(r - rs);
            for (int64_t e = beg + lane; e < end; e += 32) {
                const int32_t c = __ldg(idx + e);
                if (c >= 0 && (int64_t)c < n) atomicOr(&mask[c], bit);
            }
        }
        __syncthreads();
        for (int64_t r = rs + warp; r < re; r += nw) {
            int64_t beg, end;
            if (!row_bounds(ptr, r, nnz, beg, end)) continue;
            const uint32_t below = (1u << (unsigned)(r - rs)) - 1u;
            for (int64_t e = beg + lane; e < end; e += 32) {
                const int32_t c = __ldg(idx + e);
                if (c >= 0 && (int64_t)c < n) {
                    const int64_t pos = __ldg(cptr + c) + run[c] + __popc(mask[c] & below);
                    ridx[pos] = (int32_t)r;
                    cval[pos] = __ldg(val + e);
                }
            }
        }
        __syncthreads();
        for (int64_t c = threadIdx.x; c < n; c += blockDim.x) run[c] += __popc(mask[c]);
        __syncthreads();
    }
}

cudaError_t prepare_csr_to_csc(int64_t n_max) {
    if (n_max > CSC_MAX_N) return cudaErrorInvalidValue;
    const int nn = (int)(n_max > 6144 ? n_max : 6144);
    cudaError_t e = cudaFuncSetAttribute(k_csc_count, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(int32_t) * nn);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_csc_scatter<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             2 * (int)sizeof(int32_t) * nn);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_csc_scatter<double>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                2 * (int)sizeof(int32_t) * nn);
}

template <typename TV>
cudaError_t launch_csr_to_csc(int64_t m, int64_t n, int64_t nnz, const int64_t *ptr,
                              const int32_t *idx, const TV *val, int64_t *cptr, int32_t *ridx,
                              TV *cval, int32_t *cnt, int64_t *tot, CscPlan plan,
                              cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if (m <= 0) return cudaMemsetAsync(cptr, 0, sizeof(int64_t) * (n + 1), st);
    const int64_t nb = plan.nb;
    const size_t sm = sizeof(int32_t) * n;
    k_csc_count<<<(unsigned)nb, 256, sm, st>>>(m, n, nnz, ptr, idx, cnt, plan.rb);
    k_csc_scan_blocks<<<(unsigned)((n + 31) / 32), 1024, 0, st>>>(n, nb, cnt, tot);
    k_csc_colptr<<<1, 1024, 0, st>>>(n, tot, cptr);
    k_csc_scatter<TV><<<(unsigned)nb, 256, 2 * sm, st>>>(m, n, nnz, ptr, idx, val, cnt, cptr,
                                                        ridx, cval, plan.rb);
    return cudaGetLastError();
}

template cudaError_t launch_csr_to_csc<float>(int64_t, int64_t, int64_t, const int64_t *,
                                              const int32_t *, const float *, int64_t *,
                                              int32_t *, float *, int32_t *, int64_t *, CscPlan,
                                              cudaStream_t);
template cudaError_t launch_csr_to_csc<double>(int64_t, int64_t, int64_t, const int64_t *,
                                               const int32_t *, const double *, int64_t *,
                                               int32_t *, double *, int32_t *, int64_t *,
                                               CscPlan, cudaStream_t);

}  // namespace ocf
