// Layout and input-check kernels: padded factor rows, BF16 factor copies, the
// CSR view of a dense offline block (Eq. 1: every entry observed), and the
// device-side CSR validation behind open_cf_validate_csr.
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"

namespace ocf {

static unsigned grid_for(int64_t work, int threads) {
    int64_t b = (work + threads - 1) / threads;
    if (b > NUM_SMS_HINT * 32) b = NUM_SMS_HINT * 32;
    return (unsigned)(b < 1 ? 1 : b);
}

template <typename TV>
__global__ void k_pack_rows(const TV *__restrict__ src, int64_t rows, int64_t lds, int k,
                            TV *__restrict__ dst, int KP) {
    const int64_t total = rows * KP;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / KP;
        const int p = (int)(e % KP);
        dst[e] = p < k ? src[r * lds + p] : TV(0);
    }
}

template <typename TV>
__global__ void k_unpack_rows(const TV *__restrict__ src, int64_t rows, int KP, int k,
                              TV *__restrict__ dst) {
    const int64_t total = rows * k;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / k;
        const int p = (int)(e % k);
        dst[e] = src[r * KP + p];
    }
}

__global__ void k_to_bf16(const float *__restrict__ src, int64_t count,
                          __nv_bfloat16 *__restrict__ dst) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
         e += (int64_t)gridDim.x * blockDim.x)
        dst[e] = __float2bfloat16_rn(src[e]);
}

__global__ void k_to_bf16_split(const float *__restrict__ src, int64_t rows, int KP,
                                __nv_bfloat16 *__restrict__ dst) {
    const int64_t total = rows * KP;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / KP;
        const int p = (int)(e % KP);
        const float x = src[e];
        const __nv_bfloat16 hi = __float2bfloat16_rn(x);
        dst[r * 2 * KP + p] = hi;
        dst[r * 2 * KP + KP + p] = __float2bfloat16_rn(x - __bfloat162float(hi));
    }
}

template <typename TV>
__global__ void k_dense_to_csr(const TV *__restrict__ P, int64_t m, int64_t n, int64_t ld,
                               int64_t *__restrict__ ptr, int32_t *__restrict__ idx,
                               TV *__restrict__ val) {
    const int64_t total = m * n;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / n, j = e % n;
        idx[e] = (int32_t)j;
        val[e] = P[i * ld + j];
        if (j == 0) ptr[i] = e;
        if (e == total - 1) ptr[m] = total;
    }
}

// flag: 0 valid, else the smallest failed check code (atomicMin).
template <typename TV>
__global__ void k_validate_csr(int64_t m, int64_t n, int64_t nnz, const int64_t *__restrict__ ptr,
                               const int32_t *__restrict__ idx, const TV *__restrict__ val,
                               int32_t *__restrict__ flag) {
    const int lane = threadIdx.x & 31;
    const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    if (w == 0 && lane == 0) {
        if (ptr[0] != 0 || ptr[m] != nnz) atomicMin(flag, 1);
    }
    for (int64_t i = w; i < m; i += nw) {
        const int64_t beg = ptr[i], end = ptr[i + 1];
        if (beg < 0 || end < beg || end > nnz) {
            if (lane == 0) atomicMin(flag, 1);
            continue;
        }
        for (int64_t t = beg + lane; t < end; t += 32) {
            const int32_t c = idx[t];
            if (c < 0 || (int64_t)c >= n) atomicMin(flag, 2);
            else if (t > beg && idx[t - 1] >= c) atomicMin(flag, 3);
            if (!isfinite((double)val[t])) atomicMin(flag, 4);
        }
    }
}

template <typename TV>
cudaError_t launch_pack_rows(const TV *src, int64_t rows, int64_t lds, int k, TV *dst, int KP,
                             cudaStream_t st) {
    if (rows <= 0) return cudaSuccess;
    k_pack_rows<TV><<<grid_for(rows * KP, 256), 256, 0, st>>>(src, rows, lds, k, dst, KP);
    return cudaGetLastError();
}

template <typename TV>
cudaError_t launch_unpack_rows(const TV *src, int64_t rows, int KP, int k, TV *dst,
                               cudaStream_t st) {
    if (rows <= 0) return cudaSuccess;
    k_unpack_rows<TV><<<grid_for(rows * k, 256), 256, 0, st>>>(src, rows, KP, k, dst);
    return cudaGetLastError();
}

cudaError_t launch_to_bf16(const float *src, int64_t count, void *dst, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    k_to_bf16<<<grid_for(count, 256), 256, 0, st>>>(src, count,
                                                    reinterpret_cast<__nv_bfloat16 *>(dst));
    return cudaGetLastError();
}

cudaError_t launch_to_bf16_split(const float *src, int64_t rows, int KP, void *dst,
                                 cudaStream_t st) {
    if (rows <= 0) return cudaSuccess;
    k_to_bf16_split<<<grid_for(rows * KP, 256), 256, 0, st>>>(
        src, rows, KP, reinterpret_cast<__nv_bfloat16 *>(dst));
    return cudaGetLastError();
}

template <typename TV>
cudaError_t launch_dense_to_csr(const TV *P, int64_t m, int64_t n, int64_t ld, int64_t *ptr,
                                int32_t *idx, TV *val, cudaStream_t st) {
    if (m <= 0 || n <= 0) return cudaMemsetAsync(ptr, 0, sizeof(int64_t) * (m + 1), st);
    k_dense_to_csr<TV><<<grid_for(m * n, 256), 256, 0, st>>>(P, m, n, ld, ptr, idx, val);
    return cudaGetLastError();
}

template <typename TV>
cudaError_t launch_validate_csr(int64_t m, int64_t n, int64_t nnz, const int64_t *ptr,
                                const int32_t *idx, const TV *val, int32_t *flag,
                                cudaStream_t st) {
    k_validate_csr<TV><<<grid_for(m * 32 + 32, 256), 256, 0, st>>>(m, n, nnz, ptr, idx, val,
                                                                   flag);
    return cudaGetLastError();
}

#define OCF_INST(TV)                                                                         \
    template cudaError_t launch_pack_rows<TV>(const TV *, int64_t, int64_t, int, TV *, int,   \
                                              cudaStream_t);                                 \
    template cudaError_t launch_unpack_rows<TV>(const TV *, int64_t, int, int, TV *,          \
                                                cudaStream_t);                               \
    template cudaError_t launch_dense_to_csr<TV>(const TV *, int64_t, int64_t, int64_t,       \
                                                 int64_t *, int32_t *, TV *, cudaStream_t);  \
    template cudaError_t launch_validate_csr<TV>(int64_t, int64_t, int64_t, const int64_t *,  \
                                                 const int32_t *, const TV *, int32_t *,     \
                                                 cudaStream_t);
OCF_INST(float)
OCF_INST(double)

}  // namespace ocf
