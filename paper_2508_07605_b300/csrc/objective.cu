// ALS objective J(U, V) = sum_{(i,j) observed} (R_ij - u_i . v_j)^2
//                         + lambda (|U|_F^2 + |V|_F^2)
// and the per-row RMSE over a row's observed entries (the residual the
// learned warm start is judged by).  Dots are taken in the factor type, the
// residuals squared and summed in FP64.  Rows are assigned to CTAs and warps
// by a fixed partition of m and partial sums are combined in a fixed order,
// so J is bit-reproducible run to run.
#include "common.cuh"
#include "kernels.h"

namespace ocf {

constexpr int OBJ_WARPS = 8;

int64_t objective_parts(int64_t m) {
    int64_t g = (m + 7) / 8;
    if (g > NUM_SMS_HINT * 16) g = NUM_SMS_HINT * 16;
    if (g < 1) g = 1;
    return g;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(FULL, v, off);
    return v;
}

// Compensated (Kahan) running sum in the factor type: B300 executes FP64 at a
// small fraction of the FP32 rate, so the FP32 path accumulates in FP32 with a
// compensation term and touches FP64 only once per CTA.
template <typename T> struct KSum {
    T s = T(0), c = T(0);
    __device__ __forceinline__ void add(T x) {
        const T y = x - c;
        const T t = s + y;
        c = (t - s) - y;
        s = t;
    }
};

template <typename T> __device__ __forceinline__ T warp_sum_t(T v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(FULL, v, off);
    return v;
}

// Per CTA: a fixed contiguous range of rows (one warp per row, lanes over the
// row's entries, u held in registers, v_j read as 16-byte vectors) and a fixed
// slice of V's rows for |V|^2.  part[3b .. 3b+2] = (SSE, |U|^2, |V|^2) of CTA b.
template <typename TV, int KP>
__global__ void __launch_bounds__(OBJ_WARPS * 32)
k_objective_rows(int64_t m, int64_t nnz, const int64_t *__restrict__ ptr,
                 const int32_t *__restrict__ idx, const TV *__restrict__ val,
                 const TV *__restrict__ U, int64_t ldu, int k, const TV *__restrict__ V,
                 int64_t n, double *__restrict__ part, float *__restrict__ row_rmse,
                 const int32_t *__restrict__ ccount) {
    using VT = typename Vec4<TV>::type;
    constexpr int VN = Vec4<TV>::N;
    __shared__ double ws[OBJ_WARPS][3];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t G = gridDim.x;
    const int64_t per = (m + G - 1) / G;
    const int64_t r0 = blockIdx.x * per, r1 = min(m, r0 + per);
    KSum<TV> sse_w, nu_w;
    for (int64_t i = r0 + warp; i < r1; i += OBJ_WARPS) {
        int64_t beg, end;
        const bool ok = row_bounds(ptr, i, nnz, beg, end);
        TV u[KP];
#pragma unroll
        for (int p = 0; p < KP; ++p) u[p] = (p < k) ? U[i * ldu + p] : TV(0);
        TV sse = TV(0);
        for (int64_t t = beg + lane; t < end; t += 32) {
            const int32_t j = __ldg(idx + t);
            if (j < 0 || (int64_t)j >= n) continue;
            const VT *v = reinterpret_cast<const VT *>(V + (int64_t)j * KP);
            TV d = TV(0);
#pragma unroll
            for (int e4 = 0; e4 < KP / VN; ++e4) {
                const VT x = __ldg(v + e4);
#pragma unroll
                for (int e = 0; e < VN; ++e) d = my_fma(u[e4 * VN + e], vget(x, e), d);
            }
            const TV e = __ldg(val + t) - d;
            sse = my_fma(e, e, sse);
        }
        sse = warp_sum_t(sse);
        if (lane == 0) {
            TV nu = TV(0);
#pragma unroll
            for (int p = 0; p < KP; ++p) nu = my_fma(u[p], u[p], nu);
            if (ccount) nu *= TV(end - beg);   // weighted lambda: s_i |u_i|^2
            sse_w.add(sse);
            nu_w.add(nu);
            if (row_rmse) {
                const int64_t s = end - beg;
                row_rmse[i] = (ok && s > 0) ? (float)sqrt((double)sse / (double)s) : 0.0f;
            }
        }
    }
    // this CTA's slice of V (rows of KP elements, padding is zero)
    const int64_t vper = (n + G - 1) / G;
    const int64_t v0 = blockIdx.x * vper * KP, v1 = min(n, (blockIdx.x + 1) * vper) * KP;
    TV nv = TV(0);
    for (int64_t e = v0 + threadIdx.x; e < v1; e += blockDim.x)
        nv = ccount ? my_fma(TV(ccount[e / KP]) * V[e], V[e], nv) : my_fma(V[e], V[e], nv);
    nv = warp_sum_t(nv);
    if (lane == 0) {
        ws[warp][0] = (double)sse_w.s - (double)sse_w.c;
        ws[warp][1] = (double)nu_w.s - (double)nu_w.c;
        ws[warp][2] = (double)nv;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double sa = 0.0, sb = 0.0, sc = 0.0;
        for (int w = 0; w < OBJ_WARPS; ++w) {
            sa += ws[w][0];
            sb += ws[w][1];
            sc += ws[w][2];
        }
        part[3 * blockIdx.x] = sa;
        part[3 * blockIdx.x + 1] = sb;
        part[3 * blockIdx.x + 2] = sc;
    }
}

// One warp: a few FP64 additions per lane instead of a CTA-wide FP64 tree.
__global__ void __launch_bounds__(32)
k_objective_final(int64_t G, const double *__restrict__ part, double lambda,
                  double *__restrict__ J) {
    double a = 0.0, b = 0.0, c = 0.0;
    for (int64_t g = threadIdx.x; g < G; g += 32) {
        a += part[3 * g];
        b += part[3 * g + 1];
        c += part[3 * g + 2];
    }
    a = warp_sum(a);
    b = warp_sum(b);
    c = warp_sum(c);
    if (threadIdx.x == 0) *J = a + lambda * (b + c);
}

// Observations per column: from a CSC column pointer, or by counting a CSR.
__global__ void k_count_from_ptr(int64_t n, const int64_t *__restrict__ cptr,
                                 int32_t *__restrict__ cnt) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x)
        cnt[j] = (int32_t)(cptr[j + 1] - cptr[j]);
}

__global__ void k_count_cols(int64_t nnz, int64_t n, const int32_t *__restrict__ idx,
                             int32_t *__restrict__ cnt) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nnz;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int32_t j = idx[t];
        if (j >= 0 && (int64_t)j < n) atomicAdd(cnt + j, 1);
    }
}

cudaError_t launch_col_counts_from_ptr(int64_t n, const int64_t *cptr, int32_t *cnt,
                                       cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    int64_t b = (n + 255) / 256;
    if (b > NUM_SMS_HINT * 8) b = NUM_SMS_HINT * 8;
    k_count_from_ptr<<<(unsigned)b, 256, 0, st>>>(n, cptr, cnt);
    return cudaGetLastError();
}

cudaError_t launch_col_counts(int64_t nnz, int64_t n, const int32_t *idx, int32_t *cnt,
                              cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (n > 0 ? n : 1), st);
    if (e != cudaSuccess || nnz <= 0) return e;
    int64_t b = (nnz + 255) / 256;
    if (b > NUM_SMS_HINT * 16) b = NUM_SMS_HINT * 16;
    k_count_cols<<<(unsigned)b, 256, 0, st>>>(nnz, n, idx, cnt);
    return cudaGetLastError();
}

template <typename TV>
cudaError_t launch_objective(int64_t m, int64_t nnz, const int64_t *ptr, const int32_t *idx,
                             const TV *val, const TV *U, int64_t ldu, int k, const TV *V,
                             int64_t n, int KP, double lambda, double *part, double *J_out,
                             float *row_rmse, const int32_t *ccount, cudaStream_t st) {
    const int64_t G = objective_parts(m > n ? m : n);
    switch (KP) {
        case 8:
            k_objective_rows<TV, 8><<<(unsigned)G, OBJ_WARPS * 32, 0, st>>>(
                m, nnz, ptr, idx, val, U, ldu, k, V, n, part, row_rmse, ccount);
            break;
        case 16:
            k_objective_rows<TV, 16><<<(unsigned)G, OBJ_WARPS * 32, 0, st>>>(
                m, nnz, ptr, idx, val, U, ldu, k, V, n, part, row_rmse, ccount);
            break;
        case 32:
            k_objective_rows<TV, 32><<<(unsigned)G, OBJ_WARPS * 32, 0, st>>>(
                m, nnz, ptr, idx, val, U, ldu, k, V, n, part, row_rmse, ccount);
            break;
        default: return cudaErrorInvalidValue;
    }
    k_objective_final<<<1, 32, 0, st>>>(G, part, lambda, J_out);
    return cudaGetLastError();
}

template cudaError_t launch_objective<float>(int64_t, int64_t, const int64_t *, const int32_t *,
                                             const float *, const float *, int64_t, int,
                                             const float *, int64_t, int, double, double *,
                                             double *, float *, const int32_t *, cudaStream_t);
template cudaError_t launch_objective<double>(int64_t, int64_t, const int64_t *, const int32_t *,
                                              const double *, const double *, int64_t, int,
                                              const double *, int64_t, int, double, double *,
                                              double *, float *, const int32_t *, cudaStream_t);

}  // namespace ocf
