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

template <typename TV>
__global__ void __launch_bounds__(OBJ_WARPS * 32)
k_objective_rows(int64_t m, int64_t nnz, const int64_t *__restrict__ ptr,
                 const int32_t *__restrict__ idx, const TV *__restrict__ val,
                 const TV *__restrict__ U, int64_t ldu, int k, const TV *__restrict__ V,
                 int64_t n, int KP, double *__restrict__ part, float *__restrict__ row_rmse) {
    __shared__ double ws[OBJ_WARPS][2];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t G = gridDim.x;
    const int64_t per = (m + G - 1) / G;
    const int64_t r0 = blockIdx.x * per, r1 = min(m, r0 + per);
    double sse_w = 0.0, nu_w = 0.0;
    for (int64_t i = r0 + warp; i < r1; i += OBJ_WARPS) {
        int64_t beg, end;
        const bool ok = row_bounds(ptr, i, nnz, beg, end);
        const TV *u = U + i * ldu;
        double sse = 0.0;
        for (int64_t t = beg + lane; t < end; t += 32) {
            const int32_t j = __ldg(idx + t);
            if (j < 0 || (int64_t)j >= n) continue;
            const TV *v = V + (int64_t)j * KP;
            TV d = TV(0);
            for (int p = 0; p < k; ++p) d = my_fma(u[p], v[p], d);
            const double e = (double)__ldg(val + t) - (double)d;
            sse += e * e;
        }
        sse = warp_sum(sse);
        double nu = 0.0;
        if (lane < k) nu = (double)u[lane] * (double)u[lane];
        nu = warp_sum(nu);
        if (lane == 0) {
            sse_w += sse;
            nu_w += nu;
            if (row_rmse) {
                const int64_t s = end - beg;
                row_rmse[i] = (ok && s > 0) ? (float)sqrt(sse / (double)s) : 0.0f;
            }
        }
    }
    if (lane == 0) {
        ws[warp][0] = sse_w;
        ws[warp][1] = nu_w;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double sa = 0.0, sb = 0.0;
        for (int w = 0; w < OBJ_WARPS; ++w) {
            sa += ws[w][0];
            sb += ws[w][1];
        }
        part[2 * blockIdx.x] = sa;
        part[2 * blockIdx.x + 1] = sb;
    }
}

template <typename TV>
__global__ void __launch_bounds__(1024)
k_objective_final(int64_t G, const double *__restrict__ part, const TV *__restrict__ V,
                  int64_t n, int KP, int k, double lambda, double *__restrict__ J) {
    __shared__ double ws[32][3];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    double a = 0.0, b = 0.0, c = 0.0;
    for (int64_t g = threadIdx.x; g < G; g += blockDim.x) {
        a += part[2 * g];
        b += part[2 * g + 1];
    }
    for (int64_t e = threadIdx.x; e < n * KP; e += blockDim.x) {
        if ((int)(e % KP) < k) {
            const double v = (double)V[e];
            c += v * v;
        }
    }
    a = warp_sum(a);
    b = warp_sum(b);
    c = warp_sum(c);
    if (lane == 0) {
        ws[w][0] = a;
        ws[w][1] = b;
        ws[w][2] = c;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double sa = 0.0, sb = 0.0, sc = 0.0;
        for (int i = 0; i < 32; ++i) {
            sa += ws[i][0];
            sb += ws[i][1];
            sc += ws[i][2];
        }
        *J = sa + lambda * (sb + sc);
    }
}

template <typename TV>
cudaError_t launch_objective(int64_t m, int64_t nnz, const int64_t *ptr, const int32_t *idx,
                             const TV *val, const TV *U, int64_t ldu, int k, const TV *V,
                             int64_t n, int KP, double lambda, double *part, double *J_out,
                             float *row_rmse, cudaStream_t st) {
    const int64_t G = objective_parts(m);
    if (m > 0)
        k_objective_rows<TV><<<(unsigned)G, OBJ_WARPS * 32, 0, st>>>(
            m, nnz, ptr, idx, val, U, ldu, k, V, n, KP, part, row_rmse);
    else
        cudaMemsetAsync(part, 0, sizeof(double) * 2, st);
    k_objective_final<TV><<<1, 1024, 0, st>>>(m > 0 ? G : 1, part, V, n, KP, k, lambda, J_out);
    return cudaGetLastError();
}

template cudaError_t launch_objective<float>(int64_t, int64_t, const int64_t *, const int32_t *,
                                             const float *, const float *, int64_t, int,
                                             const float *, int64_t, int, double, double *,
                                             double *, float *, cudaStream_t);
template cudaError_t launch_objective<double>(int64_t, int64_t, const int64_t *, const int32_t *,
                                              const double *, const double *, int64_t, int,
                                              const double *, int64_t, int, double, double *,
                                              double *, float *, cudaStream_t);

}  // namespace ocf
