// FMA-loop microbenchmark: the FP32 / FP64 fused multiply-add throughput of
// this GPU, measured, as the denominator of the ALU rooflines (the row solves
// and the selection epilogues are bound by these pipes, not by memory).
// Every thread runs CHAINS independent FMA chains so that the pipe, not the
// dependency latency, limits the rate; the results are summed into one word
// so that no chain can be removed as dead code.
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"
#include "open_cf.h"

namespace ocf {

namespace {

constexpr int CHAINS = 8;

template <typename T>
__global__ void __launch_bounds__(256) k_fma_loop(int iters, T a, T b, T *out) {
    T x[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = T(threadIdx.x + c) * T(1e-3);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < CHAINS; ++c) x[c] = my_fma(x[c], a, b);
    }
    T s = T(0);
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) s += x[c];
    if (s == T(12345.678)) out[0] = s;   // practically never true; keeps the chains alive
}

template <typename T>
int measure(int device, double *tflops) {
    int sms = 0;
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
        return OPEN_CF_CUDA_ERROR;
    T *out = nullptr;
    if (cudaMalloc(&out, sizeof(T)) != cudaSuccess) return OPEN_CF_OUT_OF_MEMORY;
    const int blocks = sms * 8, threads = 256;
    const int iters = sizeof(T) == 8 ? 1 << 12 : 1 << 16;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_fma_loop<T><<<blocks, threads>>>(iters / 16, T(0.999), T(1e-4), out);   // warm-up
    cudaEventRecord(e0);
    k_fma_loop<T><<<blocks, threads>>>(iters, T(0.999), T(1e-4), out);
    cudaEventRecord(e1);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (e != cudaSuccess || !(ms > 0.f)) {
        cudaGetLastError();
        return OPEN_CF_CUDA_ERROR;
    }
    const double flop = 2.0 * CHAINS * (double)iters * blocks * threads;
    *tflops = flop / (ms * 1e-3) / 1e12;
    return OPEN_CF_OK;
}

}  // namespace

}  // namespace ocf

extern "C" int open_cf_fma_peak(int32_t fp64, int32_t device, double *tflops_host) {
    if (!tflops_host) return OPEN_CF_INVALID_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return OPEN_CF_INVALID_ARG;
    }
    int prev = 0;
    cudaGetDevice(&prev);
    const int rc = fp64 ? ocf::measure<double>(device, tflops_host)
                        : ocf::measure<float>(device, tflops_host);
    cudaSetDevice(prev);
    return rc;
}
