// Shared device helpers of the open_cf CUDA library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "open_cf.h"

namespace ocf {

constexpr unsigned FULL = 0xffffffffu;
constexpr int NUM_SMS_HINT = 148;

// Status codes mirrored from the header for device code.
constexpr int32_t ST_OK = OPEN_CF_ROW_OK;
constexpr int32_t ST_NOT_SPD = OPEN_CF_ROW_NOT_SPD;
constexpr int32_t ST_EMPTY = OPEN_CF_ROW_EMPTY;
constexpr int32_t ST_FALLBACK = OPEN_CF_ROW_FALLBACK_USED;
constexpr int32_t ST_BAD = OPEN_CF_ROW_BAD_INPUT;

// Padded rank: factors live in HBM as rows of KP elements (zero padded), so a
// row is a whole number of 16-byte vectors and the padded unknowns solve to 0.
__host__ __device__ inline int padded_k(int k) { return k <= 8 ? 8 : (k <= 16 ? 16 : 32); }

template <typename T> struct Vec4;
template <> struct Vec4<float> {
    using type = float4;
    static constexpr int N = 4;
};
template <> struct Vec4<double> {
    using type = double2;
    static constexpr int N = 2;
};

__device__ __forceinline__ float vget(const float4 &v, int e) {
    return e == 0 ? v.x : (e == 1 ? v.y : (e == 2 ? v.z : v.w));
}
__device__ __forceinline__ double vget(const double2 &v, int e) { return e == 0 ? v.x : v.y; }

__device__ __forceinline__ float my_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double my_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float my_fma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double my_fma(double a, double b, double c) { return fma(a, b, c); }

// Row bounds with validation against nnz: returns false if the row is malformed.
__device__ __forceinline__ bool row_bounds(const int64_t *__restrict__ ptr, int64_t row,
                                           int64_t nnz, int64_t &beg, int64_t &end) {
    beg = __ldg(ptr + row);
    end = __ldg(ptr + row + 1);
    bool ok = (beg >= 0) && (end >= beg) && (end <= nnz);
    if (!ok) { beg = 0; end = 0; }
    return ok;
}

}  // namespace ocf
