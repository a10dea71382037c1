// Device pieces shared by the fused tcgen05 kernels of the learned warm start:
// inference (mlp_tc.cu) and training (mlp_train_tc.cu).
//
// Operand images (no swizzle): an R x K BF16 matrix stored K-major as 8 x 8
// core matrices of 128 contiguous bytes, element (r, k) at byte
//   (r / 8) * (16 K) + (k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2.
// A tcgen05 descriptor reads it K-major with leading-dimension offset 128 B
// (next 8 columns of K) and stride-dimension offset 16 K bytes (next 8 rows).
// The same bytes read MN-major (the matrix transposed: R becomes the M or N
// extent, the rows of the image become K) with stride-dimension offset 128 B
// (next 8 of M or N) and leading-dimension offset 16 K bytes per 8 of K; the
// training kernel uses this to take activation images of the forward pass as
// operands of the weight-gradient products without rewriting them.
#pragma once
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"
#include "tc_util.cuh"

namespace ocf {
namespace mlp {

using namespace tc;

constexpr int TM = 128;   // rows per tile (UMMA M)

constexpr float SELU_L = 1.0507009873554804934193349852946f;
constexpr float SELU_A = 1.6732632423543772848170429916717f;

__device__ __forceinline__ float selu_f(float z) {
    const float e = __expf(fminf(z, 0.f)) - 1.f;
    return z > 0.f ? SELU_L * z : (SELU_L * SELU_A) * e;
}

// d selu / dz
__device__ __forceinline__ float dselu_f(float z) {
    return z > 0.f ? SELU_L : (SELU_L * SELU_A) * __expf(z);
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&h);
}

// Element offset of (r, k) in an R x K K-major image (units of BF16 elements).
__host__ __device__ constexpr int64_t kimg(int64_t r, int64_t k, int64_t K) {
    return (r / 8) * (8 * K) + (k / 8) * 64 + (r % 8) * 8 + k % 8;
}

// Positions of weight W_l[in][out] in the image buffer (element units):
//   W2F: W2 for the forward product, 4 chunks (64 inputs each) of 256 x 64;
//   W1:  256 x 64;  W3F: 32 x 256;  (R = outputs, K = inputs)
//   W2B: W2 for the backward product, 4 chunks (64 outputs each) of 256 x 64;
//   W3B: 256 x 32  (R = inputs, K = outputs).
__host__ __device__ constexpr int64_t img_w1(int64_t i, int64_t o) {
    return MLP_IMG_W1 + kimg(o, i, MLP_INP);
}
__host__ __device__ constexpr int64_t img_w2f(int64_t i, int64_t o) {
    return MLP_IMG_W2F + (i / 64) * (MLP_H * 64) + kimg(o, i % 64, 64);
}
__host__ __device__ constexpr int64_t img_w3f(int64_t i, int64_t o) {
    return MLP_IMG_W3F + kimg(o, i, MLP_H);
}
__host__ __device__ constexpr int64_t img_w2b(int64_t i, int64_t o) {
    return MLP_IMG_W2B + (o / 64) * (MLP_H * 64) + kimg(i, o % 64, 64);
}
__host__ __device__ constexpr int64_t img_w3b(int64_t i, int64_t o) {
    return MLP_IMG_W3B + kimg(i, o, MLP_K_OUT);
}

// The tile's rows are shared by groups of four lanes (row r = tid / 4, lane
// g = tid % 4): lane g takes the row's observation slots g, g + 4, g + 8,
// g + 12 (the first 16 in setting order), keeps their indices and values in
// registers (the inference kernel's residual reuses them) and writes their
// features (c_norm, g_norm, runtime) into the BF16 feature image (K = 64;
// slot s -> features 3s .. 3s + 2; features 48 .. 63 stay zero).  Rows at or
// beyond a.m get all-zero features.
struct RowObs {
    int64_t beg, end;
    bool ok;
    int32_t j[4];   // -1: no observation in the slot, or an index out of range
    float v[4];
};

template <typename Args>
__device__ __forceinline__ void features_quad(const Args &a, int64_t i, int r, int g,
                                              unsigned char *act, RowObs &o) {
    o.beg = 0;
    o.end = 0;
    o.ok = i < a.m && row_bounds(a.ptr, i, a.nnz, o.beg, o.end);
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const int64_t t = o.beg + g + 4 * b;
        o.j[b] = -1;
        o.v[b] = 0.f;
        if (o.ok && t < o.end) {
            const int32_t jj = __ldg(a.idx + t);
            o.v[b] = __ldg(a.val + t);
            if (jj >= 0 && (int64_t)jj < a.n) o.j[b] = jj;
        }
    }
    unsigned char *row = act + (r >> 3) * (MLP_INP * 16) + (r & 7) * 16;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const int s = g + 4 * b;
        float c = 0.f, gg = 0.f, v = 0.f;
        if (o.j[b] >= 0) {
            const int32_t ci = o.j[b] / a.n_gpu;
            c = __ldg(a.ccap + ci);
            gg = __ldg(a.gcap + (o.j[b] - ci * a.n_gpu));
            v = o.v[b];
        }
        const float x[3] = {c, gg, v};
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            const int f = 3 * s + e;
            *reinterpret_cast<__nv_bfloat16 *>(row + (f >> 3) * 128 + (f & 7) * 2) =
                __float2bfloat16_rn(x[e]);
        }
    }
    if (g < 2) *reinterpret_cast<uint4 *>(row + (6 + g) * 128) = make_uint4(0, 0, 0, 0);
}

// Hidden-layer epilogue: this warp's 32 rows (TMEM lane quarter q), columns
// [c0, c0 + 64) of the accumulator at TMEM column tacc: bias (shared memory)
// + SELU -> BF16 image (K = 256).  Both TMEM loads are in flight before the
// first wait.
__device__ __forceinline__ void epi_hidden(uint32_t tmem, uint32_t tacc, int q, int lane, int c0,
                                           const float *bias_s, unsigned char *act) {
    const int r = 32 * q + lane;
    unsigned char *row = act + (r >> 3) * (MLP_H * 16) + (r & 7) * 16;
    uint32_t v0[32], v1[32];
    const uint32_t ta = tmem + ((uint32_t)(32 * q) << 16) + tacc + (uint32_t)c0;
    tc_ld32(ta, v0);
    tc_ld32(ta + 32, v1);
    tc_wait_ld();
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        uint32_t pk[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int c = 8 * g + 2 * e;
            pk[e] = pack_bf16(selu_f(__uint_as_float(v0[c]) + bias_s[c0 + c]),
                              selu_f(__uint_as_float(v0[c + 1]) + bias_s[c0 + c + 1]));
        }
        *reinterpret_cast<uint4 *>(row + (c0 / 8 + g) * 128) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    }
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        uint32_t pk[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int c = 8 * g + 2 * e;
            pk[e] = pack_bf16(selu_f(__uint_as_float(v1[c]) + bias_s[c0 + 32 + c]),
                              selu_f(__uint_as_float(v1[c + 1]) + bias_s[c0 + 32 + c + 1]));
        }
        *reinterpret_cast<uint4 *>(row + ((c0 + 32) / 8 + g) * 128) =
            make_uint4(pk[0], pk[1], pk[2], pk[3]);
    }
}

// Programmatic dependent launch within a training step: the training kernel
// lets the reduction launch at once; the reduction waits for it before its
// first read of the partial sums.
__device__ __forceinline__ void pdl_trigger() {
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }

// Store (first tile of a slot's owner) or add (later tiles) one partial sum.
__device__ __forceinline__ void acc_store(float *p, float v, bool first) {
    *p = first ? v : *p + v;
}

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(FULL, x, off);
    return x;
}

}  // namespace mlp
}  // namespace ocf
