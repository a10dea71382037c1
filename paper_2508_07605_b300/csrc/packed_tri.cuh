// Rank-32 factorisation helpers shared by the fold-in solver (solve32_tc.cu)
// and the batched fit (batched.cu): packed lower triangles in shared memory,
// the packed FP32x2 update, and the back substitution of a half-warp that
// holds rows i and i + 16 of its system.
#pragma once

#include "common.cuh"

namespace ocf {
namespace pk {

constexpr int KP = 32;

// Packed lower triangles in shared memory.  By rows (A): row r holds entries
// 0 .. r padded to 4 floats; by columns (L): column p holds rows 4 floor(p/4)
// .. 31 (so 16-byte loads stay aligned).  Lanes of a quarter-warp load eight
// consecutive rows (columns) at once, so within each block of 8 rows
// (columns) every start sits in a different 4-bank group: a row (column) is
// moved forward by whole 16-byte steps until its group is free.
struct Tab {
    int v[33];
};
__host__ __device__ constexpr int colbase(int p) { return 4 * (p >> 2); }
__host__ __device__ constexpr Tab make_rows() {
    Tab t{};
    int cur = 0, used = 0;
    for (int q = 0; q < 32; ++q) {
        if ((q & 7) == 0) used = 0;
        while (used & (1 << ((cur >> 2) & 7))) cur += 4;
        t.v[q] = cur;
        used |= 1 << ((cur >> 2) & 7);
        cur += 4 * ((q + 4) >> 2);
    }
    t.v[32] = cur;
    return t;
}
__host__ __device__ constexpr Tab make_cols() {
    Tab t{};
    int cur = 0, used = 0;
    for (int q = 0; q < 32; ++q) {
        if ((q & 7) == 0) used = 0;
        while (used & (1 << (((cur - colbase(q)) >> 2) & 7))) cur += 4;
        t.v[q] = cur;
        used |= 1 << (((cur - colbase(q)) >> 2) & 7);
        cur += 32 - colbase(q);
    }
    t.v[32] = cur;
    return t;
}
constexpr int NROWP = make_rows().v[32], NCOLP = make_cols().v[32];
static_assert(NROWP == 676 && NCOLP == 672, "packed triangle sizes");
__device__ constexpr Tab ROWT = make_rows();
__device__ constexpr Tab COLT = make_cols();
// compile-time offsets (runtime, lane-dependent ones come from a shared table)
__device__ __forceinline__ constexpr int rowoff(int r) { return ROWT.v[r]; }
__device__ __forceinline__ constexpr int coloff(int p) { return COLT.v[p]; }

// a -= l * (c0, c1), two elements in one packed instruction
__device__ __forceinline__ void fma2_sub(float &a0, float &a1, float l, float c0, float c1) {
    const float2 r = __ffma2_rn(make_float2(-l, -l), make_float2(c0, c1), make_float2(a0, a1));
    a0 = r.x;
    a1 = r.y;
}

// L^T x = y for the two components (i, i + 16) a lane holds: columns i and
// i + 16 of L are loaded into registers, then x_p is formed on its lane and
// broadcast within the half-warp, p = 31 .. 0 (c0off, c1off: the columns'
// offsets, less their first stored row).  y arrives divided by nothing;
// the result is the solution.
__device__ __forceinline__ float2 back_subst(const float *L, int i, int c0off, int c1off,
                                             float y0, float y1, float inv0, float inv1) {
    float c0[KP], c1[16];
    {
        const float4 *q0 = reinterpret_cast<const float4 *>(L + c0off);
#pragma unroll
        for (int t = 0; t < KP / 4; ++t) {
            const float4 v = q0[t];
            c0[4 * t] = v.x;
            c0[4 * t + 1] = v.y;
            c0[4 * t + 2] = v.z;
            c0[4 * t + 3] = v.w;
        }
        const float4 *q1 = reinterpret_cast<const float4 *>(L + c1off);
#pragma unroll
        for (int t = 4; t < KP / 4; ++t) {
            const float4 v = q1[t];
            c1[4 * t - 16] = v.x;
            c1[4 * t - 15] = v.y;
            c1[4 * t - 14] = v.z;
            c1[4 * t - 13] = v.w;
        }
    }
    float x0 = y0, x1 = y1;
#pragma unroll
    for (int p = KP - 1; p >= 16; --p) {
        const float xp = __shfl_sync(FULL, x1 * inv1, p - 16, 16);
        x0 = fmaf(-c0[p], xp, x0);
        if (i + 16 < p) x1 = fmaf(-c1[p - 16], xp, x1);
    }
#pragma unroll
    for (int p = 15; p >= 0; --p) {
        const float xp = __shfl_sync(FULL, x0 * inv0, p, 16);
        if (i < p) x0 = fmaf(-c0[p], xp, x0);
    }
    return make_float2(x0 * inv0, x1 * inv1);
}

}  // namespace pk
}  // namespace ocf
