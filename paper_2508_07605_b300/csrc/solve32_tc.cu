// One ALS row solve per half-warp at padded rank 32 (two systems per warp),
// Gram on the tensor cores, FP32 Cholesky on packed FP32x2 FMAs, with an
// optional extended-precision normal-equation residual and one step of
// iterative refinement.
//
// Per row i of a CSR matrix with F the fixed other factor (the ridge row solve
// of ALS; Sec. "Collaborative Filtering Model", Sec. "Online Performance
// Prediction"):
//     A_i = sum_{j in Omega_i} f_j f_j^T + lambda I,   b_i = sum_{j in Omega_i} R_ij f_j,
//     A_i = L L^T,  L y = b_i,  L^T u_i = y.
//
// Work split: each warp owns a contiguous range of row pairs (7/8 of its fair
// share when the caller passes a pair counter; the rest of the pairs are then
// claimed one at a time, which evens out the row-length variance between
// warps).  While it solves one pair it already has the next pair's row
// bounds, column indices and values (the first 64 observations of each row)
// in flight into registers, so the Gram phase of the next pair starts without
// waiting on DRAM.
//
// Gram phase (whole warp): both rows' observations 32 at a time, each lane
// staging one observation's factor row with 16-byte cp.async (double-buffered,
// zero fill past the row end); S^T S and S^T r on mma.sync, either split BF16
// (m16n8k16: x = hi + lo, hi^T hi + hi^T lo + lo^T hi, FP32 accumulation) or
// 3-pass TF32 (m16n8k8), lower-triangle 16x8 blocks only.  The fragments go
// to shared memory as the packed lower triangle of A (rows padded to 4
// floats), which stays there for the residual.
//
// Solve phase: half h of the warp solves system h of the pair; lane i holds
// rows i and i + 16 of the lower triangle (16 + 32 registers; row i never
// needs a column >= 16).  Right-looking Cholesky: step p broadcasts column p
// of L through shared memory (packed by columns, each column from row
// 4 floor(p/4) on, so the 16-byte loads stay aligned), and the trailing
// update of both rows runs two elements per instruction (fma.rn.f32x2; each
// element rounds exactly like fmaf).  The forward substitution L y = b rides
// along (y_p formed on the pivot step, broadcast by a shuffle); the back
// substitution runs from columns i and i + 16 of L held in registers.
//
// Residual (optional): r = b - A u in double-FP32 arithmetic (each product
// split exactly by an FMA, sums by error-free two-sums; the two rows of a lane
// are the two halves of each packed instruction), i.e. with ~2^-44 relative
// error instead of FP32's ~k 2^-24: B300's FP64 pipe runs at ~1/75 of the FP32
// rate, so this costs a fraction of one FP64 matrix-vector product.  With
// refinement, the correction A d = r is solved with the same FP32 factor,
// u += d, and the residual of the refined u is the one reported, as
// |A u - b| / (|A|_F |u| + |b|); it is formed as r - A D with D the step taken,
// in FP32 (its error, ~k kappa eps^2 |A||u|, is far below the residual itself).
// A residual-only mode takes u as input.
#include <cuda_bf16.h>
#include <stdint.h>

#include "common.cuh"
#include "kernels.h"
#include "mma_sync.cuh"
#include "packed_tri.cuh"

namespace ocf {
namespace {

// The kernel's arguments: the fields of SolveArgs<float> this solver reads,
// packed (the 32-bit fields share one 16-byte block).
struct Fold32Args {
    int64_t m, nnz;
    const int64_t *ptr;
    const int32_t *idx;
    const float *val;
    const void *Fsrc;              // F (FP32 rows of KP) or Fb (split BF16 rows), by the build
    float *out;
    int32_t *status;
    void *outb;
    const int32_t *row_map;
    const int64_t *m_dev;
    float *resid;
    const float *u_given;
    unsigned int *work;            // pair counter, zeroed before the launch (null: static ranges)
    int32_t n_other, ldo, kout;
    float lambda;
    bool wr, refine;
};

using namespace sm;
using namespace pk;

constexpr int WARPS = 8;

template <bool BF> struct alignas(16) Smem32 {
    static constexpr int ROWB = (BF ? 2 : 4) * (KP + 8);   // padded staged row (bytes)
    struct alignas(16) Stage {
        alignas(16) unsigned char stage[2][BF ? 2 : 1][32][ROWB];
        float sr[2][32];   // values (TF32 path); BF16 path: [0..15] hi halves, [16..31] lo halves
    };
    // The two halves of the warp touch the same offsets of their own row's
    // arrays at once, so the second row's copy of each array starts 16 banks
    // after the first row's (strides of 16 mod 32 words): conflict-free.
    static constexpr int LS = NCOLP + 16, XS = KP + 16;
    struct alignas(16) Solve {
        float L[2 * LS];      // the Cholesky factors by columns (second row's at LS)
        float x[2 * XS];
        float inv[2 * XS];    // 1 / L_pp
        float b1[KP];
        float pad[16];        // puts A1 16 banks from A0
        float A1[NROWP];      // A = Gram + lambda I of the second row, lower triangle by rows
    };
    union {
        Stage ld;
        Solve sv;
    };
    float A0[NROWP];          // A and b of the first row
    float b0[KP];
    __device__ float *A(int h) { return h ? sv.A1 : A0; }
    __device__ float *b(int h) { return h ? sv.b1 : b0; }
    __device__ float *Lf(int h) { return sv.L + h * LS; }
    __device__ float *xv(int h) { return sv.x + h * XS; }
    __device__ float *iv(int h) { return sv.inv + h * XS; }
};

// lower-triangle 16x8 blocks of the 32x32 Gram: (mb, nb) = (0,0) (0,1) (1,0..3)
__device__ constexpr int mb_of(int t) { return t < 2 ? 0 : 1; }
__device__ constexpr int nb_of(int t) { return t < 2 ? t : t - 2; }

// Error-free accumulation of S - g * x on two independent chains (the two
// halves of a packed register): (S, C) is a double-FP32 value per chain.
__device__ __forceinline__ void dot2_sub(float2 &S, float2 &C, float2 g, float2 x) {
    const float2 P = __fmul2_rn(g, x);
    const float2 nP = make_float2(-P.x, -P.y);
    const float2 E = __ffma2_rn(g, x, nP);                  // g x - P, exact
    const float2 T = __fadd2_rn(S, nP);                     // two-sum(S, -P)
    const float2 Z = __fadd2_rn(T, make_float2(-S.x, -S.y));
    const float2 TZ = __fadd2_rn(T, make_float2(-Z.x, -Z.y));
    const float2 e1 = __fadd2_rn(S, make_float2(-TZ.x, -TZ.y));
    const float2 e2 = __fadd2_rn(nP, make_float2(-Z.x, -Z.y));
    C = __fadd2_rn(C, __fadd2_rn(e1, e2));
    C = __fadd2_rn(C, make_float2(-E.x, -E.y));
    S = T;
}

// Sum over the 16 lanes of a half-warp.
__device__ __forceinline__ float half_sum(float v) {
#pragma unroll
    for (int off = 8; off > 0; off >>= 1) v += __shfl_xor_sync(FULL, v, off);
    return v;
}

// Rows i and i + 16 of b - A x (o0, o1: their offsets in the packed triangle) (A symmetric from its packed lower triangle,
// x from shared memory) in double-FP32, the two rows as the two chains of
// packed instructions; with norms, also |row|^2 of both rows.  Row i + 16's
// entries below column 16 and every column-part entry of row i above it sit
// at lane-independent offsets; only the crossings of the diagonal select.
template <bool NORMS>
__device__ __forceinline__ float2 ext_residual(const float *A, const float *x, int i, int o0,
                                               int o1, float2 bq, float2 &aa) {
    float2 S = bq, C = make_float2(0.f, 0.f), A2 = make_float2(0.f, 0.f);
    const float4 *x4 = reinterpret_cast<const float4 *>(x);
    const float4 *r4 = reinterpret_cast<const float4 *>(A + o1);
#pragma unroll
    for (int t = 0; t < KP / 4; ++t) {
        const float4 xv = x4[t];
        const float xs[4] = {xv.x, xv.y, xv.z, xv.w};
        float g1v[4];
        if (t < 4) {   // row i + 16, columns 0 .. 15: its own row segment
            const float4 g = r4[t];
            g1v[0] = g.x; g1v[1] = g.y; g1v[2] = g.z; g1v[3] = g.w;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int e = 4 * t + u;
            float g0, g1;
            if (e < 16) {
                g0 = A[e <= i ? o0 + e : rowoff(e) + i];
                g1 = g1v[u];
            } else {
                g0 = A[rowoff(e) + i];                              // column part of row i
                g1 = A[e <= i + 16 ? o1 + e : rowoff(e) + i + 16];
            }
            const float2 g = make_float2(g0, g1);
            dot2_sub(S, C, g, make_float2(xs[u], xs[u]));
            if (NORMS) A2 = __ffma2_rn(g, g, A2);
        }
    }
    if (NORMS) aa = A2;
    return make_float2(S.x + C.x, S.y + C.y);
}

// Rows i and i + 16 of r - A d in FP32 (A symmetric from its packed lower
// triangle, d from shared memory; the access pattern of ext_residual).
__device__ __forceinline__ float2 residual_update(const float *A, const float *d, int i, int o0,
                                                  int o1, float2 r) {
    float2 S = r;
    const float4 *d4 = reinterpret_cast<const float4 *>(d);
    const float4 *r4 = reinterpret_cast<const float4 *>(A + o1);
#pragma unroll
    for (int t = 0; t < KP / 4; ++t) {
        const float4 dv = d4[t];
        const float ds[4] = {dv.x, dv.y, dv.z, dv.w};
        float g1v[4];
        if (t < 4) {
            const float4 g = r4[t];
            g1v[0] = g.x; g1v[1] = g.y; g1v[2] = g.z; g1v[3] = g.w;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int e = 4 * t + u;
            float g0, g1;
            if (e < 16) {
                g0 = A[e <= i ? o0 + e : rowoff(e) + i];
                g1 = g1v[u];
            } else {
                g0 = A[rowoff(e) + i];
                g1 = A[e <= i + 16 ? o1 + e : rowoff(e) + i + 16];
            }
            S = __ffma2_rn(make_float2(-g0, -g1), make_float2(ds[u], ds[u]), S);
        }
    }
    return S;
}

template <bool BF>
__device__ __forceinline__ void gram_item(const Smem32<BF> &W, int buf, int cnt,
                                          float (&d)[6][4], float (&dr)[2][4], int lane) {
    const int gid = lane >> 2, tid4 = lane & 3;
    if constexpr (BF) {
        // 16 observations per MMA step; fragments of the hi (H) and lo (L)
        // tiles by ldmatrix.trans; S^T r from the value split the same way
        const int nks = (cnt + 15) / 16;
        const __nv_bfloat16 *sH = reinterpret_cast<const __nv_bfloat16 *>(&W.ld.stage[buf][0][0][0]);
        const __nv_bfloat16 *sL = reinterpret_cast<const __nv_bfloat16 *>(&W.ld.stage[buf][1][0][0]);
        constexpr int LDE = Smem32<BF>::ROWB / 2;
        const int mi = lane >> 3, rr = lane & 7;
        for (int ks = 0; ks < nks; ++ks) {
            const int k0 = ks * 16;
            uint32_t aH[2][4], aL[2][4];
#pragma unroll
            for (int mb = 0; mb < 2; ++mb) {
                const int off = (k0 + (mi >> 1) * 8 + rr) * LDE + mb * 16 + (mi & 1) * 8;
                ldsm_x4_trans(aH[mb], sH + off);
                ldsm_x4_trans(aL[mb], sL + off);
            }
            // the values' split halves, staged as BF16 (observation t: hi at
            // element t, lo at element 32 + t of the row): B fragments of S^T r,
            // column 0 only
            uint32_t rh0 = 0u, rh1 = 0u, rl0 = 0u, rl1 = 0u;
            if (gid == 0) {
                const uint32_t *hv = reinterpret_cast<const uint32_t *>(&W.ld.sr[buf][0]);
                rh0 = hv[(k0 >> 1) + tid4];
                rh1 = hv[(k0 >> 1) + tid4 + 4];
                rl0 = hv[16 + (k0 >> 1) + tid4];
                rl1 = hv[16 + (k0 >> 1) + tid4 + 4];
            }
#pragma unroll
            for (int ps = 0; ps < 3; ++ps) {   // pass-major: consecutive MMAs on different accumulators
#pragma unroll
                for (int tb = 0; tb < 6; ++tb) {
                    const int mb = mb_of(tb), nb = nb_of(tb);
                    const uint32_t *bsrc = (ps == 1) ? aL[nb >> 1] : aH[nb >> 1];
                    mma_bf16(d[tb], ps == 0 ? aL[mb] : aH[mb], bsrc[nb & 1], bsrc[2 + (nb & 1)]);
                }
#pragma unroll
                for (int mb = 0; mb < 2; ++mb)
                    mma_bf16(dr[mb], ps == 0 ? aL[mb] : aH[mb], ps == 1 ? rl0 : rh0,
                             ps == 1 ? rl1 : rh1);
            }
        }
    } else {
        // 8 observations per MMA step, each operand split into two TF32 halves
        const int nks = (cnt + 7) / 8;
        const float *stf = reinterpret_cast<const float *>(&W.ld.stage[buf][0][0][0]);
        constexpr int LDF = Smem32<BF>::ROWB / 4;
        for (int ks = 0; ks < nks; ++ks) {
            const int k0 = ks * 8;
            uint32_t ah[2][4], al[2][4];
#pragma unroll
            for (int mb = 0; mb < 2; ++mb) {
                split_tf32(stf[(k0 + tid4) * LDF + mb * 16 + gid], ah[mb][0], al[mb][0]);
                split_tf32(stf[(k0 + tid4) * LDF + mb * 16 + gid + 8], ah[mb][1], al[mb][1]);
                split_tf32(stf[(k0 + tid4 + 4) * LDF + mb * 16 + gid], ah[mb][2], al[mb][2]);
                split_tf32(stf[(k0 + tid4 + 4) * LDF + mb * 16 + gid + 8], ah[mb][3], al[mb][3]);
            }
            uint32_t rh0, rl0, rh1, rl1;
            split_tf32(gid == 0 ? W.ld.sr[buf][k0 + tid4] : 0.0f, rh0, rl0);
            split_tf32(gid == 0 ? W.ld.sr[buf][k0 + tid4 + 4] : 0.0f, rh1, rl1);
#pragma unroll
            for (int ps = 0; ps < 3; ++ps) {
#pragma unroll
                for (int tb = 0; tb < 6; ++tb) {
                    const int mb = mb_of(tb), nb = nb_of(tb);
                    const uint32_t *bsrc = (ps == 1) ? al[nb >> 1] : ah[nb >> 1];
                    mma_tf32(d[tb], ps == 0 ? al[mb] : ah[mb], bsrc[nb & 1], bsrc[2 + (nb & 1)]);
                }
#pragma unroll
                for (int mb = 0; mb < 2; ++mb)
                    mma_tf32(dr[mb], ps == 0 ? al[mb] : ah[mb], ps == 1 ? rl0 : rh0,
                             ps == 1 ? rl1 : rh1);
            }
        }
    }
}

// A row pair's CSR bounds and the first two 32-observation items of each
// row (this lane's column index and value in each), loaded into registers one
// pair ahead.
struct PairFetch {
    int64_t beg[2], s[2], row[2];   // row < 0: no system (odd row count)
    bool bad[2];
    int32_t j[4];                   // item order: row 0 item 0, item 1, row 1 item 0, item 1
    float v[4];
};

__device__ __forceinline__ void fetch_pair(const Fold32Args &a, int64_t k, int64_t M,
                                           int lane, PairFetch &f) {
#pragma unroll
    for (int si = 0; si < 2; ++si) {
        const int64_t is = 2 * k + si;
        int64_t beg = 0, end = 0, row = -1;
        bool bad = false;
        if (is < M) {
            row = a.row_map ? a.row_map[is] : is;
            bad = !row_bounds(a.ptr, row, a.nnz, beg, end);
        }
        f.beg[si] = beg;
        f.s[si] = end - beg;
        f.row[si] = row;
        f.bad[si] = bad;
#pragma unroll
        for (int it = 0; it < 2; ++it) {
            const int64_t t = 32 * it + lane;
            int32_t j = 0;
            float v = 0.f;
            if (t < end - beg) {
                j = __ldg(a.idx + beg + t);
                v = __ldg(a.val + beg + t);
            }
            f.j[2 * si + it] = j;
            f.v[2 * si + it] = v;
        }
    }
}

// ---------------------------------------------------------------------------
// Thin rows (s_i <= 16 observations, fewer than k = 32): the same ridge
// solution from the s_i x s_i dual system.  With S the s_i x k matrix of the
// observed factor rows,
//     (S^T S + lambda I) u = S^T r   <=>   u = S^T w,  (S S^T + lambda I) w = r
// (multiply the second by S^T: S^T S S^T w + lambda S^T w = S^T r).  The dual
// matrix has the primal's nonzero eigenvalues, so its condition number is at
// most the primal's, and its factorisation is 16 x 16 instead of 32 x 32.
// Both rows of a pair must be thin (a warp-uniform choice); padded
// observations are zero rows of S with r = 0, so they solve to w = 0.
//
// Layout: row h's 16 staged observations sit in stage buffer h; G_h = S S^T
// goes to shared memory (16 rows of stride 20 floats, the two systems in the
// area of the first row's packed triangle), is overwritten by L's columns
// (same stride) during the factorisation, and w is written where the
// buffer's values were staged, so that S^T w runs on the same MMA path as
// the primal right-hand side S^T r.  Where the observed rows are nearly
// dependent, u = S^T w cancels and carries the error of w relative to |S||w|;
// in FP32 mode one refinement step (residual of the dual system from the
// staged FP32 rows, correction with the same factor, u += S^T dw) restores
// the accuracy of the normal-equation solve.
constexpr int DUAL_MAX = 16, DUAL_LD = 20, DUAL_SYS = DUAL_MAX * DUAL_LD;

// G = S S^T of the 16 staged observations of buffer buf (whole warp): the A
// fragment of S (rows = observations) also supplies the B fragments of S^T.
template <bool BF>
__device__ __forceinline__ void dual_gram(const Smem32<BF> &W, int buf, float (&d)[2][4],
                                          int lane) {
    const int gid = lane >> 2, tid4 = lane & 3;
#pragma unroll
    for (int t = 0; t < 2; ++t)
#pragma unroll
        for (int e = 0; e < 4; ++e) d[t][e] = 0.f;
    if constexpr (BF) {
        const __nv_bfloat16 *sH = reinterpret_cast<const __nv_bfloat16 *>(&W.ld.stage[buf][0][0][0]);
        const __nv_bfloat16 *sL = reinterpret_cast<const __nv_bfloat16 *>(&W.ld.stage[buf][1][0][0]);
        constexpr int LDE = Smem32<BF>::ROWB / 2;
        const int row = (lane & 7) + ((lane >> 3) & 1) * 8, cofs = (lane >> 4) * 8;
#pragma unroll
        for (int k0 = 0; k0 < KP; k0 += 16) {
            uint32_t aH[4], aL[4];
            ldsm_x4(aH, sH + row * LDE + k0 + cofs);
            ldsm_x4(aL, sL + row * LDE + k0 + cofs);
#pragma unroll
            for (int ps = 0; ps < 3; ++ps) {   // lo.hi, hi.lo, hi.hi
                const uint32_t(&A)[4] = ps == 0 ? aL : aH;
                const uint32_t(&B)[4] = ps == 1 ? aL : aH;
                mma_bf16(d[0], A, B[0], B[2]);
                mma_bf16(d[1], A, B[1], B[3]);
            }
        }
    } else {
        const float *stf = reinterpret_cast<const float *>(&W.ld.stage[buf][0][0][0]);
        constexpr int LDF = Smem32<BF>::ROWB / 4;
#pragma unroll
        for (int k0 = 0; k0 < KP; k0 += 8) {
            uint32_t h[4], l[4];
            split_tf32(stf[gid * LDF + k0 + tid4], h[0], l[0]);
            split_tf32(stf[(gid + 8) * LDF + k0 + tid4], h[1], l[1]);
            split_tf32(stf[gid * LDF + k0 + tid4 + 4], h[2], l[2]);
            split_tf32(stf[(gid + 8) * LDF + k0 + tid4 + 4], h[3], l[3]);
#pragma unroll
            for (int ps = 0; ps < 3; ++ps) {
                const uint32_t(&A)[4] = ps == 0 ? l : h;
                const uint32_t(&B)[4] = ps == 1 ? l : h;
                mma_tf32(d[0], A, B[0], B[2]);
                mma_tf32(d[1], A, B[1], B[3]);
            }
        }
    }
}

// u = S^T w over the 16 staged observations of buffer buf (split BF16 mode),
// w staged where the values were (whole warp; dr as in the primal right-hand
// side).  The FP32 mode forms S^T w with FP32 FMAs instead (see the kernel).
__device__ __forceinline__ void dual_sTw_bf16(const Smem32<true> &W, int buf, float (&dr)[2][4],
                                              int lane) {
    const int gid = lane >> 2, tid4 = lane & 3;
#pragma unroll
    for (int t = 0; t < 2; ++t)
#pragma unroll
        for (int e = 0; e < 4; ++e) dr[t][e] = 0.f;
    const __nv_bfloat16 *sH = reinterpret_cast<const __nv_bfloat16 *>(&W.ld.stage[buf][0][0][0]);
    const __nv_bfloat16 *sL = reinterpret_cast<const __nv_bfloat16 *>(&W.ld.stage[buf][1][0][0]);
    constexpr int LDE = Smem32<true>::ROWB / 2;
    const int mi = lane >> 3, rr = lane & 7;
    uint32_t aH[2][4], aL[2][4];
#pragma unroll
    for (int mb = 0; mb < 2; ++mb) {
        const int off = ((mi >> 1) * 8 + rr) * LDE + mb * 16 + (mi & 1) * 8;
        ldsm_x4_trans(aH[mb], sH + off);
        ldsm_x4_trans(aL[mb], sL + off);
    }
    uint32_t wh0 = 0u, wh1 = 0u, wl0 = 0u, wl1 = 0u;
    if (gid == 0) {
        const uint32_t *hv = reinterpret_cast<const uint32_t *>(&W.ld.sr[buf][0]);
        wh0 = hv[tid4];
        wh1 = hv[tid4 + 4];
        wl0 = hv[16 + tid4];
        wl1 = hv[16 + tid4 + 4];
    }
#pragma unroll
    for (int ps = 0; ps < 3; ++ps)
#pragma unroll
        for (int mb = 0; mb < 2; ++mb)
            mma_bf16(dr[mb], ps == 0 ? aL[mb] : aH[mb], ps == 1 ? wl0 : wh0, ps == 1 ? wl1 : wh1);
}

template <bool BF, bool DUAL>
__global__ void __launch_bounds__(32 * WARPS, 2) k_solve32_tc(Fold32Args a) {
    using WS = Smem32<BF>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gid = lane >> 2, tid4 = lane & 3;
    const int h = lane >> 4, i = lane & 15;   // solve phase: system h of the pair, rows i, i + 16
    WS &W = reinterpret_cast<WS *>(smem_raw)[warp];
    // lane-dependent offsets into the packed triangles, from a shared table
    __shared__ int s_row[33], s_col[33];
    if (threadIdx.x == 0) {
#pragma unroll
        for (int t = 0; t < 33; ++t) {
            s_row[t] = rowoff(t);
            s_col[t] = t < 32 ? coloff(t) - colbase(t) : 0;
        }
    }
    __syncthreads();
    const int ro_i = s_row[i], ro_i16 = s_row[i + 16];
    const int co_i = s_col[i], co_i16 = s_col[i + 16];
    pdl_trigger();
    if (a.m_dev || a.row_map) pdl_wait();         // the list comes from the preceding kernel
    const int64_t M = a.m_dev ? *a.m_dev : a.m;
    const int64_t P = (M + 1) / 2;                // row pairs
    const int64_t G = (int64_t)gridDim.x * WARPS, gw = (int64_t)blockIdx.x * WARPS + warp;
    // Work.  Without a counter warp gw solves the pairs [P gw / G, P (gw + 1) / G).
    // With one (a.work, zero at the launch) it first solves a contiguous range of
    // Q = floor((P - P / 8) / G) pairs, then claims the remaining pairs one at a
    // time (pair Q G + c for the counter's value c), so that row-length variance
    // does not leave SMs idle at the end (the warps then finish within about one
    // pair's time of each other).  A pair's result does not depend on the warp.
    // (pair indices fit in 32 bits: the launcher refuses more than 2^31 - 1 pairs)
    const bool dyn = a.work != nullptr;
    const int32_t P32 = (int32_t)P, G32 = (int32_t)G, gw32 = (int32_t)gw;
    const int32_t Q = dyn ? (P32 - P32 / 8) / G32 : 0;
    auto claimed = [&](unsigned int c) -> int32_t { return Q * G32 + (int32_t)c; };
    int32_t k = dyn ? Q * gw32 : (int32_t)(P * gw / G), kend = dyn ? Q * (gw32 + 1) : (int32_t)(P * (gw + 1) / G);
    if (dyn && k == kend) {   // no contiguous share: claim the first pair
        unsigned int c = 0;
        if (lane == 0) c = atomicAdd(a.work, 1u);
        k = claimed(__shfl_sync(FULL, c, 0));
        kend = k < P32 ? k + 1 : k;
    }
    PairFetch cur;
    if (k < kend) fetch_pair(a, k, M, lane, cur);
    const bool dual_ok = DUAL && !a.resid && !a.refine && !a.u_given;
    const float lam0 = a.lambda;

    while (k < kend) {
      // The pair after this one: the next of the range, else (with a counter)
      // a claimed one, whose claim is issued here and read where the next pair
      // is fetched (warp-uniform points; every path through the body has one).
      const bool need = dyn && k + 1 == kend;
      unsigned int claim = 0;
      if (need && lane == 0) claim = atomicAdd(a.work, 1u);
      int32_t kn = -1, knend = 0;
      auto next = [&]() {
          if (kn >= 0) return;
          if (k + 1 < kend) {
              kn = k + 1;
              knend = kend;
          } else if (need) {
              kn = claimed(__shfl_sync(FULL, claim, 0));
              knend = kn < P32 ? kn + 1 : kn;
          } else {
              kn = knend = kend;
          }
      };
      // A pair with one thin and one thick row runs in two passes, each row
      // with an empty partner, so that every row takes the branch its own
      // length selects and its result does not depend on the row it is paired
      // with.  Only the last pass prefetches the next pair into cur.
      const bool thin0 = cur.s[0] <= DUAL_MAX, thin1 = cur.s[1] <= DUAL_MAX;
      const bool mixed = dual_ok && thin0 != thin1;
#pragma unroll 1
      for (int pass = 0; pass < (mixed ? 2 : 1); ++pass) {
        const bool last = pass == (mixed ? 1 : 0);
        PairFetch cp = cur;
        if (mixed) {   // pass 0: the thin row alone; pass 1: the thick row alone
            const int drop = ((pass == 0) == thin0) ? 1 : 0;
#pragma unroll
            for (int x = 0; x < 2; ++x)
                if (x == drop) {
                    cp.s[x] = 0;
                    cp.row[x] = -1;
                    cp.bad[x] = false;
                }
        }
        if (dual_ok && cp.s[0] <= DUAL_MAX && cp.s[1] <= DUAL_MAX) {
            // ---------------- thin pair: the 16 x 16 dual systems
            const PairFetch pf = cp;
            bool badf[2] = {false, false};
            float vv[2];
            pdl_wait();
#pragma unroll
            for (int si = 0; si < 2; ++si) {   // row si's observations -> stage buffer si
                int32_t j = cp.j[2 * si];
                float v = cp.v[2 * si];
                const bool in = lane < pf.s[si];
                if (in && (j < 0 || (int64_t)j >= a.n_other)) {
                    badf[si] = true;
                    j = 0;
                    v = 0.f;
                }
                vv[si] = in ? v : 0.f;
                if (lane < DUAL_MAX) {
                    const int nb = in ? 16 : 0;
                    if constexpr (BF) {
                        const unsigned char *src =
                            reinterpret_cast<const unsigned char *>(a.Fsrc) + (int64_t)j * KP * 4;
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            cp_async16(&W.ld.stage[si][0][lane][16 * e], src + 16 * e, nb);
                            cp_async16(&W.ld.stage[si][1][lane][16 * e], src + 2 * KP + 16 * e, nb);
                        }
                    } else {
                        const unsigned char *src = reinterpret_cast<const unsigned char *>(a.Fsrc) + (int64_t)j * KP * 4;
#pragma unroll
                        for (int e = 0; e < 8; ++e)
                            cp_async16(&W.ld.stage[si][0][lane][16 * e], src + 16 * e, nb);
                    }
                }
            }
            cp_async_commit();
            if (last) {   // in flight during the solve
                next();
                if (kn < knend) fetch_pair(a, kn, M, lane, cur);
            }
            const bool bad0 = pf.bad[0] || (__any_sync(FULL, badf[0]) != 0);
            const bool bad1 = pf.bad[1] || (__any_sync(FULL, badf[1]) != 0);
            cp_async_wait<0>();
            __syncwarp();
            float *Gb = W.A0;
#pragma unroll
            for (int si = 0; si < 2; ++si) {
                float d[2][4];
                dual_gram<BF>(W, si, d, lane);
                float *G = Gb + si * DUAL_SYS;
#pragma unroll
                for (int nb = 0; nb < 2; ++nb) {
                    const int c = nb * 8 + 2 * tid4;
                    *reinterpret_cast<float2 *>(G + gid * DUAL_LD + c) = make_float2(d[nb][0], d[nb][1]);
                    *reinterpret_cast<float2 *>(G + (gid + 8) * DUAL_LD + c) =
                        make_float2(d[nb][2], d[nb][3]);
                }
            }
            __syncwarp();
            // half h solves system h: lane i holds row i of G_h + lambda I
            const int64_t s = h ? pf.s[1] : pf.s[0];
            const bool bad = h ? bad1 : bad0;
            const float lam = a.wr ? lam0 * (float)(int)s : lam0;   // weighted: lambda s_i
            float *G = Gb + h * DUAL_SYS;
            G[i * (DUAL_LD + 1)] += lam;
            __syncwarp();
            float g[DUAL_MAX];
#pragma unroll
            for (int t = 0; t < DUAL_MAX / 4; ++t) {
                const float4 v = *reinterpret_cast<const float4 *>(G + i * DUAL_LD + 4 * t);
                g[4 * t] = v.x;
                g[4 * t + 1] = v.y;
                g[4 * t + 2] = v.z;
                g[4 * t + 3] = v.w;
            }
            const float r0 = __shfl_sync(FULL, vv[0], i), r1 = __shfl_sync(FULL, vv[1], i);
            float y = h ? r1 : r0;
            __syncwarp();   // every row is read before L's columns overwrite G
            // Cholesky with the forward substitution riding along; column p of L
            // at G + p * DUAL_LD
            float myinv = 0.f;
#pragma unroll
            for (int p = 0; p < DUAL_MAX; ++p) {
                const float piv = __shfl_sync(FULL, g[p], p, 16);
                const float inv = rsqrtf(piv);
                const float l = g[p] * inv;
                float *Lc = G + p * DUAL_LD;
                if (i >= p) Lc[i] = l;
                if (i == p) myinv = inv;
                const float yp = __shfl_sync(FULL, y, p, 16) * inv;
                if (i > p) y = fmaf(-l, yp, y);
                __syncwarp();
#pragma unroll
                for (int r4 = ((p + 1) / 4) * 4; r4 < DUAL_MAX; r4 += 4) {
                    const float4 c4 = *reinterpret_cast<const float4 *>(Lc + r4);
                    const float cv[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
                    for (int e = 0; e < 4; e += 2) {
                        const int r = r4 + e;
                        if (r > p) fma2_sub(g[r], g[r + 1], l, cv[e], cv[e + 1]);
                        else if (r + 1 > p) g[r + 1] = fmaf(-l, cv[e + 1], g[r + 1]);
                    }
                }
            }
            // L^T w = L^{-1} r from column i of L in registers
            float c[DUAL_MAX];
#pragma unroll
            for (int t = 0; t < DUAL_MAX / 4; ++t) {
                const float4 v = *reinterpret_cast<const float4 *>(G + i * DUAL_LD + 4 * t);
                c[4 * t] = v.x;
                c[4 * t + 1] = v.y;
                c[4 * t + 2] = v.z;
                c[4 * t + 3] = v.w;
            }
            float x = y * myinv;
#pragma unroll
            for (int p = DUAL_MAX - 1; p >= 0; --p) {
                const float wp = __shfl_sync(FULL, x * myinv, p, 16);
                if (i < p) x = fmaf(-c[p], wp, x);
            }
            float w = x * myinv;
            const unsigned fb = __ballot_sync(FULL, !isfinite(w));
            const bool fail = ((fb >> (16 * h)) & 0xffffu) != 0u;
            int32_t st = ST_OK;
            if (bad) st = ST_BAD;
            else if (s == 0) st = ST_EMPTY;
            else if (fail) st = ST_NOT_SPD;
            if (st != ST_OK) w = 0.f;
            if constexpr (BF) {
                // w replaces the staged values of buffer h; u = S^T w on the MMA
                // path of the primal right-hand side (split BF16)
                __nv_bfloat16 *sb = reinterpret_cast<__nv_bfloat16 *>(&W.ld.sr[h][0]);
                const __nv_bfloat16 wh = __float2bfloat16_rn(w);
                sb[i] = wh;
                sb[32 + i] = __float2bfloat16_rn(w - __bfloat162float(wh));
                const int32_t st_r[2] = {__shfl_sync(FULL, st, 0), __shfl_sync(FULL, st, 16)};
                __syncwarp();
                const int cs[4] = {gid, gid + 8, 16 + gid, 24 + gid};   // components a lane holds
#pragma unroll
                for (int si = 0; si < 2; ++si) {
                    float ur[2][4];
                    dual_sTw_bf16(W, si, ur, lane);
                    const int64_t rw = si ? pf.row[1] : pf.row[0];
                    if (rw >= 0) {
                        if (tid4 == 0) {
                            const float us[4] = {ur[0][0], ur[0][2], ur[1][0], ur[1][2]};
#pragma unroll
                            for (int q = 0; q < 4; ++q) {
                                if (cs[q] < a.kout) a.out[rw * a.ldo + cs[q]] = us[q];
                                if (a.outb) {   // split BF16 copy [hi | lo] of the output row
                                    __nv_bfloat16 *ob = reinterpret_cast<__nv_bfloat16 *>(a.outb) + rw * 2 * KP;
                                    const __nv_bfloat16 uh = __float2bfloat16_rn(us[q]);
                                    ob[cs[q]] = uh;
                                    ob[KP + cs[q]] = __float2bfloat16_rn(us[q] - __bfloat162float(uh));
                                }
                            }
                        }
                        if (a.status && lane == 0) a.status[rw] = st_r[si];
                    }
                }
            } else {
                // FP32 mode: u = S^T w in FP32 FMAs over the staged rows (lane i of
                // half h: components ca = i + 16 h and cb = i + 16 (1 - h), so the
                // two halves' loads fall in different banks), then one refinement
                // step: rho = r - S u - lambda w from the staged FP32 rows (not the
                // split products the Gram was formed from), dw = (G + lambda I)^-1 rho
                // with the same factor, u += S^T dw.  Where the observed rows are
                // nearly dependent u = S^T w cancels; this step recovers (and
                // passes) the accuracy of the normal-equation solve.
                constexpr int LDF = WS::ROWB / 4;
                const float *sf = reinterpret_cast<const float *>(&W.ld.stage[h][0][0][0]);
                const int ca = i + 16 * h, cb = i + 16 * (1 - h);
                float uA = 0.f, uB = 0.f;
#pragma unroll
                for (int t = 0; t < DUAL_MAX; ++t) {
                    const float wt = __shfl_sync(FULL, w, t, 16);
                    uA = fmaf(sf[t * LDF + ca], wt, uA);
                    uB = fmaf(sf[t * LDF + cb], wt, uB);
                }
                float *uv = h ? W.b0 : W.A0 + 2 * DUAL_SYS;   // u of system h, 32 floats
                uv[ca] = uA;
                uv[cb] = uB;
                __syncwarp();
                const float4 *srow = reinterpret_cast<const float4 *>(sf + i * LDF);
                const float4 *u4 = reinterpret_cast<const float4 *>(uv);
                float2 acc = make_float2(fmaf(-lam, w, h ? r1 : r0), 0.f);
#pragma unroll
                for (int c4 = 0; c4 < KP / 4; ++c4) {
                    const float4 x = srow[c4], uu = u4[c4];
                    acc = __ffma2_rn(make_float2(-x.x, -x.y), make_float2(uu.x, uu.y), acc);
                    acc = __ffma2_rn(make_float2(-x.z, -x.w), make_float2(uu.z, uu.w), acc);
                }
                float z = st == ST_OK ? acc.x + acc.y : 0.f;
                // L z' = rho (column p of L at G + p * DUAL_LD), then L^T dw = z'
#pragma unroll
                for (int p = 0; p < DUAL_MAX; ++p) {
                    const float zp = __shfl_sync(FULL, z * myinv, p, 16);
                    if (i > p) z = fmaf(-G[p * DUAL_LD + i], zp, z);
                }
                float xd = z * myinv;
#pragma unroll
                for (int p = DUAL_MAX - 1; p >= 0; --p) {
                    const float wp = __shfl_sync(FULL, xd * myinv, p, 16);
                    if (i < p) xd = fmaf(-c[p], wp, xd);
                }
                const float dw = st == ST_OK ? xd * myinv : 0.f;   // (1 / L_ii may be inf there)
#pragma unroll
                for (int t = 0; t < DUAL_MAX; ++t) {
                    const float dt = __shfl_sync(FULL, dw, t, 16);
                    uA = fmaf(sf[t * LDF + ca], dt, uA);
                    uB = fmaf(sf[t * LDF + cb], dt, uB);
                }
                const int64_t rw = h ? pf.row[1] : pf.row[0];
                if (rw >= 0) {
                    if (ca < a.kout) a.out[rw * a.ldo + ca] = uA;
                    if (cb < a.kout) a.out[rw * a.ldo + cb] = uB;
                    if (a.outb) {   // split BF16 copy [hi | lo] of the output row
                        __nv_bfloat16 *ob = reinterpret_cast<__nv_bfloat16 *>(a.outb) + rw * 2 * KP;
                        const __nv_bfloat16 ha = __float2bfloat16_rn(uA), hb = __float2bfloat16_rn(uB);
                        ob[ca] = ha;
                        ob[cb] = hb;
                        ob[KP + ca] = __float2bfloat16_rn(uA - __bfloat162float(ha));
                        ob[KP + cb] = __float2bfloat16_rn(uB - __bfloat162float(hb));
                    }
                    if (a.status && i == 0) a.status[rw] = st;
                }
            }
            __syncwarp();   // the shared area is restaged by the next pair
            continue;
        }
        // ---------------- Gram phase: both rows' items, one after the other
        const int n0 = (int)((cp.s[0] + 31) / 32), n1 = (int)((cp.s[1] + 31) / 32);
        const int nit = n0 + n1;
        bool badf0 = false, badf1 = false;
        // column index and value of this lane's observation in item w
        auto item_jv = [&](int w, int32_t &j, float &v, int &buf_si) {
            const int si = w < n0 ? 0 : 1;
            const int loc = w - (si ? n0 : 0);
            buf_si = si;
            const int64_t t = (int64_t)loc * 32 + lane;
            const int64_t ss = si ? cp.s[1] : cp.s[0];
            if (loc < 2) {
                const int slot = 2 * si + loc;
                j = slot == 0 ? cp.j[0] : slot == 1 ? cp.j[1] : slot == 2 ? cp.j[2] : cp.j[3];
                v = slot == 0 ? cp.v[0] : slot == 1 ? cp.v[1] : slot == 2 ? cp.v[2] : cp.v[3];
            } else {
                j = 0;
                v = 0.f;
                if (t < ss) {
                    const int64_t bg = si ? cp.beg[1] : cp.beg[0];
                    j = __ldg(a.idx + bg + t);
                    v = __ldg(a.val + bg + t);
                }
            }
            if (t < ss && (j < 0 || (int64_t)j >= a.n_other)) {
                if (si) badf1 = true; else badf0 = true;
                j = 0;
                v = 0.f;
            }
            return t < ss;
        };
        auto issue = [&](int w, int buf) {
            int32_t j;
            float v;
            int si;
            const bool ok = item_jv(w, j, v, si);
            if constexpr (BF) {
                const unsigned char *src =
                    reinterpret_cast<const unsigned char *>(a.Fsrc) + (int64_t)j * KP * 4;
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    cp_async16(&W.ld.stage[buf][0][lane][16 * e], src + 16 * e, ok ? 16 : 0);
                    cp_async16(&W.ld.stage[buf][1][lane][16 * e], src + 2 * KP + 16 * e, ok ? 16 : 0);
                }
            } else {
                const unsigned char *src = reinterpret_cast<const unsigned char *>(a.Fsrc) + (int64_t)j * KP * 4;
#pragma unroll
                for (int e = 0; e < 8; ++e)
                    cp_async16(&W.ld.stage[buf][0][lane][16 * e], src + 16 * e, ok ? 16 : 0);
            }
            if constexpr (BF) {
                const float vv = ok ? v : 0.f;
                const __nv_bfloat16 hi = __float2bfloat16_rn(vv);
                const __nv_bfloat16 lo = __float2bfloat16_rn(vv - __bfloat162float(hi));
                __nv_bfloat16 *sb = reinterpret_cast<__nv_bfloat16 *>(&W.ld.sr[buf][0]);
                sb[lane] = hi;
                sb[32 + lane] = lo;
            } else {
                W.ld.sr[buf][lane] = ok ? v : 0.f;
            }
        };
        pdl_wait();   // from here on the other factor is read
        if (nit > 0) {
            issue(0, 0);
            cp_async_commit();
        }
#pragma unroll
        for (int si = 0; si < 2; ++si) {
            // this row's items, the next item (possibly the other row's first)
            // staged while this one is on the tensor cores
            float d[6][4], dr[2][4];
#pragma unroll
            for (int t = 0; t < 6; ++t)
#pragma unroll
                for (int e = 0; e < 4; ++e) d[t][e] = 0.f;
#pragma unroll
            for (int t = 0; t < 2; ++t)
#pragma unroll
                for (int e = 0; e < 4; ++e) dr[t][e] = 0.f;
            const int w0 = si ? n0 : 0, w1 = si ? nit : n0;
            const int64_t ss = si ? cp.s[1] : cp.s[0];
            for (int w = w0; w < w1; ++w) {
                if (w + 1 < nit) issue(w + 1, (w + 1) & 1);
                cp_async_commit();
                cp_async_wait<1>();
                __syncwarp();
                const int cnt = (int)min((int64_t)32, ss - (int64_t)(w - w0) * 32);
                gram_item<BF>(W, w & 1, cnt, d, dr, lane);
                __syncwarp();   // this buffer is refilled two items later
            }
            if (si == 1) {
                cp_async_wait<0>();   // nothing in flight before the solve area overlays the stages
                __syncwarp();
            }
            // fragments -> the row's packed lower triangle of A, and b (the first
            // row's lie outside the staging area, the second's overlay it)
            float *Ap = si ? W.sv.A1 : W.A0;
            float *bp = si ? W.sv.b1 : W.b0;
#pragma unroll
            for (int tb = 0; tb < 6; ++tb) {
                const int mb = mb_of(tb), nb = nb_of(tb);
                const int r0 = mb * 16 + gid, c = nb * 8 + 2 * tid4;
                const bool diag = (mb == 0) || (nb >= 2);   // diagonal 16x16 block
                const int o0 = s_row[r0], o8 = s_row[r0 + 8];
                if (!diag || c <= r0) Ap[o0 + c] = d[tb][0];
                if (!diag || c + 1 <= r0) Ap[o0 + c + 1] = d[tb][1];
                if (!diag || c <= r0 + 8) Ap[o8 + c] = d[tb][2];
                if (!diag || c + 1 <= r0 + 8) Ap[o8 + c + 1] = d[tb][3];
            }
            if (tid4 == 0) {
#pragma unroll
                for (int mb = 0; mb < 2; ++mb) {
                    bp[mb * 16 + gid] = dr[mb][0];
                    bp[mb * 16 + gid + 8] = dr[mb][2];
                }
            }
        }
        const PairFetch pf = cp;
        const bool bad0 = pf.bad[0] || (__any_sync(FULL, badf0) != 0);
        const bool bad1 = pf.bad[1] || (__any_sync(FULL, badf1) != 0);
        __syncwarp();
        // ---------------- solve phase: half h solves system h
        float *SA = W.A(h), *SL = W.Lf(h), *Sx = W.xv(h), *Sinv = W.iv(h);
        const int64_t s = h ? pf.s[1] : pf.s[0];
        const int64_t row = h ? pf.row[1] : pf.row[0];
        const bool bad = h ? bad1 : bad0;
        const float lam = a.wr ? lam0 * (float)(int)s : lam0;   // weighted: lambda s_i
        SA[ro_i + i] += lam;
        SA[ro_i16 + i + 16] += lam;
        __syncwarp();
        const float2 bq = make_float2(W.b(h)[i], W.b(h)[i + 16]);
        float x0, x1, inv0 = 0.f, inv1 = 0.f;
        if (!a.u_given) {
            float a0[16], a1[KP];
            {
                const float4 *q0 = reinterpret_cast<const float4 *>(SA + ro_i);
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const float4 v = q0[t];
                    a0[4 * t] = v.x;
                    a0[4 * t + 1] = v.y;
                    a0[4 * t + 2] = v.z;
                    a0[4 * t + 3] = v.w;
                }
                const float4 *q1 = reinterpret_cast<const float4 *>(SA + ro_i16);
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    const float4 v = q1[t];
                    a1[4 * t] = v.x;
                    a1[4 * t + 1] = v.y;
                    a1[4 * t + 2] = v.z;
                    a1[4 * t + 3] = v.w;
                }
            }
            // ---- Cholesky A = L L^T with the forward substitution L y = b
            float y0 = bq.x, y1 = bq.y;
#pragma unroll
            for (int p = 0; p < KP; ++p) {
                const float piv = p < 16 ? __shfl_sync(FULL, a0[p & 15], p, 16)
                                         : __shfl_sync(FULL, a1[p], p - 16, 16);
                const float inv = rsqrtf(piv);
                float *Lc = SL + coloff(p) - colbase(p);   // Lc[r] = L[r][p]
                float l0 = 0.f;
                if (p < 16) {
                    l0 = a0[p & 15] * inv;
                    a0[p & 15] = l0;
                    if (i >= colbase(p)) Lc[i] = l0;
                }
                const float l1 = a1[p] * inv;
                a1[p] = l1;
                if (colbase(p) <= 16 || i + 16 >= colbase(p)) Lc[i + 16] = l1;
                if (i == 0) Sinv[p] = inv;
                const float yp = (p < 16 ? __shfl_sync(FULL, y0, p, 16)
                                         : __shfl_sync(FULL, y1, p - 16, 16)) * inv;
                if (p < 16) {
                    if (i > p) y0 = fmaf(-l0, yp, y0);
                    y1 = fmaf(-l1, yp, y1);
                } else {
                    if (i + 16 > p) y1 = fmaf(-l1, yp, y1);
                }
                __syncwarp();
                // trailing update: row i over columns (p, 16), row i + 16 over (p, 32)
#pragma unroll
                for (int r4 = ((p + 1) / 4) * 4; r4 < KP; r4 += 4) {
                    const float4 c4 = *reinterpret_cast<const float4 *>(Lc + r4);
                    const float cv[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
                    for (int e = 0; e < 4; e += 2) {
                        const int r = r4 + e;
                        if (r > p) {
                            fma2_sub(a1[r], a1[r + 1], l1, cv[e], cv[e + 1]);
                            if (p < 16 && r < 16) fma2_sub(a0[r & 15], a0[(r + 1) & 15], l0, cv[e], cv[e + 1]);
                        } else if (r + 1 > p) {
                            a1[r + 1] = fmaf(-l1, cv[e + 1], a1[r + 1]);
                            if (p < 16 && r + 1 < 16) a0[(r + 1) & 15] = fmaf(-l0, cv[e + 1], a0[(r + 1) & 15]);
                        }
                    }
                }
            }
            // the factor is done: fetch the next pair's bounds, indices and values
            // while the substitutions and the residual run
            if (last) {
                next();
                if (kn < knend) fetch_pair(a, kn, M, lane, cur);
            }
            inv0 = Sinv[i];
            inv1 = Sinv[i + 16];
            // ---- back substitution L^T x = y
            const float2 xx = back_subst(SL, i, co_i, co_i16, y0 * inv0, y1 * inv1, inv0, inv1);
            x0 = xx.x;
            x1 = xx.y;
        } else {
            if (last) {
                next();
                if (kn < knend) fetch_pair(a, kn, M, lane, cur);
            }
            x0 = (i < a.kout && row >= 0) ? a.u_given[row * a.ldo + i] : 0.f;
            x1 = (i + 16 < a.kout && row >= 0) ? a.u_given[row * a.ldo + i + 16] : 0.f;
        }
        const unsigned fb = __ballot_sync(FULL, !isfinite(x0) || !isfinite(x1));
        const bool fail = ((fb >> (16 * h)) & 0xffffu) != 0u;
        int32_t st = ST_OK;
        if (bad) st = ST_BAD;
        else if (s == 0) st = ST_EMPTY;
        else if (fail && !a.u_given) st = ST_NOT_SPD;
        if (st != ST_OK && !a.u_given) x0 = x1 = 0.f;

        // ---- residual |A u - b| / (|A|_F |u| + |b|), optional refinement
        float rel = -1.f;
        const bool want = (a.resid || a.refine) && (st == ST_OK || a.u_given);
        if (__any_sync(FULL, want)) {   // both halves run the same instructions
            Sx[i] = x0;
            Sx[i + 16] = x1;
            __syncwarp();
            float2 aa;
            float2 r = ext_residual<true>(SA, Sx, i, ro_i, ro_i16, bq, aa);
            if (a.refine && !a.u_given) {
                // A d = r with the FP32 factor: L z = r (L[q][p] = column p, row q), L^T d = z
                // (both halves run it: the shuffles need the whole warp)
                float z0 = r.x, z1 = r.y;
#pragma unroll
                for (int p = 0; p < KP; ++p) {
                    const float *Lc = SL + coloff(p) - colbase(p);
                    if (p < 16) {
                        const float zp = __shfl_sync(FULL, z0 * inv0, p, 16);
                        if (i > p) z0 = fmaf(-Lc[i], zp, z0);
                        z1 = fmaf(-Lc[i + 16], zp, z1);
                    } else {
                        const float zp = __shfl_sync(FULL, z1 * inv1, p - 16, 16);
                        if (i + 16 > p) z1 = fmaf(-Lc[i + 16], zp, z1);
                    }
                }
                const float2 dd = back_subst(SL, i, co_i, co_i16, z0 * inv0, z1 * inv1, inv0, inv1);
                // The refined residual b - A x' = r - A D with D = x' - x, the step
                // actually taken (exact in FP32 where the correction is small next
                // to x).  |D| is ~kappa eps |x|, so A D in FP32 errs by ~k kappa eps^2
                // |A||x|, far below the residual's own size (~eps |A||x| once x' is
                // rounded to FP32): the extended-precision part is r, not A D.
                float d0 = 0.f, d1 = 0.f;
                if (want) {
                    const float n0 = x0 + dd.x, n1 = x1 + dd.y;
                    d0 = n0 - x0;
                    d1 = n1 - x1;
                    x0 = n0;
                    x1 = n1;
                }
                __syncwarp();   // every lane has read x before it is rewritten
                Sx[i] = d0;
                Sx[i + 16] = d1;
                __syncwarp();
                r = residual_update(SA, Sx, i, ro_i, ro_i16, r);
            }
            // |A|_F over the k x k system: padded rows (q >= k) hold only lambda
            const float rr = half_sum(r.x * r.x + r.y * r.y);
            const float na = half_sum((i < a.kout ? aa.x : 0.f) + (i + 16 < a.kout ? aa.y : 0.f));
            const float nu = half_sum(x0 * x0 + x1 * x1);
            const float nb = half_sum(bq.x * bq.x + bq.y * bq.y);
            const float den = sqrtf(na) * sqrtf(nu) + sqrtf(nb);
            if (want) rel = den > 0.f ? sqrtf(rr) / den : 0.f;
        }
        if (row >= 0) {
            if (!a.u_given) {
                if (i < a.kout) a.out[row * a.ldo + i] = x0;
                if (i + 16 < a.kout) a.out[row * a.ldo + i + 16] = x1;
                if (a.outb) {   // split BF16 copy [hi | lo] of the output row
                    __nv_bfloat16 *ob = reinterpret_cast<__nv_bfloat16 *>(a.outb) + row * 2 * KP;
                    const __nv_bfloat16 h0 = __float2bfloat16_rn(x0), h1 = __float2bfloat16_rn(x1);
                    ob[i] = h0;
                    ob[i + 16] = h1;
                    ob[KP + i] = __float2bfloat16_rn(x0 - __bfloat162float(h0));
                    ob[KP + i + 16] = __float2bfloat16_rn(x1 - __bfloat162float(h1));
                }
                if (a.status && i == 0) a.status[row] = st;
            }
            if (a.resid && i == 0) a.resid[row] = rel;
        }
        __syncwarp();   // the shared area is restaged by the next pair
      }
      next();
      k = kn;
      kend = knend;
    }
}

template <bool BF> size_t smem_bytes() { return sizeof(Smem32<BF>) * WARPS; }

template <bool BF, bool DUAL> cudaError_t launch32(const SolveArgs<float> &a, cudaStream_t st) {
    // a persistent grid: at most two CTAs per SM
    const int64_t pairs = (a.m + 1) / 2;
    int64_t blocks = (pairs + WARPS - 1) / WARPS;
    if (blocks > NUM_SMS_HINT * 2) blocks = NUM_SMS_HINT * 2;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)blocks);
    cfg.blockDim = dim3(32 * WARPS);
    cfg.dynamicSmemBytes = smem_bytes<BF>();
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    Fold32Args f;
    f.m = a.m; f.nnz = a.nnz; f.ptr = a.ptr; f.idx = a.idx; f.val = a.val;
    f.Fsrc = BF ? a.Fb : (const void *)a.F;
    f.out = a.out; f.status = a.status; f.outb = a.outb; f.row_map = a.row_map; f.m_dev = a.m_dev;
    f.resid = a.resid; f.u_given = a.u_given;
    // the counter only where the launch does not overlap its producer (a device
    // row list or count comes from the preceding kernel)
    f.work = (a.m_dev || a.row_map) ? nullptr : a.work;
    f.n_other = (int32_t)a.n_other; f.ldo = (int32_t)a.ldo; f.kout = a.kout;
    // lambda in FP32 once, on the host (a conversion from double on the device
    // runs on the FP64 pipe, a small fraction of the FP32 rate on this part)
    f.lambda = (float)a.lambda;
    f.wr = a.wr; f.refine = a.refine;
    return cudaLaunchKernelEx(&cfg, k_solve32_tc<BF, DUAL>, f);
}

template <bool BF> cudaError_t attr32() {
    cudaError_t e = cudaFuncSetAttribute(k_solve32_tc<BF, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem_bytes<BF>());
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_solve32_tc<BF, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem_bytes<BF>());
}

}  // namespace

cudaError_t prepare_solve32_tc() {
    cudaError_t e = attr32<true>();
    if (e != cudaSuccess) return e;
    return attr32<false>();
}

cudaError_t launch_solve32_tc(const SolveArgs<float> &a, bool bf16, cudaStream_t st) {
    if (a.m <= 0) return cudaSuccess;
    if (bf16 && !a.Fb) return cudaErrorInvalidValue;
    if (a.gram) return cudaErrorInvalidValue;   // the streaming refit's sums are not supported here
    // the packed arguments hold the setting count and the row stride in 32 bits
    if (a.n_other > INT32_MAX || a.ldo > INT32_MAX) return cudaErrorInvalidValue;
    // one build serves the plain fold-in too (a build without the residual
    // paths spilled more registers and measured slower).  The build with the
    // thin-row dual branch runs where rows average fewer than 24 observations
    // (and no residual is wanted); with longer rows few pairs are thin, and
    // the build without it keeps the normal-equation path's registers.
    const bool dual = !a.resid && !a.refine && !a.u_given && a.nnz < 24 * a.m;
    if ((a.m + 1) / 2 > INT32_MAX) return cudaErrorInvalidValue;   // pair indices are 32-bit
    if (a.work && !a.m_dev && !a.row_map) {
        cudaError_t e = cudaMemsetAsync(a.work, 0, sizeof(unsigned int), st);
        if (e != cudaSuccess) return e;
    }
    if (bf16) return dual ? launch32<true, true>(a, st) : launch32<true, false>(a, st);
    return dual ? launch32<false, true>(a, st) : launch32<false, false>(a, st);
}

}  // namespace ocf
