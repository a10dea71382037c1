// One ALS row solve per warp at padded rank 32, Gram on the tensor cores,
// FP32 Cholesky on packed FP32x2 FMAs, with an optional extended-precision
// normal-equation residual and one step of iterative refinement.
//
// Per row i of a CSR matrix with F the fixed other factor (the ridge row solve
// of ALS; Sec. "Collaborative Filtering Model", Sec. "Online Performance
// Prediction"):
//     A_i = sum_{j in Omega_i} f_j f_j^T + lambda I,   b_i = sum_{j in Omega_i} R_ij f_j,
//     A_i = L L^T,  L y = b_i,  L^T u_i = y.
//
// Gram phase: the row's observations 32 at a time, each lane staging one
// observation's factor row with 16-byte cp.async (double-buffered, zero fill
// past the row end); S^T S and S^T r on mma.sync, either split BF16
// (m16n8k16: x = hi + lo, hi^T hi + hi^T lo + lo^T hi, FP32 accumulation) or
// 3-pass TF32 (m16n8k8), lower-triangle 16x8 blocks only.  The fragments go to
// shared memory as the full symmetric A (the off-diagonal block is written
// twice), which stays there for the residual.
//
// Solve phase, lane q owning row q:
//  * right-looking Cholesky: step p broadcasts column p of L through shared
//    memory (stored column-major, so all of L stays there), and the trailing
//    update a[r] -= l_q * L[r][p], r > p, runs two elements per instruction
//    (fma.rn.f32x2; each element rounds exactly like fmaf);
//  * the forward substitution L y = b rides along: y_p is formed on the pivot
//    step and broadcast with column p;
//  * back substitution from column q of L held in registers.
// The operations and their order per element are those of the lane-per-row
// factorisation in row_solve_tc.cu.
//
// Residual (optional): r = b - A u in double-FP32 arithmetic (each product
// split exactly by an FMA, sums by error-free two-sums, two chains per
// packed instruction), i.e. with ~2^-44 relative error instead of FP32's
// ~k 2^-24: B300's FP64 pipe runs at ~1/75 of the FP32 rate, so this costs a
// fraction of one FP64 matrix-vector product.  With refinement, the
// correction A d = r is solved with the same FP32 factor, u += d, and the
// residual of the refined u is the one reported, as
// |A u - b| / (|A|_F |u| + |b|).  A residual-only mode takes u as input.
#include <cuda_bf16.h>
#include <stdint.h>

#include "common.cuh"
#include "kernels.h"
#include "mma_sync.cuh"

namespace ocf {
namespace {

using namespace sm;

constexpr int KP = 32, WARPS = 8, NST = 2, LDA = 36;

template <bool BF> struct alignas(16) Smem32 {
    static constexpr int ROWB = (BF ? 2 : 4) * (KP + 8);   // padded staged row (bytes)
    struct alignas(16) Stage {
        alignas(16) unsigned char stage[NST][BF ? 2 : 1][32][ROWB];
        float sr[NST][32];
    };
    struct alignas(16) Solve {
        float G[KP][LDA];    // A = Gram + lambda I, both triangles
        float Lc[KP][LDA];   // Lc[p][r] = L[r][p] for r >= p; Lc[p][32] = y_p
        float b[KP];
        float x[KP];
    };
    union {
        Stage ld;
        Solve sv;
    };
};

// lower-triangle 16x8 blocks of the 32x32 Gram: (mb, nb) = (0,0) (0,1) (1,0..3)
__device__ constexpr int mb_of(int t) { return t < 2 ? 0 : 1; }
__device__ constexpr int nb_of(int t) { return t < 2 ? t : t - 2; }

// a -= l * (c0, c1), two elements in one packed instruction
__device__ __forceinline__ void fma2_sub(float &a0, float &a1, float l, float c0, float c1) {
    const float2 r = __ffma2_rn(make_float2(-l, -l), make_float2(c0, c1), make_float2(a0, a1));
    a0 = r.x;
    a1 = r.y;
}

// Error-free accumulation of s - g * x on two independent chains (the two
// halves of a packed register): (S, C) is a double-FP32 value per chain.
__device__ __forceinline__ void dot2_sub(float2 &S, float2 &C, float2 g, float2 x) {
    const float2 P = __fmul2_rn(g, x);
    const float2 E = __ffma2_rn(g, x, make_float2(-P.x, -P.y));   // g x - P, exact
    const float2 nP = make_float2(-P.x, -P.y);
    const float2 T = __fadd2_rn(S, nP);                              // two-sum(S, -P)
    const float2 Z = __fadd2_rn(T, make_float2(-S.x, -S.y));
    const float2 TZ = __fadd2_rn(T, make_float2(-Z.x, -Z.y));
    const float2 e1 = __fadd2_rn(S, make_float2(-TZ.x, -TZ.y));
    const float2 e2 = __fadd2_rn(nP, make_float2(-Z.x, -Z.y));
    C = __fadd2_rn(C, __fadd2_rn(e1, e2));
    C = __fadd2_rn(C, make_float2(-E.x, -E.y));
    S = T;
}

// r_q = b_q - sum_e A[q][e] x_e in double-FP32; also |A row q|^2 (FP32).
template <typename WS>
__device__ __forceinline__ float ext_residual(const WS &W, int q, float bq, float &aa) {
    const float4 *g4 = reinterpret_cast<const float4 *>(W.sv.G[q]);
    const float4 *x4 = reinterpret_cast<const float4 *>(W.sv.x);
    float2 S0 = make_float2(bq, 0.f), C0 = make_float2(0.f, 0.f);
    float2 S1 = make_float2(0.f, 0.f), C1 = make_float2(0.f, 0.f);
    float2 A2 = make_float2(0.f, 0.f);
#pragma unroll
    for (int e4 = 0; e4 < KP / 4; ++e4) {
        const float4 g = g4[e4], x = x4[e4];
        dot2_sub(S0, C0, make_float2(g.x, g.y), make_float2(x.x, x.y));
        dot2_sub(S1, C1, make_float2(g.z, g.w), make_float2(x.z, x.w));
        A2 = __ffma2_rn(make_float2(g.x, g.y), make_float2(g.x, g.y), A2);
        A2 = __ffma2_rn(make_float2(g.z, g.w), make_float2(g.z, g.w), A2);
    }
    aa = A2.x + A2.y;
    // combine the four chains: hi parts by two-sums, lo parts plainly
    float hi = S0.x, lo = C0.x + C0.y + C1.x + C1.y;
    const float parts[3] = {S0.y, S1.x, S1.y};
#pragma unroll
    for (int t = 0; t < 3; ++t) {
        const float T = hi + parts[t];
        const float Z = T - hi;
        lo += (hi - (T - Z)) + (parts[t] - Z);
        hi = T;
    }
    return hi + lo;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(FULL, v, off);
    return v;
}

// L^T x = y for lane q's component: column q of L (L[r][q], r >= q) is loaded
// into registers, then x_p is formed on lane p and broadcast, p = 31 .. 0.
template <typename WS>
__device__ __forceinline__ float back_subst(const WS &W, int q, float yq, float myinv) {
    float c[KP];
    const float4 *c4 = reinterpret_cast<const float4 *>(W.sv.Lc[q]);
#pragma unroll
    for (int e4 = 0; e4 < KP / 4; ++e4) {
        const float4 v = c4[e4];
        c[4 * e4] = v.x;
        c[4 * e4 + 1] = v.y;
        c[4 * e4 + 2] = v.z;
        c[4 * e4 + 3] = v.w;
    }
    float x = yq;
#pragma unroll
    for (int p = KP - 1; p >= 0; --p) {
        const float xp = __shfl_sync(FULL, x * myinv, p);
        if (q < p) x = fmaf(-c[p], xp, x);
    }
    return x * myinv;
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
            float r0 = 0.f, r1 = 0.f, r2 = 0.f, r3 = 0.f;
            if (gid == 0) {
                r0 = W.ld.sr[buf][k0 + 2 * tid4];
                r1 = W.ld.sr[buf][k0 + 2 * tid4 + 1];
                r2 = W.ld.sr[buf][k0 + 2 * tid4 + 8];
                r3 = W.ld.sr[buf][k0 + 2 * tid4 + 9];
            }
            const float h0 = __bfloat162float(__float2bfloat16_rn(r0));
            const float h1 = __bfloat162float(__float2bfloat16_rn(r1));
            const float h2 = __bfloat162float(__float2bfloat16_rn(r2));
            const float h3 = __bfloat162float(__float2bfloat16_rn(r3));
            const uint32_t rh0 = pack_bf16(h0, h1), rh1 = pack_bf16(h2, h3);
            const uint32_t rl0 = pack_bf16(r0 - h0, r1 - h1), rl1 = pack_bf16(r2 - h2, r3 - h3);
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

template <bool BF>
__global__ void __launch_bounds__(32 * WARPS, 2) k_solve32_tc(SolveArgs<float> a) {
    using WS = Smem32<BF>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gid = lane >> 2, tid4 = lane & 3;
    const int q = lane;
    WS &W = reinterpret_cast<WS *>(smem_raw)[warp];
    pdl_trigger();
    if (a.m_dev || a.row_map) pdl_wait();         // the list comes from the preceding kernel
    const int64_t M = a.m_dev ? *a.m_dev : a.m;
    const int64_t stride = (int64_t)gridDim.x * WARPS;

    for (int64_t is = (int64_t)blockIdx.x * WARPS + warp; is < M; is += stride) {
        const int64_t row = a.row_map ? a.row_map[is] : is;
        int64_t beg = 0, end = 0;
        bool bad = !row_bounds(a.ptr, row, a.nnz, beg, end);
        const int64_t s = end - beg;
        const int nitems = (int)((s + 31) / 32);
        bool badf = false;

        // ---------------- Gram phase --------------------------------------
        auto load_idx = [&](int w) -> int32_t {
            const int64_t t = (int64_t)w * 32 + lane;
            int32_t j = 0;
            if (t < s) {
                j = __ldg(a.idx + beg + t);
                if (j < 0 || (int64_t)j >= a.n_other) {
                    badf = true;
                    j = 0;
                }
            }
            return j;
        };
        auto issue = [&](int w, int32_t j, int buf) {
            const int64_t t = (int64_t)w * 32 + lane;
            const bool v = t < s;
            if constexpr (BF) {
                const unsigned char *src =
                    reinterpret_cast<const unsigned char *>(a.Fb) + (int64_t)j * KP * 4;
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    cp_async16(&W.ld.stage[buf][0][lane][16 * e], src + 16 * e, v ? 16 : 0);
                    cp_async16(&W.ld.stage[buf][1][lane][16 * e], src + 2 * KP + 16 * e, v ? 16 : 0);
                }
            } else {
                const unsigned char *src = reinterpret_cast<const unsigned char *>(a.F + (int64_t)j * KP);
#pragma unroll
                for (int e = 0; e < 8; ++e)
                    cp_async16(&W.ld.stage[buf][0][lane][16 * e], src + 16 * e, v ? 16 : 0);
            }
            cp_async4(&W.ld.sr[buf][lane], v ? (const void *)(a.val + beg + t) : (const void *)a.val,
                      v ? 4 : 0);
        };
        float d[6][4], dr[2][4];
#pragma unroll
        for (int t = 0; t < 6; ++t)
#pragma unroll
            for (int e = 0; e < 4; ++e) d[t][e] = 0.f;
#pragma unroll
        for (int t = 0; t < 2; ++t)
#pragma unroll
            for (int e = 0; e < 4; ++e) dr[t][e] = 0.f;
        pdl_wait();   // from here on the other factor is read
        if (nitems > 0) {
            issue(0, load_idx(0), 0);
            cp_async_commit();
            int32_t jn = nitems > 1 ? load_idx(1) : 0;
            for (int w = 0; w < nitems; ++w) {
                if (w + 1 < nitems) issue(w + 1, jn, (w + 1) & 1);
                cp_async_commit();
                jn = (w + 2 < nitems) ? load_idx(w + 2) : 0;
                cp_async_wait<1>();
                __syncwarp();
                const int cnt = (int)min((int64_t)32, s - (int64_t)w * 32);
                gram_item<BF>(W, w & 1, cnt, d, dr, lane);
                __syncwarp();   // this buffer is refilled two items later
            }
        }
        cp_async_wait<0>();   // nothing in flight before the solve area overlays the stages
        __syncwarp();
        // fragments -> A (both triangles) and b
#pragma unroll
        for (int tb = 0; tb < 6; ++tb) {
            const int mb = mb_of(tb), nb = nb_of(tb);
            const int r0 = mb * 16 + gid, c = nb * 8 + 2 * tid4;
            W.sv.G[r0][c] = d[tb][0];
            W.sv.G[r0][c + 1] = d[tb][1];
            W.sv.G[r0 + 8][c] = d[tb][2];
            W.sv.G[r0 + 8][c + 1] = d[tb][3];
            if (mb == 1 && nb < 2) {
                W.sv.G[c][r0] = d[tb][0];
                W.sv.G[c + 1][r0] = d[tb][1];
                W.sv.G[c][r0 + 8] = d[tb][2];
                W.sv.G[c + 1][r0 + 8] = d[tb][3];
            }
        }
        if (tid4 == 0) {
#pragma unroll
            for (int mb = 0; mb < 2; ++mb) {
                W.sv.b[mb * 16 + gid] = dr[mb][0];
                W.sv.b[mb * 16 + gid + 8] = dr[mb][2];
            }
        }
        bad = bad || (__any_sync(FULL, badf) != 0);
        __syncwarp();
        const float lam = float(a.lambda) * (a.wr ? float(s) : 1.f);   // weighted: lambda s_i
        W.sv.G[q][q] += lam;
        __syncwarp();
        float ar[KP];
        {
            const float4 *g4 = reinterpret_cast<const float4 *>(W.sv.G[q]);
#pragma unroll
            for (int e4 = 0; e4 < KP / 4; ++e4) {
                const float4 v = g4[e4];
                ar[4 * e4] = v.x;
                ar[4 * e4 + 1] = v.y;
                ar[4 * e4 + 2] = v.z;
                ar[4 * e4 + 3] = v.w;
            }
        }
        const float bq = W.sv.b[q];

        float xq, myinv = 0.f;
        if (!a.u_given) {
            // ---- Cholesky A = L L^T with the forward substitution L y = b
            float y = bq;
#pragma unroll
            for (int p = 0; p < KP; ++p) {
                const float piv = __shfl_sync(FULL, ar[p], p);
                const float inv = rsqrtf(piv);
                if (q == p) myinv = inv;
                const float l = ar[p] * inv;
                ar[p] = l;
                float *cp = W.sv.Lc[p];
                cp[q] = l;
                if (q == p) cp[32] = y * inv;
                __syncwarp();
                const float yp = cp[32];
                if (q > p) y = fmaf(-l, yp, y);
                // trailing update a[r] -= l * L[r][p], r > p, from 16-byte loads of column p
#pragma unroll
                for (int r4 = ((p + 1) / 4) * 4; r4 < KP; r4 += 4) {
                    const float4 c4 = *reinterpret_cast<const float4 *>(cp + r4);
                    const float cv[4] = {c4.x, c4.y, c4.z, c4.w};
                    if (r4 > p) {
                        fma2_sub(ar[r4], ar[r4 + 1], l, cv[0], cv[1]);
                        fma2_sub(ar[r4 + 2], ar[r4 + 3], l, cv[2], cv[3]);
                    } else {
#pragma unroll
                        for (int e = 0; e < 4; e += 2) {
                            const int r = r4 + e;
                            if (r > p) {
                                fma2_sub(ar[r], ar[r + 1], l, cv[e], cv[e + 1]);
                            } else if (r + 1 > p) {
                                ar[r + 1] = fmaf(-l, cv[e + 1], ar[r + 1]);
                            }
                        }
                    }
                }
            }
            const float yq = y * myinv;
            // ---- back substitution L^T x = y
            xq = back_subst(W, q, yq, myinv);
        } else {
            xq = (q < a.kout) ? a.u_given[row * a.ldo + q] : 0.f;
        }
        bool fail = !isfinite(xq);
        fail = __any_sync(FULL, fail) != 0;
        int32_t st = ST_OK;
        if (bad) st = ST_BAD;
        else if (s == 0) st = ST_EMPTY;
        else if (fail && !a.u_given) st = ST_NOT_SPD;
        if (st != ST_OK && !a.u_given) xq = 0.f;

        // ---- residual |A u - b| / (|A|_F |u| + |b|), optional refinement
        float rel = -1.f;
        if ((a.resid || a.refine) && (st == ST_OK || a.u_given)) {
            W.sv.x[q] = xq;
            __syncwarp();
            float aa;
            float r = ext_residual(W, q, bq, aa);
            if (a.refine && !a.u_given) {
                // A d = r with the FP32 factor: L z = r (L[q][p] = Lc[p][q]), L^T d = z
                float z = r;
#pragma unroll
                for (int p = 0; p < KP; ++p) {
                    const float zp = __shfl_sync(FULL, z * myinv, p);
                    if (q > p) z = fmaf(-W.sv.Lc[p][q], zp, z);
                }
                xq = xq + back_subst(W, q, z * myinv, myinv);
                __syncwarp();   // every lane has read x before it is rewritten
                W.sv.x[q] = xq;
                __syncwarp();
                r = ext_residual(W, q, bq, aa);
            }
            // |A|_F over the k x k system: the padded rows (q >= k) hold only lambda
            const float rr = warp_sum(r * r), na = warp_sum(q < a.kout ? aa : 0.f),
                        nu = warp_sum(xq * xq), nb = warp_sum(bq * bq);
            const float den = sqrtf(na) * sqrtf(nu) + sqrtf(nb);
            rel = den > 0.f ? sqrtf(rr) / den : 0.f;
        }
        if (!a.u_given) {
            if (q < a.kout) a.out[row * a.ldo + q] = xq;
            if (a.outb) {   // split BF16 copy [hi | lo] of the output row
                const __nv_bfloat16 hi = __float2bfloat16_rn(xq);
                __nv_bfloat16 *ob = reinterpret_cast<__nv_bfloat16 *>(a.outb) + row * 2 * KP;
                ob[q] = hi;
                ob[KP + q] = __float2bfloat16_rn(xq - __bfloat162float(hi));
            }
            if (a.status && q == 0) a.status[row] = st;
        }
        if (a.resid && q == 0) a.resid[row] = rel;
        __syncwarp();   // the shared area is restaged by the next system
    }
}

template <bool BF> size_t smem_bytes() { return sizeof(Smem32<BF>) * WARPS; }

template <bool BF> cudaError_t launch32(const SolveArgs<float> &a, cudaStream_t st) {
    int64_t blocks = (a.m + WARPS - 1) / WARPS;
    if (blocks > NUM_SMS_HINT * 32) blocks = NUM_SMS_HINT * 32;
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
    return cudaLaunchKernelEx(&cfg, k_solve32_tc<BF>, a);
}

}  // namespace

cudaError_t prepare_solve32_tc() {
    cudaError_t e = cudaFuncSetAttribute(k_solve32_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem_bytes<true>());
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_solve32_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem_bytes<false>());
}

cudaError_t launch_solve32_tc(const SolveArgs<float> &a, bool bf16, cudaStream_t st) {
    if (a.m <= 0) return cudaSuccess;
    if (bf16 && !a.Fb) return cudaErrorInvalidValue;
    if (a.gram) return cudaErrorInvalidValue;   // the streaming refit's sums are not supported here
    return bf16 ? launch32<true>(a, st) : launch32<false>(a, st);
}

}  // namespace ocf
