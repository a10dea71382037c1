// One NCF training step (the paper's CF model, Sec. "Collaborative Filtering
// Model"; mean squared error over a mini-batch of observed entries, Adam) in
// two kernels.
//
// k_ncf_train_tile: one CTA per 32 batch rows runs the whole forward and
// backward pass of its rows on the SM, with the BF16 weights and every
// activation in shared memory:
//   gather   x = [Ea_i, Es_j]                        (32 x 64, BF16)
//   forward  z1 = x W1 + b1, h1 = SELU(z1)            (32 x 128)
//            z2 = h1 W2 + b2, h2 = SELU(z2)           (32 x 64)
//   head     y = h2 . w3 + b3, dy = 2 (y - r) / B, dz2 = dy w3 SELU'(z2)
//   backward dz1 = (dz2 W2^T) SELU'(z1),  dW2 += h1^T dz2,  dW1 += x^T dz1,
//            db1 += colsum dz1,  dx = dz1 W1^T -> the two embedding rows
// Every product is an mma.sync m16n8k16 (BF16 operands, FP32 accumulation)
// on operands read by ldmatrix from padded shared tiles.  The CTA's share of
// the network gradient goes to its own partial vector (in the packing of the
// parameters); the embedding gradients are added atomically into the
// gradient table (rows of different CTAs can coincide).
//
// k_ncf_reduce_adam: sums the partial vectors in CTA order (a fixed order),
// applies Adam to every parameter (network and both embedding tables, dense
// moments), refreshes the BF16 copies of W1 and W2, clears the embedding
// gradient for the next step, and records the step's loss.
//
// A step reads its batch position from a device-side counter, so one CUDA
// graph of the two kernels serves every step of a training run.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"
#include "kernels.h"

namespace ocf {

namespace {

typedef __nv_bfloat16 bf16;

constexpr float SELU_L = 1.0507009873554804934193349852946f;
constexpr float SELU_A = 1.6732632423543772848170429916717f;

__device__ __forceinline__ float selu_t(float z) {
    const float e = __expf(fminf(z, 0.f)) - 1.f;
    return z > 0.f ? SELU_L * z : (SELU_L * SELU_A) * e;
}
__device__ __forceinline__ float dselu_t(float z) {
    return z > 0.f ? SELU_L : (SELU_L * SELU_A) * __expf(z);
}

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                               uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
__device__ __forceinline__ void mma_f16_16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                              uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
__device__ __forceinline__ void ld_x4(uint32_t (&r)[4], const bf16 *p) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(s));
}
__device__ __forceinline__ void ld_x4_t(uint32_t (&r)[4], const bf16 *p) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(s));
}

// Warp tile of a shared-memory product: acc[j] += op(A)[m0 .. m0 + 16, :] op(B)[:, n0 + 8 j ..]
// over K.  A is [M][K] (row stride lda), or [K][M] when AT; B is [K][N], or
// [N][K] when BT.  acc[j][e]: row m0 + lane / 4 + 8 (e / 2), column
// n0 + 8 j + 2 (lane % 4) + e % 2.  F16: the tiles hold FP16, not BF16, values
// (same 16-bit layout; only the MMA's operand type differs).
template <bool AT, bool BT, int NT, bool F16 = false>
__device__ __forceinline__ void warp_mma(float (&acc)[NT][4], const bf16 *A, int lda,
                                         const bf16 *B, int ldb, int m0, int n0, int K,
                                         int lane) {
    const int mi = lane >> 3, rr = lane & 7;
#pragma unroll
    for (int j = 0; j < NT; ++j)
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[j][e] = 0.f;
    for (int k0 = 0; k0 < K; k0 += 16) {
        uint32_t af[4];
        if (!AT) ld_x4(af, A + (m0 + (lane & 15)) * lda + k0 + (lane >> 4) * 8);
        else ld_x4_t(af, A + (k0 + (mi >> 1) * 8 + rr) * lda + m0 + (mi & 1) * 8);
#pragma unroll
        for (int j = 0; j < NT; j += 2) {
            const int nb = n0 + 8 * j;
            uint32_t t[4];
            if (!BT) ld_x4_t(t, B + (k0 + (mi & 1) * 8 + rr) * ldb + nb + (mi >> 1) * 8);
            else ld_x4(t, B + (nb + (mi >> 1) * 8 + rr) * ldb + k0 + (mi & 1) * 8);
            if constexpr (F16) {
                mma_f16_16816(acc[j], af, t[0], t[1]);
                mma_f16_16816(acc[j + 1], af, t[2], t[3]);
            } else {
                mma_bf16_16816(acc[j], af, t[0], t[1]);
                mma_bf16_16816(acc[j + 1], af, t[2], t[3]);
            }
        }
    }
}

__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

__device__ __forceinline__ void st_pair(bf16 *p, float a, float b) {
    *reinterpret_cast<__nv_bfloat162 *>(p) = __floats2bfloat162_rn(a, b);
}

constexpr int TB = 64;                  // rows per tile of the prediction kernel
constexpr int TT = NCF_TT;              // batch rows per CTA of the training kernel
constexpr int MT = TT / 16;             // its 16-row slabs (MMA m-tiles)
constexpr int WPM = 8 / MT;             // warps sharing one slab
constexpr int NTH = 256;
constexpr int RPT = TT * 8 / NTH;       // gathered rows per thread
constexpr int SX = 2 * NCF_D + 8;       // row strides (elements) of the padded tiles
constexpr int S1 = NCF_H1 + 8;
constexpr int S2 = NCF_H2 + 8;
constexpr uint32_t O_W1 = 0;                                   // W1  [64][S1]
constexpr uint32_t O_W2 = O_W1 + 2 * NCF_D * S1 * 2;           // W2  [128][S2]
constexpr uint32_t O_X = O_W2 + NCF_H1 * S2 * 2;               // x   [64][SX]
constexpr uint32_t O_Z1 = O_X + TT * SX * 2;                   // z1, h1, dz1 [TT][S1]
constexpr uint32_t O_H1 = O_Z1 + TT * S1 * 2;
constexpr uint32_t O_DZ1 = O_H1 + TT * S1 * 2;
constexpr uint32_t O_Z2 = O_DZ1 + TT * S1 * 2;                 // z2, h2, dz2 [TT][S2]
constexpr uint32_t O_H2 = O_Z2 + TT * S2 * 2;
constexpr uint32_t O_DZ2 = O_H2 + TT * S2 * 2;
constexpr int HEADP = 2 * NCF_H2 + 2;                          // gb2 | gw3 | gb3 | sse
constexpr uint32_t O_RED = O_DZ2 + TT * S2 * 2;                // [8][HEADP] floats
constexpr uint32_t O_R = O_RED + 8 * HEADP * 4;
constexpr uint32_t O_RI = O_R + TT * 4;
constexpr uint32_t O_RJ = O_RI + TT * 4;
constexpr uint32_t O_CB = O_RJ + TT * 4;                         // [MT][128] db1 partials
constexpr uint32_t TRAIN_SMEM = O_CB + MT * NCF_H1 * 4;

__global__ void __launch_bounds__(NTH, 1) k_ncf_train_tile(NcfTrainArgs a) {
    extern __shared__ __align__(16) unsigned char sm[];
    bf16 *W1s = reinterpret_cast<bf16 *>(sm + O_W1), *W2s = reinterpret_cast<bf16 *>(sm + O_W2);
    bf16 *Xs = reinterpret_cast<bf16 *>(sm + O_X);
    bf16 *Z1s = reinterpret_cast<bf16 *>(sm + O_Z1), *H1s = reinterpret_cast<bf16 *>(sm + O_H1);
    bf16 *D1s = reinterpret_cast<bf16 *>(sm + O_DZ1);
    bf16 *Z2s = reinterpret_cast<bf16 *>(sm + O_Z2), *H2s = reinterpret_cast<bf16 *>(sm + O_H2);
    bf16 *D2s = reinterpret_cast<bf16 *>(sm + O_DZ2);
    float *red = reinterpret_cast<float *>(sm + O_RED);
    float *Rs = reinterpret_cast<float *>(sm + O_R);
    int32_t *RI = reinterpret_cast<int32_t *>(sm + O_RI), *RJ = reinterpret_cast<int32_t *>(sm + O_RJ);
    float *colp = reinterpret_cast<float *>(sm + O_CB);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int gid = lane >> 2, t4 = lane & 3;

    // batch position of this step
    const int64_t s = a.ctl->step;
    const int64_t epoch = s / a.spe, off = (s % a.spe) * (int64_t)a.B;
    const int64_t left = a.nnz - off;
    const int beff = (int)(left < a.B ? left : a.B);
    if (blockIdx.x == 0 && tid == 0) {
        a.ctl->beff = beff;
        if (a.adam) a.adam->t += 1;   // the update kernel of this step reads it
    }

    // ---- weights (BF16 copies, row-major): asynchronous copies into the padded
    // tiles, in flight while the inputs are gathered
    const bf16 *W1g = reinterpret_cast<const bf16 *>(a.W1b);
    const bf16 *W2g = reinterpret_cast<const bf16 *>(a.W2b);
    for (int v = tid; v < 2 * NCF_D * (NCF_H1 / 8); v += NTH) {
        const int r = v / (NCF_H1 / 8), c8 = (v % (NCF_H1 / 8)) * 8;
        cp_async16(W1s + r * S1 + c8, W1g + r * NCF_H1 + c8);
    }
    for (int v = tid; v < NCF_H1 * (NCF_H2 / 8); v += NTH) {
        const int r = v / (NCF_H2 / 8), c8 = (v % (NCF_H2 / 8)) * 8;
        cp_async16(W2s + r * S2 + c8, W2g + r * NCF_H2 + c8);
    }
    cp_async_commit();
    // ---- gathered inputs: thread (row rr, chunk q) takes rows rr, rr + 32, ...
    // (RPT of them), their dependent load chains (position -> indices ->
    // embedding rows) in flight together
    {
        const int q = tid & 7;
        int rr[RPT], b[RPT];
        bool ok[RPT];
        int64_t e[RPT];
        int32_t i[RPT], j[RPT];
        float rv[RPT];
#pragma unroll
        for (int h = 0; h < RPT; ++h) {
            rr[h] = (tid >> 3) + 32 * h;
            b[h] = blockIdx.x * TT + rr[h];
            ok[h] = b[h] < beff;
            e[h] = off + b[h];
        }
        if (a.perms) {
#pragma unroll
            for (int h = 0; h < RPT; ++h)
                if (ok[h]) e[h] = (int64_t)__ldg(a.perms + epoch * a.nnz + off + b[h]);
        }
#pragma unroll
        for (int h = 0; h < RPT; ++h) {
            ok[h] = ok[h] && e[h] >= 0 && e[h] < a.nnz;
            i[h] = -1;
            j[h] = -1;
            rv[h] = 0.f;
            if (ok[h] && !a.feat) {
                i[h] = __ldg(a.app + e[h]);
                j[h] = __ldg(a.set + e[h]);
            }
            if (ok[h] && a.val) rv[h] = __ldg(a.val + e[h]);   // no targets when only predicting
        }
        uint4 pk[RPT];
#pragma unroll
        for (int h = 0; h < RPT; ++h) {
            const bool live = b[h] < beff;
            if (ok[h] && !a.feat)
                ok[h] = i[h] >= 0 && (int64_t)i[h] < a.m && j[h] >= 0 && (int64_t)j[h] < a.n;
            if (ok[h] && a.feat) i[h] = 0;   // a live row (no embedding rows to update)
            if (live && !ok[h] && q == 0)
                atomicAdd(reinterpret_cast<unsigned long long *>(&a.ctl->skipped), 1ull);
            float x[8];
#pragma unroll
            for (int t = 0; t < 8; ++t) x[t] = 0.f;
            if (ok[h] && a.feat) {   // dense features, zero padded to 64 columns
#pragma unroll
                for (int t = 0; t < 8; ++t)
                    if (8 * q + t < a.nfeat) x[t] = __ldg(a.feat + e[h] * a.nfeat + 8 * q + t);
            } else if (ok[h]) {
                const float *src = q < 4 ? a.Ea + (int64_t)i[h] * NCF_D + 8 * q
                                         : a.Es + (int64_t)j[h] * NCF_D + 8 * (q - 4);
                const float4 x0 = __ldg(reinterpret_cast<const float4 *>(src));
                const float4 x1 = __ldg(reinterpret_cast<const float4 *>(src) + 1);
                x[0] = x0.x; x[1] = x0.y; x[2] = x0.z; x[3] = x0.w;
                x[4] = x1.x; x[5] = x1.y; x[6] = x1.z; x[7] = x1.w;
            }
            __nv_bfloat162 p0 = __floats2bfloat162_rn(x[0], x[1]), p1 = __floats2bfloat162_rn(x[2], x[3]);
            __nv_bfloat162 p2 = __floats2bfloat162_rn(x[4], x[5]), p3 = __floats2bfloat162_rn(x[6], x[7]);
            pk[h] = make_uint4(*reinterpret_cast<uint32_t *>(&p0), *reinterpret_cast<uint32_t *>(&p1),
                               *reinterpret_cast<uint32_t *>(&p2), *reinterpret_cast<uint32_t *>(&p3));
        }
#pragma unroll
        for (int h = 0; h < RPT; ++h) {
            *reinterpret_cast<uint4 *>(Xs + rr[h] * SX + 8 * q) = pk[h];
            if (q == 0) {
                Rs[rr[h]] = ok[h] ? rv[h] : 0.f;
                RI[rr[h]] = ok[h] ? i[h] : -1;
                RJ[rr[h]] = ok[h] ? j[h] : -1;
            }
        }
    }
    cp_async_wait_all();
    __syncthreads();

    // ---- z1 = x W1 + b1 (TT x 128, K = 64)
    {
        constexpr int NT = NCF_H1 / WPM / 8;
        const int m0 = 16 * (warp % MT), n0 = (NCF_H1 / WPM) * (warp / MT);
        float acc[NT][4];
        warp_mma<false, false, NT>(acc, Xs, SX, W1s, S1, m0, n0, 2 * NCF_D, lane);
#pragma unroll
        for (int j = 0; j < NT; ++j)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int r = m0 + gid + 8 * h, c = n0 + 8 * j + 2 * t4;
                const float z0 = acc[j][2 * h] + a.b1[c], z1 = acc[j][2 * h + 1] + a.b1[c + 1];
                st_pair(Z1s + r * S1 + c, z0, z1);
                st_pair(H1s + r * S1 + c, selu_t(z0), selu_t(z1));
            }
    }
    __syncthreads();

    // ---- z2 = h1 W2 + b2 (TT x 64, K = 128)
    {
        constexpr int NT = NCF_H2 / WPM / 8;
        const int m0 = 16 * (warp % MT), n0 = (NCF_H2 / WPM) * (warp / MT);
        float acc[NT][4];
        warp_mma<false, false, NT>(acc, H1s, S1, W2s, S2, m0, n0, NCF_H1, lane);
#pragma unroll
        for (int j = 0; j < NT; ++j)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int r = m0 + gid + 8 * h, c = n0 + 8 * j + 2 * t4;
                const float z0 = acc[j][2 * h] + a.b2[c], z1 = acc[j][2 * h + 1] + a.b2[c + 1];
                st_pair(Z2s + r * S2 + c, z0, z1);
                st_pair(H2s + r * S2 + c, selu_t(z0), selu_t(z1));
            }
    }
    __syncthreads();

    // ---- head: warp w takes rows (TT/8) w .. + TT/8 - 1, lane l hidden columns 2l, 2l + 1
    {
        const float scale = beff > 0 ? 2.f / (float)beff : 0.f;
        const float w0 = a.w3[2 * lane], w1 = a.w3[2 * lane + 1], b3 = a.b3[0];
        float gb2_0 = 0.f, gb2_1 = 0.f, gw3_0 = 0.f, gw3_1 = 0.f, gb3 = 0.f, sse = 0.f;
        for (int u = 0; u < TT / 8; ++u) {
            const int r = (TT / 8) * warp + u;
            const __nv_bfloat162 hh = *reinterpret_cast<const __nv_bfloat162 *>(H2s + r * S2 + 2 * lane);
            const __nv_bfloat162 zz = *reinterpret_cast<const __nv_bfloat162 *>(Z2s + r * S2 + 2 * lane);
            const float h0 = __low2float(hh), h1 = __high2float(hh);
            float y = fmaf(w1, h1, w0 * h0);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) y += __shfl_xor_sync(FULL, y, o);
            y += b3;
            const float e = RI[r] >= 0 ? y - Rs[r] : 0.f;
            const float dy = scale * e;
            const float d0 = dy * w0 * dselu_t(__low2float(zz));
            const float d1 = dy * w1 * dselu_t(__high2float(zz));
            st_pair(D2s + r * S2 + 2 * lane, d0, d1);
            gb2_0 += d0; gb2_1 += d1;
            gw3_0 = fmaf(dy, h0, gw3_0); gw3_1 = fmaf(dy, h1, gw3_1);
            gb3 += dy;
            sse = fmaf(e, e, sse);
        }
        float *rw = red + warp * HEADP;
        rw[2 * lane] = gb2_0;
        rw[2 * lane + 1] = gb2_1;
        rw[NCF_H2 + 2 * lane] = gw3_0;
        rw[NCF_H2 + 2 * lane + 1] = gw3_1;
        if (lane == 0) {
            rw[2 * NCF_H2] = gb3;
            rw[2 * NCF_H2 + 1] = sse;
        }
    }
    __syncthreads();
    float *part = a.part + (int64_t)blockIdx.x * a.part_stride;
    for (int c = tid; c < HEADP; c += NTH) {
        float v = 0.f;
        for (int w = 0; w < 8; ++w) v += red[w * HEADP + c];
        if (c < HEADP - 1) part[NCF_OFF_B2 + c] = v;   // gb2 | gw3 | gb3, contiguous in the packing
        else a.lpart[blockIdx.x] = v;
    }

    // ---- dz1 = (dz2 W2^T) SELU'(z1) (TT x 128, K = 64), and dW2 = h1^T dz2 (128 x 64, K = TT)
    {
        constexpr int NT = NCF_H1 / WPM / 8;
        const int m0 = 16 * (warp % MT), n0 = (NCF_H1 / WPM) * (warp / MT);
        float acc[NT][4];
        warp_mma<false, true, NT>(acc, D2s, S2, W2s, S2, m0, n0, NCF_H2, lane);
#pragma unroll
        for (int j = 0; j < NT; ++j) {
            float cs0 = 0.f, cs1 = 0.f;   // this lane's two columns over its two rows
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int r = m0 + gid + 8 * h, c = n0 + 8 * j + 2 * t4;
                const __nv_bfloat162 zz = *reinterpret_cast<const __nv_bfloat162 *>(Z1s + r * S1 + c);
                const float d0 = acc[j][2 * h] * dselu_t(__low2float(zz));
                const float d1 = acc[j][2 * h + 1] * dselu_t(__high2float(zz));
                st_pair(D1s + r * S1 + c, d0, d1);
                cs0 += d0;
                cs1 += d1;
            }
#pragma unroll
            for (int o = 4; o < 32; o <<= 1) {   // over the eight row pairs of the slab
                cs0 += __shfl_xor_sync(FULL, cs0, o);
                cs1 += __shfl_xor_sync(FULL, cs1, o);
            }
            if (gid == 0) {
                colp[(warp % MT) * NCF_H1 + n0 + 8 * j + 2 * t4] = cs0;
                colp[(warp % MT) * NCF_H1 + n0 + 8 * j + 2 * t4 + 1] = cs1;
            }
        }
    }
    {
        const int m0 = 16 * warp;
        float acc[8][4];
        warp_mma<true, false, 8>(acc, H1s, S1, D2s, S2, m0, 0, TT, lane);
#pragma unroll
        for (int j = 0; j < 8; ++j)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int r = m0 + gid + 8 * h, c = 8 * j + 2 * t4;
                *reinterpret_cast<float2 *>(part + NCF_OFF_W2 + r * NCF_H2 + c) =
                    make_float2(acc[j][2 * h], acc[j][2 * h + 1]);
            }
    }
    __syncthreads();

    // ---- dW1 = x^T dz1 (64 x 128, K = TT), db1 = column sums of dz1
    {
        const int m0 = 16 * (warp & 3), n0 = 64 * (warp >> 2);
        float acc[8][4];
        warp_mma<true, false, 8>(acc, Xs, SX, D1s, S1, m0, n0, TT, lane);
#pragma unroll
        for (int j = 0; j < 8; ++j)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int r = m0 + gid + 8 * h, c = n0 + 8 * j + 2 * t4;
                *reinterpret_cast<float2 *>(part + r * NCF_H1 + c) =
                    make_float2(acc[j][2 * h], acc[j][2 * h + 1]);
            }
    }
    if (tid < NCF_H1) {   // the 16-row slabs in order
        float v = colp[tid];
#pragma unroll
        for (int t = 1; t < MT; ++t) v += colp[t * NCF_H1 + tid];
        part[NCF_OFF_B1 + tid] = v;
    }
    // ---- dx = dz1 W1^T (TT x 64, K = 128) into the embedding gradients
    if (a.gE) {
        constexpr int NT = 2 * NCF_D / WPM / 8;
        const int m0 = 16 * (warp % MT), n0 = (2 * NCF_D / WPM) * (warp / MT);
        float acc[NT][4];
        warp_mma<false, true, NT>(acc, D1s, S1, W1s, S1, m0, n0, NCF_H1, lane);
#pragma unroll
        for (int j = 0; j < NT; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int r = m0 + gid + 8 * (e >> 1), c = n0 + 8 * j + 2 * t4 + (e & 1);
                const bool lo = c < NCF_D;
                const int32_t row = lo ? RI[r] : RJ[r];
                if (row >= 0)
                    atomicAdd(a.gE + (lo ? 0 : a.s_off) + (int64_t)row * NCF_D + (lo ? c : c - NCF_D),
                              acc[j][e]);
            }
    }
}

// Network gradient = sum of the CTA partials (CTA order); Adam on every
// parameter; BF16 copies of W1, W2; embedding gradient cleared; loss recorded.
__global__ void __launch_bounds__(256) k_ncf_reduce_adam(NcfAdamArgs a) {
    __shared__ float corr[3];   // bias corrections of step t and the step size, once per CTA
    const int64_t total = a.net_pad + a.n_emb;
    if (threadIdx.x == 0) {
        corr[0] = corr[1] = 1.f;
        corr[2] = 0.f;
        if (a.update) {   // 1 - beta^t as 1 - 2^(t log2 beta), in FP32 (accurate to ~1e-7 here)
            const float tt = (float)a.adam->t;
            corr[0] = 1.f - exp2f(tt * log2f(0.9f));
            corr[1] = 1.f - exp2f(tt * log2f(0.999f));
            corr[2] = a.adam->lr;
        }
    }
    __syncthreads();
    const float fc1 = corr[0], fc2 = corr[1], lr = corr[2];
    bf16 *bf = reinterpret_cast<bf16 *>(a.bf);
    // Work items: four per network parameter (lane q of a group of four sums
    // partials q, q + 4, q + 8, ... in order, and the four sums are combined in
    // a fixed order: one round of loads instead of parts / 8 dependent ones),
    // then the embedding table four entries at a time (it starts 16-byte
    // aligned at net_pad; the padding between is never touched).  Only an
    // update touches the embeddings.
    const int64_t n4 = a.update ? a.n_emb / 4 : 0;
    const int64_t items = 4 * NCF_NET + n4;
    const int lane = threadIdx.x & 31;
    for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < items;
         w += (int64_t)gridDim.x * blockDim.x) {
        if (w < 4 * NCF_NET) {   // 4 NCF_NET is a multiple of 4: a group never straddles
            const int64_t e = w >> 2;
            const int q = (int)(w & 3);
            const unsigned gm = 0xFu << (lane & ~3);
            float g = 0.f;
            int c = q;
            for (; c + 28 < a.parts; c += 32) {   // eight partials in flight at a time
                float v[8];
#pragma unroll
                for (int t = 0; t < 8; ++t) v[t] = a.part[(int64_t)(c + 4 * t) * a.part_stride + e];
#pragma unroll
                for (int t = 0; t < 8; ++t) g += v[t];
            }
            for (; c < a.parts; c += 4) g += a.part[(int64_t)c * a.part_stride + e];
            g += __shfl_xor_sync(gm, g, 1);   // (s0 + s1) + (s2 + s3) on every lane
            g += __shfl_xor_sync(gm, g, 2);
            if (q != 0) continue;
            a.grad[e] = g;
            if (!a.update) continue;
            const float m1 = 0.9f * a.m1[e] + 0.1f * g;
            const float m2 = 0.999f * a.m2[e] + 0.001f * g * g;
            a.m1[e] = m1;
            a.m2[e] = m2;
            const float t = a.th[e] - lr * (m1 / fc1) / (sqrtf(m2 / fc2) + 1e-8f);
            a.th[e] = t;
            if (e < NCF_OFF_B1) bf[e] = __float2bfloat16_rn(t);
            else if (e >= NCF_OFF_W2 && e < NCF_OFF_B2)
                bf[NCF_OFF_B1 + (e - NCF_OFF_W2)] = __float2bfloat16_rn(t);
        } else {   // embeddings: the same update on a float4, the gradient cleared
            const int64_t e = a.net_pad + 4 * (w - 4 * NCF_NET);
            float4 *gp = reinterpret_cast<float4 *>(a.grad + e);
            float4 *m1p = reinterpret_cast<float4 *>(a.m1 + e);
            float4 *m2p = reinterpret_cast<float4 *>(a.m2 + e);
            float4 *thp = reinterpret_cast<float4 *>(a.th + e);
            const float4 g4 = *gp, a1 = *m1p, a2 = *m2p, t4 = *thp;
            *gp = make_float4(0.f, 0.f, 0.f, 0.f);
            const float gv[4] = {g4.x, g4.y, g4.z, g4.w}, v1[4] = {a1.x, a1.y, a1.z, a1.w};
            const float v2[4] = {a2.x, a2.y, a2.z, a2.w}, vt[4] = {t4.x, t4.y, t4.z, t4.w};
            float o1[4], o2[4], ot[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float g = gv[q];
                o1[q] = 0.9f * v1[q] + 0.1f * g;
                o2[q] = 0.999f * v2[q] + 0.001f * g * g;
                ot[q] = vt[q] - lr * (o1[q] / fc1) / (sqrtf(o2[q] / fc2) + 1e-8f);
            }
            *m1p = make_float4(o1[0], o1[1], o1[2], o1[3]);
            *m2p = make_float4(o2[0], o2[1], o2[2], o2[3]);
            *thp = make_float4(ot[0], ot[1], ot[2], ot[3]);
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        double sse = 0.0;
        for (int c = 0; c < a.parts; ++c) sse += (double)a.lpart[c];
        const int beff = a.ctl->beff;
        const double L = beff > 0 ? sse / (double)beff : 0.0;
        if (a.loss_hist) a.loss_hist[a.ctl->step] = L;
        if (a.loss_last) *a.loss_last = L;
        a.ctl->step += 1;
    }
}

// BF16 copies of W1 and W2 from the FP32 parameters (after they are set).
__global__ void k_ncf_refresh_bf(const float *__restrict__ th, bf16 *__restrict__ bf) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 2 * NCF_OFF_B1;
         e += gridDim.x * blockDim.x)
        bf[e] = __float2bfloat16_rn(e < NCF_OFF_B1 ? th[e] : th[NCF_OFF_W2 + e - NCF_OFF_B1]);
}

// Prediction with the dense-feature network (the offline performance
// predictor): a persistent kernel that loads W1 (only the K1 = nfeat rounded
// up to 16 rows that meet non-zero inputs) and W2 once per CTA and walks
// 64-row tiles: gather -> z1 (K = K1) -> SELU -> z2 -> SELU -> y, the output
// dot product folded into the second layer's epilogue.  The first layer runs
// on BF16 operands like training; the hidden activations are formed in packed
// FP16 pairs (a branch-free SELU on two values per instruction: lambda
// max(z, 0) + lambda alpha (2^(log2(e) min(z, 0)) - 1)) and the second layer
// multiplies them, on FP16 operands, with W2 converted from its BF16 copy
// (exact for |w| >= 2^-14; FP16 keeps three more mantissa bits than BF16 for
// the activations).  Biases and output weights sit in registers.
constexpr uint32_t P_OFF_W1 = 0;                                  // W1 [64][S1] BF16 (K1 rows used)
constexpr uint32_t P_OFF_W2 = P_OFF_W1 + 2 * NCF_D * S1 * 2;      // W2 [128][S2] FP16
constexpr uint32_t P_OFF_X = P_OFF_W2 + NCF_H1 * S2 * 2;          // x  [64][SX] BF16
constexpr uint32_t P_OFF_H1 = P_OFF_X + TB * SX * 2;              // h1 [64][S1] FP16
constexpr uint32_t P_OFF_Y = P_OFF_H1 + TB * S1 * 2;              // [2][64] partial y
constexpr uint32_t PRED_SMEM = P_OFF_Y + 2 * TB * 4;

__device__ __forceinline__ uint32_t h2_bits(__half2 h) { return *reinterpret_cast<uint32_t *>(&h); }
__device__ __forceinline__ __half2 bits_h2(uint32_t u) { return *reinterpret_cast<__half2 *>(&u); }

__device__ __forceinline__ __half2 selu_h2(__half2 z) {
    const __half2 zero = __float2half2_rn(0.f);
    const __half2 t = __hmul2(__hmin2(z, zero), __float2half2_rn(1.4426950408889634f));
    uint32_t e;
    asm("ex2.approx.f16x2 %0, %1;" : "=r"(e) : "r"(h2_bits(t)));
    const __half2 la = __float2half2_rn(SELU_L * SELU_A);
    const __half2 neg = __hfma2(bits_h2(e), la, __hneg2(la));
    return __hfma2(__hmax2(z, zero), __float2half2_rn(SELU_L), neg);
}

__global__ void __launch_bounds__(NTH, 3) k_pred_forward(NcfTrainArgs a) {
    extern __shared__ __align__(16) unsigned char sm[];
    bf16 *W1s = reinterpret_cast<bf16 *>(sm + P_OFF_W1);
    __half *W2s = reinterpret_cast<__half *>(sm + P_OFF_W2);
    bf16 *Xs = reinterpret_cast<bf16 *>(sm + P_OFF_X);
    __half *H1s = reinterpret_cast<__half *>(sm + P_OFF_H1);
    float *yp = reinterpret_cast<float *>(sm + P_OFF_Y);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int gid = lane >> 2, t4 = lane & 3;
    const int K1 = (a.nfeat + 15) / 16 * 16;
    const bf16 *W1g = reinterpret_cast<const bf16 *>(a.W1b);
    const bf16 *W2g = reinterpret_cast<const bf16 *>(a.W2b);
    for (int v = tid; v < K1 * (NCF_H1 / 8); v += NTH) {
        const int r = v / (NCF_H1 / 8), c8 = (v % (NCF_H1 / 8)) * 8;
        *reinterpret_cast<uint4 *>(W1s + r * S1 + c8) =
            __ldg(reinterpret_cast<const uint4 *>(W1g + r * NCF_H1 + c8));
    }
    for (int v = tid; v < NCF_H1 * (NCF_H2 / 8); v += NTH) {
        const int r = v / (NCF_H2 / 8), c8 = (v % (NCF_H2 / 8)) * 8;
        const uint4 w = __ldg(reinterpret_cast<const uint4 *>(W2g + r * NCF_H2 + c8));
        const uint32_t wv[4] = {w.x, w.y, w.z, w.w};
        uint32_t hv[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&wv[q]));
            hv[q] = h2_bits(__floats2half2_rn(f.x, f.y));
        }
        *reinterpret_cast<uint4 *>(W2s + r * S2 + c8) = make_uint4(hv[0], hv[1], hv[2], hv[3]);
    }
    // this thread's columns of both epilogues: layer 1 n0 + 8 j + 2 t4 (+1),
    // layer 2 likewise with its own n0
    const int m0 = 16 * (warp & 3), n1 = 64 * (warp >> 2), n2 = 32 * (warp >> 2);
    __half2 b1h[8], b2h[4];
    float w3v[4][2];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int c = n1 + 8 * j + 2 * t4;
        b1h[j] = __floats2half2_rn(a.b1[c], a.b1[c + 1]);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int c = n2 + 8 * j + 2 * t4;
        b2h[j] = __floats2half2_rn(a.b2[c], a.b2[c + 1]);
        w3v[j][0] = a.w3[c];
        w3v[j][1] = a.w3[c + 1];
    }
    const float b3 = a.b3[0];
    const int64_t tiles = (a.nnz + TB - 1) / TB;
    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int64_t r0 = tile * TB;
        // x tile: K1 columns (features, then zeros)
        for (int v = tid; v < TB * (K1 / 8); v += NTH) {
            const int rr = v / (K1 / 8), q = v % (K1 / 8);
            const int64_t e = r0 + rr;
            float x[8];
#pragma unroll
            for (int t = 0; t < 8; ++t)
                x[t] = (e < a.nnz && 8 * q + t < a.nfeat) ? __ldg(a.feat + e * a.nfeat + 8 * q + t)
                                                          : 0.f;
#pragma unroll
            for (int t = 0; t < 8; t += 2) st_pair(Xs + rr * SX + 8 * q + t, x[t], x[t + 1]);
        }
        __syncthreads();
        {   // h1 = SELU(x W1 + b1), FP16 pairs
            float acc[8][4];
            warp_mma<false, false, 8>(acc, Xs, SX, W1s, S1, m0, n1, K1, lane);
#pragma unroll
            for (int j = 0; j < 8; ++j)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int r = m0 + gid + 8 * h, c = n1 + 8 * j + 2 * t4;
                    const __half2 z =
                        __hadd2(__floats2half2_rn(acc[j][2 * h], acc[j][2 * h + 1]), b1h[j]);
                    *reinterpret_cast<__half2 *>(H1s + r * S1 + c) = selu_h2(z);
                }
        }
        __syncthreads();
        {   // z2 = h1 W2 + b2; this warp's share of y = SELU(z2) . w3
            float acc[4][4];
            warp_mma<false, false, 4, true>(acc, reinterpret_cast<const bf16 *>(H1s), S1,
                                            reinterpret_cast<const bf16 *>(W2s), S2, m0, n2,
                                            NCF_H1, lane);
            float p[2] = {0.f, 0.f};
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const __half2 z =
                        __hadd2(__floats2half2_rn(acc[j][2 * h], acc[j][2 * h + 1]), b2h[j]);
                    const float2 hv = __half22float2(selu_h2(z));
                    p[h] = fmaf(w3v[j][0], hv.x, p[h]);
                    p[h] = fmaf(w3v[j][1], hv.y, p[h]);
                }
#pragma unroll
            for (int h = 0; h < 2; ++h) {   // the four lanes of a row hold its columns
                p[h] += __shfl_xor_sync(FULL, p[h], 1);
                p[h] += __shfl_xor_sync(FULL, p[h], 2);
                if (t4 == 0) yp[(warp >> 2) * TB + m0 + gid + 8 * h] = p[h];
            }
        }
        __syncthreads();
        if (tid < TB && r0 + tid < a.nnz) a.y_out[r0 + tid] = (yp[tid] + yp[TB + tid]) + b3;
    }
}

}  // namespace

cudaError_t prepare_ncf_train() {
    cudaError_t e = cudaFuncSetAttribute(k_ncf_train_tile,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)TRAIN_SMEM);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_pred_forward, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)PRED_SMEM);
}

cudaError_t launch_ncf_train_step(const NcfTrainArgs &t, const NcfAdamArgs &u, cudaStream_t st) {
    if (t.B % TT || t.B <= 0 || u.parts != t.B / TT) return cudaErrorInvalidValue;
    k_ncf_train_tile<<<t.B / TT, NTH, TRAIN_SMEM, st>>>(t);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (u.net_pad % 4 || u.n_emb % 4) return cudaErrorInvalidValue;   // float4 embedding updates
    int64_t blocks = (4 * NCF_NET + u.n_emb / 4 + 255) / 256;
    if (blocks > NUM_SMS_HINT * 8) blocks = NUM_SMS_HINT * 8;
    k_ncf_reduce_adam<<<(unsigned)blocks, 256, 0, st>>>(u);
    return cudaGetLastError();
}

cudaError_t launch_pred_forward(const NcfTrainArgs &t, int num_sms, cudaStream_t st) {
    if (!t.feat || !t.y_out || t.nfeat < 1 || t.nfeat > 2 * NCF_D) return cudaErrorInvalidValue;
    if (t.nnz <= 0) return cudaSuccess;
    const int64_t tiles = (t.nnz + TB - 1) / TB, cap = 3 * (int64_t)num_sms;   // 3 CTAs per SM
    k_pred_forward<<<(unsigned)(tiles < cap ? tiles : cap), NTH, PRED_SMEM, st>>>(t);
    return cudaGetLastError();
}

cudaError_t launch_ncf_refresh_bf(const float *theta, void *bf, cudaStream_t st) {
    k_ncf_refresh_bf<<<32, 256, 0, st>>>(theta, reinterpret_cast<bf16 *>(bf));
    return cudaGetLastError();
}

}  // namespace ocf
