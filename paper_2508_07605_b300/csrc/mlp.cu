// Learned warm start for the online fold-in: an MLP that maps an
// application's first 16 online-profiled (CPU cap, GPU cap, runtime) samples
// straight to its latent factor u (k = 32), trained on factors the plain ALS
// fold-in produces; ALS remains the fallback where the MLP's observed-entry
// residual is too large (engine: open_cf_mlp_infer).  SELU activations, as
// the paper's collaborative-filtering MLP uses (Sec. "Collaborative Filtering
// Model"); constants from Klambauer et al. 2017.
//
// Network: X[B,64] (48 features + 16 zero columns) -> W1[64,256] -> SELU ->
// W2[256,256] -> SELU -> W3[256,k].  Every product is a BF16 tensor-core GEMM
// (mma.sync m16n8k16, FP32 accumulation, fragments by ldmatrix) with a fused
// epilogue; weight gradients use split-K partials summed in a fixed order, so
// a training step is bit-reproducible.
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"

namespace ocf {

typedef __nv_bfloat16 bf16;

constexpr float SELU_L = 1.0507009873554804934193349852946f;
constexpr float SELU_A = 1.6732632423543772848170429916717f;

__device__ __forceinline__ float selu(float z) { return z > 0.f ? SELU_L * z : SELU_L * SELU_A * expm1f(z); }
__device__ __forceinline__ float dselu(float z) { return z > 0.f ? SELU_L : SELU_L * SELU_A * expf(z); }

// ---------------------------------------------------------------- features
// Row i of the CSR (its settings in increasing index order): triple t of the
// first 16 observations is (c_norm, g_norm, runtime); missing triples are 0.
__global__ void k_mlp_features(int64_t m, int64_t nnz, const int64_t *__restrict__ ptr,
                               const int32_t *__restrict__ idx, const float *__restrict__ val,
                               const float *__restrict__ cnorm, const float *__restrict__ gnorm,
                               int64_t n, bf16 *__restrict__ X) {
    const int64_t total = m * MLP_INP;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / MLP_INP;
        const int f = (int)(e % MLP_INP);
        float x = 0.f;
        if (f < MLP_IN) {
            int64_t beg, end;
            if (row_bounds(ptr, i, nnz, beg, end)) {
                const int t = f / 3, c = f % 3;
                if (beg + t < end) {
                    const int32_t j = idx[beg + t];
                    if (j >= 0 && j < n) x = c == 0 ? cnorm[j] : (c == 1 ? gnorm[j] : val[beg + t]);
                }
            }
        }
        X[e] = __float2bfloat16_rn(x);
    }
}

// ---------------------------------------------------------------- GEMM
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
__device__ __forceinline__ void ldsm4(uint32_t (&r)[4], const void *p) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(s));
}
__device__ __forceinline__ void ldsm4t(uint32_t (&r)[4], const void *p) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(s));
}

constexpr int GBM = 64, GBN = 64, GBK = 32;

// C[M,N] = op(A)[M,K] op(B)[K,N].  A is [M,K] row-major, or [K,M] when AT;
// B is [K,N] row-major, or [N,K] when BT.  M, K multiples of 64 / 32; N a
// multiple of 32.  blockIdx.z selects a K slice (split-K partials for EPI_PART).
template <bool AT, bool BT, int EPI>
__global__ void __launch_bounds__(128) k_gemm_bf16(GemmArgs g) {
    constexpr int AS = AT ? GBM + 8 : GBK + 8;   // shared row strides (bf16)
    constexpr int BS = BT ? GBK + 8 : GBN + 8;
    __shared__ __align__(16) bf16 As[AT ? GBK : GBM][AS];
    __shared__ __align__(16) bf16 Bs[BT ? GBN : GBK][BS];
    const bf16 *gA = reinterpret_cast<const bf16 *>(g.A);
    const bf16 *gB = reinterpret_cast<const bf16 *>(g.B);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int gid = lane >> 2, tid4 = lane & 3;
    const int m0 = blockIdx.y * GBM, n0 = blockIdx.x * GBN;
    const int kslice = g.K / (int)gridDim.z;
    const int kbeg = blockIdx.z * kslice, kend = kbeg + kslice;

    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;

    for (int k0 = kbeg; k0 < kend; k0 += GBK) {
        // A tile: 64 x 32 values = 256 vectors of 8
        for (int v = tid; v < GBM * GBK / 8; v += 128) {
            uint4 x = make_uint4(0, 0, 0, 0);
            if (!AT) {
                const int r = v / (GBK / 8), c8 = (v % (GBK / 8)) * 8;
                if (m0 + r < g.M) x = *reinterpret_cast<const uint4 *>(gA + (int64_t)(m0 + r) * g.lda + k0 + c8);
                *reinterpret_cast<uint4 *>(&As[r][c8]) = x;
            } else {
                const int r = v / (GBM / 8), c8 = (v % (GBM / 8)) * 8;
                if (m0 + c8 < g.M) x = *reinterpret_cast<const uint4 *>(gA + (int64_t)(k0 + r) * g.lda + m0 + c8);
                *reinterpret_cast<uint4 *>(&As[r][c8]) = x;
            }
        }
        for (int v = tid; v < GBN * GBK / 8; v += 128) {
            uint4 x = make_uint4(0, 0, 0, 0);
            if (!BT) {
                const int r = v / (GBN / 8), c8 = (v % (GBN / 8)) * 8;
                if (n0 + c8 < g.N) x = *reinterpret_cast<const uint4 *>(gB + (int64_t)(k0 + r) * g.ldb + n0 + c8);
                *reinterpret_cast<uint4 *>(&Bs[r][c8]) = x;
            } else {
                const int r = v / (GBK / 8), c8 = (v % (GBK / 8)) * 8;
                if (n0 + r < g.N) x = *reinterpret_cast<const uint4 *>(gB + (int64_t)(n0 + r) * g.ldb + k0 + c8);
                *reinterpret_cast<uint4 *>(&Bs[r][c8]) = x;
            }
        }
        __syncthreads();
        const int mi = lane >> 3, rr = lane & 7;
#pragma unroll
        for (int kk = 0; kk < GBK; kk += 16) {
            uint32_t af[2][4], bfr[4][2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int mb = wm + 16 * i;
                if (!AT) ldsm4(af[i], &As[mb + (lane & 15)][kk + (lane >> 4) * 8]);
                else ldsm4t(af[i], &As[kk + (mi >> 1) * 8 + rr][mb + (mi & 1) * 8]);
            }
#pragma unroll
            for (int j = 0; j < 4; j += 2) {
                const int nb = wn + 8 * j;
                uint32_t t[4];
                if (!BT) {
                    ldsm4t(t, &Bs[kk + (mi & 1) * 8 + rr][nb + (mi >> 1) * 8]);
                } else {
                    ldsm4(t, &Bs[nb + (mi >> 1) * 8 + rr][kk + (mi & 1) * 8]);
                }
                bfr[j][0] = t[0]; bfr[j][1] = t[1]; bfr[j + 1][0] = t[2]; bfr[j + 1][1] = t[3];
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) mma16816(acc[i][j], af[i], bfr[j][0], bfr[j][1]);
        }
        __syncthreads();
    }
    // fused epilogue
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int r = m0 + wm + 16 * i + gid + (e >= 2 ? 8 : 0);
                const int c = n0 + wn + 8 * j + 2 * tid4 + (e & 1);
                if (r >= g.M || c >= g.N) continue;
                const float v = acc[i][j][e];
                const int64_t o = (int64_t)r * g.ldo + c;
                if (EPI == EPI_BIAS_SELU) {
                    const float z = v + g.bias[c];
                    reinterpret_cast<bf16 *>(g.out_z)[o] = __float2bfloat16_rn(z);
                    reinterpret_cast<bf16 *>(g.out_bf)[o] = __float2bfloat16_rn(selu(z));
                } else if (EPI == EPI_BIAS) {
                    g.out_f[o] = v + g.bias[c];
                } else if (EPI == EPI_DSELU) {
                    const bf16 zb = reinterpret_cast<const bf16 *>(g.Zin)[o];
                    reinterpret_cast<bf16 *>(g.out_bf)[o] = __float2bfloat16_rn(v * dselu(__bfloat162float(zb)));
                } else {   // EPI_PART: split-K partial
                    g.out_f[(int64_t)blockIdx.z * g.M * g.N + (int64_t)r * g.N + c] = v;
                }
            }
}

template <bool AT, bool BT, int EPI>
static cudaError_t gemm(const GemmArgs &g, int splits, cudaStream_t st) {
    dim3 grid((g.N + GBN - 1) / GBN, (g.M + GBM - 1) / GBM, splits);
    k_gemm_bf16<AT, BT, EPI><<<grid, 128, 0, st>>>(g);
    return cudaGetLastError();
}

cudaError_t launch_gemm(const GemmArgs &g, bool at, bool bt, int epi, int splits,
                        cudaStream_t st) {
    if (g.M % GBM || g.K % (GBK * splits) || g.N % 32) return cudaErrorInvalidValue;
    if (!at && !bt && epi == EPI_BIAS_SELU) return gemm<false, false, EPI_BIAS_SELU>(g, splits, st);
    if (!at && !bt && epi == EPI_BIAS) return gemm<false, false, EPI_BIAS>(g, splits, st);
    if (!at && bt && epi == EPI_DSELU) return gemm<false, true, EPI_DSELU>(g, splits, st);
    if (at && !bt && epi == EPI_PART) return gemm<true, false, EPI_PART>(g, splits, st);
    return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------- reductions
// out[c] = sum_s part[s][c] in s order (split-K partials, or column sums).
__global__ void k_sum_parts(int64_t count, int splits, const float *__restrict__ part,
                            float *__restrict__ out) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < count;
         c += (int64_t)gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int p = 0; p < splits; ++p) s += part[(int64_t)p * count + c];
        out[c] = s;
    }
}

// Column sums of a [M,N] bf16 matrix in fixed order: CTA b sums rows
// [b*R, (b+1)*R) into part[b][N].
__global__ void k_colsum_part(int M, int N, int R, const bf16 *__restrict__ A,
                              float *__restrict__ part) {
    const int b = blockIdx.y;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) {
        float s = 0.f;
        const int r1 = min(M, (b + 1) * R);
        for (int r = b * R; r < r1; ++r) s += __bfloat162float(A[(int64_t)r * N + c]);
        part[(int64_t)b * N + c] = s;
    }
}

// Loss (y - t)^T G (y - t) per row, dY = (2/B) G (y - t) as BF16; per-CTA loss
// partials.  G is k x k (k <= 32), one warp per row, lane q owns component q.
__global__ void __launch_bounds__(256)
k_mlp_loss(int B, int k, const float *__restrict__ Y, const float *__restrict__ T,
           const float *__restrict__ G, bf16 *__restrict__ dY, int ldd,
           float *__restrict__ part) {
    __shared__ float Gs[32][33];
    __shared__ float ws[8];
    for (int e = threadIdx.x; e < k * k; e += blockDim.x) Gs[e / k][e % k] = G[e];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float lsum = 0.f;
    for (int r = blockIdx.x * 8 + warp; r < B; r += gridDim.x * 8) {
        const float d = lane < k ? Y[(int64_t)r * k + lane] - T[(int64_t)r * k + lane] : 0.f;
        float gd = 0.f;
        for (int p = 0; p < k; ++p) gd = fmaf(Gs[lane < k ? lane : 0][p], __shfl_sync(FULL, d, p), gd);
        if (lane < k) dY[(int64_t)r * ldd + lane] = __float2bfloat16_rn(2.f * gd / (float)B);
        float l = lane < k ? d * gd : 0.f;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) l += __shfl_xor_sync(FULL, l, off);
        lsum += l;
    }
    if (lane == 0) ws[warp] = lsum;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.f;
        for (int w = 0; w < 8; ++w) s += ws[w];
        part[blockIdx.x] = s;
    }
}

__global__ void k_loss_final(int parts, int B, const float *__restrict__ part,
                             double *__restrict__ out) {
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int p = 0; p < parts; ++p) s += part[p];
        *out = s / (double)B;
    }
}

// G = V^T V over the first k components of V rows (stride KP): CTA b sums
// the rows j = b, b + GRAM_PARTS, ... into part[b][k][k]; the parts are then
// added in b order (fixed order, reproducible).
constexpr int GRAM_PARTS = 64;
__global__ void __launch_bounds__(1024) k_gram_v_part(int64_t n, int KP, int k,
                                                      const float *__restrict__ V,
                                                      float *__restrict__ part) {
    const int p = threadIdx.x / 32, q = threadIdx.x % 32;   // 1024 threads: 32 x 32
    if (p >= k || q >= k) return;
    float s = 0.f;
    for (int64_t j = blockIdx.x; j < n; j += GRAM_PARTS) s = fmaf(V[j * KP + p], V[j * KP + q], s);
    part[(int64_t)blockIdx.x * k * k + p * k + q] = s;
}

// Adam (Kingma & Ba 2015) on FP32 master parameters; BF16 copies refreshed.
// Step counter and step size live on the device, so one captured training
// step serves every step of a schedule: the host sets lr by a launch ahead of
// the step (stream-ordered), the step's first kernel advances t.
__global__ void k_adam_tick(AdamState *s) { s->t += 1; }
__global__ void k_adam_set_lr(AdamState *s, float lr) { s->lr = lr; }

__global__ void k_adam(int64_t count, float *__restrict__ th, const float *__restrict__ gr,
                       float *__restrict__ m1, float *__restrict__ m2, float b1, float b2,
                       float eps, const AdamState *__restrict__ as,
                       const int64_t *__restrict__ bf_map, bf16 *__restrict__ thb,
                       const int64_t *__restrict__ img_map, bf16 *__restrict__ img) {
    __shared__ float corr[3];   // bias corrections of step t (after the tick), once per CTA
    if (threadIdx.x == 0) {
        const double tt = (double)as->t;
        corr[0] = (float)(1.0 - pow((double)b1, tt));
        corr[1] = (float)(1.0 - pow((double)b2, tt));
        corr[2] = as->lr;
    }
    __syncthreads();
    const float c1 = corr[0], c2 = corr[1], lr = corr[2];
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
         e += (int64_t)gridDim.x * blockDim.x) {
        const float g = gr[e];
        const float a = b1 * m1[e] + (1.f - b1) * g;
        const float b = b2 * m2[e] + (1.f - b2) * g * g;
        m1[e] = a;
        m2[e] = b;
        const float t = th[e] - lr * (a / c1) / (sqrtf(b / c2) + eps);
        th[e] = t;
        const bf16 tb = __float2bfloat16_rn(t);
        const int64_t q = bf_map ? bf_map[e] : -1, qi = img_map ? img_map[e] : -1;
        if (q >= 0) thb[q] = tb;
        if (qi >= 0) img[qi] = tb;
    }
}

__global__ void k_to_bf16_map(int64_t count, const float *__restrict__ th,
                              const int64_t *__restrict__ bf_map, bf16 *__restrict__ thb,
                              const int64_t *__restrict__ img_map, bf16 *__restrict__ img) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
         e += (int64_t)gridDim.x * blockDim.x) {
        const bf16 tb = __float2bfloat16_rn(th[e]);
        const int64_t q = bf_map ? bf_map[e] : -1, qi = img_map ? img_map[e] : -1;
        if (q >= 0) thb[q] = tb;
        if (qi >= 0) img[qi] = tb;
    }
}

// Fallback list: rows whose observed-entry RMSE exceeds thr (or is not finite).
__global__ void k_fallback_rows(int64_t m, const float *__restrict__ rmse, float thr,
                                int32_t *__restrict__ list, int64_t *__restrict__ count,
                                int32_t *__restrict__ status) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float r = rmse[i];
        const bool bad = !(r <= thr);
        if (status) status[i] = bad ? ST_FALLBACK : ST_OK;
        if (bad) list[atomicAdd(reinterpret_cast<unsigned long long *>(count), 1ull)] = (int32_t)i;
    }
}

// After the ALS solve of the listed rows (which wrote OK / NOT_SPD / EMPTY):
// a listed row solved without trouble reports FALLBACK_USED.
__global__ void k_fallback_mark(const int32_t *__restrict__ list, const int64_t *__restrict__ count,
                                int32_t *__restrict__ status) {
    const int64_t c = *count;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < c;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int32_t i = list[t];
        if (status[i] == ST_OK) status[i] = ST_FALLBACK;
    }
}

static unsigned gfor(int64_t w) {
    int64_t b = (w + 255) / 256;
    if (b > NUM_SMS_HINT * 32) b = NUM_SMS_HINT * 32;
    return (unsigned)(b < 1 ? 1 : b);
}

cudaError_t launch_mlp_features(int64_t m, int64_t nnz, const int64_t *ptr, const int32_t *idx,
                                const float *val, const float *cnorm, const float *gnorm,
                                int64_t n, void *X, cudaStream_t st) {
    if (m <= 0) return cudaSuccess;
    k_mlp_features<<<gfor(m * MLP_INP), 256, 0, st>>>(m, nnz, ptr, idx, val, cnorm, gnorm, n,
                                                      reinterpret_cast<bf16 *>(X));
    return cudaGetLastError();
}

cudaError_t launch_sum_parts(int64_t count, int splits, const float *part, float *out,
                             cudaStream_t st) {
    k_sum_parts<<<gfor(count), 256, 0, st>>>(count, splits, part, out);
    return cudaGetLastError();
}

cudaError_t launch_colsum(int M, int N, const void *A, float *part, float *out, cudaStream_t st) {
    const int R = 128, nb = (M + R - 1) / R;
    dim3 grid((N + 255) / 256, nb);
    k_colsum_part<<<grid, 256, 0, st>>>(M, N, R, reinterpret_cast<const bf16 *>(A), part);
    k_sum_parts<<<gfor(N), 256, 0, st>>>(N, nb, part, out);
    return cudaGetLastError();
}

cudaError_t launch_mlp_loss(int B, int k, const float *Y, const float *T, const float *G,
                            void *dY, int ldd, float *part, double *loss, cudaStream_t st) {
    const int blocks = (B + 7) / 8 < 512 ? (B + 7) / 8 : 512;
    k_mlp_loss<<<blocks, 256, 0, st>>>(B, k, Y, T, G, reinterpret_cast<bf16 *>(dY), ldd, part);
    if (loss) k_loss_final<<<1, 32, 0, st>>>(blocks, B, part, loss);
    return cudaGetLastError();
}

cudaError_t launch_gram_v(int64_t n, int KP, int k, const float *V, float *part, float *G,
                          cudaStream_t st) {
    k_gram_v_part<<<GRAM_PARTS, 1024, 0, st>>>(n, KP, k, V, part);
    k_sum_parts<<<gfor(k * k), 256, 0, st>>>(k * k, GRAM_PARTS, part, G);
    return cudaGetLastError();
}

cudaError_t launch_adam(int64_t count, float *th, const float *g, float *m1, float *m2, float b1,
                        float b2, float eps, void *state, const int64_t *bf_map, void *thb,
                        const int64_t *img_map, void *img, cudaStream_t st) {
    AdamState *as = reinterpret_cast<AdamState *>(state);
    k_adam_tick<<<1, 1, 0, st>>>(as);
    k_adam<<<gfor(count), 256, 0, st>>>(count, th, g, m1, m2, b1, b2, eps, as, bf_map,
                                        reinterpret_cast<bf16 *>(thb), img_map,
                                        reinterpret_cast<bf16 *>(img));
    return cudaGetLastError();
}

cudaError_t launch_adam_set_lr(void *state, float lr, cudaStream_t st) {
    k_adam_set_lr<<<1, 1, 0, st>>>(reinterpret_cast<AdamState *>(state), lr);
    return cudaGetLastError();
}

cudaError_t launch_to_bf16_map(int64_t count, const float *th, const int64_t *bf_map, void *thb,
                               const int64_t *img_map, void *img, cudaStream_t st) {
    k_to_bf16_map<<<gfor(count), 256, 0, st>>>(count, th, bf_map, reinterpret_cast<bf16 *>(thb),
                                                img_map, reinterpret_cast<bf16 *>(img));
    return cudaGetLastError();
}

cudaError_t launch_fallback_rows(int64_t m, const float *rmse, float thr, int32_t *list,
                                 int64_t *count, int32_t *status, cudaStream_t st) {
    if (m <= 0) return cudaSuccess;
    k_fallback_rows<<<gfor(m), 256, 0, st>>>(m, rmse, thr, list, count, status);
    return cudaGetLastError();
}

cudaError_t launch_fallback_mark(int64_t m, const int32_t *list, const int64_t *count,
                                 int32_t *status, cudaStream_t st) {
    if (m <= 0 || !status) return cudaSuccess;
    k_fallback_mark<<<gfor(m), 256, 0, st>>>(list, count, status);
    return cudaGetLastError();
}

}  // namespace ocf
