// Learned warm start for the online fold-in: an MLP that maps an
// application's first 16 online-profiled (CPU cap, GPU cap, runtime) samples
// straight to its latent factor u (k = 32), trained on factors the plain ALS
// fold-in produces; ALS remains the fallback where the MLP's observed-entry
// residual is too large (engine: open_cf_mlp_infer).  SELU activations, as
// the paper's collaborative-filtering MLP uses (Sec. "Collaborative Filtering
// Model"); constants from Klambauer et al. 2017.
//
// Network: features X[B,48] (padded to 64 columns) -> W1 -> SELU -> W2 ->
// SELU -> W3 -> u[B,32].  The forward pass (mlp_tc.cu) and a training step's
// forward and backward passes (mlp_train_tc.cu) run on tcgen05; this file
// holds what surrounds them: the BF16 operand images of the weights, the
// reduction of the training kernel's per-CTA partial gradients fused with
// Adam, and the fallback bookkeeping.
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"
#include "mlp_tc.cuh"

namespace ocf {

namespace {

typedef __nv_bfloat16 bf16;

// Every BF16 image position of internal parameter e (weights only; -1 none).
__device__ __forceinline__ void image_slots(int64_t e, int64_t &p0, int64_t &p1) {
    p0 = p1 = -1;
    if (e < MLP_OFF_B1) {
        p0 = mlp::img_w1(e / MLP_H, e % MLP_H);
    } else if (e >= MLP_OFF_W2 && e < MLP_OFF_B2) {
        const int64_t x = e - MLP_OFF_W2;
        p0 = mlp::img_w2f(x / MLP_H, x % MLP_H);
        p1 = mlp::img_w2b(x / MLP_H, x % MLP_H);
    } else if (e >= MLP_OFF_W3 && e < MLP_OFF_B3) {
        const int64_t x = e - MLP_OFF_W3;
        p0 = mlp::img_w3f(x / MLP_K_OUT, x % MLP_K_OUT);
        p1 = mlp::img_w3b(x / MLP_K_OUT, x % MLP_K_OUT);
    }
}

__device__ __forceinline__ void write_images(int64_t e, float w, bf16 *img) {
    int64_t p0, p1;
    image_slots(e, p0, p1);
    const bf16 b = __float2bfloat16_rn(w);
    if (p0 >= 0) img[p0] = b;
    if (p1 >= 0) img[p1] = b;
}

__global__ void k_mlp_images(const float *__restrict__ th, bf16 *__restrict__ img) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < MLP_P_INT;
         e += (int64_t)gridDim.x * blockDim.x)
        write_images(e, th[e], img);
}

// Slot offset and lane-quarter count of internal parameter e's partial sums.
__device__ __forceinline__ void part_slot(int64_t e, int64_t &off, int &nq, int64_t &qstride) {
    nq = 1;
    qstride = 0;
    if (e < MLP_OFF_B1) off = MLP_PART_W1 + e;
    else if (e < MLP_OFF_W2) { off = MLP_PART_B1 + (e - MLP_OFF_B1); nq = 4; qstride = MLP_H; }
    else if (e < MLP_OFF_B2) off = MLP_PART_W2 + (e - MLP_OFF_W2);
    else if (e < MLP_OFF_W3) { off = MLP_PART_B2 + (e - MLP_OFF_B2); nq = 4; qstride = MLP_H; }
    else if (e < MLP_OFF_B3) off = MLP_PART_W3 + (e - MLP_OFF_W3);
    else { off = MLP_PART_B3 + (e - MLP_OFF_B3); nq = 4; qstride = MLP_K_OUT; }
}

constexpr int RED_PARAMS = 64;   // parameters per CTA of the reduction; 4 slot groups each

// After k_mlp_train_tc: gradient = sum of the CTAs' partial sums; then either
// Adam (Kingma & Ba 2015) on the FP32 masters with the BF16 images
// refreshed, or the gradient written out in the external layout.  The step
// counter was advanced by the training kernel; the step size was set ahead
// of the step.  A step whose training kernel gave up (err[1]) changes
// nothing (the step counter is moved back) and reports NaN (loss and, in
// gradient mode, the gradient).
//
// Fixed summation order: warp w of a CTA takes slot group g = w / 2 and
// parameters 32 (w % 2) + lane; it adds the slots c = g, g + 4, g + 8, ...
// in increasing c (a bias slot contributes its four lane-quarter partials
// in order), with up to eight loads in flight; the four group sums are then
// added in g order.
__global__ void __launch_bounds__(256) k_mlp_reduce_adam(MlpReduceArgs a) {
    __shared__ float corr[3];
    __shared__ float gs[4][RED_PARAMS];
    mlp::pdl_wait();   // the training kernel's partial sums
    const bool failed = a.err && a.err[1] != 0;
    const float nan = __int_as_float(0x7fc00000);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0 && a.adam) {   // bias corrections 1 - beta^t in FP32 (FP64 is slow here)
        const float tt = (float)a.adam->t;
        corr[0] = 1.f - exp2f(tt * -0.15200309344504997f);    // log2(0.9)
        corr[1] = 1.f - exp2f(tt * -0.0014434168696687186f);  // log2(0.999)
        corr[2] = a.adam->lr;
        // a step that did not happen leaves the step counter as it was (the
        // other blocks' copies of t are not used when the step failed)
        if (failed && blockIdx.x == 0) a.adam->t -= 1;
    }
    if (blockIdx.x == 0 && warp == 0 && a.loss) {   // loss: warp 0, fixed order
        double s = 0.0;
        for (int64_t x = lane; x < (int64_t)a.ctas * 32; x += 32)
            s += __ldcg(a.part + (x >> 5) * MLP_PART_STRIDE + MLP_PART_LOSS + (x & 31));
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(FULL, s, off);
        if (lane == 0) *a.loss = failed ? (double)nan : s / (double)a.B;
    }
    const int g = warp >> 1, pl = 32 * (warp & 1) + lane;
    const int64_t e = (int64_t)blockIdx.x * RED_PARAMS + pl;
    float sum = 0.f;
    if (e < MLP_P_INT) {
        int64_t off, qstride;
        int nq;
        part_slot(e, off, nq, qstride);
        const float *p = a.part + off;
        for (int c0 = g; c0 < a.ctas; c0 += 32) {
            float x[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int c = c0 + 4 * u;
                x[u] = 0.f;
                if (c < a.ctas) {
                    const float *pc = p + (int64_t)c * MLP_PART_STRIDE;
                    x[u] = __ldcg(pc);
                    for (int qq = 1; qq < nq; ++qq) x[u] += __ldcg(pc + qq * qstride);
                }
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) sum += x[u];
        }
    }
    gs[g][pl] = sum;
    __syncthreads();
    if (g != 0 || e >= MLP_P_INT) return;
    const float gr = ((gs[0][pl] + gs[1][pl]) + gs[2][pl]) + gs[3][pl];
    if (!a.adam) {   // external layout: W1 has 48 input rows
        const int64_t pad = (int64_t)(MLP_INP - MLP_IN) * MLP_H;
        if (e < (int64_t)MLP_IN * MLP_H) a.grads_out[e] = failed ? nan : gr;
        else if (e >= MLP_OFF_B1) a.grads_out[e - pad] = failed ? nan : gr;
        return;
    }
    if (failed) return;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float m1 = b1 * a.m1[e] + (1.f - b1) * gr;
    const float m2 = b2 * a.m2[e] + (1.f - b2) * gr * gr;
    a.m1[e] = m1;
    a.m2[e] = m2;
    const float w = a.th[e] - corr[2] * (m1 / corr[0]) / (sqrtf(m2 / corr[1]) + eps);
    a.th[e] = w;
    write_images(e, w, reinterpret_cast<bf16 *>(a.img));
}

__global__ void k_adam_set_lr(AdamState *s, float lr) { s->lr = lr; }

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

unsigned gfor(int64_t w) {
    int64_t b = (w + 255) / 256;
    if (b > NUM_SMS_HINT * 32) b = NUM_SMS_HINT * 32;
    return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace

cudaError_t launch_mlp_images(const float *th, void *img, cudaStream_t st) {
    k_mlp_images<<<gfor(MLP_P_INT), 256, 0, st>>>(th, reinterpret_cast<bf16 *>(img));
    return cudaGetLastError();
}

cudaError_t launch_mlp_reduce_adam(const MlpReduceArgs &a, cudaStream_t st) {
    // launched as a programmatic dependent of the training kernel
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)((MLP_P_INT + RED_PARAMS - 1) / RED_PARAMS));
    cfg.blockDim = dim3(256);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_mlp_reduce_adam, a);
}

cudaError_t launch_adam_set_lr(void *state, float lr, cudaStream_t st) {
    k_adam_set_lr<<<1, 1, 0, st>>>(reinterpret_cast<AdamState *>(state), lr);
    return cudaGetLastError();
}

cudaError_t launch_fallback_mark(int64_t m, const int32_t *list, const int64_t *count,
                                 int32_t *status, cudaStream_t st) {
    if (m <= 0 || !status) return cudaSuccess;
    k_fallback_mark<<<gfor(m), 256, 0, st>>>(list, count, status);
    return cudaGetLastError();
}

}  // namespace ocf
