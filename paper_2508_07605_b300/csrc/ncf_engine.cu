// Engine behind the NCF C ABI (open_cf_ncf.h): the handle owns the FP32
// parameters, gradients and Adam moments of the model (one packed vector
// [net | Ea | Es] so that one update kernel covers all of them), the BF16
// copies of W1 and W2 the training kernel reads, the per-CTA gradient
// partials and the completion workspaces, all allocated at creation.  A
// training step (two kernels) is captured once into a CUDA graph and replayed
// for every step of every epoch: its kernels take their batch position from a
// device-side counter.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <string>
#include <vector>

#include "common.cuh"
#include "kernels.h"
#include "open_cf_ncf.h"

using namespace ocf;

namespace {

constexpr int64_t NET_PAD = (NCF_NET + 3) / 4 * 4;   // embeddings start 16-byte aligned
constexpr int STEPS_PER_GRAPH = 16;                   // training steps per graph launch
static_assert(NCF_NET == OPEN_CF_NCF_NET, "network size");

struct NBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

struct StepGraph {
    std::vector<int64_t> key;
    cudaGraphExec_t exec = nullptr;
};

}  // namespace

struct open_cf_ncf {
    int device = 0, num_sms = 0;
    int64_t m = 0, n = 0;
    int B = 0;
    std::vector<double> cpu, gpu;
    int64_t base_default = 0;
    bool params_set = false;
    NBuf theta, grad, m1, m2, bf, adam, ctl, loss1;
    NBuf part, lpart;
    NBuf A, S, w2img, T, cg, err;
    int wait_limit = OPEN_CF_WAIT_POLLS_DEFAULT;   // polls of a tensor-core pipeline wait
    cudaStream_t cap_stream = nullptr;
    std::vector<StepGraph> graphs;
    std::string msg;
};

struct open_cf_pred {
    int device = 0, nfeat = 0, B = 0, num_sms = 0;
    bool params_set = false;
    NBuf theta, grad, m1, m2, bf, adam, ctl, loss1, part, lpart;
    cudaStream_t cap_stream = nullptr;
    std::vector<StepGraph> graphs;
    std::string msg;
};

namespace {

struct Guard {
    int prev = -1;
    explicit Guard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~Guard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

template <typename H> int nfail(H *h, int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (h) h->msg = buf;
    return code;
}

template <typename H> int ncuda(H *h, cudaError_t e, const char *where) {
    cudaGetLastError();
    return nfail(h, e == cudaErrorMemoryAllocation ? OPEN_CF_OUT_OF_MEMORY : OPEN_CF_CUDA_ERROR,
                 "%s: %s", where, cudaGetErrorString(e));
}

#define NCK(h, expr)                                          \
    do {                                                      \
        cudaError_t e_ = (expr);                              \
        if (e_ != cudaSuccess) return ncuda((h), e_, #expr);  \
    } while (0)

cudaError_t alloc(NBuf &b, size_t bytes) {
    b.bytes = std::max<size_t>(bytes, 256);
    return cudaMalloc(&b.p, b.bytes);
}

void release(NBuf &b) {
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
}

cudaStream_t SS(void *s) { return reinterpret_cast<cudaStream_t>(s); }

float *F(NBuf &b) { return reinterpret_cast<float *>(b.p); }

int64_t n_emb(const open_cf_ncf_t *h) { return (h->m + h->n) * NCF_D; }

// Forward, loss and backward of one batch; with `update`, one Adam step.
cudaError_t enqueue_step(open_cf_ncf_t *h, int64_t nnz, int64_t spe, const int32_t *app,
                         const int32_t *set, const float *val, const int32_t *perms,
                         double *loss_hist, bool update, cudaStream_t st) {
    float *th = F(h->theta), *g = F(h->grad);
    NcfCtl *ctl = reinterpret_cast<NcfCtl *>(h->ctl.p);
    NcfTrainArgs t{};
    t.ctl = ctl;
    t.adam = update ? reinterpret_cast<AdamState *>(h->adam.p) : nullptr;
    t.nnz = nnz; t.spe = spe; t.m = h->m; t.n = h->n; t.B = h->B;
    t.perms = perms; t.app = app; t.set = set; t.val = val;
    t.Ea = th + NET_PAD; t.Es = th + NET_PAD + h->m * NCF_D;
    t.W1b = h->bf.p; t.W2b = reinterpret_cast<const char *>(h->bf.p) + 2 * NCF_OFF_B1;
    t.b1 = th + NCF_OFF_B1; t.b2 = th + NCF_OFF_B2; t.w3 = th + NCF_OFF_W3; t.b3 = th + NCF_OFF_B3;
    t.part = F(h->part); t.part_stride = NET_PAD; t.lpart = F(h->lpart);
    t.gE = g + NET_PAD; t.s_off = h->m * NCF_D;
    NcfAdamArgs u{};
    u.ctl = ctl;
    u.adam = reinterpret_cast<const AdamState *>(h->adam.p);
    u.update = update;
    u.parts = h->B / NCF_TT; u.part = F(h->part); u.part_stride = NET_PAD; u.lpart = F(h->lpart);
    u.th = th; u.grad = g; u.m1 = F(h->m1); u.m2 = F(h->m2);
    u.net_pad = NET_PAD; u.n_emb = n_emb(h);
    u.bf = h->bf.p;
    u.loss_hist = loss_hist; u.loss_last = (double *)h->loss1.p;
    return launch_ncf_train_step(t, u, st);
}

// Replays `steps` training steps: one graph of STEPS_PER_GRAPH consecutive
// steps as often as it fits, then single-step graphs (the steps read their
// position from the device counter, so every replay advances the run).  The
// graphs are cached by `key` and rebuilt when the arguments change.
template <typename H, typename F>
int run_steps(H *h, std::vector<int64_t> key, int64_t steps, cudaStream_t st, F &&enqueue) {
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    for (int r = 0; r < 2; ++r) {
        const int reps = r == 0 ? 1 : STEPS_PER_GRAPH;
        std::vector<int64_t> k = key;
        k.push_back(reps);
        for (auto &g : h->graphs)
            if (g.key == k) exec[r] = g.exec;
        if (exec[r] || (r == 1 && steps < STEPS_PER_GRAPH)) continue;
        NCK(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = cudaSuccess;
        for (int t = 0; t < reps && e == cudaSuccess; ++t) e = enqueue(h->cap_stream);
        cudaGraph_t graph = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(h->cap_stream, &graph);
        if (e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return ncuda(h, e, "training step capture");
        }
        if (e2 != cudaSuccess) return ncuda(h, e2, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&exec[r], graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return ncuda(h, e, "cudaGraphInstantiate");
        if (h->graphs.size() >= 8) {
            cudaGraphExecDestroy(h->graphs.front().exec);
            h->graphs.erase(h->graphs.begin());
        }
        h->graphs.push_back(StepGraph{k, exec[r]});
    }
    int64_t s = 0;
    for (; s + STEPS_PER_GRAPH <= steps; s += STEPS_PER_GRAPH) NCK(h, cudaGraphLaunch(exec[1], st));
    for (; s < steps; ++s) NCK(h, cudaGraphLaunch(exec[0], st));
    return OPEN_CF_OK;
}

}  // namespace

extern "C" {

int open_cf_ncf_create(int64_t m, int32_t n_cpu, const double *cpu_caps_w_host, int32_t n_gpu,
                       const double *gpu_caps_w_host, int32_t batch, int device,
                       open_cf_ncf_t **out) {
    if (!out) return OPEN_CF_INVALID_ARG;
    *out = nullptr;
    if (m < 1 || m > (int64_t)1 << 31 || n_cpu < 1 || n_gpu < 1 || !cpu_caps_w_host ||
        !gpu_caps_w_host || (int64_t)n_cpu * n_gpu > (int64_t)1 << 24)
        return OPEN_CF_INVALID_ARG;
    if (batch < 64 || batch > 65536 || batch % 64) return OPEN_CF_INVALID_ARG;
    for (int c = 0; c < n_cpu; ++c)
        if (!std::isfinite(cpu_caps_w_host[c])) return OPEN_CF_INVALID_ARG;
    for (int c = 0; c < n_gpu; ++c)
        if (!std::isfinite(gpu_caps_w_host[c])) return OPEN_CF_INVALID_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return OPEN_CF_INVALID_ARG;
    }
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return OPEN_CF_CUDA_ERROR;
    if (!(prop.major == 10 && prop.minor == 3)) return OPEN_CF_UNSUPPORTED;
    open_cf_ncf_t *h = new open_cf_ncf();
    h->device = device;
    h->m = m;
    h->n = (int64_t)n_cpu * n_gpu;
    h->B = batch;
    h->cpu.assign(cpu_caps_w_host, cpu_caps_w_host + n_cpu);
    h->gpu.assign(gpu_caps_w_host, gpu_caps_w_host + n_gpu);
    const int64_t ci = std::max_element(h->cpu.begin(), h->cpu.end()) - h->cpu.begin();
    const int64_t gi = std::max_element(h->gpu.begin(), h->gpu.end()) - h->gpu.begin();
    h->base_default = ci * n_gpu + gi;
    Guard gd(device);
    const int64_t P = NET_PAD + n_emb(h);
    std::vector<float> cg(h->n);
    for (int64_t j = 0; j < h->n; ++j)
        cg[j] = (float)h->cpu[j / n_gpu] + (float)h->gpu[j % n_gpu];
    cudaError_t e = cudaSuccess;
    auto A = [&](NBuf &b, size_t bytes) {
        if (e == cudaSuccess) e = alloc(b, bytes);
    };
    A(h->theta, sizeof(float) * P); A(h->grad, sizeof(float) * P);
    A(h->m1, sizeof(float) * P); A(h->m2, sizeof(float) * P);
    A(h->bf, 2 * 2 * NCF_OFF_B1);
    A(h->adam, 16); A(h->ctl, sizeof(NcfCtl)); A(h->loss1, sizeof(double));
    A(h->part, sizeof(float) * (batch / NCF_TT) * NET_PAD); A(h->lpart, sizeof(float) * (batch / NCF_TT));
    A(h->A, sizeof(float) * m * NCF_H1); A(h->S, sizeof(float) * h->n * NCF_H1);
    A(h->w2img, 2 * NCF_H1 * NCF_H2); A(h->cg, sizeof(float) * h->n); A(h->err, 16);
    if (e == cudaSuccess) e = cudaMemcpy(h->cg.p, cg.data(), sizeof(float) * h->n,
                                         cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(h->err.p, 0, 16);
    if (e == cudaSuccess) e = cudaMemset(h->ctl.p, 0, sizeof(NcfCtl));
    if (e == cudaSuccess) e = prepare_ncf_predict_tc();
    if (e == cudaSuccess) e = prepare_ncf_train();
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        cudaGetLastError();
        open_cf_ncf_destroy(h);
        return e == cudaErrorMemoryAllocation ? OPEN_CF_OUT_OF_MEMORY : OPEN_CF_CUDA_ERROR;
    }
    *out = h;
    return OPEN_CF_OK;
}

void open_cf_ncf_destroy(open_cf_ncf_t *h) {
    if (!h) return;
    {
        Guard gd(h->device);
        cudaDeviceSynchronize();
        for (auto &g : h->graphs) cudaGraphExecDestroy(g.exec);
        if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
        for (NBuf *b : {&h->theta, &h->grad, &h->m1, &h->m2, &h->bf, &h->adam, &h->ctl,
                        &h->loss1, &h->part, &h->lpart, &h->A, &h->S, &h->w2img, &h->T, &h->cg,
                        &h->err})
            release(*b);
    }
    delete h;
}

const char *open_cf_ncf_last_error(const open_cf_ncf_t *h) { return h ? h->msg.c_str() : ""; }

int open_cf_ncf_set_params(open_cf_ncf_t *h, const float *net, const float *Ea, const float *Es,
                           void *stream) {
    if (!h) return OPEN_CF_INVALID_ARG;
    h->msg.clear();
    if (!net || !Ea || !Es) return nfail(h, OPEN_CF_INVALID_ARG, "net, Ea and Es are required");
    Guard gd(h->device);
    cudaStream_t st = SS(stream);
    float *th = F(h->theta);
    const int64_t P = NET_PAD + n_emb(h);
    NCK(h, cudaMemsetAsync(th, 0, sizeof(float) * NET_PAD, st));
    NCK(h, cudaMemcpyAsync(th, net, sizeof(float) * NCF_NET, cudaMemcpyDeviceToDevice, st));
    NCK(h, cudaMemcpyAsync(th + NET_PAD, Ea, sizeof(float) * h->m * NCF_D,
                           cudaMemcpyDeviceToDevice, st));
    NCK(h, cudaMemcpyAsync(th + NET_PAD + h->m * NCF_D, Es, sizeof(float) * h->n * NCF_D,
                           cudaMemcpyDeviceToDevice, st));
    NCK(h, cudaMemsetAsync(h->m1.p, 0, sizeof(float) * P, st));
    NCK(h, cudaMemsetAsync(h->m2.p, 0, sizeof(float) * P, st));
    NCK(h, cudaMemsetAsync(h->adam.p, 0, 16, st));
    NCK(h, cudaMemsetAsync(h->ctl.p, 0, sizeof(NcfCtl), st));
    NCK(h, cudaMemsetAsync(h->grad.p, 0, sizeof(float) * P, st));   // embedding rows accumulate
    NCK(h, launch_ncf_refresh_bf(th, h->bf.p, st));
    h->params_set = true;
    return OPEN_CF_OK;
}

int open_cf_ncf_get_params(open_cf_ncf_t *h, float *net, float *Ea, float *Es, void *stream) {
    if (!h) return OPEN_CF_INVALID_ARG;
    h->msg.clear();
    if (!h->params_set) return nfail(h, OPEN_CF_NOT_FITTED, "set the parameters first");
    Guard gd(h->device);
    cudaStream_t st = SS(stream);
    const float *th = F(h->theta);
    if (net) NCK(h, cudaMemcpyAsync(net, th, sizeof(float) * NCF_NET, cudaMemcpyDeviceToDevice, st));
    if (Ea)
        NCK(h, cudaMemcpyAsync(Ea, th + NET_PAD, sizeof(float) * h->m * NCF_D,
                               cudaMemcpyDeviceToDevice, st));
    if (Es)
        NCK(h, cudaMemcpyAsync(Es, th + NET_PAD + h->m * NCF_D, sizeof(float) * h->n * NCF_D,
                               cudaMemcpyDeviceToDevice, st));
    return OPEN_CF_OK;
}

int open_cf_ncf_train(open_cf_ncf_t *h, int64_t nnz, const int32_t *app, const int32_t *setting,
                      const float *val, int32_t epochs, const int32_t *perms, float lr,
                      double *loss_out, void *stream) {
    if (!h) return OPEN_CF_INVALID_ARG;
    h->msg.clear();
    if (!h->params_set) return nfail(h, OPEN_CF_NOT_FITTED, "set the parameters first");
    if (nnz < 1 || nnz > INT32_MAX || epochs < 0 || !app || !setting || !val ||
        (epochs > 0 && !perms))
        return nfail(h, OPEN_CF_INVALID_ARG, "bad nnz, epochs or array");
    if (!(lr >= 0.0f) || !std::isfinite(lr)) return nfail(h, OPEN_CF_INVALID_ARG, "bad lr");
    if (epochs == 0) return OPEN_CF_OK;
    Guard gd(h->device);
    cudaStream_t st = SS(stream);
    const int64_t spe = (nnz + h->B - 1) / h->B, steps = spe * epochs;
    NCK(h, cudaMemsetAsync(h->ctl.p, 0, sizeof(int64_t), st));   // step = 0
    NCK(h, cudaMemsetAsync(F(h->grad) + NET_PAD, 0, sizeof(float) * n_emb(h), st));
    NCK(h, launch_adam_set_lr(h->adam.p, lr, st));
    return run_steps(h, {nnz, spe, (int64_t)app, (int64_t)setting, (int64_t)val, (int64_t)perms,
                         (int64_t)loss_out},
                     steps, st, [&](cudaStream_t cs) {
                         return enqueue_step(h, nnz, spe, app, setting, val, perms, loss_out, true,
                                             cs);
                     });
}

int open_cf_ncf_grad(open_cf_ncf_t *h, int64_t B, const int32_t *app, const int32_t *setting,
                     const float *val, double *loss_out, float *g_net, float *g_Ea, float *g_Es,
                     void *stream) {
    if (!h) return OPEN_CF_INVALID_ARG;
    h->msg.clear();
    if (!h->params_set) return nfail(h, OPEN_CF_NOT_FITTED, "set the parameters first");
    if (B < 1 || B > h->B || !app || !setting || !val)
        return nfail(h, OPEN_CF_INVALID_ARG, "B must be in [1, batch] and the arrays given");
    Guard gd(h->device);
    cudaStream_t st = SS(stream);
    NCK(h, cudaMemsetAsync(h->ctl.p, 0, sizeof(int64_t), st));
    NCK(h, cudaMemsetAsync(F(h->grad) + NET_PAD, 0, sizeof(float) * n_emb(h), st));
    NCK(h, enqueue_step(h, B, 1, app, setting, val, nullptr, nullptr, false, st));
    const float *g = F(h->grad);
    if (loss_out)
        NCK(h, cudaMemcpyAsync(loss_out, h->loss1.p, sizeof(double), cudaMemcpyDeviceToDevice, st));
    if (g_net)
        NCK(h, cudaMemcpyAsync(g_net, g, sizeof(float) * NCF_NET, cudaMemcpyDeviceToDevice, st));
    if (g_Ea)
        NCK(h, cudaMemcpyAsync(g_Ea, g + NET_PAD, sizeof(float) * h->m * NCF_D,
                               cudaMemcpyDeviceToDevice, st));
    if (g_Es)
        NCK(h, cudaMemcpyAsync(g_Es, g + NET_PAD + h->m * NCF_D, sizeof(float) * h->n * NCF_D,
                               cudaMemcpyDeviceToDevice, st));
    return OPEN_CF_OK;
}

int open_cf_ncf_predict(open_cf_ncf_t *h, float *T_out, float gamma, int32_t baseline_setting,
                        int32_t *best, float *saving, void *stream) {
    if (!h) return OPEN_CF_INVALID_ARG;
    h->msg.clear();
    if (!h->params_set) return nfail(h, OPEN_CF_NOT_FITTED, "set the parameters first");
    const bool sel = best || saving;
    if (!sel && !T_out) return OPEN_CF_OK;
    if (!std::isfinite(gamma)) return nfail(h, OPEN_CF_INVALID_ARG, "gamma is not finite");
    const int64_t base = baseline_setting < 0 ? h->base_default : baseline_setting;
    if (base >= h->n) return nfail(h, OPEN_CF_INVALID_ARG, "baseline setting out of range");
    Guard gd(h->device);
    cudaStream_t st = SS(stream);
    float *T = T_out;
    if (!T) {
        const size_t bytes = sizeof(float) * (size_t)h->m * (size_t)h->n;
        if (h->T.bytes < bytes) {
            NCK(h, cudaStreamSynchronize(st));
            release(h->T);
            NCK(h, alloc(h->T, bytes));
        }
        T = F(h->T);
    }
    float *th = F(h->theta);
    const float *Ea = th + NET_PAD, *Es = Ea + h->m * NCF_D;
    NCK(h, launch_ncf_w2_image(th + NCF_OFF_W2, h->w2img.p, st));
    NCK(h, launch_ncf_first_layer(h->m, Ea, th, th + NCF_OFF_B1, F(h->A), st));
    NCK(h, launch_ncf_first_layer(h->n, Es, th + NCF_D * NCF_H1, nullptr, F(h->S), st));
    NcfPredArgs a{h->m, h->n, F(h->A), F(h->S), h->w2img.p, th + NCF_OFF_B2, th + NCF_OFF_W3,
                  th + NCF_OFF_B3, T, (int *)h->err.p, h->wait_limit};
    NCK(h, launch_ncf_predict_tc(a, h->num_sms, st));
    if (sel) {
        const int ng = (int)h->gpu.size();
        const float Eb = (float)h->cpu[base / ng] + (float)h->gpu[base % ng];
        NCK(h, launch_select(h->m, h->n, T, h->n, F(h->cg), base, Eb, gamma, best, saving, st));
    }
    return OPEN_CF_OK;
}

int open_cf_ncf_skipped(open_cf_ncf_t *h, int64_t *count_host) {
    if (!h || !count_host) return OPEN_CF_INVALID_ARG;
    Guard gd(h->device);
    NcfCtl c{};
    NCK(h, cudaDeviceSynchronize());
    NCK(h, cudaMemcpy(&c, h->ctl.p, sizeof(NcfCtl), cudaMemcpyDeviceToHost));
    *count_host = (int64_t)c.skipped;
    return OPEN_CF_OK;
}

int open_cf_ncf_set_wait_limit(open_cf_ncf_t *h, int32_t polls) {
    if (!h) return OPEN_CF_INVALID_ARG;
    h->msg.clear();
    if (polls < -1) return nfail(h, OPEN_CF_INVALID_ARG, "polls must be >= -1");
    h->wait_limit = polls < 0 ? OPEN_CF_WAIT_POLLS_DEFAULT : polls;
    return OPEN_CF_OK;
}

int open_cf_ncf_check(open_cf_ncf_t *h) {
    if (!h) return OPEN_CF_INVALID_ARG;
    Guard gd(h->device);
    int flag = 0;
    NCK(h, cudaDeviceSynchronize());
    NCK(h, cudaMemcpy(&flag, h->err.p, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
        NCK(h, cudaMemset(h->err.p, 0, 16));
        return nfail(h, OPEN_CF_TIMEOUT, "a completion kernel gave up on a tensor-core wait");
    }
    return OPEN_CF_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- predictor
// The offline performance predictor (Sec. "Performance Prediction Model"):
// the same network on n_features dense inputs (zero padded to 64), trained
// and evaluated by the NCF training kernel in its dense-feature mode.
namespace {

int64_t pred_count(int nf) { return (int64_t)nf * NCF_H1 + (NCF_NET - NCF_OFF_B1); }

cudaError_t pred_step(open_cf_pred_t *h, int64_t N, int64_t spe, const float *X, const float *y,
                      const int32_t *perms, double *loss_hist, bool update, cudaStream_t st) {
    float *th = F(h->theta), *g = F(h->grad);
    NcfCtl *ctl = reinterpret_cast<NcfCtl *>(h->ctl.p);
    NcfTrainArgs t{};
    t.ctl = ctl;
    t.adam = update ? reinterpret_cast<AdamState *>(h->adam.p) : nullptr;
    t.nnz = N; t.spe = spe; t.m = 0; t.n = 0; t.B = h->B;
    t.perms = perms; t.val = y;
    t.feat = X; t.nfeat = h->nfeat;
    t.W1b = h->bf.p; t.W2b = reinterpret_cast<const char *>(h->bf.p) + 2 * NCF_OFF_B1;
    t.b1 = th + NCF_OFF_B1; t.b2 = th + NCF_OFF_B2; t.w3 = th + NCF_OFF_W3; t.b3 = th + NCF_OFF_B3;
    t.part = F(h->part); t.part_stride = NET_PAD; t.lpart = F(h->lpart);
    NcfAdamArgs u{};
    u.ctl = ctl;
    u.adam = reinterpret_cast<const AdamState *>(h->adam.p);
    u.update = update;
    u.parts = h->B / NCF_TT; u.part = F(h->part); u.part_stride = NET_PAD; u.lpart = F(h->lpart);
    u.th = th; u.grad = g; u.m1 = F(h->m1); u.m2 = F(h->m2);
    u.net_pad = NET_PAD; u.n_emb = 0;
    u.bf = h->bf.p;
    u.loss_hist = loss_hist; u.loss_last = (double *)h->loss1.p;
    return launch_ncf_train_step(t, u, st);
}

}  // namespace

extern "C" {

int open_cf_pred_create(int32_t n_features, int32_t batch, int device, open_cf_pred_t **out) {
    if (!out) return OPEN_CF_INVALID_ARG;
    *out = nullptr;
    if (n_features < 1 || n_features > 2 * NCF_D) return OPEN_CF_INVALID_ARG;
    if (batch < 64 || batch > 65536 || batch % 64) return OPEN_CF_INVALID_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return OPEN_CF_INVALID_ARG;
    }
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return OPEN_CF_CUDA_ERROR;
    if (!(prop.major == 10 && prop.minor == 3)) return OPEN_CF_UNSUPPORTED;
    open_cf_pred_t *h = new open_cf_pred();
    h->device = device;
    h->nfeat = n_features;
    h->B = batch;
    Guard gd(device);
    cudaError_t e = cudaSuccess;
    auto A = [&](NBuf &b, size_t bytes) {
        if (e == cudaSuccess) e = alloc(b, bytes);
    };
    A(h->theta, sizeof(float) * NET_PAD); A(h->grad, sizeof(float) * NET_PAD);
    A(h->m1, sizeof(float) * NET_PAD); A(h->m2, sizeof(float) * NET_PAD);
    A(h->bf, 2 * 2 * NCF_OFF_B1);
    A(h->adam, 16); A(h->ctl, sizeof(NcfCtl)); A(h->loss1, sizeof(double));
    A(h->part, sizeof(float) * (batch / NCF_TT) * NET_PAD); A(h->lpart, sizeof(float) * (batch / NCF_TT));
    if (e == cudaSuccess) e = cudaMemset(h->ctl.p, 0, sizeof(NcfCtl));
    if (e == cudaSuccess) e = prepare_ncf_train();
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        cudaGetLastError();
        open_cf_pred_destroy(h);
        return e == cudaErrorMemoryAllocation ? OPEN_CF_OUT_OF_MEMORY : OPEN_CF_CUDA_ERROR;
    }
    *out = h;
    return OPEN_CF_OK;
}

void open_cf_pred_destroy(open_cf_pred_t *h) {
    if (!h) return;
    {
        Guard gd(h->device);
        cudaDeviceSynchronize();
        for (auto &g : h->graphs) cudaGraphExecDestroy(g.exec);
        if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
        for (NBuf *b : {&h->theta, &h->grad, &h->m1, &h->m2, &h->bf, &h->adam, &h->ctl, &h->loss1,
                        &h->part, &h->lpart})
            release(*b);
    }
    delete h;
}

const char *open_cf_pred_last_error(const open_cf_pred_t *h) { return h ? h->msg.c_str() : ""; }

int open_cf_pred_set_params(open_cf_pred_t *h, const float *params, void *stream) {
    if (!h) return OPEN_CF_INVALID_ARG;
    h->msg.clear();
    if (!params) return nfail(h, OPEN_CF_INVALID_ARG, "params is NULL");
    Guard gd(h->device);
    cudaStream_t st = SS(stream);
    float *th = F(h->theta);
    const int64_t w1 = (int64_t)h->nfeat * NCF_H1;
    NCK(h, cudaMemsetAsync(th, 0, sizeof(float) * NET_PAD, st));
    NCK(h, cudaMemcpyAsync(th, params, sizeof(float) * w1, cudaMemcpyDeviceToDevice, st));
    NCK(h, cudaMemcpyAsync(th + NCF_OFF_B1, params + w1, sizeof(float) * (NCF_NET - NCF_OFF_B1),
                           cudaMemcpyDeviceToDevice, st));
    NCK(h, cudaMemsetAsync(h->m1.p, 0, sizeof(float) * NET_PAD, st));
    NCK(h, cudaMemsetAsync(h->m2.p, 0, sizeof(float) * NET_PAD, st));
    NCK(h, cudaMemsetAsync(h->adam.p, 0, 16, st));
    NCK(h, cudaMemsetAsync(h->ctl.p, 0, sizeof(NcfCtl), st));
    NCK(h, launch_ncf_refresh_bf(th, h->bf.p, st));
    h->params_set = true;
    return OPEN_CF_OK;
}

int open_cf_pred_get_params(open_cf_pred_t *h, float *params, void *stream) {
    if (!h) return OPEN_CF_INVALID_ARG;
    h->msg.clear();
    if (!h->params_set) return nfail(h, OPEN_CF_NOT_FITTED, "set the parameters first");
    if (!params) return nfail(h, OPEN_CF_INVALID_ARG, "params is NULL");
    Guard gd(h->device);
    cudaStream_t st = SS(stream);
    const float *th = F(h->theta);
    const int64_t w1 = (int64_t)h->nfeat * NCF_H1;
    NCK(h, cudaMemcpyAsync(params, th, sizeof(float) * w1, cudaMemcpyDeviceToDevice, st));
    NCK(h, cudaMemcpyAsync(params + w1, th + NCF_OFF_B1, sizeof(float) * (NCF_NET - NCF_OFF_B1),
                           cudaMemcpyDeviceToDevice, st));
    return OPEN_CF_OK;
}

int open_cf_pred_train(open_cf_pred_t *h, int64_t N, const float *X, const float *y,
                       int32_t epochs, const int32_t *perms, float lr, double *loss_out,
                       void *stream) {
    if (!h) return OPEN_CF_INVALID_ARG;
    h->msg.clear();
    if (!h->params_set) return nfail(h, OPEN_CF_NOT_FITTED, "set the parameters first");
    if (N < 1 || N > INT32_MAX || epochs < 0 || !X || !y || (epochs > 0 && !perms))
        return nfail(h, OPEN_CF_INVALID_ARG, "bad N, epochs or array");
    if (!(lr >= 0.0f) || !std::isfinite(lr)) return nfail(h, OPEN_CF_INVALID_ARG, "bad lr");
    if (epochs == 0) return OPEN_CF_OK;
    Guard gd(h->device);
    cudaStream_t st = SS(stream);
    const int64_t spe = (N + h->B - 1) / h->B, steps = spe * epochs;
    NCK(h, cudaMemsetAsync(h->ctl.p, 0, sizeof(int64_t), st));
    NCK(h, launch_adam_set_lr(h->adam.p, lr, st));
    return run_steps(h, {N, spe, (int64_t)X, (int64_t)y, (int64_t)perms, (int64_t)loss_out}, steps,
                     st, [&](cudaStream_t cs) {
                         return pred_step(h, N, spe, X, y, perms, loss_out, true, cs);
                     });
}

int open_cf_pred_grad(open_cf_pred_t *h, int64_t B, const float *X, const float *y,
                      double *loss_out, float *g_params, void *stream) {
    if (!h) return OPEN_CF_INVALID_ARG;
    h->msg.clear();
    if (!h->params_set) return nfail(h, OPEN_CF_NOT_FITTED, "set the parameters first");
    if (B < 1 || B > h->B || !X || !y)
        return nfail(h, OPEN_CF_INVALID_ARG, "B must be in [1, batch] and the arrays given");
    Guard gd(h->device);
    cudaStream_t st = SS(stream);
    NCK(h, cudaMemsetAsync(h->ctl.p, 0, sizeof(int64_t), st));
    NCK(h, pred_step(h, B, 1, X, y, nullptr, nullptr, false, st));
    const float *g = F(h->grad);
    const int64_t w1 = (int64_t)h->nfeat * NCF_H1;
    if (loss_out)
        NCK(h, cudaMemcpyAsync(loss_out, h->loss1.p, sizeof(double), cudaMemcpyDeviceToDevice, st));
    if (g_params) {
        NCK(h, cudaMemcpyAsync(g_params, g, sizeof(float) * w1, cudaMemcpyDeviceToDevice, st));
        NCK(h, cudaMemcpyAsync(g_params + w1, g + NCF_OFF_B1,
                               sizeof(float) * (NCF_NET - NCF_OFF_B1), cudaMemcpyDeviceToDevice,
                               st));
    }
    return OPEN_CF_OK;
}

int open_cf_pred_infer(open_cf_pred_t *h, int64_t N, const float *X, float *y_out, void *stream) {
    if (!h) return OPEN_CF_INVALID_ARG;
    h->msg.clear();
    if (!h->params_set) return nfail(h, OPEN_CF_NOT_FITTED, "set the parameters first");
    if (N < 0 || (N > 0 && (!X || !y_out)))
        return nfail(h, OPEN_CF_INVALID_ARG, "bad N or array");
    if (N == 0) return OPEN_CF_OK;
    Guard gd(h->device);
    float *th = F(h->theta);
    NcfTrainArgs t{};
    t.nnz = N;
    t.feat = X; t.nfeat = h->nfeat; t.y_out = y_out;
    t.W1b = h->bf.p; t.W2b = reinterpret_cast<const char *>(h->bf.p) + 2 * NCF_OFF_B1;
    t.b1 = th + NCF_OFF_B1; t.b2 = th + NCF_OFF_B2; t.w3 = th + NCF_OFF_W3; t.b3 = th + NCF_OFF_B3;
    NCK(h, launch_pred_forward(t, h->num_sms, SS(stream)));
    return OPEN_CF_OK;
}

}  // extern "C"
