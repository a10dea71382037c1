// Engine behind the open_cf C ABI: the handle owns V, the cap grid, the CSC
// copy and every workspace, validates arguments on the host, and enqueues the
// kernels on the caller's stream.  A fit (CSC build + all ALS sweeps + unpack)
// is captured once into a CUDA graph per argument set and replayed, so a
// 15-sweep fit costs one graph launch instead of ~35 kernel launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "common.cuh"
#include "kernels.h"
#include "open_cf.h"

using namespace ocf;

namespace {

struct Buf {
    void *p = nullptr;
    size_t bytes = 0;
};

struct GraphEntry {
    std::vector<int64_t> key;
    cudaGraphExec_t exec = nullptr;
};

}  // namespace

struct open_cf {
    open_cf_config cfg{};
    std::vector<double> cpu_caps, gpu_caps;
    int device = 0;
    int k = 0, KP = 8;
    bool f64 = false;
    size_t esz = 4;           // element size of "real"
    int64_t n = -1;           // settings (rows of V)
    bool V_set = false;
    Buf V, Vb16, cg;          // V: n x KP real; Vb16: BF16 copy; cg: n floats
    int64_t base_default = -1;
    // offline block kept for joint refits (CSR of the dense block)
    Buf off_ptr, off_idx, off_val;
    int64_t m_off = 0, nnz_off = 0;
    // workspaces
    Buf U_w, csc_ptr, csc_idx, csc_val, cnt, tot, part, flag, j_ptr, j_idx, j_val, Ub16;
    // batched fits: planned metadata (device), workspaces, tuned warps per class
    Buf b_meta, b_Uw, b_Vw, b_cptr, b_cidx, b_cval, b_counter;
    std::vector<int64_t> b_key;       // host description of the planned batch
    int32_t b_W[2] = {8, 2};          // warps per problem: large class, small class
    int32_t b_cut = 50;               // % of a padded rank's cost in its large class
    int32_t b_ctas = 2;               // CTAs per SM of the persistent launch
    int32_t b_nclass = 0;             // classes of the planned batch
    int32_t b_class_end[BATCH_MAX_CLASSES] = {};
    int32_t b_class_W[BATCH_MAX_CLASSES] = {};
    int64_t b_Um = 0, b_Vn = 0;       // padded factor sizes (floats)
    // learned warm start: FP32 master parameters, Adam moments, BF16 weights, scratch
    Buf mlp_th, mlp_m1, mlp_m2, mlp_t, mlp_cn, mlp_scr;   // masters, moments, Adam state, caps, step scratch
    Buf mlp_img, mlp_err;   // tcgen05 weight images, timeout flags
    // V changes (set, fit, streaming refit) advance v_epoch; the MLP loss matrix
    // G = V^T V in the step scratch is current while mlp_g_epoch == v_epoch
    uint64_t v_epoch = 1, mlp_g_epoch = 0;
    Buf vimg, pt_err;                 // split BF16 operand images of V, timeout flag (predict)
    int wait_limit = OPEN_CF_WAIT_POLLS_DEFAULT;   // polls of a tensor-core pipeline wait
    Buf work_ctr;                     // the rank-32 fold-in's pair counter (allocated at creation)
    uint64_t vimg_epoch = 0;          // the images are of V while vimg_epoch == v_epoch
    void *vimg_at = nullptr;          // ... and they are still at this address
    Buf ccount;                       // observations per column (weighted-lambda objective)
    Buf sg, sb, sn;                   // streaming refit: per-setting Gram, RHS, count sums
    bool stream_on = false;
    int num_sms = 0;
    bool mlp_ready = false;
    uint64_t generation = 0;  // bumps whenever a workspace moves
    cudaStream_t cap_stream = nullptr;
    std::vector<GraphEntry> graphs;
    // host-buffer completion: device copies of the inputs and outputs, a copy
    // stream and per-chunk events (created on first use)
    Buf hs_ptr, hs_rptr, hs_col, hs_col16, hs_val, hs_U, hs_best, hs_sav, hs_st, hs_res;
    cudaStream_t hs_copy = nullptr;
    std::vector<cudaEvent_t> hs_ev;
    std::string err;
};

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

// An NVTX range over each compute entry point (header-only NVTX: without an
// attached tool the push and pop do nothing), so a timeline shows which call
// enqueued which kernels.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

int fail(open_cf_t *h, int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (h) h->err = buf;
    return code;
}

int cuda_fail(open_cf_t *h, cudaError_t e, const char *where) {
    cudaGetLastError();  // clear the sticky-free error state of the runtime
    return fail(h, e == cudaErrorMemoryAllocation ? OPEN_CF_OUT_OF_MEMORY : OPEN_CF_CUDA_ERROR,
                "%s: %s", where, cudaGetErrorString(e));
}

#define CK(h, expr)                                             \
    do {                                                        \
        cudaError_t e_ = (expr);                                \
        if (e_ != cudaSuccess) return cuda_fail((h), e_, #expr); \
    } while (0)

cudaError_t ensure(open_cf_t *h, Buf &b, size_t bytes) {
    if (bytes <= b.bytes && b.p) return cudaSuccess;
    size_t want = std::max<size_t>(bytes + bytes / 4, 256);
    if (b.p) {
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return e;
        cudaFree(b.p);
        b.p = nullptr;
        b.bytes = 0;
    }
    cudaError_t e = cudaMalloc(&b.p, want);
    if (e != cudaSuccess) return e;
    b.bytes = want;
    h->generation++;
    return cudaSuccess;
}

void free_buf(Buf &b) {
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
}

cudaStream_t S(void *s) { return reinterpret_cast<cudaStream_t>(s); }

// Run `enqueue` on `stream` through a cached CUDA graph keyed by `key`.
template <typename F>
int run_graph(open_cf_t *h, std::vector<int64_t> key, cudaStream_t stream, F &&enqueue) {
    key.push_back((int64_t)h->generation);
    for (auto &g : h->graphs)
        if (g.key == key) {
            CK(h, cudaGraphLaunch(g.exec, stream));
            return OPEN_CF_OK;
        }
    if (!h->cap_stream) CK(h, cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    CK(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = enqueue(h->cap_stream);
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(h->cap_stream, &graph);
    if (e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return cuda_fail(h, e, "enqueue during capture");
    }
    if (e2 != cudaSuccess) return cuda_fail(h, e2, "cudaStreamEndCapture");
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphInstantiate");
    if (h->graphs.size() >= 16) {
        cudaGraphExecDestroy(h->graphs.front().exec);
        h->graphs.erase(h->graphs.begin());
    }
    h->graphs.push_back(GraphEntry{std::move(key), exec});
    CK(h, cudaGraphLaunch(exec, stream));
    return OPEN_CF_OK;
}

// One ALS half-step with the handle's precision.  In BF16-Gram mode a.Fb is
// the BF16 copy of a.F (and a.outb, if set, receives the BF16 copy of the output).
template <typename TV>
cudaError_t half_step(open_cf_t *h, const SolveArgs<TV> &a, cudaStream_t st) {
    if constexpr (sizeof(TV) == 8) {
        return launch_row_solve<double, double>(a, h->KP, st);
    } else {
        const bool bf = h->cfg.precision == OPEN_CF_BF16_GRAM;
        if (bf || h->KP >= 16) {
            SolveArgs<TV> b = a;
            b.work = (unsigned int *)h->work_ctr.p;   // used by the rank-32 FP32 solver
            return launch_row_solve_tc(b, h->KP, h->cfg.cholesky_fp64 != 0, bf, st);
        }
        if (h->cfg.cholesky_fp64) return launch_row_solve<float, double>(a, h->KP, st);
        return launch_row_solve<float, float>(a, h->KP, st);
    }
}

int check_csr_args(open_cf_t *h, int64_t m, int64_t nnz, const void *ptr, const void *idx,
                   const void *val) {
    if (m < 0 || nnz < 0) return fail(h, OPEN_CF_INVALID_ARG, "negative m or nnz");
    if (m > 0 && !ptr) return fail(h, OPEN_CF_INVALID_ARG, "row_ptr is NULL");
    if (nnz > 0 && (!idx || !val)) return fail(h, OPEN_CF_INVALID_ARG, "col or val is NULL");
    if (nnz > INT64_C(0x7fffffff) * 64) return fail(h, OPEN_CF_UNSUPPORTED, "nnz too large");
    return OPEN_CF_OK;
}

// ALS sweeps on a CSR matrix (rows m, columns n == h->n) starting from h->V.
template <typename TV>
int fit_sweeps(open_cf_t *h, int64_t m, int64_t nnz, const int64_t *ptr, const int32_t *idx,
               const TV *val, TV *U_out, int64_t u_row0, int64_t u_rows, int32_t *row_status,
               int32_t *col_status, double *J_hist, cudaStream_t stream) {
    h->v_epoch++;   // the sweeps rewrite V
    const int64_t n = h->n;
    const int KP = h->KP;
    const CscPlan plan = csc_plan(m, n, nnz, 0);
    const int64_t nb = plan.nb;
    CK(h, ensure(h, h->U_w, sizeof(TV) * std::max<int64_t>(m, 1) * KP));
    CK(h, ensure(h, h->csc_ptr, sizeof(int64_t) * (n + 1)));
    CK(h, ensure(h, h->csc_idx, sizeof(int32_t) * std::max<int64_t>(nnz, 1)));
    CK(h, ensure(h, h->csc_val, sizeof(TV) * std::max<int64_t>(nnz, 1)));
    CK(h, ensure(h, h->cnt, sizeof(int32_t) * n * nb));
    CK(h, ensure(h, h->tot, sizeof(int64_t) * n));
    CK(h, ensure(h, h->part, sizeof(double) * 3 * objective_parts(std::max<int64_t>(m, n))));
    const bool bf = h->cfg.precision == OPEN_CF_BF16_GRAM;
    if (bf) CK(h, ensure(h, h->Ub16, 4 * std::max<int64_t>(m, 1) * KP));   // split BF16 rows
    TV *Uw = (TV *)h->U_w.p;
    TV *V = (TV *)h->V.p;
    int64_t *cptr = (int64_t *)h->csc_ptr.p;
    int32_t *cidx = (int32_t *)h->csc_idx.p;
    TV *cval = (TV *)h->csc_val.p;
    const int sweeps = h->cfg.sweeps;
    const int k = h->k;
    const double lam = h->cfg.lambda;
    const bool wr = h->cfg.weighted_lambda != 0;
    if (wr && J_hist) CK(h, ensure(h, h->ccount, sizeof(int32_t) * std::max<int64_t>(n, 1)));
    const int32_t *ccount = (wr && J_hist) ? (const int32_t *)h->ccount.p : nullptr;
    auto enqueue = [&](cudaStream_t st) -> cudaError_t {
        cudaError_t e = cudaMemsetAsync(Uw, 0, sizeof(TV) * m * KP, st);
        if (e != cudaSuccess) return e;
        e = launch_csr_to_csc<TV>(m, n, nnz, ptr, idx, val, cptr, cidx, cval, (int32_t *)h->cnt.p,
                                  (int64_t *)h->tot.p, plan, st);
        if (e != cudaSuccess) return e;
        if (ccount &&
            (e = launch_col_counts_from_ptr(n, cptr, (int32_t *)ccount, st)) != cudaSuccess)
            return e;
        for (int s = 0; s < sweeps; ++s) {
            SolveArgs<TV> ua{m, nnz, ptr, idx, val, V, n, Uw, KP, KP, row_status, lam};
            ua.wr = wr;
            if (bf) {
                ua.Fb = h->Vb16.p;
                ua.outb = h->Ub16.p;
            }
            if ((e = half_step<TV>(h, ua, st)) != cudaSuccess) return e;
            if (J_hist &&
                (e = launch_objective<TV>(m, nnz, ptr, idx, val, Uw, KP, k, V, n, KP, lam,
                                          (double *)h->part.p, J_hist + 2 * s, nullptr, ccount,
                                          st)) != cudaSuccess)
                return e;
            SolveArgs<TV> va{n, nnz, cptr, cidx, cval, Uw, m, V, KP, KP, col_status, lam};
            va.wr = wr;
            if (bf) {
                va.Fb = h->Ub16.p;
                va.outb = h->Vb16.p;
            }
            if ((e = half_step<TV>(h, va, st)) != cudaSuccess) return e;
            if (J_hist &&
                (e = launch_objective<TV>(m, nnz, ptr, idx, val, Uw, KP, k, V, n, KP, lam,
                                          (double *)h->part.p, J_hist + 2 * s + 1, nullptr,
                                          ccount, st)) != cudaSuccess)
                return e;
        }
        if (U_out && u_rows > 0)
            return launch_unpack_rows<TV>(Uw + u_row0 * KP, u_rows, KP, k, U_out, st);
        return cudaSuccess;
    };
    std::vector<int64_t> key = {1,
                                m,
                                nnz,
                                (int64_t)ptr,
                                (int64_t)idx,
                                (int64_t)val,
                                (int64_t)U_out,
                                u_row0,
                                u_rows,
                                (int64_t)row_status,
                                (int64_t)col_status,
                                (int64_t)J_hist};
    return run_graph(h, key, stream, enqueue);
}

template <typename TV> TV *as(const void *p) { return (TV *)p; }

}  // namespace

namespace {

// Device layout of the planned batch metadata (one buffer of int64 words).
struct BatchPlan {
    int64_t P, nnz, sum_m, sum_n;
    // word offsets inside b_meta
    int64_t o_m, o_n, o_k, o_rowoff, o_coloff, o_fu, o_fv, o_tu, o_tv, o_order;
};

BatchPlan batch_layout(int64_t P) {
    BatchPlan L{};
    L.P = P;
    int64_t w = 0;
    L.o_m = w; w += P;
    L.o_n = w; w += P;
    L.o_k = w; w += (P + 1) / 2;          // int32
    L.o_rowoff = w; w += P + 1;
    L.o_coloff = w; w += P + 1;
    L.o_fu = w; w += P + 1;
    L.o_fv = w; w += P + 1;
    L.o_tu = w; w += P + 1;
    L.o_tv = w; w += P + 1;
    L.o_order = w; w += (P + 1) / 2;      // int32
    L.sum_m = w;                          // total words (reused below)
    return L;
}

// Validate, plan (offsets, cost order, classes) and upload the batch when its
// description changed since the last call.
int batch_plan(open_cf_t *h, int64_t P, const int64_t *m, const int64_t *n, const int32_t *k,
               const int64_t *nnz_p, int64_t nnz, BatchPlan &L) {
    if (P <= 0 || !m || !n || !k || !nnz_p) return fail(h, OPEN_CF_INVALID_ARG, "bad batch description");
    int64_t tot = 0;
    for (int64_t p = 0; p < P; ++p) {
        if (m[p] < 0 || n[p] < 1 || nnz_p[p] < 0 || nnz_p[p] > m[p] * n[p])
            return fail(h, OPEN_CF_INVALID_ARG, "problem %lld: bad m, n or nnz", (long long)p);
        if (n[p] > BATCH_MAX_N)
            return fail(h, OPEN_CF_UNSUPPORTED, "problem %lld: n > %lld", (long long)p,
                        (long long)BATCH_MAX_N);
        if (k[p] < 1 || k[p] > OPEN_CF_MAX_K)
            return fail(h, OPEN_CF_UNSUPPORTED, "problem %lld: k out of range", (long long)p);
        tot += nnz_p[p];
    }
    if (tot != nnz) return fail(h, OPEN_CF_INVALID_ARG, "sum of per-problem nnz != nnz");
    L = batch_layout(P);
    const int64_t words = L.sum_m;
    std::vector<int64_t> key;
    key.reserve(4 * P + 4);
    key.push_back(P);
    key.push_back(nnz);
    key.push_back(h->b_W[0]);
    key.push_back(h->b_W[1]);
    key.push_back(h->b_cut);
    for (int64_t p = 0; p < P; ++p) {
        key.push_back(m[p]);
        key.push_back(n[p]);
        key.push_back(k[p]);
        key.push_back(nnz_p[p]);
    }
    std::vector<int64_t> meta(words, 0);
    int32_t *k32 = reinterpret_cast<int32_t *>(meta.data() + L.o_k);
    int32_t *ord = reinterpret_cast<int32_t *>(meta.data() + L.o_order);
    int64_t sm = 0, sn = 0, fu = 0, fv = 0, tu = 0, tv = 0;
    std::vector<double> cost(P);
    for (int64_t p = 0; p < P; ++p) {
        const int KP = padded_k(k[p]);
        meta[L.o_m + p] = m[p];
        meta[L.o_n + p] = n[p];
        k32[p] = k[p];
        meta[L.o_rowoff + p] = sm;
        meta[L.o_coloff + p] = sn;
        meta[L.o_fu + p] = fu;
        meta[L.o_fv + p] = fv;
        meta[L.o_tu + p] = tu;
        meta[L.o_tv + p] = tv;
        sm += m[p];
        sn += n[p];
        fu += m[p] * KP;
        fv += n[p] * KP;
        tu += m[p] * k[p];
        tv += n[p] * k[p];
        // cost of one sweep: masked Grams + factorisations
        cost[p] = (double)nnz_p[p] * 2.0 * KP * KP + (double)(m[p] + n[p]) * KP * KP * KP / 3.0;
    }
    meta[L.o_rowoff + P] = sm;
    meta[L.o_coloff + P] = sn;
    meta[L.o_fu + P] = fu;
    meta[L.o_fv + P] = fv;
    meta[L.o_tu + P] = tu;
    meta[L.o_tv + P] = tv;
    // Order: padded rank first (32, 16, 8), then cost, largest first (LPT).
    // Keeping one padded rank together keeps the warps of an SM in one unrolled
    // solver at a time (mixing the three thrashed the instruction cache).  Per
    // padded rank, class "large" holds the costliest problems that take about
    // a share of that rank's work (b_cut %, tuned), class "small" the rest.
    std::vector<int32_t> order(P);
    for (int64_t p = 0; p < P; ++p) order[p] = (int32_t)p;
    std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) {
        const int kx = padded_k(k[x]), ky = padded_k(k[y]);
        if (kx != ky) return kx > ky;
        return cost[x] > cost[y];
    });
    for (int64_t p = 0; p < P; ++p) ord[p] = order[p];
    h->b_nclass = 0;
    for (int64_t g0 = 0; g0 < P;) {
        const int kp = padded_k(k[order[g0]]);
        int64_t g1 = g0;
        double total = 0.0;
        while (g1 < P && padded_k(k[order[g1]]) == kp) total += cost[order[g1++]];
        double acc = 0.0;
        int64_t split = g0;
        while (split < g1 && acc < 0.01 * h->b_cut * total) acc += cost[order[split++]];
        if (split > g0) {
            h->b_class_end[h->b_nclass] = (int32_t)split;
            h->b_class_W[h->b_nclass++] = h->b_W[0];
        }
        if (g1 > split) {
            h->b_class_end[h->b_nclass] = (int32_t)g1;
            h->b_class_W[h->b_nclass++] = h->b_W[1];
        }
        g0 = g1;
    }
    h->b_Um = fu;
    h->b_Vn = fv;
    L.nnz = nnz;
    L.sum_n = sn;
    const int64_t sum_m = sm;
    CK(h, ensure(h, h->b_Uw, sizeof(float) * std::max<int64_t>(fu, 1)));
    CK(h, ensure(h, h->b_Vw, sizeof(float) * std::max<int64_t>(fv, 1)));
    CK(h, ensure(h, h->b_cptr, sizeof(int64_t) * (sn + P)));
    CK(h, ensure(h, h->b_cidx, sizeof(int32_t) * std::max<int64_t>(nnz, 1)));
    CK(h, ensure(h, h->b_cval, sizeof(float) * std::max<int64_t>(nnz, 1)));
    CK(h, ensure(h, h->b_counter, sizeof(int32_t) * BATCH_MAX_CLASSES));
    CK(h, ensure(h, h->b_meta, sizeof(int64_t) * words));
    if (key != h->b_key) {
        CK(h, cudaMemcpy(h->b_meta.p, meta.data(), sizeof(int64_t) * words,
                         cudaMemcpyHostToDevice));
        h->b_key.swap(key);
    }
    L.sum_m = sum_m;
    return OPEN_CF_OK;
}

BatchArgs batch_args(open_cf_t *h, const BatchPlan &L, const int64_t *row_ptr, const int32_t *col,
                     const float *val, int sweeps) {
    const int64_t *meta = (const int64_t *)h->b_meta.p;
    BatchArgs b{};
    b.P = L.P;
    b.order = reinterpret_cast<const int32_t *>(meta + L.o_order);
    b.m = meta + L.o_m;
    b.n = meta + L.o_n;
    b.k = reinterpret_cast<const int32_t *>(meta + L.o_k);
    b.row_off = meta + L.o_rowoff;
    b.col_off = meta + L.o_coloff;
    b.fu_off = meta + L.o_fu;
    b.fv_off = meta + L.o_fv;
    b.row_ptr = row_ptr;
    b.col = col;
    b.val = val;
    b.nnz = L.nnz;
    b.Uw = (float *)h->b_Uw.p;
    b.Vw = (float *)h->b_Vw.p;
    b.cptr = (int64_t *)h->b_cptr.p;
    b.cidx = (int32_t *)h->b_cidx.p;
    b.cval = (float *)h->b_cval.p;
    b.counter = (int32_t *)h->b_counter.p;
    b.sweeps = sweeps;
    b.lambda = h->cfg.lambda;
    b.wr = h->cfg.weighted_lambda != 0;
    b.n_classes = h->b_nclass;
    for (int c = 0; c < h->b_nclass; ++c) {
        b.class_end[c] = h->b_class_end[c];
        b.class_W[c] = h->b_class_W[c];
    }
    return b;
}

// Persistent grid: as many CTAs as fit on every SM at once (shared memory
// bound; at most 2 per SM with 128 registers x 256 threads).
int batched_grid(open_cf_t *h) {
    cudaDeviceProp prop;
    cudaGetDeviceProperties(&prop, h->device);
    const size_t smem = batched_smem_bytes();
    int per_sm = (int)std::max<size_t>(1, (size_t)prop.sharedMemPerMultiprocessor / (smem + 1024));
    if (per_sm > 2) per_sm = 2;
    if (per_sm > h->b_ctas) per_sm = h->b_ctas;
    return prop.multiProcessorCount * per_sm;
}

// Enqueue one batched fit: pack V, the persistent kernel, unpack U and V.
cudaError_t batch_enqueue(open_cf_t *h, const BatchPlan &L, const BatchArgs &b, float *V_inout,
                          float *U_out, int grid, cudaStream_t st) {
    const int64_t *meta = (const int64_t *)h->b_meta.p;
    const int32_t *k32 = reinterpret_cast<const int32_t *>(meta + L.o_k);
    cudaError_t e = cudaMemsetAsync(h->b_counter.p, 0, sizeof(int32_t) * BATCH_MAX_CLASSES, st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(h->b_Uw.p, 0, sizeof(float) * std::max<int64_t>(h->b_Um, 1), st);
    if (e != cudaSuccess) return e;
    e = launch_batched_pack(L.P, meta + L.o_n, k32, meta + L.o_tv, meta + L.o_fv, V_inout,
                            (float *)h->b_Vw.p, true, st);
    if (e != cudaSuccess) return e;
    e = launch_batched(b, grid, st);
    if (e != cudaSuccess) return e;
    if (U_out) {
        e = launch_batched_pack(L.P, meta + L.o_m, k32, meta + L.o_tu, meta + L.o_fu,
                                (const float *)h->b_Uw.p, U_out, false, st);
        if (e != cudaSuccess) return e;
    }
    return launch_batched_pack(L.P, meta + L.o_n, k32, meta + L.o_tv, meta + L.o_fv,
                               (const float *)h->b_Vw.p, V_inout, false, st);
}

}  // namespace

namespace {

// Parameter layout.  External (the caller's, and the oracle's): W1[48][256],
// b1[256], W2[256][256], b2[256], W3[256][32], b3[32] = 86,560 floats.
// Internal (MLP_OFF_*): W1 padded to [64][256] (rows 48..63 stay zero), rest identical.
constexpr int64_t MLP_K = 32;
constexpr int64_t P_EXT = MLP_IN * MLP_H + MLP_H + MLP_H * MLP_H + MLP_H + MLP_H * MLP_K + MLP_K;
static_assert(P_EXT == OPEN_CF_MLP_PARAMS, "parameter count of the C ABI");
static_assert(MLP_P_INT == P_EXT + (MLP_INP - MLP_IN) * MLP_H, "internal parameter count");

int mlp_check(open_cf_t *h) {
    if (h->k != MLP_K) return fail(h, OPEN_CF_UNSUPPORTED, "the learned warm start has k = 32");
    if (h->f64) return fail(h, OPEN_CF_UNSUPPORTED, "the learned warm start runs in FP32 modes");
    if (!h->V_set) return fail(h, OPEN_CF_NOT_FITTED, "set or fit V first");
    if (h->cpu_caps.empty()) return fail(h, OPEN_CF_INVALID_ARG, "features need the cap grid");
    if ((int64_t)h->cpu_caps.size() * (int64_t)h->gpu_caps.size() != h->n)
        return fail(h, OPEN_CF_INVALID_ARG, "cap grid size differs from the settings of V");
    if (!h->mlp_ready) return fail(h, OPEN_CF_NOT_FITTED, "set the MLP parameters first");
    return OPEN_CF_OK;
}

}  // namespace

extern "C" {

int open_cf_create(const open_cf_config *cfg, open_cf_t **out) {
    if (!cfg || !out) return OPEN_CF_INVALID_ARG;
    *out = nullptr;
    if (cfg->k < 1 || cfg->k > OPEN_CF_MAX_K) return OPEN_CF_UNSUPPORTED;
    if (!(cfg->lambda > 0.0) || !std::isfinite(cfg->lambda)) return OPEN_CF_INVALID_ARG;
    if (cfg->sweeps < 0) return OPEN_CF_INVALID_ARG;
    if (cfg->precision != OPEN_CF_FP64 && cfg->precision != OPEN_CF_FP32 &&
        cfg->precision != OPEN_CF_BF16_GRAM)
        return OPEN_CF_INVALID_ARG;
    if (cfg->n_cpu_caps < 0 || cfg->n_gpu_caps < 0 ||
        ((cfg->n_cpu_caps > 0) != (cfg->n_gpu_caps > 0)))
        return OPEN_CF_INVALID_ARG;
    if (cfg->n_cpu_caps > 0 && (!cfg->cpu_caps_w_host || !cfg->gpu_caps_w_host))
        return OPEN_CF_INVALID_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || cfg->device < 0 || cfg->device >= ndev) {
        cudaGetLastError();
        return OPEN_CF_UNSUPPORTED;
    }
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, cfg->device) != cudaSuccess) return OPEN_CF_CUDA_ERROR;
    if (!(prop.major == 10 && prop.minor == 3)) return OPEN_CF_UNSUPPORTED;

    open_cf_t *h = new open_cf();
    h->cfg = *cfg;
    h->device = cfg->device;
    h->k = cfg->k;
    h->KP = padded_k(cfg->k);
    if (cfg->precision == OPEN_CF_BF16_GRAM && h->KP < 16) h->KP = 16;   // tensor-core tiles
    h->f64 = cfg->precision == OPEN_CF_FP64;
    h->esz = h->f64 ? 8 : 4;
    if (cfg->n_cpu_caps > 0) {
        h->cpu_caps.assign(cfg->cpu_caps_w_host, cfg->cpu_caps_w_host + cfg->n_cpu_caps);
        h->gpu_caps.assign(cfg->gpu_caps_w_host, cfg->gpu_caps_w_host + cfg->n_gpu_caps);
        for (double c : h->cpu_caps)
            if (!std::isfinite(c)) { delete h; return OPEN_CF_INVALID_ARG; }
        for (double g : h->gpu_caps)
            if (!std::isfinite(g)) { delete h; return OPEN_CF_INVALID_ARG; }
        h->cfg.cpu_caps_w_host = nullptr;
        h->cfg.gpu_caps_w_host = nullptr;
        const int64_t ci = std::max_element(h->cpu_caps.begin(), h->cpu_caps.end()) -
                           h->cpu_caps.begin();
        const int64_t gi = std::max_element(h->gpu_caps.begin(), h->gpu_caps.end()) -
                           h->gpu_caps.begin();
        h->base_default = ci * cfg->n_gpu_caps + gi;
    }
    DeviceGuard g(h->device);
    if (prepare_csr_to_csc(CSC_MAX_N) != cudaSuccess || prepare_row_solve() != cudaSuccess ||
        prepare_row_solve_tc() != cudaSuccess || prepare_solve32_tc() != cudaSuccess ||
        prepare_batched() != cudaSuccess ||
        prepare_mlp_forward_tc() != cudaSuccess || prepare_mlp_train_tc() != cudaSuccess ||
        prepare_predict_tc() != cudaSuccess ||
        cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device) !=
            cudaSuccess ||
        ensure(h, h->work_ctr, 16) != cudaSuccess) {
        free_buf(h->work_ctr);
        cudaGetLastError();
        delete h;
        return OPEN_CF_CUDA_ERROR;
    }
    *out = h;
    return OPEN_CF_OK;
}

void open_cf_destroy(open_cf_t *h) {
    if (!h) return;
    {
        DeviceGuard g(h->device);
        cudaDeviceSynchronize();
        for (auto &ge : h->graphs) cudaGraphExecDestroy(ge.exec);
        if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
        if (h->hs_copy) cudaStreamDestroy(h->hs_copy);
        for (cudaEvent_t e : h->hs_ev) cudaEventDestroy(e);
        for (Buf *b : {&h->V, &h->Vb16, &h->cg, &h->off_ptr, &h->off_idx, &h->off_val, &h->U_w,
                       &h->csc_ptr, &h->csc_idx, &h->csc_val, &h->cnt, &h->tot, &h->part,
                       &h->flag, &h->j_ptr, &h->j_idx, &h->j_val, &h->Ub16, &h->b_meta, &h->b_Uw,
                       &h->b_Vw, &h->b_cptr, &h->b_cidx, &h->b_cval, &h->b_counter, &h->mlp_th,
                       &h->mlp_m1, &h->mlp_m2, &h->mlp_t, &h->mlp_cn, &h->mlp_scr, &h->mlp_img,
                       &h->mlp_err, &h->vimg, &h->pt_err, &h->ccount, &h->sg, &h->sb,
                       &h->sn, &h->hs_ptr, &h->hs_rptr, &h->hs_col, &h->hs_col16, &h->hs_val, &h->hs_U, &h->hs_best,
                       &h->hs_sav, &h->hs_st, &h->hs_res, &h->work_ctr})
            free_buf(*b);
    }
    delete h;
}

const char *open_cf_last_error(const open_cf_t *h) { return h ? h->err.c_str() : ""; }

int open_cf_set_wait_limit(open_cf_t *h, int32_t polls) {
    if (!h) return OPEN_CF_INVALID_ARG;
    h->err.clear();
    if (polls < -1) return fail(h, OPEN_CF_INVALID_ARG, "polls must be >= -1");
    h->wait_limit = polls < 0 ? OPEN_CF_WAIT_POLLS_DEFAULT : polls;
    return OPEN_CF_OK;
}

int open_cf_check(open_cf_t *h) {
    if (!h) return OPEN_CF_INVALID_ARG;
    h->err.clear();
    DeviceGuard g(h->device);
    CK(h, cudaDeviceSynchronize());
    int flags[8] = {};
    if (h->pt_err.p) CK(h, cudaMemcpy(flags, h->pt_err.p, 16, cudaMemcpyDeviceToHost));
    if (h->mlp_err.p) CK(h, cudaMemcpy(flags + 4, h->mlp_err.p, 16, cudaMemcpyDeviceToHost));
    if (!(flags[0] | flags[4] | flags[5])) return OPEN_CF_OK;
    if (h->pt_err.p) CK(h, cudaMemset(h->pt_err.p, 0, 16));
    if (h->mlp_err.p) CK(h, cudaMemset(h->mlp_err.p, 0, 16));
    std::string what;
    if (flags[0]) what += " reconstruction";
    if (flags[4]) what += " learned-inference";
    if (flags[5]) what += " learned-training";
    return fail(h, OPEN_CF_TIMEOUT, "a tensor-core pipeline wait gave up in:%s", what.c_str());
}

int open_cf_set_V(open_cf_t *h, const void *V, int64_t n, void *stream) {
    if (!h) return OPEN_CF_INVALID_ARG;
    h->err.clear();
    if (!V || n <= 0) return fail(h, OPEN_CF_INVALID_ARG, "V is NULL or n <= 0");
    if (n > CSC_MAX_N)
        return fail(h, OPEN_CF_UNSUPPORTED, "n = %lld settings exceeds %lld", (long long)n,
                    (long long)CSC_MAX_N);
    if (!h->cpu_caps.empty() && n != (int64_t)h->cpu_caps.size() * (int64_t)h->gpu_caps.size())
        return fail(h, OPEN_CF_INVALID_ARG, "n = %lld != n_cpu_caps * n_gpu_caps", (long long)n);
    DeviceGuard g(h->device);
    CK(h, ensure(h, h->V, h->esz * n * h->KP));
    cudaStream_t st = S(stream);
    if (h->f64)
        CK(h, launch_pack_rows<double>(as<double>(V), n, h->k, h->k, (double *)h->V.p, h->KP, st));
    else
        CK(h, launch_pack_rows<float>(as<float>(V), n, h->k, h->k, (float *)h->V.p, h->KP, st));
    if (h->cfg.precision == OPEN_CF_BF16_GRAM) {
        CK(h, ensure(h, h->Vb16, 4 * n * h->KP));   // split BF16 rows [hi | lo]
        CK(h, launch_to_bf16_split((const float *)h->V.p, n, h->KP, h->Vb16.p, st));
    }
    if (!h->cpu_caps.empty() && h->n != n) {
        std::vector<float> cg(n);
        const int ng = (int)h->gpu_caps.size();
        for (int64_t j = 0; j < n; ++j)
            cg[j] = (float)h->cpu_caps[j / ng] + (float)h->gpu_caps[j % ng];
        CK(h, ensure(h, h->cg, sizeof(float) * n));
        CK(h, cudaMemcpyAsync(h->cg.p, cg.data(), sizeof(float) * n, cudaMemcpyHostToDevice, st));
        CK(h, cudaStreamSynchronize(st));  // host vector goes out of scope
    }
    h->n = n;
    h->stream_on = false;   // a new V starts a new stream
    h->V_set = true;
    h->v_epoch++;
    return OPEN_CF_OK;
}

int open_cf_get_V(open_cf_t *h, void *V_out, void *stream) {
    if (!h) return OPEN_CF_INVALID_ARG;
    h->err.clear();
    if (!h->V_set) return fail(h, OPEN_CF_NOT_FITTED, "V was never set");
    if (!V_out) return fail(h, OPEN_CF_INVALID_ARG, "V_out is NULL");
    DeviceGuard g(h->device);
    if (h->f64)
        CK(h, launch_unpack_rows<double>((double *)h->V.p, h->n, h->KP, h->k, (double *)V_out,
                                         S(stream)));
    else
        CK(h, launch_unpack_rows<float>((float *)h->V.p, h->n, h->KP, h->k, (float *)V_out,
                                        S(stream)));
    return OPEN_CF_OK;
}

int open_cf_fit_csr(open_cf_t *h, int64_t m, int64_t n, int64_t nnz, const int64_t *row_ptr,
                    const int32_t *col, const void *val, void *U_out, int32_t *row_status,
                    int32_t *col_status, double *J_hist, void *stream) {
    NvtxRange nvtx_("open_cf_fit_csr");
    if (!h) return OPEN_CF_INVALID_ARG;
    h->err.clear();
    int rc = check_csr_args(h, m, nnz, row_ptr, col, val);
    if (rc) return rc;
    if (!h->V_set) return fail(h, OPEN_CF_NOT_FITTED, "set the initial V before a fit");
    if (n != h->n) return fail(h, OPEN_CF_INVALID_ARG, "n = %lld but V has %lld rows",
                               (long long)n, (long long)h->n);
    DeviceGuard g(h->device);
    if (h->f64)
        return fit_sweeps<double>(h, m, nnz, row_ptr, col, as<double>(val), (double *)U_out, 0,
                                  m, row_status, col_status, J_hist, S(stream));
    return fit_sweeps<float>(h, m, nnz, row_ptr, col, as<float>(val), (float *)U_out, 0, m,
                             row_status, col_status, J_hist, S(stream));
}

int open_cf_fit_offline(open_cf_t *h, const void *P, int64_t m_off, int64_t n, int64_t ld,
                        void *U_out, double *J_hist, void *stream) {
    NvtxRange nvtx_("open_cf_fit_offline");
    if (!h) return OPEN_CF_INVALID_ARG;
    h->err.clear();
    if (!P || m_off <= 0 || n <= 0 || ld < n)
        return fail(h, OPEN_CF_INVALID_ARG, "bad dense block (P, m_off, n, ld)");
    if (!h->V_set) return fail(h, OPEN_CF_NOT_FITTED, "set the initial V before a fit");
    if (n != h->n) return fail(h, OPEN_CF_INVALID_ARG, "n = %lld but V has %lld rows",
                               (long long)n, (long long)h->n);
    if (m_off * n > INT64_C(0x7fffffff) * 8)
        return fail(h, OPEN_CF_UNSUPPORTED, "dense block too large");
    DeviceGuard g(h->device);
    cudaStream_t st = S(stream);
    const int64_t nnz = m_off * n;
    CK(h, ensure(h, h->off_ptr, sizeof(int64_t) * (m_off + 1)));
    CK(h, ensure(h, h->off_idx, sizeof(int32_t) * nnz));
    CK(h, ensure(h, h->off_val, h->esz * nnz));
    h->m_off = 0;
    if (h->f64)
        CK(h, launch_dense_to_csr<double>(as<double>(P), m_off, n, ld, (int64_t *)h->off_ptr.p,
                                          (int32_t *)h->off_idx.p, (double *)h->off_val.p, st));
    else
        CK(h, launch_dense_to_csr<float>(as<float>(P), m_off, n, ld, (int64_t *)h->off_ptr.p,
                                         (int32_t *)h->off_idx.p, (float *)h->off_val.p, st));
    int rc;
    if (h->f64)
        rc = fit_sweeps<double>(h, m_off, nnz, (int64_t *)h->off_ptr.p, (int32_t *)h->off_idx.p,
                                (double *)h->off_val.p, (double *)U_out, 0, m_off, nullptr,
                                nullptr, J_hist, st);
    else
        rc = fit_sweeps<float>(h, m_off, nnz, (int64_t *)h->off_ptr.p, (int32_t *)h->off_idx.p,
                               (float *)h->off_val.p, (float *)U_out, 0, m_off, nullptr, nullptr,
                               J_hist, st);
    if (rc == OPEN_CF_OK) {
        h->m_off = m_off;
        h->nnz_off = nnz;
    }
    return rc;
}

namespace {
__global__ void k_offset_copy(const int64_t *__restrict__ src, int64_t count, int64_t add,
                              int64_t *__restrict__ dst) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
         e += (int64_t)gridDim.x * blockDim.x)
        dst[e] = src[e] + add;
}
}  // namespace

int open_cf_complete_rows(open_cf_t *h, int64_t m_new, int64_t nnz, const int64_t *row_ptr,
                          const int32_t *col, const void *val, void *U_out, int32_t *status,
                          int32_t joint, void *stream) {
    NvtxRange nvtx_("open_cf_complete_rows");
    if (!h) return OPEN_CF_INVALID_ARG;
    h->err.clear();
    int rc = check_csr_args(h, m_new, nnz, row_ptr, col, val);
    if (rc) return rc;
    if (!h->V_set) return fail(h, OPEN_CF_NOT_FITTED, "no V: fit or set V first");
    if (m_new > 0 && !U_out) return fail(h, OPEN_CF_INVALID_ARG, "U_out is NULL");
    DeviceGuard g(h->device);
    cudaStream_t st = S(stream);
    if (!joint) {
        if (h->f64) {
            SolveArgs<double> a{m_new, nnz, row_ptr, col, as<double>(val), (double *)h->V.p,
                                h->n, (double *)U_out, h->k, h->k, status, h->cfg.lambda};
            a.wr = h->cfg.weighted_lambda != 0;
            CK(h, half_step<double>(h, a, st));
        } else {
            SolveArgs<float> a{m_new, nnz, row_ptr, col, as<float>(val), (float *)h->V.p,
                               h->n, (float *)U_out, h->k, h->k, status, h->cfg.lambda};
            a.wr = h->cfg.weighted_lambda != 0;
            if (h->cfg.precision == OPEN_CF_BF16_GRAM) a.Fb = h->Vb16.p;
            CK(h, half_step<float>(h, a, st));
        }
        return OPEN_CF_OK;
    }
    // joint: [offline block ; new rows] as one CSR in handle workspaces
    const int64_t m = h->m_off + m_new, nz = h->nnz_off + nnz;
    CK(h, ensure(h, h->j_ptr, sizeof(int64_t) * (m + 1)));
    CK(h, ensure(h, h->j_idx, sizeof(int32_t) * std::max<int64_t>(nz, 1)));
    CK(h, ensure(h, h->j_val, h->esz * std::max<int64_t>(nz, 1)));
    int64_t *jp = (int64_t *)h->j_ptr.p;
    if (h->m_off > 0) {
        CK(h, cudaMemcpyAsync(jp, h->off_ptr.p, sizeof(int64_t) * h->m_off,
                              cudaMemcpyDeviceToDevice, st));
        CK(h, cudaMemcpyAsync(h->j_idx.p, h->off_idx.p, sizeof(int32_t) * h->nnz_off,
                              cudaMemcpyDeviceToDevice, st));
        CK(h, cudaMemcpyAsync(h->j_val.p, h->off_val.p, h->esz * h->nnz_off,
                              cudaMemcpyDeviceToDevice, st));
    }
    k_offset_copy<<<(unsigned)std::min<int64_t>((m_new + 256) / 256 + 1, 4096), 256, 0, st>>>(
        row_ptr, m_new + 1, h->nnz_off, jp + h->m_off);
    CK(h, cudaGetLastError());
    if (nnz > 0) {
        CK(h, cudaMemcpyAsync((int32_t *)h->j_idx.p + h->nnz_off, col, sizeof(int32_t) * nnz,
                              cudaMemcpyDeviceToDevice, st));
        CK(h, cudaMemcpyAsync((char *)h->j_val.p + h->esz * h->nnz_off, val, h->esz * nnz,
                              cudaMemcpyDeviceToDevice, st));
    }
    if (status && m_new > 0) CK(h, cudaMemsetAsync(status, 0, sizeof(int32_t) * m_new, st));
    if (h->f64)
        return fit_sweeps<double>(h, m, nz, jp, (int32_t *)h->j_idx.p, (double *)h->j_val.p,
                                  (double *)U_out, h->m_off, m_new, nullptr, nullptr, nullptr,
                                  st);
    return fit_sweeps<float>(h, m, nz, jp, (int32_t *)h->j_idx.p, (float *)h->j_val.p,
                             (float *)U_out, h->m_off, m_new, nullptr, nullptr, nullptr, st);
}

int open_cf_complete_rows_checked(open_cf_t *h, int64_t m_new, int64_t nnz,
                                  const int64_t *row_ptr, const int32_t *col, const float *val,
                                  float *U_out, int32_t *status, float *resid, int32_t refine,
                                  void *stream) {
    NvtxRange nvtx_("open_cf_complete_rows_checked");
    if (!h) return OPEN_CF_INVALID_ARG;
    h->err.clear();
    int rc = check_csr_args(h, m_new, nnz, row_ptr, col, val);
    if (rc) return rc;
    if (h->f64 || h->KP != 32 || h->cfg.cholesky_fp64)
        return fail(h, OPEN_CF_UNSUPPORTED,
                    "the residual check needs 16 < k <= 32, FP32 or BF16-Gram precision and the "
                    "FP32 factorisation");
    if (!h->V_set) return fail(h, OPEN_CF_NOT_FITTED, "no V: fit or set V first");
    if (m_new > 0 && !U_out) return fail(h, OPEN_CF_INVALID_ARG, "U_out is NULL");
    if (refine != 0 && refine != 1) return fail(h, OPEN_CF_INVALID_ARG, "refine must be 0 or 1");
    DeviceGuard g(h->device);
    SolveArgs<float> a{m_new, nnz, row_ptr, col, val, (float *)h->V.p, h->n, U_out, h->k, h->k,
                       status, h->cfg.lambda};
    a.wr = h->cfg.weighted_lambda != 0;
    const bool bf = h->cfg.precision == OPEN_CF_BF16_GRAM;
    if (bf) a.Fb = h->Vb16.p;
    a.resid = resid;
    a.refine = refine != 0;
    a.work = (unsigned int *)h->work_ctr.p;
    CK(h, launch_solve32_tc(a, bf, S(stream)));
    return OPEN_CF_OK;
}

int open_cf_normal_residual(open_cf_t *h, int64_t m, int64_t nnz, const int64_t *row_ptr,
                            const int32_t *col, const float *val, const float *U, float *resid,
                            void *stream) {
    NvtxRange nvtx_("open_cf_normal_residual");
    if (!h) return OPEN_CF_INVALID_ARG;
    h->err.clear();
    int rc = check_csr_args(h, m, nnz, row_ptr, col, val);
    if (rc) return rc;
    if (h->f64 || h->KP != 32)
        return fail(h, OPEN_CF_UNSUPPORTED,
                    "the residual needs 16 < k <= 32 and FP32 or BF16-Gram precision");
    if (!h->V_set) return fail(h, OPEN_CF_NOT_FITTED, "no V: fit or set V first");
    if (m > 0 && (!U || !resid)) return fail(h, OPEN_CF_INVALID_ARG, "U or resid is NULL");
    DeviceGuard g(h->device);
    SolveArgs<float> a{m, nnz, row_ptr, col, val, (float *)h->V.p, h->n, nullptr, h->k, h->k,
                       nullptr, h->cfg.lambda};
    a.wr = h->cfg.weighted_lambda != 0;
    const bool bf = h->cfg.precision == OPEN_CF_BF16_GRAM;
    if (bf) a.Fb = h->Vb16.p;
    a.resid = resid;
    a.u_given = U;
    a.work = (unsigned int *)h->work_ctr.p;
    CK(h, launch_solve32_tc(a, bf, S(stream)));
    return OPEN_CF_OK;
}

}  // extern "C"

namespace {

// Streaming refit: CSC of a batch of rows with (padded) factors Uw, then the
// V-half-step with the stored sums added and kept (every setting re-solved).
// stream_vhalf_ws sizes the workspaces (not capturable: it may allocate);
// stream_vhalf_enqueue only launches kernels.
template <typename TV>
int stream_vhalf_ws(open_cf_t *h, int64_t m, int64_t nnz) {
    const int64_t n = h->n;
    const CscPlan plan = csc_plan(m, n, nnz, 0);
    CK(h, ensure(h, h->csc_ptr, sizeof(int64_t) * (n + 1)));
    CK(h, ensure(h, h->csc_idx, sizeof(int32_t) * std::max<int64_t>(nnz, 1)));
    CK(h, ensure(h, h->csc_val, sizeof(TV) * std::max<int64_t>(nnz, 1)));
    CK(h, ensure(h, h->cnt, sizeof(int32_t) * n * plan.nb));
    CK(h, ensure(h, h->tot, sizeof(int64_t) * n));
    return OPEN_CF_OK;
}

template <typename TV>
cudaError_t stream_vhalf_enqueue(open_cf_t *h, int64_t m, int64_t nnz, const int64_t *ptr,
                                 const int32_t *idx, const TV *val, const TV *Uw, cudaStream_t st) {
    const int64_t n = h->n;
    const CscPlan plan = csc_plan(m, n, nnz, 0);
    int64_t *cptr = (int64_t *)h->csc_ptr.p;
    cudaError_t e = launch_csr_to_csc<TV>(m, n, nnz, ptr, idx, val, cptr, (int32_t *)h->csc_idx.p,
                                          (TV *)h->csc_val.p, (int32_t *)h->cnt.p,
                                          (int64_t *)h->tot.p, plan, st);
    if (e != cudaSuccess) return e;
    SolveArgs<TV> va{n, nnz, cptr, (const int32_t *)h->csc_idx.p, (const TV *)h->csc_val.p, Uw,
                     m, (TV *)h->V.p, h->KP, h->KP, nullptr, h->cfg.lambda};
    va.wr = h->cfg.weighted_lambda != 0;
    va.gram = (TV *)h->sg.p;
    va.gram_b = (TV *)h->sb.p;
    va.gram_n = (int64_t *)h->sn.p;
    va.gram_keep = true;
    return half_step<TV>(h, va, st);
}

template <typename TV>
int stream_vhalf(open_cf_t *h, int64_t m, int64_t nnz, const int64_t *ptr, const int32_t *idx,
                 const TV *val, const TV *Uw, cudaStream_t st) {
    h->v_epoch++;   // the refit rewrites V
    int rc = stream_vhalf_ws<TV>(h, m, nnz);
    if (rc) return rc;
    CK(h, stream_vhalf_enqueue<TV>(h, m, nnz, ptr, idx, val, Uw, st));
    return OPEN_CF_OK;
}

template <typename TV>
int stream_begin_t(open_cf_t *h, int64_t m, int64_t nnz, const int64_t *ptr, const int32_t *idx,
                   const TV *val, const TV *U, cudaStream_t st) {
    const int KP = h->KP;
    CK(h, ensure(h, h->U_w, sizeof(TV) * std::max<int64_t>(m, 1) * KP));
    TV *Uw = (TV *)h->U_w.p;
    if (m > 0) CK(h, launch_pack_rows<TV>(U, m, h->k, h->k, Uw, KP, st));
    return stream_vhalf<TV>(h, m, nnz, ptr, idx, val, Uw, st);
}

template <typename TV>
int stream_ingest_t(open_cf_t *h, int64_t m, int64_t nnz, const int64_t *ptr, const int32_t *idx,
                    const TV *val, TV *U_out, int32_t *status, cudaStream_t st) {
    h->v_epoch++;   // the refit rewrites V
    const int KP = h->KP;
    CK(h, ensure(h, h->U_w, sizeof(TV) * std::max<int64_t>(m, 1) * KP));
    int rc = stream_vhalf_ws<TV>(h, m, nnz);
    if (rc) return rc;
    TV *Uw = (TV *)h->U_w.p;
    // fold-in against the current V, the factors out, the V-half with the
    // stored sums: one captured graph per argument set, replayed
    auto enqueue = [&](cudaStream_t cs) -> cudaError_t {
        SolveArgs<TV> ua{m, nnz, ptr, idx, val, (const TV *)h->V.p, h->n, Uw, KP, KP, status,
                         h->cfg.lambda};
        ua.wr = h->cfg.weighted_lambda != 0;
        cudaError_t e = half_step<TV>(h, ua, cs);
        if (e != cudaSuccess) return e;
        if (m > 0 && (e = launch_unpack_rows<TV>(Uw, m, KP, h->k, U_out, cs)) != cudaSuccess)
            return e;
        return stream_vhalf_enqueue<TV>(h, m, nnz, ptr, idx, val, Uw, cs);
    };
    std::vector<int64_t> key = {6, m, nnz, (int64_t)ptr, (int64_t)idx, (int64_t)val,
                                (int64_t)U_out, (int64_t)status};
    return run_graph(h, key, st, enqueue);
}

}  // namespace

extern "C" {

int open_cf_stream_begin(open_cf_t *h, int64_t m, int64_t nnz, const int64_t *row_ptr,
                         const int32_t *col, const void *val, const void *U, void *stream) {
    NvtxRange nvtx_("open_cf_stream_begin");
    if (!h) return OPEN_CF_INVALID_ARG;
    h->err.clear();
    if (h->cfg.precision == OPEN_CF_BF16_GRAM)
        return fail(h, OPEN_CF_UNSUPPORTED, "the streaming refit runs in FP32 or FP64 mode");
    int rc = check_csr_args(h, m, nnz, row_ptr, col, val);
    if (rc) return rc;
    if (!h->V_set) return fail(h, OPEN_CF_NOT_FITTED, "no V: the number of settings is unknown");
    if (m > 0 && !U) return fail(h, OPEN_CF_INVALID_ARG, "U is NULL");
    DeviceGuard g(h->device);
    cudaStream_t st = S(stream);
    const int64_t n = h->n, KP = h->KP;
    CK(h, ensure(h, h->sg, h->esz * n * KP * KP));
    CK(h, ensure(h, h->sb, h->esz * n * KP));
    CK(h, ensure(h, h->sn, sizeof(int64_t) * n));
    CK(h, cudaMemsetAsync(h->sg.p, 0, h->esz * n * KP * KP, st));
    CK(h, cudaMemsetAsync(h->sb.p, 0, h->esz * n * KP, st));
    CK(h, cudaMemsetAsync(h->sn.p, 0, sizeof(int64_t) * n, st));
    rc = h->f64 ? stream_begin_t<double>(h, m, nnz, row_ptr, col, as<double>(val), as<double>(U), st)
                : stream_begin_t<float>(h, m, nnz, row_ptr, col, as<float>(val), as<float>(U), st);
    if (rc == OPEN_CF_OK) h->stream_on = true;
    return rc;
}

int open_cf_stream_ingest(open_cf_t *h, int64_t m_new, int64_t nnz, const int64_t *row_ptr,
                          const int32_t *col, const void *val, void *U_out, int32_t *status,
                          void *stream) {
    NvtxRange nvtx_("open_cf_stream_ingest");
    if (!h) return OPEN_CF_INVALID_ARG;
    h->err.clear();
    if (!h->stream_on) return fail(h, OPEN_CF_NOT_FITTED, "call open_cf_stream_begin first");
    int rc = check_csr_args(h, m_new, nnz, row_ptr, col, val);
    if (rc) return rc;
    if (m_new > 0 && !U_out) return fail(h, OPEN_CF_INVALID_ARG, "U_out is NULL");
    DeviceGuard g(h->device);
    cudaStream_t st = S(stream);
    return h->f64 ? stream_ingest_t<double>(h, m_new, nnz, row_ptr, col, as<double>(val),
                                            (double *)U_out, status, st)
                  : stream_ingest_t<float>(h, m_new, nnz, row_ptr, col, as<float>(val),
                                           (float *)U_out, status, st);
}

int open_cf_stream_sums(open_cf_t *h, void *G_out, void *b_out, int64_t *n_out, void *stream) {
    if (!h) return OPEN_CF_INVALID_ARG;
    h->err.clear();
    if (!h->stream_on) return fail(h, OPEN_CF_NOT_FITTED, "call open_cf_stream_begin first");
    DeviceGuard g(h->device);
    cudaStream_t st = S(stream);
    const int64_t n = h->n, KP = h->KP;
    if (G_out)
        CK(h, cudaMemcpyAsync(G_out, h->sg.p, h->esz * n * KP * KP, cudaMemcpyDeviceToDevice, st));
    if (b_out)
        CK(h, cudaMemcpyAsync(b_out, h->sb.p, h->esz * n * KP, cudaMemcpyDeviceToDevice, st));
    if (n_out)
        CK(h, cudaMemcpyAsync(n_out, h->sn.p, sizeof(int64_t) * n, cudaMemcpyDeviceToDevice, st));
    return OPEN_CF_OK;
}

int open_cf_stream_set_sums(open_cf_t *h, const void *G, const void *b, const int64_t *n_obs,
                            void *stream) {
    if (!h) return OPEN_CF_INVALID_ARG;
    h->err.clear();
    if (!h->stream_on) return fail(h, OPEN_CF_NOT_FITTED, "call open_cf_stream_begin first");
    if (!G || !b || !n_obs) return fail(h, OPEN_CF_INVALID_ARG, "G, b and n_obs are required");
    DeviceGuard g(h->device);
    cudaStream_t st = S(stream);
    const int64_t n = h->n, KP = h->KP;
    CK(h, cudaMemcpyAsync(h->sg.p, G, h->esz * n * KP * KP, cudaMemcpyDeviceToDevice, st));
    CK(h, cudaMemcpyAsync(h->sb.p, b, h->esz * n * KP, cudaMemcpyDeviceToDevice, st));
    CK(h, cudaMemcpyAsync(h->sn.p, n_obs, sizeof(int64_t) * n, cudaMemcpyDeviceToDevice, st));
    // every setting re-solved from the sums alone (a batch of no rows)
    CK(h, ensure(h, h->U_w, h->esz * KP));
    CK(h, ensure(h, h->j_ptr, sizeof(int64_t)));
    CK(h, cudaMemsetAsync(h->j_ptr.p, 0, sizeof(int64_t), st));
    const int64_t *p0 = (const int64_t *)h->j_ptr.p;
    return h->f64 ? stream_vhalf<double>(h, 0, 0, p0, nullptr, nullptr, (const double *)h->U_w.p, st)
                  : stream_vhalf<float>(h, 0, 0, p0, nullptr, nullptr, (const float *)h->U_w.p, st);
}

int open_cf_predict(open_cf_t *h, const void *U, int64_t m, void *T_out, int32_t *best,
                    float *saving, float gamma, int32_t baseline_setting, void *stream) {
    NvtxRange nvtx_("open_cf_predict");
    if (!h) return OPEN_CF_INVALID_ARG;
    h->err.clear();
    if (!h->V_set) return fail(h, OPEN_CF_NOT_FITTED, "no V: fit or set V first");
    if (m < 0 || (m > 0 && !U)) return fail(h, OPEN_CF_INVALID_ARG, "bad U or m");
    const bool sel = best || saving;
    if (sel && h->cpu_caps.empty())
        return fail(h, OPEN_CF_INVALID_ARG, "selection needs a cap grid");
    if (!std::isfinite(gamma)) return fail(h, OPEN_CF_INVALID_ARG, "gamma is not finite");
    int64_t base = baseline_setting < 0 ? h->base_default : baseline_setting;
    if (sel && (base < 0 || base >= h->n))
        return fail(h, OPEN_CF_INVALID_ARG, "baseline setting out of range");
    float Eb = 0.0f;
    if (sel) {
        const int ng = (int)h->gpu_caps.size();
        Eb = (float)h->cpu_caps[base / ng] + (float)h->gpu_caps[base % ng];
    }
    DeviceGuard g(h->device);
    if (h->f64) {
        PredictArgs<double> a{m, h->n, h->KP, h->k, as<double>(U), h->k, (double *)h->V.p,
                              sel ? (float *)h->cg.p : nullptr, base, Eb, gamma,
                              (double *)T_out, best, saving};
        CK(h, launch_predict_select<double>(a, S(stream)));
    } else if (h->cfg.precision == OPEN_CF_BF16_GRAM && h->KP == 32 &&
               h->n <= PREDICT_TC_CG_MAX) {
        // tensor cores: split-BF16 U V^T in TMEM, Algorithm 2 in the epilogue
        if (m == 0) return OPEN_CF_OK;
        cudaStream_t st = S(stream);
        if (!h->pt_err.p) {
            CK(h, ensure(h, h->pt_err, 16));
            CK(h, cudaMemsetAsync(h->pt_err.p, 0, 16, st));
        }
        CK(h, ensure(h, h->vimg, predict_tc_image_bytes(h->n)));
        if (h->vimg_epoch != h->v_epoch || h->vimg_at != h->vimg.p) {   // V's images, once per V
            CK(h, launch_v_image((const float *)h->V.p, h->n, h->vimg.p, st));
            h->vimg_epoch = h->v_epoch;
            h->vimg_at = h->vimg.p;
        }
        PredictTcArgs a{};
        a.m = m; a.n = h->n; a.U = as<float>(U); a.ldu = h->k; a.k = h->k;
        a.Vimg = h->vimg.p; a.cg = sel ? (const float *)h->cg.p : nullptr;
        a.base = sel ? base : 0; a.Ebase = Eb; a.gamma = gamma; a.select = sel;
        a.T = (float *)T_out;
        a.t_vec = T_out && (reinterpret_cast<uintptr_t>(T_out) % 16 == 0) && (h->n % 4 == 0);
        a.best = best; a.saving = saving; a.err = (int *)h->pt_err.p;
        a.wait_limit = h->wait_limit;
        CK(h, launch_predict_select_tc(a, h->num_sms, st));
    } else {
        PredictArgs<float> a{m, h->n, h->KP, h->k, as<float>(U), h->k, (float *)h->V.p,
                             sel ? (float *)h->cg.p : nullptr, base, Eb, gamma, (float *)T_out,
                             best, saving};
        CK(h, launch_predict_select<float>(a, S(stream)));
    }
    return OPEN_CF_OK;
}

namespace {
// 16-bit setting indices of one chunk widened to the solvers' int32 (kept as
// unsigned: up to 65,535 settings)
__global__ void k_widen_u16(const uint16_t *__restrict__ src, int64_t count,
                            int32_t *__restrict__ dst) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
         e += (int64_t)gridDim.x * blockDim.x)
        dst[e] = (int32_t)src[e];
}
}  // namespace

int open_cf_complete_select_host(open_cf_t *h, int64_t m, int64_t nnz, const int64_t *row_ptr,
                                 const void *col, int32_t col_bytes, const float *val,
                                 int32_t check,
                                 float gamma, int32_t baseline_setting, int32_t *best,
                                 float *saving, int32_t *status, float *resid,
                                 int64_t chunk_rows, void *stream) {
    NvtxRange nvtx_("open_cf_complete_select_host");
    if (!h) return OPEN_CF_INVALID_ARG;
    h->err.clear();
    if (m < 0 || nnz < 0) return fail(h, OPEN_CF_INVALID_ARG, "negative m or nnz");
    if (m > 0 && (!row_ptr || !best || !saving))
        return fail(h, OPEN_CF_INVALID_ARG, "row_ptr, best or saving is NULL");
    if (nnz > 0 && (!col || !val)) return fail(h, OPEN_CF_INVALID_ARG, "col or val is NULL");
    if (check < 0 || check > 2) return fail(h, OPEN_CF_INVALID_ARG, "check must be 0, 1 or 2");
    if (col_bytes != 2 && col_bytes != 4)
        return fail(h, OPEN_CF_INVALID_ARG, "col_bytes must be 2 or 4");
    if (check == 0 && resid) return fail(h, OPEN_CF_INVALID_ARG, "resid needs check >= 1");
    if (h->f64) return fail(h, OPEN_CF_UNSUPPORTED, "host-buffer completion is FP32 / BF16-Gram only");
    if (check > 0 && (h->KP != 32 || h->cfg.cholesky_fp64))
        return fail(h, OPEN_CF_UNSUPPORTED,
                    "the residual check needs 16 < k <= 32 and the FP32 factorisation");
    if (!h->V_set) return fail(h, OPEN_CF_NOT_FITTED, "no V: fit or set V first");
    if (h->cpu_caps.empty()) return fail(h, OPEN_CF_INVALID_ARG, "selection needs a cap grid");
    if (chunk_rows < 0) return fail(h, OPEN_CF_INVALID_ARG, "chunk_rows < 0");
    if (m == 0) return OPEN_CF_OK;
    if (row_ptr[0] != 0 || row_ptr[m] != nnz)
        return fail(h, OPEN_CF_INVALID_ARG, "row_ptr[0] must be 0 and row_ptr[m] == nnz");
    // chunks: about 16 per call, at least 32768 rows; by default a whole number
    // of 128-row reconstruction tiles per SM, so each chunk's persistent
    // reconstruction ends with every SM busy
    int64_t rows;
    if (chunk_rows > 0) {
        rows = (chunk_rows + 255) / 256 * 256;
    } else {
        const int64_t unit = 128 * (int64_t)std::max(1, h->num_sms);
        rows = std::max<int64_t>(32768, (m + 15) / 16);
        rows = (rows + unit - 1) / unit * unit;
    }
    rows = std::max<int64_t>(rows, ((m + 1023) / 1024 + 255) / 256 * 256);   // at most 1024 chunks
    const int64_t nch = (m + rows - 1) / rows;
    // chunk boundaries in the entry arrays, read on the host; a non-decreasing
    // sequence inside [0, nnz] is required here.  Each chunk is solved as a CSR
    // of its own (row pointers rebased to the chunk's first entry), so rows
    // inside it are checked against its own entries, as a separate call would.
    std::vector<int64_t> eb((size_t)nch + 1);
    for (int64_t c = 0; c <= nch; ++c) eb[(size_t)c] = row_ptr[std::min(m, c * rows)];
    for (int64_t c = 0; c < nch; ++c)
        if (eb[(size_t)c] < 0 || eb[(size_t)c + 1] < eb[(size_t)c] || eb[(size_t)c + 1] > nnz)
            return fail(h, OPEN_CF_INVALID_ARG, "row_ptr is not non-decreasing within [0, nnz]");
    DeviceGuard g(h->device);
    cudaStream_t st = S(stream);
    CK(h, ensure(h, h->hs_ptr, sizeof(int64_t) * (m + 1)));
    CK(h, ensure(h, h->hs_rptr, sizeof(int64_t) * (m + nch)));
    CK(h, ensure(h, h->hs_col, sizeof(int32_t) * std::max<int64_t>(nnz, 1)));
    if (col_bytes == 2) CK(h, ensure(h, h->hs_col16, sizeof(uint16_t) * std::max<int64_t>(nnz, 1)));
    CK(h, ensure(h, h->hs_val, sizeof(float) * std::max<int64_t>(nnz, 1)));
    CK(h, ensure(h, h->hs_U, sizeof(float) * m * h->k));
    CK(h, ensure(h, h->hs_best, sizeof(int32_t) * m));
    CK(h, ensure(h, h->hs_sav, sizeof(float) * m));
    CK(h, ensure(h, h->hs_st, sizeof(int32_t) * m));
    if (check > 0) CK(h, ensure(h, h->hs_res, sizeof(float) * m));
    if (!h->hs_copy) CK(h, cudaStreamCreateWithFlags(&h->hs_copy, cudaStreamNonBlocking));
    while ((int64_t)h->hs_ev.size() < 2 * nch + 2) {   // copies, start, solves, end
        cudaEvent_t e;
        CK(h, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        h->hs_ev.push_back(e);
    }
    // the copies may overwrite the device buffers only after the work queued
    // before this call on the caller's stream (an earlier call's solves)
    CK(h, cudaEventRecord(h->hs_ev[(size_t)nch], st));
    CK(h, cudaStreamWaitEvent(h->hs_copy, h->hs_ev[(size_t)nch], 0));
    int64_t *dptr = (int64_t *)h->hs_ptr.p, *drp = (int64_t *)h->hs_rptr.p;
    int32_t *dcol = (int32_t *)h->hs_col.p;
    float *dval = (float *)h->hs_val.p, *dU = (float *)h->hs_U.p;
    int32_t *dbest = (int32_t *)h->hs_best.p, *dst = (int32_t *)h->hs_st.p;
    float *dsav = (float *)h->hs_sav.p, *dres = (float *)h->hs_res.p;
    // copy stream: every chunk's copies in order, then its row pointers rebased
    // to its first entry (and 16-bit indices widened), then an event
    for (int64_t c = 0; c < nch; ++c) {
        const int64_t r0 = c * rows, r1 = std::min(m, r0 + rows), mc = r1 - r0;
        const int64_t e0 = eb[(size_t)c], e1 = eb[(size_t)c + 1];
        CK(h, cudaMemcpyAsync(dptr + r0, row_ptr + r0, sizeof(int64_t) * (mc + 1),
                              cudaMemcpyHostToDevice, h->hs_copy));
        if (e1 > e0) {
            if (col_bytes == 2)
                CK(h, cudaMemcpyAsync((uint16_t *)h->hs_col16.p + e0,
                                      (const uint16_t *)col + e0, sizeof(uint16_t) * (e1 - e0),
                                      cudaMemcpyHostToDevice, h->hs_copy));
            else
                CK(h, cudaMemcpyAsync(dcol + e0, (const int32_t *)col + e0,
                                      sizeof(int32_t) * (e1 - e0), cudaMemcpyHostToDevice,
                                      h->hs_copy));
            CK(h, cudaMemcpyAsync(dval + e0, val + e0, sizeof(float) * (e1 - e0),
                                  cudaMemcpyHostToDevice, h->hs_copy));
        }
        k_offset_copy<<<(unsigned)std::min<int64_t>((mc + 256) / 256 + 1, 4096), 256, 0,
                        h->hs_copy>>>(dptr + r0, mc + 1, -e0, drp + r0 + c);
        CK(h, cudaGetLastError());
        if (col_bytes == 2 && e1 > e0) {
            k_widen_u16<<<(unsigned)std::min<int64_t>((e1 - e0 + 255) / 256, 4 * 148), 256, 0,
                          h->hs_copy>>>((const uint16_t *)h->hs_col16.p + e0, e1 - e0, dcol + e0);
            CK(h, cudaGetLastError());
        }
        CK(h, cudaEventRecord(h->hs_ev[(size_t)c], h->hs_copy));
    }
    // the caller's stream: chunk c's solves wait for its copies only, then an event
    for (int64_t c = 0; c < nch; ++c) {
        const int64_t r0 = c * rows, r1 = std::min(m, r0 + rows), mc = r1 - r0;
        const int64_t e0 = eb[(size_t)c], e1 = eb[(size_t)c + 1];
        CK(h, cudaStreamWaitEvent(st, h->hs_ev[(size_t)c], 0));
        int64_t *rp = drp + r0 + c;   // this chunk's rebased row pointers (mc + 1)
        int rc;
        if (check > 0)
            rc = open_cf_complete_rows_checked(h, mc, e1 - e0, rp, dcol + e0, dval + e0,
                                               dU + r0 * h->k, dst + r0, dres + r0,
                                               check == 2 ? 1 : 0, st);
        else
            rc = open_cf_complete_rows(h, mc, e1 - e0, rp, dcol + e0, dval + e0,
                                       dU + r0 * h->k, dst + r0, 0, st);
        if (rc) return rc;
        rc = open_cf_predict(h, dU + r0 * h->k, mc, nullptr, dbest + r0, dsav + r0, gamma,
                             baseline_setting, st);
        if (rc) return rc;
        CK(h, cudaEventRecord(h->hs_ev[(size_t)(nch + 1 + c)], st));
    }
    // copy stream again (after all input copies): each chunk's decisions back
    // once its solves are done, then the caller's stream waits for the last
    for (int64_t c = 0; c < nch; ++c) {
        const int64_t r0 = c * rows, mc = std::min(m, r0 + rows) - r0;
        CK(h, cudaStreamWaitEvent(h->hs_copy, h->hs_ev[(size_t)(nch + 1 + c)], 0));
        CK(h, cudaMemcpyAsync(best + r0, dbest + r0, sizeof(int32_t) * mc,
                              cudaMemcpyDeviceToHost, h->hs_copy));
        CK(h, cudaMemcpyAsync(saving + r0, dsav + r0, sizeof(float) * mc,
                              cudaMemcpyDeviceToHost, h->hs_copy));
        if (status)
            CK(h, cudaMemcpyAsync(status + r0, dst + r0, sizeof(int32_t) * mc,
                                  cudaMemcpyDeviceToHost, h->hs_copy));
        if (resid)
            CK(h, cudaMemcpyAsync(resid + r0, dres + r0, sizeof(float) * mc,
                                  cudaMemcpyDeviceToHost, h->hs_copy));
    }
    CK(h, cudaEventRecord(h->hs_ev[(size_t)(2 * nch + 1)], h->hs_copy));
    CK(h, cudaStreamWaitEvent(st, h->hs_ev[(size_t)(2 * nch + 1)], 0));
    return OPEN_CF_OK;
}

int open_cf_select(open_cf_t *h, const float *T, int64_t m, int64_t ld, int32_t *best,
                   float *saving, float gamma, int32_t baseline_setting, void *stream) {
    NvtxRange nvtx_("open_cf_select");
    if (!h) return OPEN_CF_INVALID_ARG;
    h->err.clear();
    if (h->cpu_caps.empty()) return fail(h, OPEN_CF_INVALID_ARG, "selection needs a cap grid");
    const int64_t n = (int64_t)h->cpu_caps.size() * (int64_t)h->gpu_caps.size();
    if (m < 0 || (m > 0 && !T) || ld < n) return fail(h, OPEN_CF_INVALID_ARG, "bad T, m or ld");
    if (!std::isfinite(gamma)) return fail(h, OPEN_CF_INVALID_ARG, "gamma is not finite");
    int64_t base = baseline_setting < 0 ? h->base_default : baseline_setting;
    if (base < 0 || base >= n) return fail(h, OPEN_CF_INVALID_ARG, "baseline out of range");
    DeviceGuard g(h->device);
    if (h->n != n) {
        std::vector<float> cg(n);
        const int ng = (int)h->gpu_caps.size();
        for (int64_t j = 0; j < n; ++j)
            cg[j] = (float)h->cpu_caps[j / ng] + (float)h->gpu_caps[j % ng];
        CK(h, ensure(h, h->cg, sizeof(float) * n));
        CK(h, cudaMemcpy(h->cg.p, cg.data(), sizeof(float) * n, cudaMemcpyHostToDevice));
    }
    const int ng = (int)h->gpu_caps.size();
    const float Eb = (float)h->cpu_caps[base / ng] + (float)h->gpu_caps[base % ng];
    CK(h, launch_select(m, n, T, ld, (float *)h->cg.p, base, Eb, gamma, best, saving,
                        S(stream)));
    return OPEN_CF_OK;
}

int open_cf_objective(open_cf_t *h, int64_t m, int64_t nnz, const int64_t *row_ptr,
                      const int32_t *col, const void *val, const void *U, double *J_out,
                      float *row_rmse, void *stream) {
    NvtxRange nvtx_("open_cf_objective");
    if (!h) return OPEN_CF_INVALID_ARG;
    h->err.clear();
    int rc = check_csr_args(h, m, nnz, row_ptr, col, val);
    if (rc) return rc;
    if (!h->V_set) return fail(h, OPEN_CF_NOT_FITTED, "no V: fit or set V first");
    if (!J_out || (m > 0 && !U)) return fail(h, OPEN_CF_INVALID_ARG, "J_out or U is NULL");
    DeviceGuard g(h->device);
    CK(h, ensure(h, h->part, sizeof(double) * 3 * objective_parts(std::max<int64_t>(m, h->n))));
    const int32_t *ccount = nullptr;
    if (h->cfg.weighted_lambda) {   // observations per column of this matrix
        CK(h, ensure(h, h->ccount, sizeof(int32_t) * std::max<int64_t>(h->n, 1)));
        CK(h, launch_col_counts(nnz, h->n, col, (int32_t *)h->ccount.p, S(stream)));
        ccount = (const int32_t *)h->ccount.p;
    }
    if (h->f64)
        CK(h, launch_objective<double>(m, nnz, row_ptr, col, as<double>(val), as<double>(U), h->k,
                                       h->k, (double *)h->V.p, h->n, h->KP, h->cfg.lambda,
                                       (double *)h->part.p, J_out, row_rmse, ccount, S(stream)));
    else
        CK(h, launch_objective<float>(m, nnz, row_ptr, col, as<float>(val), as<float>(U), h->k,
                                      h->k, (float *)h->V.p, h->n, h->KP, h->cfg.lambda,
                                      (double *)h->part.p, J_out, row_rmse, ccount, S(stream)));
    return OPEN_CF_OK;
}

int open_cf_csr_to_csc(open_cf_t *h, int64_t m, int64_t n, int64_t nnz, const int64_t *row_ptr,
                       const int32_t *col, const void *val, int64_t *col_ptr, int32_t *row_idx,
                       void *cval, void *stream) {
    NvtxRange nvtx_("open_cf_csr_to_csc");
    if (!h) return OPEN_CF_INVALID_ARG;
    h->err.clear();
    int rc = check_csr_args(h, m, nnz, row_ptr, col, val);
    if (rc) return rc;
    if (n <= 0 || !col_ptr || (nnz > 0 && (!row_idx || !cval)))
        return fail(h, OPEN_CF_INVALID_ARG, "bad n or output arrays");
    if (n > CSC_MAX_N) return fail(h, OPEN_CF_UNSUPPORTED, "n exceeds %lld columns",
                                   (long long)CSC_MAX_N);
    DeviceGuard g(h->device);
    const CscPlan plan = csc_plan(m, n, nnz, 0);
    const int64_t nb = plan.nb;
    CK(h, ensure(h, h->cnt, sizeof(int32_t) * n * nb));
    CK(h, ensure(h, h->tot, sizeof(int64_t) * n));
    if (h->f64)
        CK(h, launch_csr_to_csc<double>(m, n, nnz, row_ptr, col, as<double>(val), col_ptr, row_idx,
                                        (double *)cval, (int32_t *)h->cnt.p,
                                        (int64_t *)h->tot.p, plan, S(stream)));
    else
        CK(h, launch_csr_to_csc<float>(m, n, nnz, row_ptr, col, as<float>(val), col_ptr, row_idx,
                                       (float *)cval, (int32_t *)h->cnt.p, (int64_t *)h->tot.p,
                                       plan, S(stream)));
    return OPEN_CF_OK;
}

int open_cf_validate_csr(open_cf_t *h, int64_t m, int64_t n, int64_t nnz, const int64_t *row_ptr,
                         const int32_t *col, const void *val, int32_t *result_host,
                         void *stream) {
    if (!h) return OPEN_CF_INVALID_ARG;
    h->err.clear();
    int rc = check_csr_args(h, m, nnz, row_ptr, col, val);
    if (rc) return rc;
    if (!result_host || n <= 0) return fail(h, OPEN_CF_INVALID_ARG, "bad result pointer or n");
    DeviceGuard g(h->device);
    cudaStream_t st = S(stream);
    CK(h, ensure(h, h->flag, sizeof(int32_t)));
    CK(h, cudaMemsetAsync(h->flag.p, 0x7f, sizeof(int32_t), st));
    if (h->f64)
        CK(h, launch_validate_csr<double>(m, n, nnz, row_ptr, col, as<double>(val),
                                          (int32_t *)h->flag.p, st));
    else
        CK(h, launch_validate_csr<float>(m, n, nnz, row_ptr, col, as<float>(val),
                                         (int32_t *)h->flag.p, st));
    int32_t f = 0;
    CK(h, cudaMemcpyAsync(&f, h->flag.p, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CK(h, cudaStreamSynchronize(st));
    *result_host = (f == 0x7f7f7f7f) ? 0 : f;
    return OPEN_CF_OK;
}

int open_cf_batched_fit(open_cf_t *h, int64_t P, const int64_t *m_host, const int64_t *n_host,
                        const int32_t *k_host, const int64_t *nnz_host, int64_t nnz,
                        const int64_t *row_ptr, const int32_t *col, const float *val,
                        float *V_inout, float *U_out, void *stream) {
    NvtxRange nvtx_("open_cf_batched_fit");
    if (!h) return OPEN_CF_INVALID_ARG;
    h->err.clear();
    if (h->cfg.precision != OPEN_CF_FP32)
        return fail(h, OPEN_CF_UNSUPPORTED, "batched fits run in OPEN_CF_FP32 precision");
    if (!row_ptr || !V_inout || (nnz > 0 && (!col || !val)))
        return fail(h, OPEN_CF_INVALID_ARG, "NULL array");
    DeviceGuard g(h->device);
    BatchPlan L;
    int rc = batch_plan(h, P, m_host, n_host, k_host, nnz_host, nnz, L);
    if (rc) return rc;
    const BatchArgs b = batch_args(h, L, row_ptr, col, val, h->cfg.sweeps);
    const int grid = batched_grid(h);
    std::vector<int64_t> key = {2, P, nnz, (int64_t)row_ptr, (int64_t)col, (int64_t)val,
                                (int64_t)V_inout, (int64_t)U_out, h->b_nclass, grid};
    for (int c = 0; c < h->b_nclass; ++c) {   // the classes are baked into the graph
        key.push_back(h->b_class_end[c]);
        key.push_back(h->b_class_W[c]);
    }
    return run_graph(h, key, S(stream), [&](cudaStream_t st) {
        return batch_enqueue(h, L, b, V_inout, U_out, grid, st);
    });
}

int open_cf_batched_tune(open_cf_t *h, int64_t P, const int64_t *m_host, const int64_t *n_host,
                         const int32_t *k_host, const int64_t *nnz_host, int64_t nnz,
                         const int64_t *row_ptr, const int32_t *col, const float *val,
                         float *V_scratch, int32_t *W_out_host, void *stream) {
    NvtxRange nvtx_("open_cf_batched_tune");
    if (!h) return OPEN_CF_INVALID_ARG;
    h->err.clear();
    if (h->cfg.precision != OPEN_CF_FP32)
        return fail(h, OPEN_CF_UNSUPPORTED, "batched fits run in OPEN_CF_FP32 precision");
    if (!row_ptr || !V_scratch || (nnz > 0 && (!col || !val)))
        return fail(h, OPEN_CF_INVALID_ARG, "NULL array");
    DeviceGuard g(h->device);
    cudaStream_t st = S(stream);
    cudaEvent_t e0, e1;
    CK(h, cudaEventCreate(&e0));
    CK(h, cudaEventCreate(&e1));
    // one 2-sweep trial of the current setting (the first run warms caches)
    auto trial = [&](float &ms) -> int {
        BatchPlan L;
        int rc = batch_plan(h, P, m_host, n_host, k_host, nnz_host, nnz, L);
        if (rc) return rc;
        const BatchArgs b = batch_args(h, L, row_ptr, col, val, 2);
        const int grid = batched_grid(h);
        for (int rep = 0; rep < 2; ++rep) {
            CK(h, cudaEventRecord(e0, st));
            CK(h, batch_enqueue(h, L, b, V_scratch, nullptr, grid, st));
            CK(h, cudaEventRecord(e1, st));
            CK(h, cudaEventSynchronize(e1));
            CK(h, cudaEventElapsedTime(&ms, e0, e1));
        }
        return OPEN_CF_OK;
    };
    // coordinate search: warps per problem of both classes, then the class cut,
    // then the CTAs per SM, each stage from the best of the previous one
    float best_ms = 0.0f;
    bool first = true;
    int32_t best[4] = {h->b_W[0], h->b_W[1], h->b_cut, h->b_ctas};
    auto consider = [&]() -> int {
        float ms = 0.0f;
        int rc = trial(ms);
        if (rc) return rc;
        if (first || ms < best_ms) {
            best_ms = ms;
            best[0] = h->b_W[0];
            best[1] = h->b_W[1];
            best[2] = h->b_cut;
            best[3] = h->b_ctas;
            first = false;
        }
        return OPEN_CF_OK;
    };
    auto restore = [&]() {
        h->b_W[0] = best[0];
        h->b_W[1] = best[1];
        h->b_cut = best[2];
        h->b_ctas = best[3];
    };
    const int cand_large[3] = {2, 4, 8}, cand_small[3] = {1, 2, 4};
    const int cand_cut[3] = {30, 50, 70}, cand_ctas[2] = {1, 2};
    int rc = OPEN_CF_OK;
    for (int a = 0; a < 3 && !rc; ++a)
        for (int c = 0; c < 3 && !rc; ++c) {
            h->b_W[0] = cand_large[a];
            h->b_W[1] = cand_small[c];
            rc = consider();
        }
    restore();
    for (int c = 0; c < 3 && !rc; ++c) {
        h->b_cut = cand_cut[c];
        rc = consider();
    }
    restore();
    for (int c = 0; c < 2 && !rc; ++c) {
        h->b_ctas = cand_ctas[c];
        rc = consider();
    }
    restore();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    if (W_out_host)
        for (int t = 0; t < 4; ++t) W_out_host[t] = best[t];
    return OPEN_CF_OK;
}

static int mlp_caps_table(open_cf_t *h);

int open_cf_mlp_set_params(open_cf_t *h, const float *params, void *stream) {
    int rc_caps;
    if (!h) return OPEN_CF_INVALID_ARG;
    h->err.clear();
    if (h->k != MLP_K) return fail(h, OPEN_CF_UNSUPPORTED, "the learned warm start has k = 32");
    if (h->f64) return fail(h, OPEN_CF_UNSUPPORTED, "the learned warm start runs in FP32 modes");
    if (!params) return fail(h, OPEN_CF_INVALID_ARG, "params is NULL");
    DeviceGuard g(h->device);
    cudaStream_t st = S(stream);
    CK(h, ensure(h, h->mlp_th, 4 * MLP_P_INT));
    CK(h, ensure(h, h->mlp_m1, 4 * MLP_P_INT));
    CK(h, ensure(h, h->mlp_m2, 4 * MLP_P_INT));
    CK(h, ensure(h, h->mlp_img, 2 * MLP_IMG_TOTAL));
    CK(h, ensure(h, h->mlp_err, 16));
    CK(h, cudaMemsetAsync(h->mlp_err.p, 0, 16, st));
    CK(h, ensure(h, h->mlp_t, 16));
    float *th = (float *)h->mlp_th.p;
    CK(h, cudaMemsetAsync(th, 0, 4 * MLP_P_INT, st));
    CK(h, cudaMemcpyAsync(th, params, 4 * MLP_IN * MLP_H, cudaMemcpyDeviceToDevice, st));
    CK(h, cudaMemcpyAsync(th + MLP_OFF_B1, params + MLP_IN * MLP_H, 4 * (P_EXT - MLP_IN * MLP_H),
                          cudaMemcpyDeviceToDevice, st));
    CK(h, cudaMemsetAsync(h->mlp_m1.p, 0, 4 * MLP_P_INT, st));
    CK(h, cudaMemsetAsync(h->mlp_m2.p, 0, 4 * MLP_P_INT, st));
    CK(h, cudaMemsetAsync(h->mlp_t.p, 0, 16, st));
    CK(h, launch_mlp_images(th, h->mlp_img.p, st));   // the tensor cores' BF16 operand images
    rc_caps = mlp_caps_table(h);
    if (rc_caps) return rc_caps;
    CK(h, cudaStreamSynchronize(st));
    h->mlp_ready = true;
    return OPEN_CF_OK;
}

// normalised caps of every setting (the learned path's features), FP32
static int mlp_caps_table(open_cf_t *h) {
    const int64_t ns = (int64_t)h->cpu_caps.size() * (int64_t)h->gpu_caps.size();
    if (ns > 0) {
        const double cmin = *std::min_element(h->cpu_caps.begin(), h->cpu_caps.end());
        const double cmax = *std::max_element(h->cpu_caps.begin(), h->cpu_caps.end());
        const double gmin = *std::min_element(h->gpu_caps.begin(), h->gpu_caps.end());
        const double gmax = *std::max_element(h->gpu_caps.begin(), h->gpu_caps.end());
        const int nc = (int)h->cpu_caps.size(), ng = (int)h->gpu_caps.size();
        // [c_norm per CPU cap | g_norm per GPU cap]
        std::vector<float> cn(nc + ng);
        auto cnorm = [&](double c) { return (float)(cmax > cmin ? (c - cmin) / (cmax - cmin) : 0.0); };
        auto gnorm = [&](double g) { return (float)(gmax > gmin ? (g - gmin) / (gmax - gmin) : 0.0); };
        for (int c = 0; c < nc; ++c) cn[c] = cnorm(h->cpu_caps[c]);
        for (int g = 0; g < ng; ++g) cn[nc + g] = gnorm(h->gpu_caps[g]);
        CK(h, ensure(h, h->mlp_cn, 4 * cn.size()));
        CK(h, cudaMemcpy(h->mlp_cn.p, cn.data(), 4 * cn.size(), cudaMemcpyHostToDevice));
    }
    return OPEN_CF_OK;
}

int open_cf_mlp_get_params(open_cf_t *h, float *params_out, void *stream) {
    if (!h) return OPEN_CF_INVALID_ARG;
    h->err.clear();
    if (!h->mlp_ready) return fail(h, OPEN_CF_NOT_FITTED, "set the MLP parameters first");
    if (!params_out) return fail(h, OPEN_CF_INVALID_ARG, "params_out is NULL");
    DeviceGuard g(h->device);
    const float *th = (const float *)h->mlp_th.p;
    CK(h, cudaMemcpyAsync(params_out, th, 4 * MLP_IN * MLP_H, cudaMemcpyDeviceToDevice, S(stream)));
    CK(h, cudaMemcpyAsync(params_out + MLP_IN * MLP_H, th + MLP_OFF_B1, 4 * (P_EXT - MLP_IN * MLP_H),
                          cudaMemcpyDeviceToDevice, S(stream)));
    return OPEN_CF_OK;
}

int open_cf_mlp_train_step(open_cf_t *h, int64_t B, int64_t nnz, const int64_t *row_ptr,
                           const int32_t *col, const float *val, const float *U_target, float lr,
                           double *loss_out, float *grads_out, void *stream) {
    NvtxRange nvtx_("open_cf_mlp_train_step");
    if (!h) return OPEN_CF_INVALID_ARG;
    h->err.clear();
    int rc = mlp_check(h);
    if (rc) return rc;
    rc = check_csr_args(h, B, nnz, row_ptr, col, val);
    if (rc) return rc;
    if (B <= 0 || !U_target) return fail(h, OPEN_CF_INVALID_ARG, "empty batch or no targets");
    if (!(lr >= 0.0f) || !std::isfinite(lr)) return fail(h, OPEN_CF_INVALID_ARG, "bad lr");
    if (B > (1 << 20)) return fail(h, OPEN_CF_UNSUPPORTED, "batch above 2^20 rows");
    if ((uintptr_t)U_target % 16) return fail(h, OPEN_CF_INVALID_ARG, "U_target not 16-byte aligned");
    DeviceGuard g(h->device);
    // scratch: the slices of G = V^T V, G, the slices' ticket (zero between
    // launches), then one slot of partial sums per CTA
    const size_t g_floats = (size_t)MLP_GRAM_PARTS * MLP_K * MLP_K + MLP_K * MLP_K + 64;
    const int slots = mlp_train_tc_slots(B, h->num_sms);
    const size_t p_floats = (size_t)slots * MLP_PART_STRIDE;
    const size_t cap0 = h->mlp_scr.bytes;
    CK(h, ensure(h, h->mlp_scr, 4 * (g_floats + p_floats)));
    float *Gpart = (float *)h->mlp_scr.p, *Gfin = Gpart + MLP_GRAM_PARTS * MLP_K * MLP_K;
    unsigned int *ticket = (unsigned int *)(Gfin + MLP_K * MLP_K);
    float *part = Gpart + g_floats;
    if (h->mlp_scr.bytes != cap0) {   // a new scratch: the ticket is zeroed, G recomputed
        CK(h, cudaMemsetAsync(ticket, 0, 4, S(stream)));
        h->mlp_g_epoch = 0;
    }
    if (h->mlp_g_epoch != h->v_epoch) {   // G = V^T V, once per V
        CK(h, launch_mlp_gram(h->n, h->KP, (const float *)h->V.p, Gpart, Gfin, ticket, S(stream)));
        h->mlp_g_epoch = h->v_epoch;
    }
    std::vector<int64_t> key = {3, B, nnz, (int64_t)row_ptr, (int64_t)col, (int64_t)val,
                                (int64_t)U_target, (int64_t)loss_out, (int64_t)grads_out,
                                h->wait_limit};
    if (!grads_out) CK(h, launch_adam_set_lr(h->mlp_t.p, lr, S(stream)));
    return run_graph(h, key, S(stream), [&](cudaStream_t st) -> cudaError_t {
        float *th = (float *)h->mlp_th.p;
        MlpTrainArgs ta{};
        ta.m = B; ta.nnz = nnz; ta.ptr = row_ptr; ta.idx = col; ta.val = val;
        ta.ccap = (const float *)h->mlp_cn.p;
        ta.gcap = ta.ccap + h->cpu_caps.size();
        ta.n_gpu = (int32_t)h->gpu_caps.size();
        ta.n = h->n;
        ta.img = h->mlp_img.p;
        ta.b1 = th + MLP_OFF_B1; ta.b2 = th + MLP_OFF_B2; ta.b3 = th + MLP_OFF_B3;
        ta.T = U_target; ta.G = Gfin; ta.scale = 2.0f / (float)B; ta.part = part;
        ta.adam = grads_out ? nullptr : (AdamState *)h->mlp_t.p;
        ta.err = (int *)h->mlp_err.p;
        ta.wait_limit = h->wait_limit;
        cudaError_t e = launch_mlp_train_tc(ta, h->num_sms, false, st);
        if (e != cudaSuccess) return e;
        MlpReduceArgs ra{};
        ra.part = part; ra.ctas = slots;
        ra.th = th; ra.m1 = (float *)h->mlp_m1.p; ra.m2 = (float *)h->mlp_m2.p;
        ra.adam = grads_out ? nullptr : (AdamState *)h->mlp_t.p;
        ra.img = h->mlp_img.p; ra.grads_out = grads_out; ra.loss = loss_out; ra.B = B;
        ra.err = (const int *)h->mlp_err.p;
        return launch_mlp_reduce_adam(ra, st);
    });
}

int open_cf_mlp_infer(open_cf_t *h, int64_t m, int64_t nnz, const int64_t *row_ptr,
                      const int32_t *col, const float *val, float *U_out, int32_t *status,
                      float *row_rmse, void *stream) {
    NvtxRange nvtx_("open_cf_mlp_infer");
    if (!h) return OPEN_CF_INVALID_ARG;
    h->err.clear();
    int rc = mlp_check(h);
    if (rc) return rc;
    rc = check_csr_args(h, m, nnz, row_ptr, col, val);
    if (rc) return rc;
    if (m > 0 && !U_out) return fail(h, OPEN_CF_INVALID_ARG, "U_out is NULL");
    if (m == 0) return OPEN_CF_OK;
    if (reinterpret_cast<uintptr_t>(U_out) % 16)
        return fail(h, OPEN_CF_INVALID_ARG, "U_out must be 16-byte aligned");
    DeviceGuard g(h->device);
    cudaStream_t st = S(stream);
    CK(h, ensure(h, h->flag, 64));
    CK(h, ensure(h, h->j_idx, sizeof(int32_t) * m));   // fallback row list
    // fused forward pass on the tensor cores (tcgen05), straight into U_out
    MlpTcArgs ta{};
    ta.m = m; ta.nnz = nnz; ta.ptr = row_ptr; ta.idx = col; ta.val = val;
    ta.ccap = (const float *)h->mlp_cn.p;
    ta.gcap = ta.ccap + h->cpu_caps.size();
    ta.n_gpu = (int32_t)h->gpu_caps.size();
    ta.n = h->n;
    ta.img = h->mlp_img.p;
    const float *th = (const float *)h->mlp_th.p;
    ta.b1 = th + MLP_OFF_B1; ta.b2 = th + MLP_OFF_B2; ta.b3 = th + MLP_OFF_B3;
    ta.Y = U_out; ta.err = (int *)h->mlp_err.p; ta.wait_limit = h->wait_limit;
    // the kernel also evaluates each row's observed-entry RMSE and lists the
    // rows above the threshold; those are re-solved by the ridge fold-in
    int64_t *cnt = (int64_t *)h->flag.p;
    ta.V = (const float *)h->V.p; ta.threshold = h->cfg.mlp_fallback_threshold;
    ta.row_rmse = row_rmse; ta.status = status; ta.list = (int32_t *)h->j_idx.p; ta.count = cnt;
    CK(h, cudaMemsetAsync(cnt, 0, sizeof(int64_t), st));
    CK(h, launch_mlp_forward_tc(ta, h->num_sms, st));
    SolveArgs<float> a{m, nnz, row_ptr, col, val, (const float *)h->V.p, h->n, U_out, MLP_K,
                       MLP_K, status, h->cfg.lambda};
    a.row_map = (const int32_t *)h->j_idx.p;
    a.m_dev = cnt;
    a.wr = h->cfg.weighted_lambda != 0;
    if (h->cfg.precision == OPEN_CF_BF16_GRAM) a.Fb = h->Vb16.p;
    CK(h, half_step<float>(h, a, st));
    CK(h, launch_fallback_mark(m, (const int32_t *)h->j_idx.p, cnt, status, st));
    return OPEN_CF_OK;
}

int open_cf_phase_detect(const float *power, int64_t n_traces, int64_t len, int64_t ld,
                         float p_th, int32_t window, int64_t *first, void *stream) {
    if (n_traces < 0 || len < 0 || ld < len || window < 1) return OPEN_CF_INVALID_ARG;
    if (n_traces > 0 && (!first || (len > 0 && !power))) return OPEN_CF_INVALID_ARG;
    if (!std::isfinite(p_th)) return OPEN_CF_INVALID_ARG;
    if (launch_phase_detect(power, n_traces, len, ld, p_th, window, first, S(stream)) !=
        cudaSuccess)
        return OPEN_CF_CUDA_ERROR;
    return OPEN_CF_OK;
}

// ---------------------------------------------------------------------------
// Checkpoint and resume of a handle's state: a header, the cap grid, then the
// sections the handle holds (V in its padded device layout; the learned warm
// start's FP32 masters, Adam moments and step state; the streaming refit's
// per-setting sums), and an FNV-1a 64-bit checksum of all that precedes it.
// Little-endian, as the hosts this library runs on.
static const char CKPT_MAGIC[8] = {'O', 'P', 'E', 'N', 'C', 'F', 'c', 'k'};
static const uint32_t CKPT_VERSION = 1;
enum : uint32_t { CKPT_V = 1u, CKPT_MLP = 2u, CKPT_STREAM = 4u };
struct CkptHeader {
    char magic[8];
    uint32_t version, flags;
    int32_t k, KP, precision, cholesky_fp64, weighted_lambda, sweeps;
    double lambda;
    int64_t n;
    int32_t n_cpu, n_gpu, esz, reserved;
    int64_t bytes;   // the whole checkpoint, checksum included
};
static_assert(sizeof(CkptHeader) == 80, "checkpoint header layout");

static uint64_t fnv1a64(const unsigned char *p, size_t n) {
    uint64_t x = 0xcbf29ce484222325ull;
    for (size_t i = 0; i < n; ++i) {
        x ^= p[i];
        x *= 0x100000001b3ull;
    }
    return x;
}

static int64_t ckpt_bytes(const open_cf_t *h, uint32_t flags) {
    const int64_t n = h->n, KP = h->KP, e = (int64_t)h->esz;
    int64_t b = (int64_t)sizeof(CkptHeader) + 8 * (int64_t)(h->cpu_caps.size() + h->gpu_caps.size());
    if (flags & CKPT_V) b += e * n * KP;
    if (flags & CKPT_MLP) b += 3 * 4 * MLP_P_INT + 16;
    if (flags & CKPT_STREAM) b += e * n * KP * KP + e * n * KP + 8 * n;
    return b + 8;
}

int open_cf_save(open_cf_t *h, void *buf, int64_t cap, int64_t *size_out) {
    NvtxRange nvtx_("open_cf_save");
    if (!h) return OPEN_CF_INVALID_ARG;
    h->err.clear();
    const uint32_t flags = (h->V_set ? CKPT_V : 0u) | (h->mlp_ready ? CKPT_MLP : 0u) |
                           (h->stream_on ? CKPT_STREAM : 0u);
    const int64_t total = ckpt_bytes(h, flags);
    if (size_out) *size_out = total;
    if (!buf) return OPEN_CF_OK;
    if (cap < total) return fail(h, OPEN_CF_INVALID_ARG, "buffer of %lld bytes, %lld needed",
                                 (long long)cap, (long long)total);
    DeviceGuard g(h->device);
    CK(h, cudaDeviceSynchronize());   // the state is complete on every stream
    unsigned char *p = (unsigned char *)buf;
    CkptHeader hd{};
    memcpy(hd.magic, CKPT_MAGIC, 8);
    hd.version = CKPT_VERSION;
    hd.flags = flags;
    hd.k = h->k; hd.KP = h->KP; hd.precision = (int32_t)h->cfg.precision;
    hd.cholesky_fp64 = h->cfg.cholesky_fp64; hd.weighted_lambda = h->cfg.weighted_lambda;
    hd.sweeps = h->cfg.sweeps; hd.lambda = h->cfg.lambda;
    hd.n = h->V_set ? h->n : 0;
    hd.n_cpu = (int32_t)h->cpu_caps.size(); hd.n_gpu = (int32_t)h->gpu_caps.size();
    hd.esz = (int32_t)h->esz; hd.bytes = total;
    memcpy(p, &hd, sizeof(hd));
    p += sizeof(hd);
    for (double c : h->cpu_caps) { memcpy(p, &c, 8); p += 8; }
    for (double c : h->gpu_caps) { memcpy(p, &c, 8); p += 8; }
    const int64_t n = h->n, KP = h->KP, e = (int64_t)h->esz;
    auto d2h = [&](const void *src, int64_t bytes) -> cudaError_t {
        cudaError_t r = cudaMemcpy(p, src, (size_t)bytes, cudaMemcpyDeviceToHost);
        p += bytes;
        return r;
    };
    if (flags & CKPT_V) CK(h, d2h(h->V.p, e * n * KP));
    if (flags & CKPT_MLP) {
        CK(h, d2h(h->mlp_th.p, 4 * MLP_P_INT));
        CK(h, d2h(h->mlp_m1.p, 4 * MLP_P_INT));
        CK(h, d2h(h->mlp_m2.p, 4 * MLP_P_INT));
        CK(h, d2h(h->mlp_t.p, 16));
    }
    if (flags & CKPT_STREAM) {
        CK(h, d2h(h->sg.p, e * n * KP * KP));
        CK(h, d2h(h->sb.p, e * n * KP));
        CK(h, d2h(h->sn.p, 8 * n));
    }
    const uint64_t sum = fnv1a64((const unsigned char *)buf, (size_t)(total - 8));
    memcpy(p, &sum, 8);
    return OPEN_CF_OK;
}

int open_cf_load(open_cf_t *h, const void *buf, int64_t size) {
    NvtxRange nvtx_("open_cf_load");
    if (!h) return OPEN_CF_INVALID_ARG;
    h->err.clear();
    if (!buf || size < (int64_t)sizeof(CkptHeader) + 8)
        return fail(h, OPEN_CF_INVALID_ARG, "no checkpoint or too short");
    const unsigned char *p = (const unsigned char *)buf;
    CkptHeader hd;
    memcpy(&hd, p, sizeof(hd));
    if (memcmp(hd.magic, CKPT_MAGIC, 8) != 0) return fail(h, OPEN_CF_INVALID_ARG, "not a checkpoint");
    if (hd.version != CKPT_VERSION)
        return fail(h, OPEN_CF_UNSUPPORTED, "checkpoint version %u", hd.version);
    if (hd.bytes != size) return fail(h, OPEN_CF_INVALID_ARG, "checkpoint size mismatch");
    uint64_t sum;
    memcpy(&sum, p + size - 8, 8);
    if (sum != fnv1a64(p, (size_t)(size - 8)))
        return fail(h, OPEN_CF_INVALID_ARG, "checkpoint checksum mismatch");
    // the state belongs to a handle of the same model configuration
    if (hd.k != h->k || hd.KP != h->KP || hd.precision != (int32_t)h->cfg.precision ||
        hd.cholesky_fp64 != h->cfg.cholesky_fp64 || hd.weighted_lambda != h->cfg.weighted_lambda ||
        hd.lambda != h->cfg.lambda || hd.esz != (int32_t)h->esz)
        return fail(h, OPEN_CF_INVALID_ARG,
                    "checkpoint of another configuration (k, precision, lambda or weighting)");
    if (hd.n_cpu != (int32_t)h->cpu_caps.size() || hd.n_gpu != (int32_t)h->gpu_caps.size())
        return fail(h, OPEN_CF_INVALID_ARG, "checkpoint of another cap grid");
    p += sizeof(hd);
    for (int i = 0; i < hd.n_cpu + hd.n_gpu; ++i) {
        double c;
        memcpy(&c, p, 8);
        p += 8;
        const double mine = i < hd.n_cpu ? h->cpu_caps[i] : h->gpu_caps[i - hd.n_cpu];
        if (c != mine) return fail(h, OPEN_CF_INVALID_ARG, "checkpoint of another cap grid");
    }
    if ((hd.flags & ~(CKPT_V | CKPT_MLP | CKPT_STREAM)) ||
        ((hd.flags & CKPT_STREAM) && !(hd.flags & CKPT_V)))
        return fail(h, OPEN_CF_INVALID_ARG, "checkpoint sections inconsistent");
    const int64_t n = hd.n, KP = h->KP, e = (int64_t)h->esz;
    if ((hd.flags & CKPT_V) && (n <= 0 || n > CSC_MAX_N ||
                                (!h->cpu_caps.empty() &&
                                 n != (int64_t)h->cpu_caps.size() * (int64_t)h->gpu_caps.size())))
        return fail(h, OPEN_CF_INVALID_ARG, "checkpoint V has a bad number of settings");
    if ((hd.flags & CKPT_MLP) && (h->k != MLP_K || h->f64))
        return fail(h, OPEN_CF_INVALID_ARG, "checkpoint holds a learned warm start this handle cannot run");
    {   // the declared sections must account for every byte
        const int64_t saved_n = h->n;
        h->n = n;
        const int64_t want = ckpt_bytes(h, hd.flags);
        h->n = saved_n;
        if (want != size) return fail(h, OPEN_CF_INVALID_ARG, "checkpoint sections inconsistent");
    }
    DeviceGuard g(h->device);
    CK(h, cudaDeviceSynchronize());
    auto h2d = [&](void *dst, int64_t bytes) -> cudaError_t {
        cudaError_t r = cudaMemcpy(dst, p, (size_t)bytes, cudaMemcpyHostToDevice);
        p += bytes;
        return r;
    };
    if (hd.flags & CKPT_V) {
        CK(h, ensure(h, h->V, e * n * KP));
        CK(h, h2d(h->V.p, e * n * KP));
        if (h->cfg.precision == OPEN_CF_BF16_GRAM) {
            CK(h, ensure(h, h->Vb16, 4 * n * KP));
            CK(h, launch_to_bf16_split((const float *)h->V.p, n, KP, h->Vb16.p, 0));
        }
        if (!h->cpu_caps.empty() && h->n != n) {
            std::vector<float> cg(n);
            const int ng = (int)h->gpu_caps.size();
            for (int64_t j = 0; j < n; ++j)
                cg[j] = (float)h->cpu_caps[j / ng] + (float)h->gpu_caps[j % ng];
            CK(h, ensure(h, h->cg, sizeof(float) * n));
            CK(h, cudaMemcpy(h->cg.p, cg.data(), sizeof(float) * n, cudaMemcpyHostToDevice));
        }
        h->n = n;
        h->V_set = true;
        h->stream_on = false;
        h->v_epoch++;
    }
    if (hd.flags & CKPT_MLP) {
        CK(h, ensure(h, h->mlp_th, 4 * MLP_P_INT));
        CK(h, ensure(h, h->mlp_m1, 4 * MLP_P_INT));
        CK(h, ensure(h, h->mlp_m2, 4 * MLP_P_INT));
        CK(h, ensure(h, h->mlp_img, 2 * MLP_IMG_TOTAL));
        CK(h, ensure(h, h->mlp_err, 16));
        CK(h, ensure(h, h->mlp_t, 16));
        CK(h, cudaMemset(h->mlp_err.p, 0, 16));
        CK(h, h2d(h->mlp_th.p, 4 * MLP_P_INT));
        CK(h, h2d(h->mlp_m1.p, 4 * MLP_P_INT));
        CK(h, h2d(h->mlp_m2.p, 4 * MLP_P_INT));
        CK(h, h2d(h->mlp_t.p, 16));
        CK(h, launch_mlp_images((const float *)h->mlp_th.p, h->mlp_img.p, 0));
        const int rc = mlp_caps_table(h);
        if (rc) return rc;
        h->mlp_ready = true;
    }
    if (hd.flags & CKPT_STREAM) {
        CK(h, ensure(h, h->sg, e * n * KP * KP));
        CK(h, ensure(h, h->sb, e * n * KP));
        CK(h, ensure(h, h->sn, 8 * n));
        CK(h, h2d(h->sg.p, e * n * KP * KP));
        CK(h, h2d(h->sb.p, e * n * KP));
        CK(h, h2d(h->sn.p, 8 * n));
        h->stream_on = true;
    }
    CK(h, cudaDeviceSynchronize());
    return OPEN_CF_OK;
}

}  // extern "C"
