// Internal launcher declarations shared by the engine (open_cf.cu) and the
// kernel translation units.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ocf {

// One ALS half-step over the rows of a CSR matrix against a fixed factor F.
template <typename TV> struct SolveArgs {
    int64_t m;            // number of systems (rows)
    int64_t nnz;          // entries of the CSR arrays (bounds for row_ptr)
    const int64_t *ptr;   // row_ptr [m+1]
    const int32_t *idx;   // column indices [nnz]
    const TV *val;        // observed values [nnz]
    const TV *F;          // other factor, n_other rows of KP elements (zero padded)
    int64_t n_other;
    TV *out;              // output rows: out[i * ldo + q], q < kout
    int64_t ldo;
    int kout;
    int32_t *status;      // per-row status or null
    double lambda;
    const void *Fb = nullptr;   // BF16 split copy of F: rows [hi (KP) | lo (KP)], BF16 path
    void *outb = nullptr;       // optional split BF16 copy of the output rows (stride 2*KP)
    const int32_t *row_map = nullptr;   // optional: system i is CSR row row_map[i]
    const int64_t *m_dev = nullptr;     // optional: number of systems read on the device
    bool wr = false;                    // weighted lambda: the diagonal gets lambda * s_i
    // Streaming refit: per-system stored sums of earlier rows' normal equations
    // (Gram [KP][KP], right-hand side [KP], observation count), indexed by the
    // CSR row; they are added to this call's sums before lambda, and with
    // gram_keep the totals are written back.
    TV *gram = nullptr;
    TV *gram_b = nullptr;
    int64_t *gram_n = nullptr;
    bool gram_keep = false;
    // Rank-32 FP32-Cholesky solver only (solve32_tc.cu): per-row relative
    // normal-equation residual |A u - b| / (|A|_F |u| + |b|) (null: none), one
    // refinement step, or the residual of a given u (rows of stride ldo) with
    // nothing solved or written but the residual.
    float *resid = nullptr;
    bool refine = false;
    const TV *u_given = nullptr;
    // Rank-32 FP32-Cholesky solver only: a device word it may use as a pair
    // counter (zeroed on the stream before each launch) to balance the warps'
    // work; null: fixed ranges.
    unsigned int *work = nullptr;
};

template <typename TV, typename TC>
cudaError_t launch_row_solve(const SolveArgs<TV> &a, int KP, cudaStream_t st);

// CSR -> CSC stable counting sort.  Rows are cut into nb blocks of rb rows
// (rb a multiple of 32).  Scratch: cnt int32[n * nb] and tot int64[n].
// nb_cap > 0 bounds nb (and so the scratch); 0 = no bound.
struct CscPlan {
    int64_t rb, nb;
};
CscPlan csc_plan(int64_t m, int64_t n, int64_t nnz, int64_t nb_cap);
constexpr int64_t CSC_MAX_N = 25000;   // two 4-byte shared counters per column
template <typename TV>
cudaError_t launch_csr_to_csc(int64_t m, int64_t n, int64_t nnz, const int64_t *ptr,
                              const int32_t *idx, const TV *val, int64_t *cptr, int32_t *ridx,
                              TV *cval, int32_t *cnt, int64_t *tot, CscPlan plan,
                              cudaStream_t st);
cudaError_t prepare_csr_to_csc(int64_t n_max);
cudaError_t prepare_row_solve();

// FP32 path with the Gram and RHS on tensor cores, KP in {16, 32}: 3-pass TF32
// mma.sync (FP32 accuracy), or BF16 operands (bf16 = true; a.Fb required).
cudaError_t launch_row_solve_tc(const SolveArgs<float> &a, int KP, bool chol_fp64, bool bf16,
                                cudaStream_t st);
cudaError_t prepare_row_solve_tc();
// Padded rank 32, FP32 Cholesky, one system per warp (bf16: split-BF16 Gram,
// else 3-pass TF32), with the optional residual / refinement of SolveArgs.
cudaError_t launch_solve32_tc(const SolveArgs<float> &a, bool bf16, cudaStream_t st);
cudaError_t prepare_solve32_tc();

// Batched ALS over independent problems (batched.cu).  Per-problem arrays are
// indexed by problem id p; order[] lists problem ids in processing order;
// classes are consecutive ranges of order[] with their own warps per problem
// (per padded rank, largest first: a "large" and a "small" class each).
constexpr int BATCH_MAX_CLASSES = 6;
constexpr int64_t BATCH_MAX_N = 1024;
struct BatchArgs {
    int64_t P;
    const int32_t *order;
    const int64_t *m, *n;
    const int32_t *k;
    const int64_t *row_off;   // first global row of p (index into row_ptr)
    const int64_t *col_off;   // prefix sum of n: p's columns in the global CSC
    const int64_t *fu_off;    // p's padded U rows (KP_p floats each) in Uw
    const int64_t *fv_off;    // p's padded V rows in Vw
    const int64_t *row_ptr;   // global CSR row pointer (global entry offsets)
    const int32_t *col;       // local column indices
    const float *val;
    int64_t nnz;
    float *Uw, *Vw;
    int64_t *cptr;            // CSC pointers: problem p uses [col_off[p] + p, +n_p] (global offsets)
    int32_t *cidx;            // CSC local row indices (same entry ranges as the CSR)
    float *cval;
    int32_t *counter;         // work queue position per class (zeroed before launch)
    int sweeps;
    double lambda;
    bool wr;                  // weighted lambda (lambda * observations of the row / column)
    int n_classes;
    int32_t class_end[BATCH_MAX_CLASSES];
    int32_t class_W[BATCH_MAX_CLASSES];
};
cudaError_t prepare_batched();
size_t batched_smem_bytes();
cudaError_t launch_batched(const BatchArgs &b, int grid, cudaStream_t st);
cudaError_t launch_batched_pack(int64_t P, const int64_t *rows, const int32_t *k,
                                const int64_t *t_off, const int64_t *f_off, const float *src,
                                float *dst, bool to_padded, cudaStream_t st);

// MLP warm start (mlp.cu, mlp_tc.cu, mlp_train_tc.cu).
constexpr int MLP_IN = 48, MLP_INP = 64, MLP_H = 256, MLP_SIN = 16, MLP_K_OUT = 32;
// Internal parameter layout (FP32 masters): W1[64][256] (input rows 48 .. 63
// stay zero), b1[256], W2[256][256], b2[256], W3[256][32], b3[32]; W[in][out].
constexpr int64_t MLP_OFF_W1 = 0, MLP_OFF_B1 = MLP_INP * MLP_H,
                  MLP_OFF_W2 = MLP_OFF_B1 + MLP_H, MLP_OFF_B2 = MLP_OFF_W2 + MLP_H * MLP_H,
                  MLP_OFF_W3 = MLP_OFF_B2 + MLP_H, MLP_OFF_B3 = MLP_OFF_W3 + MLP_H * MLP_K_OUT,
                  MLP_P_INT = MLP_OFF_B3 + MLP_K_OUT;
// BF16 weight images (element offsets; layouts in mlp_tc.cuh): W2 for the
// forward product (4 chunks of 256 x 64), W1 (256 x 64), W3 forward (32 x 256),
// W2 for the backward product (4 chunks of 256 x 64), W3 backward (256 x 32).
constexpr int64_t MLP_IMG_W2F = 0, MLP_IMG_W1 = MLP_IMG_W2F + MLP_H * MLP_H,
                  MLP_IMG_W3F = MLP_IMG_W1 + MLP_INP * MLP_H,
                  MLP_IMG_W2B = MLP_IMG_W3F + MLP_H * MLP_K_OUT,
                  MLP_IMG_W3B = MLP_IMG_W2B + MLP_H * MLP_H,
                  MLP_IMG_TOTAL = MLP_IMG_W3B + MLP_H * MLP_K_OUT;
// Adam step counter and step size in device memory (zero = before step 1).
struct AdamState {
    int64_t t;
    float lr;
};
// state: 16 bytes of device memory holding an AdamState
cudaError_t launch_adam_set_lr(void *state, float lr, cudaStream_t st);
cudaError_t launch_fallback_mark(int64_t m, const int32_t *list, const int64_t *count,
                                 int32_t *status, cudaStream_t st);
// img (MLP_IMG_TOTAL BF16) from the FP32 masters th (MLP_P_INT)
cudaError_t launch_mlp_images(const float *th, void *img, cudaStream_t st);

// One CTA's slot of partial sums of a training step (floats): dW2 [256][256],
// dW1 [64][256], dW3 [256][32], db1 [4][256], db2 [4][256], db3 [4][32] (per
// TMEM lane quarter), loss [32] (per warp of the two CTAs of a cluster pair).
constexpr int64_t MLP_PART_W2 = 0, MLP_PART_W1 = MLP_PART_W2 + MLP_H * MLP_H,
                  MLP_PART_W3 = MLP_PART_W1 + MLP_INP * MLP_H,
                  MLP_PART_B1 = MLP_PART_W3 + MLP_H * MLP_K_OUT,
                  MLP_PART_B2 = MLP_PART_B1 + 4 * MLP_H, MLP_PART_B3 = MLP_PART_B2 + 4 * MLP_H,
                  MLP_PART_LOSS = MLP_PART_B3 + 4 * MLP_K_OUT, MLP_PART_STRIDE = 92416;
constexpr int MLP_GRAM_PARTS = 32;   // slices of G = V^T V, added in order
struct MlpTrainArgs {
    int64_t m, nnz;                   // batch rows B and their observations
    const int64_t *ptr;
    const int32_t *idx;
    const float *val;
    const float *ccap, *gcap;         // normalised CPU caps [n_cpu], GPU caps [n_gpu]
    int32_t n_gpu;                    // setting j = c * n_gpu + g
    int wait_limit;                   // polls of each pipeline wait before it gives up
    int64_t n;
    const void *img;                  // BF16 weight images
    const float *b1, *b2, *b3;        // FP32 biases
    const float *T;                   // B x 32 targets, 16-byte aligned
    const float *G;                   // 32 x 32, G = V^T V (launch_mlp_gram)
    float scale;                      // 2 / B
    float *part;                      // slots x MLP_PART_STRIDE (mlp_train_tc_slots)
    AdamState *adam;                  // advanced once (NULL: gradient only)
    int *err;                         // err[1] set when a bounded wait ran out
};
// slots of partial sums: one per cluster pair (at most num_sms / 2 tiles),
// else one per CTA of the one-CTA-per-tile kernel (mlp_train_tc1.cu)
int mlp_train_tc_slots(int64_t B, int num_sms);
cudaError_t prepare_mlp_train_tc();
cudaError_t prepare_mlp_train_tc1();
// pdl: launched as a programmatic dependent of the preceding kernel
cudaError_t launch_mlp_train_tc(const MlpTrainArgs &a, int num_sms, bool pdl, cudaStream_t st);
cudaError_t launch_mlp_train_tc1(const MlpTrainArgs &a, int grid, bool pdl, cudaStream_t st);
// G = V^T V (32 x 32) via MLP_GRAM_PARTS slices; ticket: one zeroed word, left zero
cudaError_t launch_mlp_gram(int64_t n, int KP, const float *V, float *Gpart, float *G,
                            unsigned int *ticket, cudaStream_t st);
struct MlpReduceArgs {
    const float *part;                // slots of the training kernel
    int ctas;
    float *th, *m1, *m2;              // FP32 masters and moments (MLP_P_INT)
    AdamState *adam;                  // NULL: gradient only (t moved back if the step failed)
    void *img;                        // BF16 images refreshed after the update
    float *grads_out;                 // gradient-only mode: external layout
    double *loss;                     // may be NULL
    int64_t B;
    const int *err;
};
cudaError_t launch_mlp_reduce_adam(const MlpReduceArgs &a, cudaStream_t st);

// Fused tcgen05 forward pass (mlp_tc.cu) over the images above.
struct MlpTcArgs {
    int64_t m, nnz;
    const int64_t *ptr;
    const int32_t *idx;
    const float *val;
    const float *ccap, *gcap;     // normalised CPU caps [n_cpu], GPU caps [n_gpu]
    int32_t n_gpu;                // setting j = c * n_gpu + g
    int wait_limit;               // polls of each pipeline wait before it gives up
    int64_t n;
    const void *img;              // BF16 weight images
    const float *b1, *b2, *b3;
    float *Y;                     // m x 32, 16-byte aligned
    const float *V;               // n x 32 setting factors (observed-entry residual)
    float threshold;              // fallback when the row's RMSE is above it (or not finite)
    float *row_rmse;              // m, may be null
    int32_t *status;              // m, may be null: OK or FALLBACK_USED
    int32_t *list;                // fallback rows, appended at list[*count]
    int64_t *count;
    int *err;                     // set to 1 when a bounded wait ran out
};
size_t mlp_forward_tc_smem();
cudaError_t prepare_mlp_forward_tc();
cudaError_t launch_mlp_forward_tc(const MlpTcArgs &a, int num_sms, cudaStream_t st);

// Reconstruction on the tensor cores fused with Algorithm 2 (predict_tc.cu):
// BF16-Gram precision mode, KP = 32.  Vimg: split BF16 operand images of V in
// chunks of 256 settings (launch_v_image; predict_tc_image_bytes(n) bytes).
constexpr int64_t PREDICT_TC_CG_MAX = 16384;   // c + g table kept in shared memory up to here
struct PredictTcArgs {
    int64_t m, n;
    const float *U;       // m rows of k floats, stride ldu
    int64_t ldu;
    int k;
    int wait_limit;       // polls of each pipeline wait before it gives up (fills the
                          // padding: the struct stays at 128 bytes, the size it was
                          // timed at)
    const void *Vimg;
    const float *cg;      // n: c_j + g_j
    const float *cg_pad;  // the same, zero-padded to whole chunks of 256 (used when n > PREDICT_TC_CG_MAX)
    int64_t base;
    float Ebase, gamma;
    bool select;          // run Algorithm 2
    float *T;             // m x n or null
    bool t_vec;           // T 16-byte aligned and n % 4 == 0
    int32_t *best;
    float *saving;
    int *err;
};
size_t predict_tc_image_bytes(int64_t n);
cudaError_t prepare_predict_tc();
cudaError_t launch_v_image(const float *V, int64_t n, void *img, cudaStream_t st);
cudaError_t launch_predict_select_tc(const PredictTcArgs &a, int num_sms, cudaStream_t st);

// Algorithm 1 over many power traces (phase.cu).
cudaError_t launch_phase_detect(const float *power, int64_t n_traces, int64_t len, int64_t ld,
                                float p_th, int32_t window, int64_t *first, cudaStream_t st);


// Reconstruction T = U V^T fused with Algorithm 2.
template <typename TV> struct PredictArgs {
    int64_t m, n;
    int KP, k;
    const TV *U;          // m rows, stride ldu
    int64_t ldu;
    const TV *V;          // n rows of KP (padded)
    const float *cg;      // [n] c_j + g_j in FP32 (null: no selection)
    int64_t base;         // baseline setting
    float Ebase;          // C_b + G_b in FP32
    float gamma;
    TV *T;                // [m, n] or null
    int32_t *best;        // [m] or null
    float *saving;        // [m] or null
};
template <typename TV> cudaError_t launch_predict_select(const PredictArgs<TV> &a, cudaStream_t st);

// Algorithm 2 on a given dense FP32 matrix.
cudaError_t launch_select(int64_t m, int64_t n, const float *T, int64_t ld, const float *cg,
                          int64_t base, float Ebase, float gamma, int32_t *best, float *saving,
                          cudaStream_t st);

// Objective J and per-row observed RMSE.  part: double[3 * objective_parts(max(m, n))].
int64_t objective_parts(int64_t m);
template <typename TV>
cudaError_t launch_objective(int64_t m, int64_t nnz, const int64_t *ptr, const int32_t *idx,
                             const TV *val, const TV *U, int64_t ldu, int k, const TV *V,
                             int64_t n, int KP, double lambda, double *part, double *J_out,
                             float *row_rmse, const int32_t *ccount, cudaStream_t st);
// ccount (int32[n], null = unweighted): observations per column for the
// weighted-lambda objective sum s_i |u_i|^2 + sum_j s_j |v_j|^2.
cudaError_t launch_col_counts_from_ptr(int64_t n, const int64_t *cptr, int32_t *cnt,
                                       cudaStream_t st);
cudaError_t launch_col_counts(int64_t nnz, int64_t n, const int32_t *idx, int32_t *cnt,
                              cudaStream_t st);

// Layout helpers.
template <typename TV>
cudaError_t launch_pack_rows(const TV *src, int64_t rows, int64_t lds, int k, TV *dst, int KP,
                             cudaStream_t st);                    // [rows,k] -> [rows,KP]
template <typename TV>
cudaError_t launch_unpack_rows(const TV *src, int64_t rows, int KP, int k, TV *dst,
                               cudaStream_t st);                  // [rows,KP] -> [rows,k]
cudaError_t launch_to_bf16(const float *src, int64_t count, void *dst, cudaStream_t st);
// rows of KP floats -> rows [bf16(x) (KP) | bf16(x - bf16(x)) (KP)]
cudaError_t launch_to_bf16_split(const float *src, int64_t rows, int KP, void *dst,
                                 cudaStream_t st);
template <typename TV>
cudaError_t launch_dense_to_csr(const TV *P, int64_t m, int64_t n, int64_t ld, int64_t *ptr,
                                int32_t *idx, TV *val, cudaStream_t st);
template <typename TV>
cudaError_t launch_validate_csr(int64_t m, int64_t n, int64_t nnz, const int64_t *ptr,
                                const int32_t *idx, const TV *val, int32_t *flag,
                                cudaStream_t st);


// Neural collaborative filtering (ncf.cu): embeddings d = 32 per side,
// MLP 64 -> 128 -> 64 -> 1 with SELU hidden units.
constexpr int NCF_D = 32, NCF_H1 = 128, NCF_H2 = 64;
constexpr int64_t NCF_OFF_B1 = 2 * NCF_D * NCF_H1;                   // net = W1 | b1 | W2 | b2 | w3 | b3
constexpr int64_t NCF_OFF_W2 = NCF_OFF_B1 + NCF_H1;
constexpr int64_t NCF_OFF_B2 = NCF_OFF_W2 + NCF_H1 * NCF_H2;
constexpr int64_t NCF_OFF_W3 = NCF_OFF_B2 + NCF_H2;
constexpr int64_t NCF_OFF_B3 = NCF_OFF_W3 + NCF_H2;
constexpr int64_t NCF_NET = NCF_OFF_B3 + 1;                            // 16641
constexpr int NCF_TT = 32;   // batch rows per CTA of the training kernel (partials per step: B / 32)
struct NcfCtl {                 // device-side position of a training run
    int64_t step;               // steps done (epoch = step / steps_per_epoch)
    unsigned long long skipped; // batch entries skipped for out-of-range indices
    int32_t beff;               // rows of the current batch
    int32_t pad;
};
struct NcfTrainArgs {            // k_ncf_train_tile: forward + backward of one batch
    NcfCtl *ctl;
    AdamState *adam;            // advanced once per step (NULL: gradient only)
    int64_t nnz, spe, m, n;     // entries, steps per epoch, applications, settings
    int B;                      // batch capacity (multiple of 64)
    const int32_t *perms;       // [epochs][nnz] visiting orders, or NULL (entries in order)
    const int32_t *app, *set;   // [nnz] indices of the observed entries
    const float *val;           // [nnz]
    const float *Ea, *Es;       // FP32 embedding tables [m][32], [n][32]
    const void *W1b, *W2b;      // BF16 copies of W1 [64][128] and W2 [128][64]
    const float *b1, *b2, *w3, *b3;   // FP32 parameters
    float *part;                // [B/32][part_stride] network-gradient partials (packed order)
    int64_t part_stride;
    float *lpart;               // [B/32] sums of squared residuals
    float *gE;                  // embedding gradients: Ea rows, then Es rows at s_off (NULL: none)
    int64_t s_off;
    // Dense-feature mode (the offline performance predictor): row e of the
    // input is feat[e][0 .. nfeat) padded with zeros to 64 (app, set, Ea, Es
    // unused).  y_out: the predictions of launch_pred_forward.
    const float *feat = nullptr;
    int nfeat = 0;
    float *y_out = nullptr;
};
struct NcfAdamArgs {            // k_ncf_reduce_adam: partials -> gradient -> Adam
    NcfCtl *ctl;
    const AdamState *adam;
    bool update;                // false: write the network gradient only
    int parts;
    const float *part;
    int64_t part_stride;
    const float *lpart;
    float *th, *grad, *m1, *m2; // packed [net (net_pad) | Ea | Es]
    int64_t net_pad, n_emb;
    void *bf;                   // BF16 W1 | W2
    double *loss_hist, *loss_last;
};
struct NcfPredArgs {
    int64_t m, n;
    const float *A;                 // [m][128] Ea W1[0:32] + b1
    const float *S;                 // [n][128] Es W1[32:64]
    const void *w2img;              // W2 as a UMMA operand image (16 KB)
    const float *b2, *w3, *b3;
    float *T;                       // [m][n]
    int *err;                       // set to 1 if a tensor-core wait ran out
    int wait_limit;                 // polls of each pipeline wait before it gives up
};
cudaError_t prepare_ncf_train();
cudaError_t launch_ncf_train_step(const NcfTrainArgs &t, const NcfAdamArgs &u, cudaStream_t st);
cudaError_t launch_ncf_refresh_bf(const float *theta, void *bf, cudaStream_t st);
// Predictions of the dense-feature network for t.nnz rows of t.feat into t.y_out
// (persistent: weights loaded once per CTA).
cudaError_t launch_pred_forward(const NcfTrainArgs &t, int num_sms, cudaStream_t st);
cudaError_t launch_ncf_first_layer(int64_t rows, const float *E, const float *W, const float *bias,
                                   float *out, cudaStream_t st);
cudaError_t launch_ncf_w2_image(const float *W2, void *img, cudaStream_t st);
cudaError_t prepare_ncf_predict_tc();
cudaError_t launch_ncf_predict_tc(const NcfPredArgs &a, int num_sms, cudaStream_t st);

}  // namespace ocf
