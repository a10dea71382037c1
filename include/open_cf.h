/*
 * open_cf.h -- C ABI of the B300 engine for the collaborative-filtering step
 * of OPEN's online phase (Zheng, Lan, Wu, Taylor, Papka: "Coordinated Power
 * Management on Heterogeneous Systems", arXiv 2508.07605).
 *
 * The paper's problem (Sec. "Putting it all together", Eq. 1; Sec. "Online
 * Performance Prediction"): a dense offline performance matrix P with one row
 * per profiled application and one column per (CPU cap, GPU cap) setting; a
 * new application is profiled online under a few settings, which appends a
 * sparse row; collaborative filtering fills in the rest of the row; and
 * Algorithm 2 picks the most energy-efficient setting within a loss bound.
 *
 * This library does the filling-in by regularised matrix factorisation
 * P ~ U V^T fitted with alternating least squares (the model of the
 * Netflix-prize work the paper cites for collaborative filtering, Sec.
 * "Collaborative Filtering Model"):
 *     J(U,V) = sum_{(i,j) observed} (R_ij - u_i . v_j)^2 + lambda (|U|_F^2 + |V|_F^2),
 * each half-step solving, per row i,
 *     (sum_{j in Omega_i} v_j v_j^T + lambda I) u_i = sum_{j in Omega_i} R_ij v_j.
 *
 * Conventions shared by every call
 *  - Settings are indexed CPU-major: j = c_idx * n_gpu_caps + g_idx.
 *  - Matrix entries are normalised runtimes (lower is faster).
 *  - Every array argument is a DEVICE pointer on cfg.device unless its name
 *    ends in _host.  The caller owns all arrays; nothing is retained after a
 *    call returns.  Arrays are C-contiguous (row-major).
 *  - "real" below means double when the handle's precision is OPEN_CF_FP64
 *    and float otherwise (OPEN_CF_FP32, OPEN_CF_BF16_GRAM).
 *  - Sparse inputs are CSR: row_ptr int64[m+1] with row_ptr[0] = 0,
 *    non-decreasing, row_ptr[m] = nnz; col int32[nnz] strictly increasing
 *    within a row, each in [0, n); val real[nnz], finite.  Kernels bounds-check
 *    row_ptr against nnz and col against n and mark offending rows with
 *    OPEN_CF_ROW_BAD_INPUT instead of reading out of bounds;
 *    open_cf_validate_csr checks every stated property.
 *  - Calls are asynchronous on `stream` (a cudaStream_t; NULL = legacy default
 *    stream).  A return of OPEN_CF_OK means the work is enqueued.  Argument
 *    errors are detected synchronously on the host and leave the handle
 *    unchanged.
 *  - A handle may be used by one host thread at a time.  What a handle keeps
 *    between calls (V and its BF16 copies and operand images, workspaces, the
 *    rank-32 row solver's pair counter) is written on the stream of the call
 *    that uses it; calls on different streams must be ordered by the caller
 *    (events), as for any shared buffer -- two row solves of one handle
 *    running at once on two streams would share that counter.  Use one handle
 *    per stream for concurrent solves.
 *  - Calls that run many kernels (fits, joint refits, streaming ingests, the
 *    learned path's training step) capture them once into a CUDA graph kept
 *    per argument set (sizes and array addresses; up to 16 per handle) and
 *    replay it: repeated calls on the same buffers cost one graph launch,
 *    new buffers a new capture.
 *  - There is no CPU fallback: every computation runs in this library's CUDA
 *    kernels for sm_103a.
 */
#ifndef OPEN_CF_H
#define OPEN_CF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Return codes. */
#define OPEN_CF_OK 0
#define OPEN_CF_INVALID_ARG (-1)
#define OPEN_CF_NOT_FITTED (-2)   /* no V set or fitted yet */
#define OPEN_CF_CUDA_ERROR (-3)
#define OPEN_CF_OUT_OF_MEMORY (-4)
#define OPEN_CF_UNSUPPORTED (-5)  /* k > OPEN_CF_MAX_K, device not sm_103 */
#define OPEN_CF_TIMEOUT (-6)

/* Per-row status codes written to status arrays. */
#define OPEN_CF_ROW_OK 0
#define OPEN_CF_ROW_NOT_SPD 1        /* a Cholesky pivot was not > 0; u = 0 */
#define OPEN_CF_ROW_EMPTY 2          /* no observation; u = 0 */
#define OPEN_CF_ROW_FALLBACK_USED 3  /* learned factor rejected, ALS used */
#define OPEN_CF_ROW_BAD_INPUT 4      /* row_ptr / col out of range; u = 0 */

#define OPEN_CF_MAX_K 32
/* Default bound of a tensor-core pipeline wait, in polls of mbarrier.try_wait. */
#define OPEN_CF_WAIT_POLLS_DEFAULT (1 << 22)

typedef struct open_cf open_cf_t; /* opaque: owns V, workspaces, CUDA graphs */

typedef enum {
    OPEN_CF_FP64 = 0,      /* FP64 values, factors, Gram and Cholesky */
    OPEN_CF_FP32 = 1,      /* FP32 values, factors, Gram and Cholesky */
    OPEN_CF_BF16_GRAM = 2  /* FP32 values and factors; Gram from BF16 copies of
                              the factors on tensor cores, FP32 accumulation */
} open_cf_precision;

typedef struct {
    int32_t k;                 /* latent rank, 1..OPEN_CF_MAX_K */
    double lambda;             /* ridge regulariser, > 0 */
    int32_t sweeps;            /* ALS sweeps of a fit (U-half then V-half), >= 0 */
    uint64_t seed;             /* reserved: random draws are passed in as inputs */
    open_cf_precision precision;
    int32_t cholesky_fp64;     /* 1: k x k factorisation in FP64 (FP32/BF16 modes) */
    int32_t n_cpu_caps;        /* cap grid for Algorithm 2; 0 = no grid */
    int32_t n_gpu_caps;
    const double *cpu_caps_w_host; /* n_cpu_caps watts, copied at create */
    const double *gpu_caps_w_host; /* n_gpu_caps watts, copied at create */
    int32_t device;            /* CUDA device ordinal */
    float mlp_fallback_threshold; /* observed-entry RMSE above which the learned
                                     factor is replaced by the ALS solve */
    int32_t weighted_lambda;   /* 1: weighted-lambda regularisation (ALS-WR of the
                                  ALS work the paper cites): every row / column
                                  solve uses lambda * (its observation count), and
                                  J weights |u_i|^2, |v_j|^2 by those counts */
} open_cf_config;

/* Create a handle.  Copies cfg and the cap grids.  Fails with
 * OPEN_CF_UNSUPPORTED if the device is not compute capability 10.3 or k is out
 * of range, OPEN_CF_INVALID_ARG for lambda <= 0 or a malformed cap grid. */
int open_cf_create(const open_cf_config *cfg, open_cf_t **out);

/* Release the handle and every device buffer it owns (synchronises the
 * device first).  NULL is ignored. */
void open_cf_destroy(open_cf_t *h);

/* Text of the last error on this handle ("" if none).  Valid until the next
 * call on the handle. */
const char *open_cf_last_error(const open_cf_t *h);

/* Watchdog of the tensor-core pipelines (reconstruction/selection, the
 * learned warm start's inference and training).  Every wait of those kernels
 * on an mbarrier (a bulk copy landing, tensor-core products finishing, a
 * buffer being released) is bounded; a wait that runs out sets a flag on the
 * device, the kernel stops issuing work, waits (again with a bound) for the
 * copies and products it already issued, frees its tensor memory and returns,
 * so the context stays usable.  What the flag means for the outputs:
 *   - open_cf_predict (tensor-core path): the rows of the CTAs that gave up
 *     hold unspecified values;
 *   - open_cf_mlp_infer: the rows of the tiles that gave up are solved by the
 *     ALS fold-in instead (status OPEN_CF_ROW_FALLBACK_USED), so U is correct;
 *   - open_cf_mlp_train_step: the step changes no parameter and reports NaN;
 *     while the flag is set every later step does the same.
 *
 * open_cf_set_wait_limit: the bound of those waits, in polls (0: a wait gives
 * up without polling, which makes every launch take its timeout path; -1: the
 * default, OPEN_CF_WAIT_POLLS_DEFAULT).  Host state only; applies to launches
 * enqueued after the call.  INVALID_ARG for polls < -1.
 *
 * open_cf_check: synchronises the device, then returns OPEN_CF_TIMEOUT (and
 * clears the flags; the text of open_cf_last_error names the kernels) if a
 * wait gave up since the last check, else OPEN_CF_OK. */
int open_cf_set_wait_limit(open_cf_t *h, int32_t polls);
int open_cf_check(open_cf_t *h);

/* Set the handle's V (n x k real): the initial V of the next fit (the random
 * draw of ALS's initialisation is passed in), or the fixed V of a fold-in.
 * If a cap grid was given, n must equal n_cpu_caps * n_gpu_caps. */
int open_cf_set_V(open_cf_t *h, const void *V, int64_t n, void *stream);

/* Copy the handle's current V (n x k real) out. */
int open_cf_get_V(open_cf_t *h, void *V_out, void *stream);

/* Offline fit on the dense offline block (Eq. 1; every entry observed):
 * P is m_off x n real with leading dimension ld >= n.  Runs cfg.sweeps ALS
 * sweeps from the V set by open_cf_set_V, keeps the fitted V (and the block,
 * for later joint refits) in the handle, and writes the offline factors to
 * U_out (m_off x k real, may be NULL).  J_hist (2 * sweeps doubles, may be
 * NULL) receives J after every half-step. */
int open_cf_fit_offline(open_cf_t *h, const void *P, int64_t m_off, int64_t n, int64_t ld,
                        void *U_out, double *J_hist, void *stream);

/* Sparse fit (extension): ALS sweeps on a CSR matrix of m rows and n columns
 * from the handle's V.  The CSC copy of the matrix is built on the device by
 * a stable counting sort.  U_out: m x k real (may be NULL); row_status and
 * col_status (int32, may be NULL) receive the codes of the last sweep;
 * J_hist as for open_cf_fit_offline. */
int open_cf_fit_csr(open_cf_t *h, int64_t m, int64_t n, int64_t nnz, const int64_t *row_ptr,
                    const int32_t *col, const void *val, void *U_out, int32_t *row_status,
                    int32_t *col_status, double *J_hist, void *stream);

/* Online completion (Sec. "Online Performance Prediction"): m_new new
 * applications, each with its few online-profiled entries as a CSR row.
 * joint = 0 (fold-in): every row is one independent ridge solve against the
 *   handle's fixed V; writes U_out (m_new x k real) and status (may be NULL).
 * joint = 1: re-runs cfg.sweeps sweeps over the offline block of the last
 *   open_cf_fit_offline plus the new rows, starting from the current V, and
 *   updates V; U_out receives the factors of the new rows. */
int open_cf_complete_rows(open_cf_t *h, int64_t m_new, int64_t nnz, const int64_t *row_ptr,
                          const int32_t *col, const void *val, void *U_out, int32_t *status,
                          int32_t joint, void *stream);

/* Online fold-in with the final residual check (extension of
 * open_cf_complete_rows with joint = 0; Sec. "Online Performance Prediction"
 * completes the new rows, the check verifies each row's normal equations).
 * For handles with 16 < k <= 32 in OPEN_CF_FP32 or OPEN_CF_BF16_GRAM precision
 * and the FP32 k x k factorisation (cholesky_fp64 = 0); other handles return
 * OPEN_CF_UNSUPPORTED.  U_out (m_new x k float) and status (may be NULL) as
 * for open_cf_complete_rows.
 *  resid (float[m_new], may be NULL): per row the relative residual of the
 *    normal equations the library formed (A_i = its Gram + lambda I, b_i its
 *    right-hand side, in the handle's Gram precision):
 *        |A_i u_i - b_i| / (|A_i|_F |u_i| + |b_i|),
 *    with b_i - A_i u_i evaluated in double-FP32 arithmetic (error-free
 *    products and sums, ~2^-44 relative), -1 for rows whose status is not OK.
 *  refine = 1: one step of iterative refinement: the correction A_i d = r_i
 *    (r_i that residual) is solved with the same FP32 factor and u_i += d;
 *    resid then reports the refined u_i, its residual formed as r_i - A_i D
 *    (D the step actually taken, in FP32: an error of ~k kappa eps^2 |A_i||u_i|,
 *    well below the residual of an FP32 u_i).  refine = 0: no refinement. */
int open_cf_complete_rows_checked(open_cf_t *h, int64_t m_new, int64_t nnz,
                                  const int64_t *row_ptr, const int32_t *col, const float *val,
                                  float *U_out, int32_t *status, float *resid, int32_t refine,
                                  void *stream);

/* The same relative normal-equation residual for given factors U (m x k float)
 * of the CSR rows against the handle's V (the residual part of the a9
 * objective/residual step): resid float[m], every row computed (an empty row
 * gives |lambda u| / (lambda sqrt(k) |u|)).  Same handle requirements as
 * open_cf_complete_rows_checked. */
int open_cf_normal_residual(open_cf_t *h, int64_t m, int64_t nnz, const int64_t *row_ptr,
                            const int32_t *col, const float *val, const float *U, float *resid,
                            void *stream);

/* Reconstruction and Algorithm 2 (energy-efficient power-cap selection) on
 * the predicted rows T = U V^T, U m x k real.  T_out (m x n real) may be NULL,
 * in which case the dense prediction never leaves the chip; best (int32[m])
 * and saving (float[m]) may be NULL.  Per row, with t the predicted runtimes:
 *   p_j = t_base / t_j, valid if t_j > 0 and 1 - p_j <= gamma,
 *   E_j = (c_j + g_j) / p_j, saving_j = (E_base - E_j) / E_base,
 *   E_base = C_b + G_b, best = argmax saving (ties: smaller c + g, then smaller j).
 * The selection is evaluated in FP32 in exactly that operation order.
 * baseline_setting = -1 selects (max CPU cap, max GPU cap).  A row whose
 * baseline runtime is not > 0 gets best = -1 and saving = 0.  Needs a cap grid
 * when best or saving is requested.
 * Precision: FP32 / FP64 modes form T with FMA chains in the handle's type.
 * OPEN_CF_BF16_GRAM with 16 < k <= 32 forms T on the tensor cores from split
 * BF16 copies of U and V (hi + lo, FP32 accumulation; predicted runtimes
 * within ~2^-16 relative of FP32); the selection is then exact on that T,
 * the values T_out receives. */
int open_cf_predict(open_cf_t *h, const void *U, int64_t m, void *T_out, int32_t *best,
                    float *saving, float gamma, int32_t baseline_setting, void *stream);

/* The online phase end to end from HOST memory (Sec. "Online Performance
 * Prediction" then Sec. "Optimal Power setting Selection"): the fold-in of m new
 * rows (open_cf_complete_rows with joint = 0, or open_cf_complete_rows_checked)
 * followed by open_cf_predict's Algorithm 2, for a caller whose CSR lives in
 * host memory and who wants the decisions back in host memory.  The rows are
 * processed in chunks (chunk_rows rows, rounded up to a multiple of 256 and to
 * at most 1024 chunks; 0 = about m / 16, at least 32,768, rounded up to 128 rows
 * per SM): the
 * host-to-device copies of chunk c + 1 run on a copy
 * stream of the handle while chunk c is solved on `stream`, so the copies
 * overlap the solves.  Every chunk is solved as its own CSR, giving the results
 * separate calls on its rows would give.
 *  row_ptr (int64[m + 1], host; row_ptr[0] = 0, row_ptr[m] = nnz,
 *    non-decreasing), col (host; col_bytes = 4: int32[nnz]; col_bytes = 2:
 *    uint16[nnz], for up to 65,535 settings, a quarter fewer bytes over the host
 *    link; widened on the device), val (float[nnz], host): the CSR.
 *    Page-locked (pinned) host memory is needed for the copies to overlap
 *    anything; pageable memory works but serialises them.
 *  check = 0: plain fold-in; 1: with the residual check; 2: with the residual
 *    check and one refinement step (check >= 1: same handle requirements as
 *    open_cf_complete_rows_checked).
 *  gamma, baseline_setting: as for open_cf_predict (a cap grid is required).
 *  best (int32[m], host), saving (float[m], host): Algorithm 2's decisions;
 *  status (int32[m], host, may be NULL), resid (float[m], host, may be NULL;
 *    check >= 1 only): as for open_cf_complete_rows_checked.
 * The host arrays must stay valid and unchanged, and the outputs unread, until
 * `stream` has completed the call's work (the call only enqueues; row_ptr is
 * read on the host at the chunk boundaries during the call).  The handle keeps
 * device copies of the inputs and outputs (grown to the largest call) and the
 * factors of the last call; calls on one handle must not overlap on different
 * streams.  FP32 / BF16-Gram handles; FP64 handles return OPEN_CF_UNSUPPORTED. */
int open_cf_complete_select_host(open_cf_t *h, int64_t m, int64_t nnz, const int64_t *row_ptr,
                                 const void *col, int32_t col_bytes, const float *val,
                                 int32_t check,
                                 float gamma, int32_t baseline_setting, int32_t *best,
                                 float *saving, int32_t *status, float *resid,
                                 int64_t chunk_rows, void *stream);

/* Algorithm 2 alone on a given dense matrix T (m x n float, ld >= n), as in
 * open_cf_predict. */
int open_cf_select(open_cf_t *h, const float *T, int64_t m, int64_t ld, int32_t *best,
                   float *saving, float gamma, int32_t baseline_setting, void *stream);

/* Objective J(U, V) of the CSR matrix against the given U (m x k real) and the
 * handle's V, accumulated in FP64 in a fixed order: J_out (one double) and
 * row_rmse (float[m], may be NULL: RMSE over each row's observed entries). */
int open_cf_objective(open_cf_t *h, int64_t m, int64_t nnz, const int64_t *row_ptr,
                      const int32_t *col, const void *val, const void *U, double *J_out,
                      float *row_rmse, void *stream);

/* CSR -> CSC by a stable counting sort on the device (entries of a column in
 * increasing row order): col_ptr int64[n+1], row_idx int32[nnz], cval real[nnz].
 * Uses handle-owned scratch of n * nb int32 counters (nb <= 4096 row blocks). */
int open_cf_csr_to_csc(open_cf_t *h, int64_t m, int64_t n, int64_t nnz, const int64_t *row_ptr,
                       const int32_t *col, const void *val, int64_t *col_ptr, int32_t *row_idx,
                       void *cval, void *stream);

/* Check every stated CSR property on the device; synchronises `stream` and
 * writes 0 (valid) or the first failed check to *result_host:
 * 1 row_ptr, 2 column range, 3 column order/duplicate, 4 non-finite value. */
int open_cf_validate_csr(open_cf_t *h, int64_t m, int64_t n, int64_t nnz, const int64_t *row_ptr,
                         const int32_t *col, const void *val, int32_t *result_host,
                         void *stream);

/* Batched completion (extension): P independent completion problems of
 * uneven size -- each its own apps x settings matrix with its own rank k_p --
 * fitted with cfg.sweeps ALS sweeps each (cfg.lambda) in one persistent,
 * graph-captured launch.  Handle precision must be OPEN_CF_FP32.
 *  m_host, n_host, k_host, nnz_host: per-problem sizes (host, P entries);
 *    1 <= n_p <= 1024, 1 <= k_p <= OPEN_CF_MAX_K, sum of nnz_host = nnz.
 *  row_ptr: int64[sum m_p + 1], the problems' CSR rows stacked in problem
 *    order, with global entry offsets; col: int32[nnz] column indices LOCAL to
 *    each problem (0 <= col < n_p); val: float[nnz].
 *  V_inout: float, the problems' n_p x k_p initial V stacked in problem order
 *    (the random initialisation is passed in); overwritten with the fitted V.
 *  U_out: float, the problems' m_p x k_p factors stacked (may be NULL).
 * Problems are ordered by estimated cost and split into a large and a small
 * class with their own warps per problem (see open_cf_batched_tune). */
int open_cf_batched_fit(open_cf_t *h, int64_t P, const int64_t *m_host, const int64_t *n_host,
                        const int32_t *k_host, const int64_t *nnz_host, int64_t nnz,
                        const int64_t *row_ptr, const int32_t *col, const float *val,
                        float *V_inout, float *U_out, void *stream);

/* Autotuner of the batched fit: times 2-sweep trial runs in a coordinate
 * search over the launch's tile shape -- warps per problem of the large class
 * {2, 4, 8} and of the small class {1, 2, 4} (9 pairs), then the share of each
 * padded rank's cost given to the large class {30, 50, 70} %, then the CTAs
 * per SM {1, 2} -- keeps the fastest setting in the handle for later
 * open_cf_batched_fit calls and writes it to W_out_host[4] = {warps large,
 * warps small, cut %, CTAs per SM} (may be NULL).
 * V_scratch receives trial results (same layout as V_inout; pass a copy of
 * the initial V).  Synchronises `stream`. */
int open_cf_batched_tune(open_cf_t *h, int64_t P, const int64_t *m_host, const int64_t *n_host,
                         const int32_t *k_host, const int64_t *nnz_host, int64_t nnz,
                         const int64_t *row_ptr, const int32_t *col, const float *val,
                         float *V_scratch, int32_t *W_out_host, void *stream);

/* Algorithm 1 (phase-transition detection, Sec. "Online Performance
 * Prediction") over many monitored jobs at once.  power: n_traces rows of len
 * GPU power readings (float watts, one every delta seconds; row t starts at
 * power + t * ld, ld >= len), device memory.  window = W / delta (25 for the
 * paper's delta = 0.2 s, W = 5 s); p_th the power threshold (60 W).
 * first (int64[n_traces], device) receives, per trace, the index of the
 * reading on which the algorithm reports a transition -- the first reading
 * that ends `window` consecutive readings none of which is below p_th -- or
 * -1.  A reading that is not a number is not below p_th.  Needs no handle;
 * OPEN_CF_INVALID_ARG for window < 1, ld < len, a non-finite p_th or NULL
 * arrays, OPEN_CF_CUDA_ERROR if the launch fails. */
int open_cf_phase_detect(const float *power, int64_t n_traces, int64_t len, int64_t ld,
                         float p_th, int32_t window, int64_t *first, void *stream);

/* ---- Learned warm start (Sec. "Collaborative Filtering Model": the paper's
 * CF model is an MLP with SELU activations; Sec. "Online Performance
 * Prediction": fill in a new application's row from its online profile).
 * An MLP maps an application's first 16 observed settings, each encoded as
 * (CPU cap, GPU cap, runtime) with caps scaled to [0, 1] over the grid (48
 * inputs), through 256 -> 256 SELU units to its factor u (k = 32 outputs).
 * Training targets are factors from the ALS fold-in; the loss is
 * (1/B) sum_r (u_r - u*_r)^T (V^T V) (u_r - u*_r), the squared error of the
 * predicted row u V^T.  Products run on BF16 tensor cores with FP32
 * accumulation; parameters, gradients and Adam moments are FP32.
 * Requirements: k = 32, precision FP32 or BF16_GRAM, V set, cap grid given
 * in the config; otherwise OPEN_CF_UNSUPPORTED / OPEN_CF_NOT_FITTED /
 * OPEN_CF_INVALID_ARG. */

/* Parameter vector (float, device), 86,560 entries in this order:
 * W1[48][256], b1[256], W2[256][256], b2[256], W3[256][32], b3[32]; each W is
 * [inputs][outputs] row-major.  Setting the parameters resets Adam. */
#define OPEN_CF_MLP_PARAMS 86560
int open_cf_mlp_set_params(open_cf_t *h, const float *params, void *stream);
int open_cf_mlp_get_params(open_cf_t *h, float *params_out, void *stream);

/* One training step on a batch of B rows (CSR as everywhere; the first 16
 * entries of each row form its features) with targets U_target (B x 32
 * float).  loss_out (one double, device, may be NULL) receives the loss
 * before the update.  grads_out NULL: Adam update (beta1 0.9, beta2 0.999,
 * eps 1e-8, step size lr).  grads_out non-NULL (OPEN_CF_MLP_PARAMS floats):
 * the gradient is written there and the parameters are left unchanged.
 * B <= 2^20. */
int open_cf_mlp_train_step(open_cf_t *h, int64_t B, int64_t nnz, const int64_t *row_ptr,
                           const int32_t *col, const float *val, const float *U_target, float lr,
                           double *loss_out, float *grads_out, void *stream);

/* Warm-started online completion: U_out (m x 32 float) = MLP(features of
 * each row); then the observed-entry RMSE of every row under U_out V^T
 * (row_rmse, m floats, may be NULL) decides the fallback: a row whose RMSE is
 * above cfg.mlp_fallback_threshold (or not finite) is re-solved by the ridge
 * fold-in of open_cf_complete_rows.  status (int32[m], may be NULL):
 * OPEN_CF_ROW_OK (MLP factor kept), OPEN_CF_ROW_FALLBACK_USED (ALS factor),
 * or the fold-in's own code for a fallback row it could not solve.  A row
 * with no observations keeps the MLP's output (RMSE 0). */
int open_cf_mlp_infer(open_cf_t *h, int64_t m, int64_t nnz, const int64_t *row_ptr,
                      const int32_t *col, const float *val, float *U_out, int32_t *status,
                      float *row_rmse, void *stream);

/* Streaming refit of V (Sec. "Online Performance Prediction": new
 * applications join the matrix and V is refitted with them), done
 * incrementally.  The handle keeps, for every setting j, the sums of the
 * V-half-step's normal equations over all rows ingested so far,
 *     G_j = sum_i u_i u_i^T,  b_j = sum_i R_ij u_i,  s_j = observations,
 * so that V = argmin over every ingested row with its factor held fixed:
 *     v_j = (G_j + lambda_j I)^{-1} b_j   (lambda_j = lambda, or lambda s_j when
 *                                          cfg.weighted_lambda), 0 if s_j = 0.
 * FP32 or FP64 precision (UNSUPPORTED in BF16_GRAM mode); workspace
 * n * KP * (KP + 1) reals + 8n bytes (KP = k padded to 8, 16 or 32).
 *
 * open_cf_stream_begin: seed the sums with m rows (CSR as everywhere) and their
 * factors U (m x k real, e.g. the offline block and the U of its fit), then
 * solve V.  Needs V set (it fixes n); a later open_cf_set_V ends the stream.
 * open_cf_stream_ingest: a batch of new applications: fold-in of each row
 * against the current V (U_out m_new x k real, status as open_cf_complete_rows),
 * their terms added to the sums, every v_j re-solved into the handle's V. */
int open_cf_stream_begin(open_cf_t *h, int64_t m, int64_t nnz, const int64_t *row_ptr,
                         const int32_t *col, const void *val, const void *U, void *stream);
int open_cf_stream_ingest(open_cf_t *h, int64_t m_new, int64_t nnz, const int64_t *row_ptr,
                          const int32_t *col, const void *val, void *U_out, int32_t *status,
                          void *stream);
/* The sums themselves, for a refit sharded over several processes (each adds
 * its rows' terms, the processes sum their increments, each installs the
 * totals): open_cf_stream_sums copies G (n x KP x KP real, row-major per
 * setting), b (n x KP real) and the counts (n int64) out (any output may be
 * NULL); open_cf_stream_set_sums installs such sums and re-solves every v_j
 * from them.  NOT_FITTED before open_cf_stream_begin. */
int open_cf_stream_sums(open_cf_t *h, void *G_out, void *b_out, int64_t *n_out, void *stream);
int open_cf_stream_set_sums(open_cf_t *h, const void *G, const void *b, const int64_t *n_obs,
                            void *stream);

/* FMA-loop microbenchmark (a measurement service, no counterpart in the
 * paper): the FP32 (fp64 = 0) or FP64 (fp64 = 1) fused multiply-add
 * throughput of `device` in TFLOP/s (2 FLOP per FMA), measured with CUDA
 * events over one launch of independent FMA chains on every SM; the
 * denominator of the ALU rooflines.  Synchronous; runs on the legacy default
 * stream of `device`. */
int open_cf_fma_peak(int32_t fp64, int32_t device, double *tflops_host);

/* Allocation-free CSR -> CSC (no counterpart in the paper; a service of this
 * library).  Some callers cannot allocate device memory: their host framework
 * owns every device allocation through its own pool and forbids direct
 * cudaMalloc, their latency path cannot absorb the device-wide
 * synchronisation of cudaMalloc/cudaFree, or they run under a fixed memory
 * budget set at start-up.  This call performs the same stable counting sort as
 * open_cf_csr_to_csc on FP32 values, needs no handle and allocates nothing:
 * its scratch (column totals and per-row-block column counters) is one
 * file-scope device array of OPEN_CF_NOALLOC_SCRATCH_BYTES that every GPU
 * loading this library holds until the process exits.  The caller still
 * provides every input and output (device pointers on the current device):
 * row_ptr int64[m+1], col int32[nnz], val float[nnz]; col_ptr int64[n+1],
 * row_idx int32[nnz], cval float[nnz].
 *  - Every call looks up the array's device address on the current device
 *    and sets the sort kernels' shared-memory limit (host-side calls that
 *    allocate nothing, repeated so that a device reset cannot leave a stale
 *    address).  The first call on a device also loads this library's module
 *    there: make that first call before any stream capture begins.
 *  - All calls share the one array, so calls whose work overlaps on the GPU
 *    (different streams, or different host threads) race and corrupt each
 *    other's results; serialise them.  Each call overwrites every counter it
 *    reads, so nothing has to be cleared between calls.
 *  - n > OPEN_CF_NOALLOC_MAX_COLUMNS returns OPEN_CF_UNSUPPORTED (the sort's
 *    per-column shared-memory counters bound n, as for the handle path); the
 *    outputs are then left untouched.
 *  - Speed: rows are sorted in at most (4 MiB - 8n rounded up to 256 B) / 4n
 *    row blocks of one CTA each (254 at n = 4096, 39 at n = 25,000), where
 *    the handle path uses up to 4096; wide matrices with many rows therefore
 *    sort more slowly through this call.  Bad sizes or NULL pointers return
 *    OPEN_CF_INVALID_ARG; a CUDA failure returns OPEN_CF_CUDA_ERROR.
 * Work is enqueued on `stream` (NULL = legacy default stream). */
#define OPEN_CF_NOALLOC_SCRATCH_BYTES (4 * 1024 * 1024)
#define OPEN_CF_NOALLOC_MAX_COLUMNS 25000 /* the transpose's shared-memory counter limit */
int open_cf_csr_to_csc_noalloc(int64_t m, int64_t n, int64_t nnz, const int64_t *row_ptr,
                               const int32_t *col, const float *val, int64_t *col_ptr,
                               int32_t *row_idx, float *cval, void *stream);

/* Checkpoint and resume (extension; the paper has no counterpart): the state
 * a handle has learned or accumulated, written to host memory and restored
 * into a handle of the same configuration, so that a fit, the learned path's
 * training or the streaming refit can stop and continue with results
 * bit-identical to an uninterrupted run.  The checkpoint holds a header (the
 * configuration: k, precision, factorisation, lambda, weighting; the number of
 * settings; the cap grid), then each part the handle has: V (as the handle
 * keeps it), the learned warm start's FP32 parameters with their Adam moments
 * and step state, the streaming refit's per-setting sums; and an FNV-1a 64-bit
 * checksum of all of it.  Little-endian.
 * open_cf_save: buf (host, cap bytes) receives the checkpoint; with buf NULL
 *   only *size_out is set (the size needed).  Waits for all work on the device
 *   (cudaDeviceSynchronize) first.  OPEN_CF_INVALID_ARG if cap is too small.
 * open_cf_load: restores a checkpoint of `size` bytes (host) into h, which must
 *   have been created with the same k, precision, cholesky_fp64, lambda,
 *   weighted_lambda and cap grid; anything else, a bad checksum or a truncated
 *   buffer returns OPEN_CF_INVALID_ARG and leaves h unchanged.  Synchronous.
 *   The offline block kept for joint refits, workspaces and captured graphs
 *   are not part of a checkpoint. */
int open_cf_save(open_cf_t *h, void *buf, int64_t cap, int64_t *size_out);
int open_cf_load(open_cf_t *h, const void *buf, int64_t size);

#ifdef __cplusplus
}
#endif

#endif /* OPEN_CF_H */
