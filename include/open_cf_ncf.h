/*
 * open_cf_ncf.h -- C ABI of neural collaborative filtering on the B300, the
 * CF model of OPEN (arXiv 2508.07605, Sec. "Collaborative Filtering Model";
 * He et al., "Neural Collaborative Filtering", 2017).
 *
 * Model.  The application index i and the power-cap-pair index j select rows
 * of two embedding tables, Ea [m][32] and Es [n][32]; the rows are
 * concatenated into x = [Ea_i, Es_j] (64 values) and passed through an MLP
 * with SELU hidden units (Klambauer et al. 2017 constants) and one linear
 * output, the predicted entry P_ij of the performance matrix (Eq. 1):
 *     z1 = x W1 + b1 (128),  z2 = SELU(z1) W2 + b2 (64),  y = SELU(z2) . w3 + b3.
 * Training minimises the mean squared error over mini-batches of observed
 * entries with Adam (beta1 0.9, beta2 0.999, eps 1e-8) on all parameters,
 * embeddings included (dense moments, as torch.optim.Adam on dense tensors).
 * Completion evaluates y for every application and setting and, optionally,
 * runs Algorithm 2 on each application's row (same FP32 evaluation and tie
 * rules as open_cf_predict / open_cf_select).
 *
 * Precision.  Parameters, gradients and Adam moments are FP32.  Products run
 * on tensor cores with FP32 accumulation: training on BF16 operands (mma.sync,
 * forward and backward of 32 batch rows per CTA in one kernel); completion on
 * FP16 operands (tcgen05, TMEM accumulators), its hidden activations formed in
 * packed FP16 pairs.  The first layer of the completion is evaluated in FP32
 * as Ea_i W1[0:32] + b1 plus Es_j W1[32:64] (the same value as the
 * concatenated product up to rounding).
 *
 * Conventions (as in open_cf.h): array arguments are DEVICE pointers on the
 * handle's device unless the name ends in _host; the caller owns them; calls
 * are asynchronous on `stream` (a cudaStream_t, NULL = legacy default
 * stream); argument errors are reported synchronously and leave the handle
 * unchanged; one host thread at a time per handle; no CPU fallback.
 * Return codes are the OPEN_CF_* codes of open_cf.h.
 */
#ifndef OPEN_CF_NCF_H
#define OPEN_CF_NCF_H

#include <stdint.h>

#include "open_cf.h"

#ifdef __cplusplus
extern "C" {
#endif

#define OPEN_CF_NCF_D 32     /* embedding width per side */
#define OPEN_CF_NCF_H1 128   /* first hidden layer */
#define OPEN_CF_NCF_H2 64    /* second hidden layer */
/* Network parameters, float, in this order: W1[64][128], b1[128],
 * W2[128][64], b2[64], w3[64], b3[1] (W as [inputs][outputs] row-major). */
#define OPEN_CF_NCF_NET 16641

typedef struct open_cf_ncf open_cf_ncf_t;

/* m applications; the n = n_cpu * n_gpu settings of the cap grid (watts, on
 * the host, CPU-major: j = c_idx * n_gpu + g_idx; the grid is used by
 * Algorithm 2, the baseline setting defaults to (max CPU cap, max GPU cap));
 * batch: training mini-batch capacity, a multiple of 64 in [64, 65536].
 * Allocates every workspace (about 4 (m + n) * 32 * 4 bytes of parameters and
 * moments plus O(batch) bytes).  UNSUPPORTED if the device is not sm_103. */
int open_cf_ncf_create(int64_t m, int32_t n_cpu, const double *cpu_caps_w_host, int32_t n_gpu,
                       const double *gpu_caps_w_host, int32_t batch, int device,
                       open_cf_ncf_t **out);
void open_cf_ncf_destroy(open_cf_ncf_t *h);
const char *open_cf_ncf_last_error(const open_cf_ncf_t *h);

/* Parameters in: net (OPEN_CF_NCF_NET floats), Ea (m x 32), Es (n x 32).
 * Resets Adam (moments and step count). */
int open_cf_ncf_set_params(open_cf_ncf_t *h, const float *net, const float *Ea, const float *Es,
                           void *stream);
/* Parameters out (any of the three may be NULL). NOT_FITTED before set_params. */
int open_cf_ncf_get_params(open_cf_ncf_t *h, float *net, float *Ea, float *Es, void *stream);

/* Mini-batch training over the nnz observed entries (app[e], setting[e],
 * val[e]) (int32, int32, float): epoch t visits them in the order
 * perms[t * nnz + 0 .. nnz - 1] (int32, a permutation of 0 .. nnz - 1 per
 * epoch; the random draw of the method is an input) in consecutive batches
 * of the handle's batch size, the last one of an epoch shorter; each batch is
 * one Adam step of step size lr on L = (1/B) sum_b (y_b - r_b)^2.
 * loss_out (double[epochs * ceil(nnz / batch)], may be NULL) receives each
 * step's loss before its update.  An entry whose application, setting or
 * position is out of range is skipped (it contributes nothing; B still counts
 * it) and counted (open_cf_ncf_skipped).  nnz in [1, 2^31 - 1], epochs >= 0. */
int open_cf_ncf_train(open_cf_ncf_t *h, int64_t nnz, const int32_t *app, const int32_t *setting,
                      const float *val, int32_t epochs, const int32_t *perms, float lr,
                      double *loss_out, void *stream);

/* The gradient of L on one batch of B <= batch entries (taken in order), with
 * no update: loss_out (1 double, may be NULL), g_net (OPEN_CF_NCF_NET floats),
 * g_Ea (m x 32), g_Es (n x 32) (each may be NULL). */
int open_cf_ncf_grad(open_cf_ncf_t *h, int64_t B, const int32_t *app, const int32_t *setting,
                     const float *val, double *loss_out, float *g_net, float *g_Ea, float *g_Es,
                     void *stream);

/* Completion of every application's row: T_out (m x n float, may be NULL)
 * receives y(i, j); best (int32[m]) and saving (float[m]) (either may be
 * NULL) receive Algorithm 2's choice with loss bound gamma and the baseline
 * setting (-1: the default).  With T_out NULL and a selection requested, T is
 * kept in a workspace of m * n floats. */
int open_cf_ncf_predict(open_cf_ncf_t *h, float *T_out, float gamma, int32_t baseline_setting,
                        int32_t *best, float *saving, void *stream);

/* Synchronising queries: entries skipped for out-of-range indices since the
 * last set_params (*count_host), and the tensor-core watchdog: returns
 * OPEN_CF_TIMEOUT (and clears the flag) if a completion kernel gave up on a
 * wait (its tiles are then NaN), else OPEN_CF_OK. */
int open_cf_ncf_skipped(open_cf_ncf_t *h, int64_t *count_host);
int open_cf_ncf_check(open_cf_ncf_t *h);
/* Bound of the completion kernel's tensor-core waits, in polls (0: every wait
 * gives up at once; -1: OPEN_CF_WAIT_POLLS_DEFAULT), as open_cf_set_wait_limit
 * does for the ALS handle.  Host state only.  INVALID_ARG for polls < -1. */
int open_cf_ncf_set_wait_limit(open_cf_ncf_t *h, int32_t polls);

/* ------------------------------------------------------------------------
 * Offline performance predictor (Sec. "Performance Prediction Model"): an MLP
 * from n_features per-run inputs (the paper's seven: CPU cap, GPU cap, memory
 * throughput, IPS, SM clock, DRAM active, FP active, each scaled by the caller)
 * to the run's normalised performance, the same network shape as the NCF
 * model's MLP (inputs zero padded to 64, 128 -> 64 SELU units, one linear
 * output), trained with the same kernels on the mean squared error.  Its
 * predictions for an application's online-profiled runs are the observed
 * entries of the sparse row the completion fills in (Sec. "Online Performance
 * Prediction").
 *
 * Parameters (float), n_features * 128 + 8449 entries in this order:
 * W1[n_features][128], b1[128], W2[128][64], b2[64], w3[64], b3[1]. */
typedef struct open_cf_pred open_cf_pred_t;

/* n_features in [1, 64]; batch a multiple of 64 in [64, 65536]. */
int open_cf_pred_create(int32_t n_features, int32_t batch, int device, open_cf_pred_t **out);
void open_cf_pred_destroy(open_cf_pred_t *h);
const char *open_cf_pred_last_error(const open_cf_pred_t *h);
/* Resets Adam. */
int open_cf_pred_set_params(open_cf_pred_t *h, const float *params, void *stream);
int open_cf_pred_get_params(open_cf_pred_t *h, float *params, void *stream);
/* N samples: X [N][n_features] (float), y [N] (float); epochs of mini-batch
 * Adam as open_cf_ncf_train (perms [epochs][N] int32; loss_out
 * double[epochs * ceil(N / batch)] or NULL). */
int open_cf_pred_train(open_cf_pred_t *h, int64_t N, const float *X, const float *y,
                       int32_t epochs, const int32_t *perms, float lr, double *loss_out,
                       void *stream);
/* Gradient of one batch of B <= batch samples, no update (g_params in the
 * parameter layout above; either output may be NULL). */
int open_cf_pred_grad(open_cf_pred_t *h, int64_t B, const float *X, const float *y,
                      double *loss_out, float *g_params, void *stream);
/* y_out[N] = the predicted normalised performance of every sample. */
int open_cf_pred_infer(open_cf_pred_t *h, int64_t N, const float *X, float *y_out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* OPEN_CF_NCF_H */
