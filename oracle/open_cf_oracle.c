/*
 * FP64 CPU oracle for the OPEN online-phase completion path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product (the CUDA library and its
 * Python binding) links, includes or calls this file; only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark use it.  It shares
 * no source with the CUDA path.
 *
 * What it computes, in plain loops, in the order the method states it:
 *
 *  - Matrix completion of the performance matrix P (Eq. 1; rows are
 *    applications, columns are CPU x GPU power-cap settings) from its observed
 *    entries, the collaborative-filtering step of the online phase (Sec.
 *    "Collaborative Filtering Model", Sec. "Online Performance Prediction").
 *    The factorisation model is the one of the cited Netflix-prize paper
 *    (Zhou et al. 2008): P ~ U V^T, fitted by alternating least squares with
 *    a ridge term, objective
 *        J(U,V) = sum_{(i,j) observed} (R_ij - u_i.v_j)^2
 *                 + lambda (sum_i |u_i|^2 + sum_j |v_j|^2)        (unweighted lambda)
 *    Each half-step solves, for every row i independently,
 *        (sum_{j in Omega_i} v_j v_j^T + lambda I) u_i = sum_{j in Omega_i} R_ij v_j
 *    by a Cholesky factorisation (no explicit inverse).
 *  - Algorithm 2 (energy-efficient power-cap selection) on a completed matrix,
 *    in FP64 and, for bit-exact comparison of the integer decision, in FP32.
 *  - The MLP of the learned warm start (SELU activations as named in Sec.
 *    "Collaborative Filtering Model"), forward, backward and Adam, in FP64.
 *  - The streaming refit of V: per-setting sums of the V-half-step's normal
 *    equations, grown by each batch of new applications, and the re-solve.
 *  - Neural collaborative filtering, the CF model that section describes
 *    (application and power-cap-pair embeddings, concatenated, through a SELU
 *    MLP to one predicted entry): forward, mean-squared-error gradient incl.
 *    the embedding rows, and the completed matrix.
 *
 * Parity pins (tests/test_oracle_*.py) check this code against numpy's lstsq
 * and cholesky, closed forms (Sherman-Morrison, soft-thresholded SVD),
 * objective monotonicity, normal-equation residuals, exact recovery,
 * hand-computed Algorithm 2 tables and finite differences; the NCF routines
 * against PyTorch's FP64 autograd and Adam, finite differences and invariants
 * (tests/test_oracle_ncf.py); the streaming refit against the batch half-step
 * over the union of ingested rows and numpy's lstsq (tests/test_oracle_stream.py).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_NOT_SPD 1
#define ORC_EMPTY_ROW 2
#define ORC_FALLBACK_USED 3

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_num_threads(int t) {
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

/* ------------------------------------------------------------------------ */
/* Cholesky factorisation A = L L^T of a k x k SPD matrix (row-major),
 * Cholesky-Banachiewicz order.  L is written row-major, upper part zeroed.
 * Returns ORC_NOT_SPD when a pivot is not strictly positive. */
int orc_cholesky(int k, const double *A, double *L) {
    memset(L, 0, sizeof(double) * (size_t)k * k);
    for (int i = 0; i < k; ++i) {
        for (int j = 0; j <= i; ++j) {
            double s = A[i * k + j];
            for (int p = 0; p < j; ++p) s -= L[i * k + p] * L[j * k + p];
            if (i == j) {
                if (!(s > 0.0)) return ORC_NOT_SPD;
                L[i * k + i] = sqrt(s);
            } else {
                L[i * k + j] = s / L[j * k + j];
            }
        }
    }
    return ORC_OK;
}

/* Solve L L^T x = b: forward substitution L y = b, then back substitution
 * L^T x = y. */
void orc_chol_solve(int k, const double *L, const double *b, double *x) {
    double y[256];
    double *yy = (k <= 256) ? y : (double *)malloc(sizeof(double) * k);
    for (int i = 0; i < k; ++i) {
        double s = b[i];
        for (int p = 0; p < i; ++p) s -= L[i * k + p] * yy[p];
        yy[i] = s / L[i * k + i];
    }
    for (int i = k - 1; i >= 0; --i) {
        double s = yy[i];
        for (int p = i + 1; p < k; ++p) s -= L[p * k + i] * x[p];
        x[i] = s / L[i * k + i];
    }
    if (yy != y) free(yy);
}

/* Normal equations of one row: A = sum_{t} v_{j_t} v_{j_t}^T + lambda I and
 * b = sum_t r_t v_{j_t}, with v_j the j-th row of F (n_other x k). */
void orc_normal_equations(int k, double lambda, int64_t s, const int32_t *idx,
                          const double *val, const double *F, double *A, double *b) {
    memset(A, 0, sizeof(double) * (size_t)k * k);
    memset(b, 0, sizeof(double) * (size_t)k);
    for (int64_t t = 0; t < s; ++t) {
        const double *v = F + (int64_t)idx[t] * k;
        for (int p = 0; p < k; ++p) {
            b[p] += val[t] * v[p];
            for (int q = 0; q < k; ++q) A[p * k + q] += v[p] * v[q];
        }
    }
    for (int p = 0; p < k; ++p) A[p * k + p] += lambda;
}

/* One ridge row solve: u = (V_O^T V_O + lambda I)^{-1} V_O^T r.
 * An empty row gives u = 0 (status EMPTY_ROW); a non-SPD system gives u = 0
 * (status NOT_SPD). */
int orc_row_solve(int k, double lambda, int64_t s, const int32_t *idx, const double *val,
                  const double *F, double *u) {
    if (s == 0) {
        memset(u, 0, sizeof(double) * k);
        return ORC_EMPTY_ROW;
    }
    double *A = (double *)malloc(sizeof(double) * (size_t)k * k * 2 + sizeof(double) * k);
    double *L = A + (size_t)k * k;
    double *b = L + (size_t)k * k;
    orc_normal_equations(k, lambda, s, idx, val, F, A, b);
    int st = orc_cholesky(k, A, L);
    if (st == ORC_OK)
        orc_chol_solve(k, L, b, u);
    else
        memset(u, 0, sizeof(double) * k);
    free(A);
    return st;
}

/* Half-step: every row of a CSR matrix against the fixed other factor F.
 * out is m x k row-major; status (may be NULL) receives per-row codes. */
void orc_half_step(int64_t m, const int64_t *ptr, const int32_t *idx, const double *val,
                   const double *F, int k, double lambda, double *out, int32_t *status) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < m; ++i) {
        int st = orc_row_solve(k, lambda, ptr[i + 1] - ptr[i], idx + ptr[i], val + ptr[i], F,
                               out + i * k);
        if (status) status[i] = st;
    }
}

/* CSR -> CSC by a stable counting sort on the column index: entries of one
 * column keep increasing row order. */
void orc_transpose(int64_t m, int64_t n, const int64_t *ptr, const int32_t *idx,
                   const double *val, int64_t *cptr, int32_t *cidx, double *cval) {
    int64_t *cursor = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    for (int64_t i = 0; i < m; ++i)
        for (int64_t t = ptr[i]; t < ptr[i + 1]; ++t) cursor[idx[t] + 1]++;
    for (int64_t j = 0; j < n; ++j) cursor[j + 1] += cursor[j];
    memcpy(cptr, cursor, sizeof(int64_t) * ((size_t)n + 1));
    for (int64_t i = 0; i < m; ++i)
        for (int64_t t = ptr[i]; t < ptr[i + 1]; ++t) {
            int64_t q = cursor[idx[t]]++;
            cidx[q] = (int32_t)i;
            cval[q] = val[t];
        }
    free(cursor);
}

/* The objective J(U, V) above.  Per-row partial sums are added in row order,
 * so the value does not depend on the thread count. */
double orc_objective(int64_t m, int64_t n, const int64_t *ptr, const int32_t *idx,
                     const double *val, const double *U, const double *V, int k,
                     double lambda) {
    double *part = (double *)malloc(sizeof(double) * 2 * (size_t)(m > 0 ? m : 1));
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i) {
        const double *u = U + i * k;
        double sse = 0.0, nu = 0.0;
        for (int64_t t = ptr[i]; t < ptr[i + 1]; ++t) {
            const double *v = V + (int64_t)idx[t] * k;
            double d = 0.0;
            for (int p = 0; p < k; ++p) d += u[p] * v[p];
            double e = val[t] - d;
            sse += e * e;
        }
        for (int p = 0; p < k; ++p) nu += u[p] * u[p];
        part[2 * i] = sse;
        part[2 * i + 1] = nu;
    }
    double sse = 0.0, nu = 0.0, nv = 0.0;
    for (int64_t i = 0; i < m; ++i) {
        sse += part[2 * i];
        nu += part[2 * i + 1];
    }
    free(part);
    for (int64_t j = 0; j < n * k; ++j) nv += V[j] * V[j];
    return sse + lambda * (nu + nv);
}

/* Per-row root-mean-square residual over the observed entries of a row. */
void orc_row_rmse(int64_t m, const int64_t *ptr, const int32_t *idx, const double *val,
                  const double *U, const double *V, int k, double *out) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i) {
        int64_t s = ptr[i + 1] - ptr[i];
        double sse = 0.0;
        for (int64_t t = ptr[i]; t < ptr[i + 1]; ++t) {
            double d = 0.0;
            for (int p = 0; p < k; ++p) d += U[i * k + p] * V[(int64_t)idx[t] * k + p];
            double e = val[t] - d;
            sse += e * e;
        }
        out[i] = s > 0 ? sqrt(sse / (double)s) : 0.0;
    }
}

/* Relative normal-equation residual |A u - b| / (|A| |u| + |b|) of one row
 * (Frobenius / Euclidean norms). */
double orc_normal_residual(int k, double lambda, int64_t s, const int32_t *idx,
                           const double *val, const double *F, const double *u) {
    double *A = (double *)malloc(sizeof(double) * ((size_t)k * k + k));
    double *b = A + (size_t)k * k;
    orc_normal_equations(k, lambda, s, idx, val, F, A, b);
    double nr = 0.0, na = 0.0, nu = 0.0, nb = 0.0;
    for (int p = 0; p < k; ++p) {
        double r = -b[p];
        for (int q = 0; q < k; ++q) {
            r += A[p * k + q] * u[q];
            na += A[p * k + q] * A[p * k + q];
        }
        nr += r * r;
        nu += u[p] * u[p];
        nb += b[p] * b[p];
    }
    free(A);
    double den = sqrt(na) * sqrt(nu) + sqrt(nb);
    return den > 0.0 ? sqrt(nr) / den : 0.0;
}

/* Alternating least squares: V starts at the given V (in/out), each sweep is
 * the U-half (all rows, V fixed) then the V-half (all columns, U fixed), for
 * a fixed number of sweeps with no early stop.  J_hist (may be NULL) gets
 * 2 * sweeps values: J after every half-step. */
void orc_als(int64_t m, int64_t n, const int64_t *ptr, const int32_t *idx, const double *val,
             int k, double lambda, int sweeps, double *U, double *V, double *J_hist,
             int32_t *row_status, int32_t *col_status) {
    int64_t nnz = ptr[m];
    int64_t *cptr = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
    int32_t *cidx = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
    double *cval = (double *)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
    orc_transpose(m, n, ptr, idx, val, cptr, cidx, cval);
    for (int s = 0; s < sweeps; ++s) {
        orc_half_step(m, ptr, idx, val, V, k, lambda, U, row_status);
        if (J_hist) J_hist[2 * s] = orc_objective(m, n, ptr, idx, val, U, V, k, lambda);
        orc_half_step(n, cptr, cidx, cval, U, k, lambda, V, col_status);
        if (J_hist) J_hist[2 * s + 1] = orc_objective(m, n, ptr, idx, val, U, V, k, lambda);
    }
    free(cptr);
    free(cidx);
    free(cval);
}

/* Dense ALS on a fully observed block: identical to orc_als with every entry
 * observed (kept separate so a test can compare the two). */
void orc_als_dense(int64_t m, int64_t n, const double *P, int k, double lambda, int sweeps,
                   double *U, double *V, double *J_hist) {
    int64_t *ptr = (int64_t *)malloc(sizeof(int64_t) * ((size_t)m + 1));
    int32_t *idx = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m * n > 0 ? m * n : 1));
    for (int64_t i = 0; i <= m; ++i) ptr[i] = i * n;
    for (int64_t i = 0; i < m; ++i)
        for (int64_t j = 0; j < n; ++j) idx[i * n + j] = (int32_t)j;
    orc_als(m, n, ptr, idx, P, k, lambda, sweeps, U, V, J_hist, NULL, NULL);
    free(ptr);
    free(idx);
}

/* Reconstruction T = U V^T (m x n, row-major). */
void orc_predict(int64_t m, int64_t n, int k, const double *U, const double *V, double *T) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i)
        for (int64_t j = 0; j < n; ++j) {
            double s = 0.0;
            for (int p = 0; p < k; ++p) s += U[i * k + p] * V[j * k + p];
            T[i * n + j] = s;
        }
}

/* ------------------------------------------------------------------------ */
/* Algorithm 2, energy-efficient power-cap selection, on a completed matrix of
 * predicted normalised runtimes t (rows: apps, columns: settings j =
 * c_idx * n_gpu + g_idx).  Predicted normalised performance relative to the
 * baseline is p_j = t_base / t_j (so p_base = 1, matching E_base = (C_b+G_b)*1).
 * For each setting with t_j > 0:
 *     pred_loss = 1 - p_j;  valid if pred_loss <= gamma (inclusive);
 *     E_pred = (c + g) / p_j;  saving = (E_base - E_pred) / E_base.
 * The selected setting maximises saving; ties go to the smaller c + g, then
 * the smaller j.  A row whose baseline runtime is not > 0 gets best = -1 and
 * saving = 0.  The arithmetic order above is the one the FP32 variant fixes
 * for bit-exact comparison of the chosen index. */
#define ORC_SELECT_BODY(REAL)                                                              \
    for (int64_t i = 0; i < m; ++i) {                                                      \
        const REAL *t = T + i * n;                                                         \
        REAL tb = t[base];                                                                 \
        int32_t bj = -1;                                                                   \
        REAL bs = (REAL)0, bcg = (REAL)0;                                                  \
        if (tb > (REAL)0) {                                                                \
            REAL Eb = (REAL)(cpu[base / n_gpu]) + (REAL)(gpu[base % n_gpu]);               \
            for (int64_t j = 0; j < n; ++j) {                                              \
                REAL tj = t[j];                                                            \
                if (!(tj > (REAL)0)) continue;                                             \
                REAL p = tb / tj;                                                          \
                REAL loss = (REAL)1 - p;                                                   \
                if (!(loss <= g_)) continue;                                               \
                REAL cg = (REAL)(cpu[j / n_gpu]) + (REAL)(gpu[j % n_gpu]);                 \
                REAL E = cg / p;                                                           \
                REAL sv = (Eb - E) / Eb;                                                   \
                if (bj < 0 || sv > bs || (sv == bs && cg < bcg)) {                         \
                    bj = (int32_t)j;                                                       \
                    bs = sv;                                                               \
                    bcg = cg;                                                              \
                }                                                                          \
            }                                                                              \
        }                                                                                  \
        best[i] = bj;                                                                      \
        saving[i] = bj >= 0 ? bs : (REAL)0;                                                \
    }

void orc_select_f64(int64_t m, int64_t n, const double *T, int32_t n_gpu, const double *cpu,
                    const double *gpu, double gamma, int64_t base, int32_t *best,
                    double *saving) {
    const double g_ = gamma;
    ORC_SELECT_BODY(double)
}

void orc_select_f32(int64_t m, int64_t n, const float *T, int32_t n_gpu, const float *cpu,
                    const float *gpu, float gamma, int64_t base, int32_t *best, float *saving) {
    const float g_ = gamma;
    ORC_SELECT_BODY(float)
}

/* ------------------------------------------------------------------------ */
/* Learned warm start: MLP 48 -> 256 -> 256 -> k with SELU (Klambauer et al.
 * 2017 constants) on the two hidden layers and a linear output.  Weights W_l
 * are [in, out] row-major, biases [out]. */
static const double SELU_L = 1.0507009873554804934193349852946;
static const double SELU_A = 1.6732632423543772848170429916717;

static double selu(double x) { return x > 0.0 ? SELU_L * x : SELU_L * SELU_A * expm1(x); }
static double selu_grad(double x) { return x > 0.0 ? SELU_L : SELU_L * SELU_A * exp(x); }

/* Y[B, o] = X[B, i] W[i, o] + b[o] */
static void dense_fwd(int64_t B, int din, int dout, const double *X, const double *W,
                      const double *bias, double *Y) {
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < B; ++r)
        for (int o = 0; o < dout; ++o) {
            double s = bias[o];
            for (int i = 0; i < din; ++i) s += X[r * din + i] * W[(int64_t)i * dout + o];
            Y[r * dout + o] = s;
        }
}

/* Forward pass; Z1, Z2 (pre-activations) and Y may be kept for backward. */
void orc_mlp_forward(int64_t B, int din, int h1, int h2, int dout, const double *X,
                     const double *W1, const double *b1, const double *W2, const double *b2,
                     const double *W3, const double *b3, double *Z1, double *Z2, double *Y) {
    double *H1 = (double *)malloc(sizeof(double) * (size_t)B * h1);
    double *H2 = (double *)malloc(sizeof(double) * (size_t)B * h2);
    dense_fwd(B, din, h1, X, W1, b1, Z1);
    for (int64_t t = 0; t < B * h1; ++t) H1[t] = selu(Z1[t]);
    dense_fwd(B, h1, h2, H1, W2, b2, Z2);
    for (int64_t t = 0; t < B * h2; ++t) H2[t] = selu(Z2[t]);
    dense_fwd(B, h2, dout, H2, W3, b3, Y);
    free(H1);
    free(H2);
}

/* Loss L = (1/B) sum_r (y_r - y*_r)^T G (y_r - y*_r) with G = V^T V (the
 * squared error of the predicted rows y V^T) and its gradient w.r.t. every
 * parameter.  Returns L. */
double orc_mlp_loss_grad(int64_t B, int din, int h1, int h2, int dout, const double *X,
                         const double *W1, const double *b1, const double *W2,
                         const double *b2, const double *W3, const double *b3,
                         const double *Ytgt, const double *G, double *gW1, double *gb1,
                         double *gW2, double *gb2, double *gW3, double *gb3) {
    double *Z1 = (double *)malloc(sizeof(double) * (size_t)B * h1);
    double *Z2 = (double *)malloc(sizeof(double) * (size_t)B * h2);
    double *Y = (double *)malloc(sizeof(double) * (size_t)B * dout);
    double *H1 = (double *)malloc(sizeof(double) * (size_t)B * h1);
    double *H2 = (double *)malloc(sizeof(double) * (size_t)B * h2);
    double *dY = (double *)malloc(sizeof(double) * (size_t)B * dout);
    double *dZ2 = (double *)malloc(sizeof(double) * (size_t)B * h2);
    double *dZ1 = (double *)malloc(sizeof(double) * (size_t)B * h1);
    orc_mlp_forward(B, din, h1, h2, dout, X, W1, b1, W2, b2, W3, b3, Z1, Z2, Y);
    for (int64_t t = 0; t < B * h1; ++t) H1[t] = selu(Z1[t]);
    for (int64_t t = 0; t < B * h2; ++t) H2[t] = selu(Z2[t]);
    double L = 0.0;
    for (int64_t r = 0; r < B; ++r) {
        for (int p = 0; p < dout; ++p) {
            double gd = 0.0;
            for (int q = 0; q < dout; ++q)
                gd += G[p * dout + q] * (Y[r * dout + q] - Ytgt[r * dout + q]);
            L += (Y[r * dout + p] - Ytgt[r * dout + p]) * gd;
            dY[r * dout + p] = 2.0 * gd / (double)B;
        }
    }
    L /= (double)B;
    /* layer 3 */
    for (int i = 0; i < h2; ++i)
        for (int o = 0; o < dout; ++o) {
            double s = 0.0;
            for (int64_t r = 0; r < B; ++r) s += H2[r * h2 + i] * dY[r * dout + o];
            gW3[(int64_t)i * dout + o] = s;
        }
    for (int o = 0; o < dout; ++o) {
        double s = 0.0;
        for (int64_t r = 0; r < B; ++r) s += dY[r * dout + o];
        gb3[o] = s;
    }
    for (int64_t r = 0; r < B; ++r)
        for (int i = 0; i < h2; ++i) {
            double s = 0.0;
            for (int o = 0; o < dout; ++o) s += dY[r * dout + o] * W3[(int64_t)i * dout + o];
            dZ2[r * h2 + i] = s * selu_grad(Z2[r * h2 + i]);
        }
    /* layer 2 */
    for (int i = 0; i < h1; ++i)
        for (int o = 0; o < h2; ++o) {
            double s = 0.0;
            for (int64_t r = 0; r < B; ++r) s += H1[r * h1 + i] * dZ2[r * h2 + o];
            gW2[(int64_t)i * h2 + o] = s;
        }
    for (int o = 0; o < h2; ++o) {
        double s = 0.0;
        for (int64_t r = 0; r < B; ++r) s += dZ2[r * h2 + o];
        gb2[o] = s;
    }
    for (int64_t r = 0; r < B; ++r)
        for (int i = 0; i < h1; ++i) {
            double s = 0.0;
            for (int o = 0; o < h2; ++o) s += dZ2[r * h2 + o] * W2[(int64_t)i * h2 + o];
            dZ1[r * h1 + i] = s * selu_grad(Z1[r * h1 + i]);
        }
    /* layer 1 */
    for (int i = 0; i < din; ++i)
        for (int o = 0; o < h1; ++o) {
            double s = 0.0;
            for (int64_t r = 0; r < B; ++r) s += X[r * din + i] * dZ1[r * h1 + o];
            gW1[(int64_t)i * h1 + o] = s;
        }
    for (int o = 0; o < h1; ++o) {
        double s = 0.0;
        for (int64_t r = 0; r < B; ++r) s += dZ1[r * h1 + o];
        gb1[o] = s;
    }
    free(Z1); free(Z2); free(Y); free(H1); free(H2); free(dY); free(dZ2); free(dZ1);
    return L;
}

/* Adam (Kingma & Ba 2015) on a flat parameter vector; step t >= 1. */
void orc_adam(int64_t count, double *theta, const double *g, double *m1, double *m2, int64_t t,
              double lr, double beta1, double beta2, double eps) {
    double c1 = 1.0 - pow(beta1, (double)t), c2 = 1.0 - pow(beta2, (double)t);
    for (int64_t q = 0; q < count; ++q) {
        m1[q] = beta1 * m1[q] + (1.0 - beta1) * g[q];
        m2[q] = beta2 * m2[q] + (1.0 - beta2) * g[q] * g[q];
        double mh = m1[q] / c1, vh = m2[q] / c2;
        theta[q] -= lr * mh / (sqrt(vh) + eps);
    }
}

/* Input encoding of the learned warm start: the first s_in observations of
 * each row (settings in increasing index order) become triples
 * (c_norm, g_norm, r) with caps scaled to [0, 1] over their grid; missing
 * triples are zero.  X is [m, 3 * s_in]. */
void orc_mlp_features(int64_t m, const int64_t *ptr, const int32_t *idx, const double *val,
                      int32_t n_cpu, int32_t n_gpu, const double *cpu, const double *gpu,
                      int s_in, double *X) {
    double cmin = cpu[0], cmax = cpu[0], gmin = gpu[0], gmax = gpu[0];
    for (int c = 1; c < n_cpu; ++c) { cmin = fmin(cmin, cpu[c]); cmax = fmax(cmax, cpu[c]); }
    for (int g = 1; g < n_gpu; ++g) { gmin = fmin(gmin, gpu[g]); gmax = fmax(gmax, gpu[g]); }
    for (int64_t i = 0; i < m; ++i) {
        double *x = X + i * 3 * s_in;
        memset(x, 0, sizeof(double) * 3 * s_in);
        int64_t s = ptr[i + 1] - ptr[i];
        if (s > s_in) s = s_in;
        for (int64_t t = 0; t < s; ++t) {
            int32_t j = idx[ptr[i] + t];
            double c = cpu[j / n_gpu], g = gpu[j % n_gpu];
            x[3 * t + 0] = cmax > cmin ? (c - cmin) / (cmax - cmin) : 0.0;
            x[3 * t + 1] = gmax > gmin ? (g - gmin) / (gmax - gmin) : 0.0;
            x[3 * t + 2] = val[ptr[i] + t];
        }
    }
}

/* Algorithm 1 (phase-transition detection), followed step by step for each
 * of n_traces power traces (row t of `power`, ld floats apart, len samples
 * taken every delta seconds): samples enter a circular buffer Q of capacity
 * N = W / delta; whenever Q is full it is divided into n_int consecutive
 * intervals of N / n_int samples, and a transition is reported when no
 * sample of any interval lies below p_th.  first[t] is the index of the
 * sample whose arrival produced the first report, or -1. */
void orc_phase_detect(int64_t n_traces, int64_t len, int64_t ld, const float *power, float p_th,
                      int32_t N, int32_t n_int, int64_t *first) {
    float *Q = (float *)malloc(sizeof(float) * (size_t)(N > 0 ? N : 1));
    for (int64_t t = 0; t < n_traces; ++t) {
        const float *pw = power + t * ld;
        int32_t head = 0, count = 0;   /* oldest sample at Q[head] */
        first[t] = -1;
        for (int64_t s = 0; s < len; ++s) {
            /* append p, removing the oldest if full */
            if (count < N) {
                Q[(head + count) % N] = pw[s];
                ++count;
            } else {
                Q[head] = pw[s];
                head = (head + 1) % N;
            }
            if (count == N) {
                int flag = 1;
                const int32_t per = N / n_int;
                for (int32_t k = 0; k < n_int && flag; ++k) {       /* each interval I */
                    for (int32_t e = 0; e < per; ++e) {
                        if (Q[(head + k * per + e) % N] < p_th) {    /* any value below */
                            flag = 0;
                            break;
                        }
                    }
                }
                if (flag) {
                    first[t] = s;
                    break;
                }
            }
        }
    }
    free(Q);
}

/* ALS with weighted-lambda regularisation (ALS-WR, the variant of the ALS
 * work the paper cites for collaborative filtering): the regulariser of each
 * factor is lambda times its number of observations,
 *   J_wr = sum (R_ij - u_i . v_j)^2 + lambda (sum_i s_i |u_i|^2 + sum_j s_j |v_j|^2),
 * so each row solve is (sum_{j in Omega_i} v_j v_j^T + lambda s_i I) u_i = b_i. */
void orc_half_step_wr(int64_t m, const int64_t *ptr, const int32_t *idx, const double *val,
                      const double *F, int k, double lambda, double *out, int32_t *status) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < m; ++i) {
        const int64_t s = ptr[i + 1] - ptr[i];
        int st = orc_row_solve(k, lambda * (double)s, s, idx + ptr[i], val + ptr[i], F,
                               out + i * k);
        if (status) status[i] = st;
    }
}

double orc_objective_wr(int64_t m, int64_t n, const int64_t *ptr, const int32_t *idx,
                        const double *val, const double *U, const double *V, int k,
                        double lambda) {
    double sse = 0.0, nu = 0.0, nv = 0.0;
    int64_t *cnt = (int64_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
    for (int64_t i = 0; i < m; ++i) {
        const double *u = U + i * k;
        double ui = 0.0;
        for (int64_t t = ptr[i]; t < ptr[i + 1]; ++t) {
            const double *v = V + (int64_t)idx[t] * k;
            double d = 0.0;
            for (int p = 0; p < k; ++p) d += u[p] * v[p];
            const double e = val[t] - d;
            sse += e * e;
            cnt[idx[t]]++;
        }
        for (int p = 0; p < k; ++p) ui += u[p] * u[p];
        nu += (double)(ptr[i + 1] - ptr[i]) * ui;
    }
    for (int64_t j = 0; j < n; ++j) {
        double vj = 0.0;
        for (int p = 0; p < k; ++p) vj += V[j * k + p] * V[j * k + p];
        nv += (double)cnt[j] * vj;
    }
    free(cnt);
    return sse + lambda * (nu + nv);
}

void orc_als_wr(int64_t m, int64_t n, const int64_t *ptr, const int32_t *idx, const double *val,
                int k, double lambda, int sweeps, double *U, double *V, double *J_hist) {
    int64_t nnz = ptr[m];
    int64_t *cptr = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
    int32_t *cidx = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
    double *cval = (double *)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
    orc_transpose(m, n, ptr, idx, val, cptr, cidx, cval);
    for (int s = 0; s < sweeps; ++s) {
        orc_half_step_wr(m, ptr, idx, val, V, k, lambda, U, NULL);
        if (J_hist) J_hist[2 * s] = orc_objective_wr(m, n, ptr, idx, val, U, V, k, lambda);
        orc_half_step_wr(n, cptr, cidx, cval, U, k, lambda, V, NULL);
        if (J_hist) J_hist[2 * s + 1] = orc_objective_wr(m, n, ptr, idx, val, U, V, k, lambda);
    }
    free(cptr);
    free(cidx);
    free(cval);
}

/* ------------------------------------------------------------------------ */
/* Neural collaborative filtering, the paper's CF model (Sec. "Collaborative
 * Filtering Model"): the application index i and the power-cap-pair index j
 * select rows of two embedding tables, Ea[m, d] and Es[n, d]; the two rows
 * are concatenated into x = [Ea_i, Es_j] (2d values) and passed through an
 * MLP with SELU hidden activations whose single linear output is the
 * predicted entry P_ij:
 *     z1 = x W1 + b1,  z2 = selu(z1) W2 + b2,  y = selu(z2) . w3 + b3
 * with W1 [2d, h1], W2 [h1, h2], w3 [h2] (weights [in, out] row-major).
 * Training minimises the mean squared error over a batch of observed
 * entries, L = (1/B) sum_b (y_b - r_b)^2.  net = {W1, b1, W2, b2, w3, b3}
 * packed in that order. */
static void ncf_unpack(int d, int h1, int h2, const double *net, const double **W1,
                       const double **b1, const double **W2, const double **b2,
                       const double **w3, const double **b3) {
    *W1 = net;
    *b1 = *W1 + (int64_t)2 * d * h1;
    *W2 = *b1 + h1;
    *b2 = *W2 + (int64_t)h1 * h2;
    *w3 = *b2 + h2;
    *b3 = *w3 + h2;
}

int64_t orc_ncf_net_size(int d, int h1, int h2) {
    return (int64_t)2 * d * h1 + h1 + (int64_t)h1 * h2 + h2 + h2 + 1;
}

/* y[b] for the pairs (ai[b], sj[b]); Z1 [B, h1] and Z2 [B, h2] optional. */
void orc_ncf_forward(int64_t B, const int32_t *ai, const int32_t *sj, int d, int h1, int h2,
                     const double *Ea, const double *Es, const double *net, double *y,
                     double *Z1_out, double *Z2_out) {
    const double *W1, *b1, *W2, *b2, *w3, *b3;
    ncf_unpack(d, h1, h2, net, &W1, &b1, &W2, &b2, &w3, &b3);
#pragma omp parallel
    {
        double *x = (double *)malloc(sizeof(double) * 2 * (size_t)d);
        double *z1 = (double *)malloc(sizeof(double) * (size_t)h1);
        double *z2 = (double *)malloc(sizeof(double) * (size_t)h2);
#pragma omp for schedule(static)
        for (int64_t b = 0; b < B; ++b) {
            for (int t = 0; t < d; ++t) {   /* concatenation of the two embeddings */
                x[t] = Ea[(int64_t)ai[b] * d + t];
                x[d + t] = Es[(int64_t)sj[b] * d + t];
            }
            for (int o = 0; o < h1; ++o) {
                double s = b1[o];
                for (int t = 0; t < 2 * d; ++t) s += x[t] * W1[(int64_t)t * h1 + o];
                z1[o] = s;
            }
            for (int o = 0; o < h2; ++o) {
                double s = b2[o];
                for (int t = 0; t < h1; ++t) s += selu(z1[t]) * W2[(int64_t)t * h2 + o];
                z2[o] = s;
            }
            double s = b3[0];
            for (int t = 0; t < h2; ++t) s += selu(z2[t]) * w3[t];
            y[b] = s;
            if (Z1_out) memcpy(Z1_out + b * h1, z1, sizeof(double) * (size_t)h1);
            if (Z2_out) memcpy(Z2_out + b * h2, z2, sizeof(double) * (size_t)h2);
        }
        free(x); free(z1); free(z2);
    }
}

/* L = (1/B) sum_b (y_b - r_b)^2 and its gradient: g_net (same packing as net)
 * and the embedding gradients gEa [m, d], gEs [n, d] (rows of indices that do
 * not occur in the batch stay 0).  Returns L. */
double orc_ncf_loss_grad(int64_t B, const int32_t *ai, const int32_t *sj, const double *r, int64_t m,
                         int64_t n, int d, int h1, int h2, const double *Ea, const double *Es,
                         const double *net, double *g_net, double *gEa, double *gEs) {
    const double *W1, *b1, *W2, *b2, *w3, *b3;
    ncf_unpack(d, h1, h2, net, &W1, &b1, &W2, &b2, &w3, &b3);
    double *gW1 = g_net, *gb1 = gW1 + (int64_t)2 * d * h1, *gW2 = gb1 + h1;
    double *gb2 = gW2 + (int64_t)h1 * h2, *gw3 = gb2 + h2, *gb3 = gw3 + h2;
    memset(g_net, 0, sizeof(double) * (size_t)orc_ncf_net_size(d, h1, h2));
    memset(gEa, 0, sizeof(double) * (size_t)(m * d));
    memset(gEs, 0, sizeof(double) * (size_t)(n * d));
    double *Z1 = (double *)malloc(sizeof(double) * (size_t)(B * h1));
    double *Z2 = (double *)malloc(sizeof(double) * (size_t)(B * h2));
    double *y = (double *)malloc(sizeof(double) * (size_t)(B > 0 ? B : 1));
    double *dz1 = (double *)malloc(sizeof(double) * (size_t)h1);
    double *dz2 = (double *)malloc(sizeof(double) * (size_t)h2);
    orc_ncf_forward(B, ai, sj, d, h1, h2, Ea, Es, net, y, Z1, Z2);
    double L = 0.0;
    /* samples in order, so every accumulation has a fixed order */
    for (int64_t b = 0; b < B; ++b) {
        const double e = y[b] - r[b];
        L += e * e;
        const double dy = 2.0 * e / (double)B;
        const double *z1 = Z1 + b * h1, *z2 = Z2 + b * h2;
        gb3[0] += dy;
        for (int t = 0; t < h2; ++t) {
            gw3[t] += dy * selu(z2[t]);
            dz2[t] = dy * w3[t] * selu_grad(z2[t]);
            gb2[t] += dz2[t];
        }
        for (int t = 0; t < h1; ++t) {
            const double a = selu(z1[t]);
            double s = 0.0;
            for (int o = 0; o < h2; ++o) {
                gW2[(int64_t)t * h2 + o] += a * dz2[o];
                s += W2[(int64_t)t * h2 + o] * dz2[o];
            }
            dz1[t] = s * selu_grad(z1[t]);
            gb1[t] += dz1[t];
        }
        const double *ea = Ea + (int64_t)ai[b] * d, *es = Es + (int64_t)sj[b] * d;
        double *gea = gEa + (int64_t)ai[b] * d, *ges = gEs + (int64_t)sj[b] * d;
        for (int t = 0; t < d; ++t) {
            double sa = 0.0, ss = 0.0;
            for (int o = 0; o < h1; ++o) {
                gW1[(int64_t)t * h1 + o] += ea[t] * dz1[o];
                gW1[(int64_t)(d + t) * h1 + o] += es[t] * dz1[o];
                sa += W1[(int64_t)t * h1 + o] * dz1[o];
                ss += W1[(int64_t)(d + t) * h1 + o] * dz1[o];
            }
            gea[t] += sa;
            ges[t] += ss;
        }
    }
    free(Z1); free(Z2); free(y); free(dz1); free(dz2);
    return B > 0 ? L / (double)B : 0.0;
}

/* The completed matrix: T[i, j] = y(i, j) for every application and setting. */
void orc_ncf_predict(int64_t m, int64_t n, int d, int h1, int h2, const double *Ea,
                     const double *Es, const double *net, double *T) {
    int32_t *ai = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *sj = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t j = 0; j < n; ++j) sj[j] = (int32_t)j;
    for (int64_t i = 0; i < m; ++i) {
        for (int64_t j = 0; j < n; ++j) ai[j] = (int32_t)i;
        orc_ncf_forward(n, ai, sj, d, h1, h2, Ea, Es, net, T + i * n, NULL, NULL);
    }
    free(ai); free(sj);
}

/* ------------------------------------------------------------------------ */
/* Streaming refit of V (the joint online refit of Sec. "Online Performance
 * Prediction" done incrementally): for every setting j the normal equations
 * of the V-half-step over all rows ingested so far are kept as sums,
 *     G_j = sum_{i in Omega_j} u_i u_i^T,   b_j = sum_{i in Omega_j} R_ij u_i,
 *     s_j = |Omega_j|,
 * so a batch of new applications adds its rank-one terms (its rows' factors
 * u_i, from the fold-in against the current V) and V is re-solved as
 *     v_j = (G_j + lambda_j I)^{-1} b_j,  lambda_j = lambda (or lambda s_j, weighted),
 * with v_j = 0 for a setting no row has observed (as the half-step does). */
void orc_stream_accumulate(int64_t m, const int64_t *ptr, const int32_t *idx, const double *val,
                           const double *U, int k, double *G, double *b, int64_t *cnt) {
    for (int64_t i = 0; i < m; ++i) {
        const double *u = U + i * k;
        for (int64_t t = ptr[i]; t < ptr[i + 1]; ++t) {
            const int64_t j = idx[t];
            double *Gj = G + j * k * k, *bj = b + j * k;
            for (int p = 0; p < k; ++p) {
                bj[p] += val[t] * u[p];
                for (int q = 0; q < k; ++q) Gj[p * k + q] += u[p] * u[q];
            }
            cnt[j] += 1;
        }
    }
}

void orc_stream_solve(int64_t n, int k, const double *G, const double *b, const int64_t *cnt,
                      double lambda, int weighted, double *V, int32_t *status) {
#pragma omp parallel
    {
        double *A = (double *)malloc(sizeof(double) * (size_t)k * k * 2);
        double *L = A + (size_t)k * k;
#pragma omp for schedule(static)
        for (int64_t j = 0; j < n; ++j) {
            int st = ORC_OK;
            if (cnt[j] == 0) {
                st = ORC_EMPTY_ROW;
            } else {
                const double lam = weighted ? lambda * (double)cnt[j] : lambda;
                memcpy(A, G + j * k * k, sizeof(double) * (size_t)k * k);
                for (int p = 0; p < k; ++p) A[p * k + p] += lam;
                st = orc_cholesky(k, A, L);
                if (st == ORC_OK) orc_chol_solve(k, L, b + j * k, V + j * k);
            }
            if (st != ORC_OK) memset(V + j * k, 0, sizeof(double) * (size_t)k);
            if (status) status[j] = st;
        }
        free(A);
    }
}
