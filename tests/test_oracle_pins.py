"""Pins of the FP64 oracle against things other than itself.

Each test checks the oracle against a textbook or library routine, a closed
form, an invariant of the method, or a hand-computed table.  Chosen so that a
dropped term, a wrong sign or index, or a transposed operand in the oracle
fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp

import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_csr(rng, m, n, density, min_per_row=0):
    rows, cols = [], []
    for i in range(m):
        mask = rng.random(n) < density
        if mask.sum() < min_per_row:
            mask[rng.choice(n, min_per_row, replace=False)] = True
        c = np.nonzero(mask)[0]
        rows.append(np.full(len(c), i)); cols.append(c)
    rows = np.concatenate(rows); cols = np.concatenate(cols).astype(np.int32)
    ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=m), out=ptr[1:])
    return ptr, cols


# --- P1: each row solve is ridge regression, i.e. lstsq of [V_O; sqrt(l) I] u = [r; 0]
@pytest.mark.parametrize("seed", range(6))
def test_row_solve_equals_augmented_lstsq(orc, seed):
    rng = np.random.default_rng(seed)
    m, n, k = int(rng.integers(2, 7)), int(rng.integers(3, 9)), int(rng.integers(1, 4))
    lam = float(rng.uniform(0.01, 1.0))
    ptr, col = _rand_csr(rng, m, n, 0.6, min_per_row=1)
    val = rng.standard_normal(len(col))
    F = rng.standard_normal((n, k))
    U, st = orc.half_step(ptr, col, val, F, lam)
    assert (st == 0).all()
    for i in range(m):
        c = col[ptr[i]:ptr[i + 1]]
        Aaug = np.vstack([F[c], math.sqrt(lam) * np.eye(k)])
        baug = np.concatenate([val[ptr[i]:ptr[i + 1]], np.zeros(k)])
        ref = np.linalg.lstsq(Aaug, baug, rcond=None)[0]
        assert np.abs(U[i] - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())


# --- P2 + P3: monotone objective; normal-equation residual per row
@pytest.mark.parametrize("which", ["small", "sparse"])
def test_objective_monotone_and_normal_residual(orc, which):
    if which == "small":
        prob = synth.make_small_offline_online(seed=0).joint
    else:
        prob = synth.make_sparse_problem(seed=1, m=300, n_cpu=4, n_gpu=30, rank=6,
                                         density=0.1, k=8, lam=0.05, sweeps=8)
    U, V, J, rs, cs = orc.als(prob.row_ptr, prob.col, prob.val, prob.n, prob.V0, prob.lam,
                              prob.sweeps, history=True)
    J0 = orc.objective(prob.row_ptr, prob.col, prob.val, np.zeros((prob.m, prob.k)), prob.V0,
                       prob.lam)
    seq = np.concatenate([[J0], J])
    assert (np.diff(seq) <= 1e-12 * seq[:-1]).all(), seq
    assert seq[-1] < 0.5 * seq[0]
    # normal equations of the final V-half hold for every column, U-half for rows
    cptr, cidx, cval = orc.transpose(prob.row_ptr, prob.col, prob.val, prob.n)
    for j in range(prob.n):
        s = slice(cptr[j], cptr[j + 1])
        if cptr[j + 1] > cptr[j]:
            assert orc.normal_residual(U, cidx[s], cval[s], prob.lam, V[j]) < 1e-10
    # U is the U-half of the last sweep, taken against the V before the last V-half:
    # re-solve rows against the final V and check the residual of that solve
    U2, _ = orc.half_step(prob.row_ptr, prob.col, prob.val, V, prob.lam)
    for i in range(prob.m):
        s = slice(prob.row_ptr[i], prob.row_ptr[i + 1])
        assert orc.normal_residual(V, prob.col[s], prob.val[s], prob.lam, U2[i]) < 1e-10


def test_objective_closed_forms(orc):
    rng = np.random.default_rng(3)
    ptr, col = _rand_csr(rng, 20, 15, 0.3, min_per_row=1)
    val = rng.standard_normal(len(col))
    V = rng.standard_normal((15, 4))
    # U = 0: every residual is the observed value itself
    J = orc.objective(ptr, col, val, np.zeros((20, 4)), V, 0.7)
    assert abs(J - (np.sum(val ** 2) + 0.7 * np.sum(V ** 2))) < 1e-12 * J
    # a factorisation that reproduces the observations exactly leaves only the ridge term
    U = rng.standard_normal((20, 4))
    rows = np.repeat(np.arange(20), np.diff(ptr))
    exact = np.einsum("tk,tk->t", U[rows], V[col])
    J = orc.objective(ptr, col, exact, U, V, 0.3)
    assert abs(J - 0.3 * (np.sum(U ** 2) + np.sum(V ** 2))) < 1e-10


# --- P4: exact recovery of a noiseless rank-k matrix
def test_exact_recovery_rank_k(orc):
    rng = np.random.default_rng(7)
    m_off, n, k = 40, 60, 5
    Ut = rng.standard_normal((m_off + 10, k)); Vt = rng.standard_normal((n, k))
    T = Ut @ Vt.T
    V0 = 0.1 * rng.standard_normal((n, k))
    _, V, _ = orc.als_dense(T[:m_off], V0, 1e-10, 3)
    # new rows with s_i >= k generic observations, V fixed (fold-in)
    ptr = [0]; cols = []; vals = []
    for i in range(m_off, m_off + 10):
        c = np.sort(rng.choice(n, size=k + 2, replace=False))
        cols.append(c); vals.append(T[i, c]); ptr.append(ptr[-1] + len(c))
    U_new, st = orc.half_step(np.array(ptr), np.concatenate(cols).astype(np.int32),
                              np.concatenate(vals), V, 1e-10)
    assert (st == 0).all()
    pred = orc.predict(U_new, V)
    assert np.abs(pred - T[m_off:]).max() < 1e-6


# --- P5: fully observed matrix -> soft-thresholded SVD (Hastie et al. 2015)
def test_fully_observed_matches_soft_thresholded_svd(orc):
    rng = np.random.default_rng(11)
    m, n, k, lam = 30, 20, 3, 0.5
    A, _ = np.linalg.qr(rng.standard_normal((m, m)))
    B, _ = np.linalg.qr(rng.standard_normal((n, n)))
    sig = np.zeros(n); sig[:6] = [10.0, 9.0, 8.0, 1.0, 0.5, 0.2]
    T = A[:, :n] @ np.diag(sig) @ B.T
    V0 = 0.1 * rng.standard_normal((n, k))
    U, V, _ = orc.als_dense(T, V0, lam, 200)
    Uu, s, Vh = np.linalg.svd(T, full_matrices=False)
    ref = (Uu[:, :k] * np.maximum(s[:k] - lam, 0.0)) @ Vh[:k]
    assert np.abs(U @ V.T - ref).max() < 1e-10


def test_dense_and_csr_als_agree(orc):
    rng = np.random.default_rng(5)
    P = rng.random((12, 9))
    V0 = 0.1 * rng.standard_normal((9, 3))
    U1, V1, J1 = orc.als_dense(P, V0, 0.2, 4, history=True)
    ptr = np.arange(13, dtype=np.int64) * 9
    col = np.tile(np.arange(9, dtype=np.int32), 12)
    U2, V2, J2, _, _ = orc.als(ptr, col, P.ravel(), 9, V0, 0.2, 4, history=True)
    assert np.array_equal(U1, U2) and np.array_equal(V1, V2) and np.array_equal(J1, J2)


# --- P6: special cases
def test_special_cases(orc):
    rng = np.random.default_rng(2)
    F = rng.standard_normal((10, 4))
    u, st = orc.row_solve(F, np.zeros(0, dtype=np.int32), np.zeros(0), 0.3)
    assert st == orc.EMPTY_ROW and np.all(u == 0)
    # one observation: Sherman-Morrison gives u = r v / (lambda + |v|^2)
    v = F[6]; r = 0.7
    u, st = orc.row_solve(F, np.array([6], dtype=np.int32), np.array([r]), 0.3)
    assert st == orc.OK
    assert np.abs(u - r * v / (0.3 + v @ v)).max() < 1e-14
    # fully observed rows with fixed V share one system (V^T V + lambda I)
    R = rng.standard_normal((5, 10))
    ptr = np.arange(6, dtype=np.int64) * 10
    col = np.tile(np.arange(10, dtype=np.int32), 5)
    U, st = orc.half_step(ptr, col, R.ravel(), F, 0.3)
    ref = np.linalg.solve(F.T @ F + 0.3 * np.eye(4), F.T @ R.T).T
    assert np.abs(U - ref).max() < 1e-12


# --- P7: Cholesky against numpy
@pytest.mark.parametrize("k", [1, 3, 8, 17, 32])
def test_cholesky(orc, k):
    rng = np.random.default_rng(k)
    X = rng.standard_normal((k + 5, k))
    A = X.T @ X + 0.1 * np.eye(k)
    L, st = orc.cholesky(A)
    assert st == 0
    assert np.linalg.norm(L @ L.T - A) / np.linalg.norm(A) <= 1e-14
    assert np.abs(L - np.linalg.cholesky(A)).max() <= 1e-12 * np.abs(L).max()
    b = rng.standard_normal(k)
    assert np.abs(orc.chol_solve(L, b) - np.linalg.solve(A, b)).max() < 1e-10
    Abad = A.copy(); Abad[k - 1, k - 1] = -1.0
    assert orc.cholesky(Abad)[1] == orc.NOT_SPD


def test_transpose_matches_scipy(orc):
    rng = np.random.default_rng(9)
    ptr, col = _rand_csr(rng, 50, 37, 0.2)
    val = rng.standard_normal(len(col))
    cptr, cidx, cval = orc.transpose(ptr, col, val, 37)
    ref = sp.csr_matrix((val, col, ptr), shape=(50, 37)).tocsc()
    ref.sort_indices()
    assert np.array_equal(cptr, ref.indptr) and np.array_equal(cidx, ref.indices)
    assert np.array_equal(cval, ref.data)


def test_predict_is_matmul(orc):
    rng = np.random.default_rng(4)
    U = rng.standard_normal((13, 5)); V = rng.standard_normal((7, 5))
    assert np.abs(orc.predict(U, V) - U @ V.T).max() < 1e-13


# --- P8: Algorithm 2 on hand-computed tables, in FP64 and FP32
def test_algorithm2_golden_tables(orc):
    cases = json.load(open(os.path.join(GOLDEN, "alg2_tables.json")))["cases"]
    for c in cases:
        T = np.array([c["t"]], dtype=np.float64)
        for fn, tol in ((orc.select_f64, 1e-12), (orc.select_f32, 1e-6)):
            best, sav = fn(T, np.array(c["cpu"], float), np.array(c["gpu"], float), c["gamma"])
            assert best[0] == c["best"], (c["name"], fn.__name__, best[0])
            assert abs(float(sav[0]) - c["saving"]) <= tol, (c["name"], float(sav[0]))


def test_algorithm2_rows_independent_and_baseline_override(orc):
    cases = json.load(open(os.path.join(GOLDEN, "alg2_tables.json")))["cases"]
    c3 = [c for c in cases if c["name"].startswith("3x3")]
    T = np.array([c3[0]["t"]] * 3)
    best, sav = orc.select_f64(T, np.array(c3[0]["cpu"], float), np.array(c3[0]["gpu"], float),
                               0.2)
    assert list(best) == [1, 1, 1]
    # explicit baseline index equal to the default gives the same answer
    b2, s2 = orc.select_f64(T, np.array(c3[0]["cpu"], float), np.array(c3[0]["gpu"], float),
                            0.2, base=8)
    assert list(b2) == [1, 1, 1] and np.array_equal(sav, s2)


# --- P9: MLP forward against SELU closed forms, backward against finite differences
SELU_LAMBDA = 1.0507009873554804934193349852946   # Klambauer et al. 2017
SELU_ALPHA = 1.6732632423543772848170429916717


def test_mlp_forward_selu_closed_form(orc):
    I2 = np.eye(2)
    params = [I2, np.zeros(2), I2, np.zeros(2), I2, np.array([0.5, -0.25])]
    X = np.array([[1.0, -1.0]])
    Z1, Z2, Y = orc.mlp_forward(X, params)
    h1 = np.array([SELU_LAMBDA, SELU_LAMBDA * SELU_ALPHA * (math.exp(-1.0) - 1.0)])
    assert np.abs(Z1 - X).max() < 1e-15
    assert np.abs(Z2[0] - h1).max() < 1e-15
    h2 = np.array([SELU_LAMBDA * h1[0],
                   SELU_LAMBDA * SELU_ALPHA * (math.exp(h1[1]) - 1.0)])
    assert np.abs(Y[0] - (h2 + [0.5, -0.25])).max() < 1e-14


def test_mlp_gradients_finite_differences(orc):
    rng = np.random.default_rng(1)
    sizes = (6, 5, 4, 3)
    params = synth.mlp_init(rng, sizes)
    params = [p + 0.1 * rng.standard_normal(p.shape) for p in params]
    X = rng.standard_normal((4, 6)); Yt = rng.standard_normal((4, 3))
    Vg = rng.standard_normal((7, 3)); G = Vg.T @ Vg
    L, grads = orc.mlp_loss_grad(X, params, Yt, G)
    # loss value against its definition via the forward pass
    _, _, Y = orc.mlp_forward(X, params)
    D = Y - Yt
    assert abs(L - np.mean(np.einsum("bp,pq,bq->b", D, G, D))) < 1e-12 * abs(L)
    h = 1e-6
    for pi, p in enumerate(params):
        for idx in np.ndindex(p.shape):
            old = p[idx]
            p[idx] = old + h; Lp, _ = orc.mlp_loss_grad(X, params, Yt, G)
            p[idx] = old - h; Lm, _ = orc.mlp_loss_grad(X, params, Yt, G)
            p[idx] = old
            fd = (Lp - Lm) / (2 * h)
            assert abs(fd - grads[pi][idx]) <= 1e-6 * max(1.0, abs(fd)), (pi, idx)


def test_adam_first_step_closed_form(orc):
    # with zero moments, the bias-corrected first step is lr * g / (|g| + eps)
    g = np.array([0.5, -2.0, 1e-3])
    th = np.array([1.0, 1.0, 1.0]); m1 = np.zeros(3); m2 = np.zeros(3)
    orc.adam(th, g, m1, m2, 1, lr=0.01)
    assert np.abs(th - (1.0 - 0.01 * g / (np.abs(g) + 1e-8))).max() < 1e-15
    # a second identical gradient keeps m_hat = g and v_hat = g^2
    orc.adam(th, g, m1, m2, 2, lr=0.01)
    assert np.abs(th - (1.0 - 2 * 0.01 * g / (np.abs(g) + 1e-8))).max() < 1e-14


def test_mlp_features_hand_example(orc):
    cpu = np.array([100.0, 200.0, 300.0]); gpu = np.array([50.0, 150.0])
    ptr = np.array([0, 2, 2], dtype=np.int64)
    col = np.array([1, 4], dtype=np.int32); val = np.array([0.3, 0.9])
    X = orc.mlp_features(ptr, col, val, cpu, gpu, s_in=3)
    # setting 1 = (100 W, 150 W) -> (0, 1); setting 4 = (300 W, 50 W) -> (1, 0)
    assert np.array_equal(X[0], [0, 1, 0.3, 1, 0, 0.9, 0, 0, 0])
    assert np.array_equal(X[1], np.zeros(9))


# ---------------------------------------------------------------- Algorithm 1
def _phase_trace(segments):
    """Concatenate (value, count) segments into one float32 power trace."""
    return np.concatenate([np.full(c, v, np.float32) for v, c in segments])


def test_phase_detection_hand_cases(orc):
    """Algorithm 1 (Sec. "Online Performance Prediction"): delta 0.2 s,
    W 5 s -> N = 25 samples, P_th 60 W, five 1-s intervals; a transition is
    reported on the sample that completes 25 consecutive readings none of
    which is below 60 W (a reading of exactly 60 W is not below)."""
    cases = [
        (_phase_trace([(100.0, 24)]), -1),                       # buffer never full
        (_phase_trace([(100.0, 25)]), 24),                       # full at sample 24
        (_phase_trace([(60.0, 30)]), 24),                        # equal to P_th passes
        (_phase_trace([(40.0, 10), (75.0, 25), (40.0, 5)]), 34),
        (_phase_trace([(40.0, 5), (90.0, 15), (59.9, 1), (90.0, 30)]), 45),
        (_phase_trace([(40.0, 3), (90.0, 24), (50.0, 1), (90.0, 24)]), -1),
    ]
    got = [int(orc.phase_detect(tr)[0]) for tr, _ in cases]
    assert got == [want for _, want in cases]


def test_phase_detection_equals_sliding_window_minimum(orc):
    """The five-interval check is the same as 'the minimum of the last 25
    readings is not below P_th': compare with that plain definition on
    random traces, and with one interval instead of five."""
    rng = np.random.default_rng(0)
    P = rng.uniform(40.0, 80.0, (200, 300)).astype(np.float32)
    P[rng.random((200, 300)) < 0.7] += 30.0
    got = orc.phase_detect(P)
    assert np.array_equal(got, orc.phase_detect(P, intervals=1))
    for t in range(200):
        ok = P[t] >= np.float32(60.0)
        want = -1
        for s in range(24, 300):
            if ok[s - 24:s + 1].all():
                want = s
                break
        assert got[t] == want


# ---------------------------------------------------------------- ALS-WR
def test_wr_row_solve_is_ridge_with_count_scaled_lambda(orc):
    """Each weighted-lambda row solve is the least-squares solution of the
    augmented system [V_Omega; sqrt(lambda s_i) I] u = [r; 0] (brute force by
    numpy's lstsq on tiny inputs)."""
    rng = np.random.default_rng(5)
    m, n, k, lam = 6, 9, 3, 0.3
    counts = np.array([0, 1, 2, 4, 6, 9])
    ptr = np.concatenate([[0], np.cumsum(counts)])
    col = np.concatenate([np.sort(rng.choice(n, c, replace=False)) for c in counts]).astype(np.int32)
    val = rng.standard_normal(ptr[-1])
    V = rng.standard_normal((n, k))
    U, st = orc.half_step_wr(ptr, col, val, V, lam)
    for i in range(m):
        c, r = col[ptr[i]:ptr[i + 1]], val[ptr[i]:ptr[i + 1]]
        if len(c) == 0:
            assert st[i] == 2 and np.all(U[i] == 0)
            continue
        A = np.vstack([V[c], np.sqrt(lam * len(c)) * np.eye(k)])
        b = np.concatenate([r, np.zeros(k)])
        ref = np.linalg.lstsq(A, b, rcond=None)[0]
        assert np.allclose(U[i], ref, rtol=1e-12, atol=1e-12)


def test_wr_objective_monotone_and_closed_form(orc):
    """Every weighted-lambda half-step minimises J_wr exactly in its block, so
    J_wr never increases; J_wr at given factors equals the definition written
    out with numpy."""
    prob = synth.make_sparse_problem(seed=7, m=120, n_cpu=4, n_gpu=10, rank=4, density=0.3,
                                     k=4, lam=0.05, n_heldout=8)
    U, V, J = orc.als_wr(prob.row_ptr, prob.col, prob.val, prob.n, prob.V0, prob.lam, 8,
                         history=True)
    assert np.all(np.diff(J) <= 1e-12 * np.abs(J[:-1]))
    rows = np.repeat(np.arange(prob.m), np.diff(prob.row_ptr))
    res = prob.val - np.einsum("tk,tk->t", U[rows], V[prob.col])
    s_i = np.diff(prob.row_ptr)
    s_j = np.bincount(prob.col, minlength=prob.n)
    want = (res ** 2).sum() + prob.lam * ((s_i * (U ** 2).sum(1)).sum() +
                                          (s_j * (V ** 2).sum(1)).sum())
    assert abs(orc.objective_wr(prob.row_ptr, prob.col, prob.val, U, V, prob.lam) - want) <= \
        1e-10 * abs(want)


# --- per-row observed RMSE (the learned path's fallback judge, the objective's
# per-row figure): a hand-computed 3 x 3 example with k = 2, then a plain numpy
# expression of the definition on a random problem
def test_row_rmse_hand_example(orc):
    U = np.array([[1.0, 2.0], [3.0, -1.0], [5.0, 5.0]])
    V = np.array([[1.0, 0.0], [0.0, 1.0], [2.0, 1.0]])
    ptr = np.array([0, 2, 3, 3], dtype=np.int64)
    col = np.array([0, 2, 1], dtype=np.int32)
    val = np.array([2.0, 6.0, 1.0])
    # row 0: predictions 1 and 4, errors 1 and 2 -> sqrt(5 / 2)
    # row 1: prediction -1, error 2 -> 2;  row 2 has no observations -> 0
    got = orc.row_rmse(ptr, col, val, U, V)
    assert np.allclose(got, [math.sqrt(2.5), 2.0, 0.0], rtol=0, atol=1e-15), got


def test_row_rmse_matches_numpy_definition(orc):
    rng = np.random.default_rng(11)
    m, n, k = 40, 25, 6
    ptr, col = _rand_csr(rng, m, n, 0.3)
    val = rng.standard_normal(len(col))
    U, V = rng.standard_normal((m, k)), rng.standard_normal((n, k))
    rows = np.repeat(np.arange(m), np.diff(ptr))
    e2 = (val - np.sum(U[rows] * V[col], axis=1)) ** 2
    cnt = np.diff(ptr)
    ref = np.sqrt(np.bincount(rows, weights=e2, minlength=m) / np.maximum(cnt, 1))
    got = orc.row_rmse(ptr, col, val, U, V)
    assert np.abs(got - ref).max() <= 1e-13 * max(1.0, ref.max())
    assert (got[cnt == 0] == 0).all()


# --- P3's checker: the relative normal-equation residual |A u - b| / (|A| |u| + |b|)
# on a hand-built system.  Observed settings 1, 2, 3 (setting 0 is not observed),
# v1 = (1, 0), v2 = (0, 2), v3 = (3, 0), r = (1, 2, 3), lambda = 1:
#   A = diag(1 + 9 + 1, 4 + 1) = diag(11, 5),  b = (1 + 9, 4) = (10, 4),
#   |A|_F = sqrt(146), |b| = sqrt(116), exact solution u* = (10/11, 4/5).
def test_normal_residual_hand_system(orc):
    F = np.array([[7.0, 7.0], [1.0, 0.0], [0.0, 2.0], [3.0, 0.0]])
    idx = np.array([1, 2, 3], dtype=np.int32)
    val = np.array([1.0, 2.0, 3.0])
    lam = 1.0
    u_star = np.array([10.0 / 11.0, 0.8])
    assert orc.normal_residual(F, idx, val, lam, u_star) < 1e-16
    # u = (1, 1): A u - b = (1, 1)
    want = math.sqrt(2.0) / (math.sqrt(146.0) * math.sqrt(2.0) + math.sqrt(116.0))
    got = orc.normal_residual(F, idx, val, lam, np.array([1.0, 1.0]))
    assert abs(got - want) <= 1e-15, (got, want)
    # u = u* + d with d = (0.5, -0.25): A d = (5.5, -1.25)
    u = u_star + np.array([0.5, -0.25])
    want = math.sqrt(5.5 ** 2 + 1.25 ** 2) / (math.sqrt(146.0) * np.linalg.norm(u) +
                                              math.sqrt(116.0))
    got = orc.normal_residual(F, idx, val, lam, u)
    assert abs(got - want) <= 1e-15, (got, want)


def test_normal_residual_separates_solved_from_perturbed(orc):
    # the ridge solution from lstsq (P1's independent routine) has a residual at
    # rounding level; any perturbation of it must show, so P3 can fail
    rng = np.random.default_rng(12)
    for k in (1, 4, 9):
        F = rng.standard_normal((30, k))
        idx = np.sort(rng.choice(30, size=12, replace=False)).astype(np.int32)
        val = rng.standard_normal(12)
        lam = 0.3
        Aaug = np.vstack([F[idx], math.sqrt(lam) * np.eye(k)])
        u = np.linalg.lstsq(Aaug, np.concatenate([val, np.zeros(k)]), rcond=None)[0]
        assert orc.normal_residual(F, idx, val, lam, u) < 1e-14
        for scale in (1e-8, 1e-4):
            d = scale * rng.standard_normal(k)
            assert orc.normal_residual(F, idx, val, lam, u + d) > 1e-3 * scale
