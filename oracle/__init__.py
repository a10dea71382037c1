"""FP64 CPU oracle (ctypes binding of ``open_cf_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the CPU-baseline
leg of ``bench.py`` are the only users.  The product library never imports
this package, and this package imports nothing from the product.

Every function takes and returns numpy arrays; floating point is FP64 except
``select_f32`` (Algorithm 2 evaluated in FP32 so that the chosen index can be
compared bit-exactly with a kernel that decides in FP32).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "open_cf_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")

OK, NOT_SPD, EMPTY_ROW, FALLBACK_USED = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP, no fast-math, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=gnu11", "-O2", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None

_d = ctypes.POINTER(ctypes.c_double)
_f = ctypes.POINTER(ctypes.c_float)
_i64 = ctypes.POINTER(ctypes.c_int64)
_i32 = ctypes.POINTER(ctypes.c_int32)
_I64, _I32, _D, _F = ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_float


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        sig = {
            "orc_num_threads": (ctypes.c_int, []),
            "orc_set_num_threads": (None, [ctypes.c_int]),
            "orc_cholesky": (ctypes.c_int, [ctypes.c_int, _d, _d]),
            "orc_chol_solve": (None, [ctypes.c_int, _d, _d, _d]),
            "orc_normal_equations": (None, [ctypes.c_int, _D, _I64, _i32, _d, _d, _d, _d]),
            "orc_row_solve": (ctypes.c_int, [ctypes.c_int, _D, _I64, _i32, _d, _d, _d]),
            "orc_half_step": (None, [_I64, _i64, _i32, _d, _d, ctypes.c_int, _D, _d, _i32]),
            "orc_transpose": (None, [_I64, _I64, _i64, _i32, _d, _i64, _i32, _d]),
            "orc_objective": (_D, [_I64, _I64, _i64, _i32, _d, _d, _d, ctypes.c_int, _D]),
            "orc_row_rmse": (None, [_I64, _i64, _i32, _d, _d, _d, ctypes.c_int, _d]),
            "orc_normal_residual": (_D, [ctypes.c_int, _D, _I64, _i32, _d, _d, _d]),
            "orc_als": (None, [_I64, _I64, _i64, _i32, _d, ctypes.c_int, _D, ctypes.c_int,
                               _d, _d, _d, _i32, _i32]),
            "orc_als_dense": (None, [_I64, _I64, _d, ctypes.c_int, _D, ctypes.c_int, _d, _d,
                                     _d]),
            "orc_predict": (None, [_I64, _I64, ctypes.c_int, _d, _d, _d]),
            "orc_select_f64": (None, [_I64, _I64, _d, _I32, _d, _d, _D, _I64, _i32, _d]),
            "orc_select_f32": (None, [_I64, _I64, _f, _I32, _f, _f, _F, _I64, _i32, _f]),
            "orc_mlp_forward": (None, [_I64] + [ctypes.c_int] * 4 + [_d] * 10),
            "orc_mlp_loss_grad": (_D, [_I64] + [ctypes.c_int] * 4 + [_d] * 15),
            "orc_adam": (None, [_I64, _d, _d, _d, _d, _I64, _D, _D, _D, _D]),
            "orc_mlp_features": (None, [_I64, _i64, _i32, _d, _I32, _I32, _d, _d,
                                        ctypes.c_int, _d]),
            "orc_phase_detect": (None, [_I64, _I64, _I64, _f, _F, _I32, _I32, _i64]),
            "orc_half_step_wr": (None, [_I64, _i64, _i32, _d, _d, ctypes.c_int, _D, _d, _i32]),
            "orc_objective_wr": (_D, [_I64, _I64, _i64, _i32, _d, _d, _d, ctypes.c_int, _D]),
            "orc_als_wr": (None, [_I64, _I64, _i64, _i32, _d, ctypes.c_int, _D, ctypes.c_int,
                                  _d, _d, _d]),
            "orc_stream_accumulate": (None, [_I64, _i64, _i32, _d, _d, ctypes.c_int, _d, _d,
                                             _i64]),
            "orc_stream_solve": (None, [_I64, ctypes.c_int, _d, _d, _i64, _D, ctypes.c_int, _d,
                                        _i32]),
            "orc_ncf_net_size": (_I64, [ctypes.c_int] * 3),
            "orc_ncf_forward": (None, [_I64, _i32, _i32] + [ctypes.c_int] * 3 + [_d] * 6),
            "orc_ncf_loss_grad": (_D, [_I64, _i32, _i32, _d, _I64, _I64] + [ctypes.c_int] * 3 +
                                  [_d] * 6),
            "orc_ncf_predict": (None, [_I64, _I64] + [ctypes.c_int] * 3 + [_d] * 4),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def num_threads() -> int:
    return int(lib().orc_num_threads())


def set_num_threads(t: int) -> None:
    lib().orc_set_num_threads(int(t))


def cholesky(A):
    A = _c(A, np.float64)
    k = A.shape[0]
    L = np.zeros((k, k))
    st = lib().orc_cholesky(k, _p(A, _d), _p(L, _d))
    return L, st


def chol_solve(L, b):
    L = _c(L, np.float64); b = _c(b, np.float64)
    x = np.zeros_like(b)
    lib().orc_chol_solve(L.shape[0], _p(L, _d), _p(b, _d), _p(x, _d))
    return x


def normal_equations(F, idx, val, lam):
    F = _c(F, np.float64); idx = _c(idx, np.int32); val = _c(val, np.float64)
    k = F.shape[1]
    A = np.zeros((k, k)); b = np.zeros(k)
    lib().orc_normal_equations(k, lam, len(idx), _p(idx, _i32), _p(val, _d), _p(F, _d),
                               _p(A, _d), _p(b, _d))
    return A, b


def row_solve(F, idx, val, lam):
    F = _c(F, np.float64); idx = _c(idx, np.int32); val = _c(val, np.float64)
    u = np.zeros(F.shape[1])
    st = lib().orc_row_solve(F.shape[1], lam, len(idx), _p(idx, _i32), _p(val, _d), _p(F, _d),
                             _p(u, _d))
    return u, st


def half_step(row_ptr, col, val, F, lam):
    """Solve every CSR row against the fixed other factor F; returns (out, status)."""
    row_ptr = _c(row_ptr, np.int64); col = _c(col, np.int32); val = _c(val, np.float64)
    F = _c(F, np.float64)
    m = len(row_ptr) - 1
    k = F.shape[1]
    out = np.zeros((m, k)); st = np.zeros(m, dtype=np.int32)
    lib().orc_half_step(m, _p(row_ptr, _i64), _p(col, _i32), _p(val, _d), _p(F, _d), k, lam,
                        _p(out, _d), _p(st, _i32))
    return out, st


def transpose(row_ptr, col, val, n):
    row_ptr = _c(row_ptr, np.int64); col = _c(col, np.int32); val = _c(val, np.float64)
    m = len(row_ptr) - 1
    nnz = int(row_ptr[-1])
    cptr = np.zeros(n + 1, dtype=np.int64)
    cidx = np.zeros(max(nnz, 1), dtype=np.int32)
    cval = np.zeros(max(nnz, 1))
    lib().orc_transpose(m, n, _p(row_ptr, _i64), _p(col, _i32), _p(val, _d), _p(cptr, _i64),
                        _p(cidx, _i32), _p(cval, _d))
    return cptr, cidx[:nnz], cval[:nnz]


def objective(row_ptr, col, val, U, V, lam):
    row_ptr = _c(row_ptr, np.int64); col = _c(col, np.int32); val = _c(val, np.float64)
    U = _c(U, np.float64); V = _c(V, np.float64)
    return float(lib().orc_objective(len(row_ptr) - 1, V.shape[0], _p(row_ptr, _i64),
                                     _p(col, _i32), _p(val, _d), _p(U, _d), _p(V, _d),
                                     U.shape[1], lam))


def row_rmse(row_ptr, col, val, U, V):
    row_ptr = _c(row_ptr, np.int64); col = _c(col, np.int32); val = _c(val, np.float64)
    U = _c(U, np.float64); V = _c(V, np.float64)
    out = np.zeros(len(row_ptr) - 1)
    lib().orc_row_rmse(len(row_ptr) - 1, _p(row_ptr, _i64), _p(col, _i32), _p(val, _d),
                       _p(U, _d), _p(V, _d), U.shape[1], _p(out, _d))
    return out


def normal_residual(F, idx, val, lam, u):
    F = _c(F, np.float64); idx = _c(idx, np.int32); val = _c(val, np.float64)
    u = _c(u, np.float64)
    return float(lib().orc_normal_residual(F.shape[1], lam, len(idx), _p(idx, _i32),
                                           _p(val, _d), _p(F, _d), _p(u, _d)))


def als(row_ptr, col, val, n, V0, lam, sweeps, history=False):
    """ALS from V0; returns (U, V, J_hist or None, row_status, col_status)."""
    row_ptr = _c(row_ptr, np.int64); col = _c(col, np.int32); val = _c(val, np.float64)
    V = np.array(V0, dtype=np.float64, copy=True, order="C")
    m = len(row_ptr) - 1
    k = V.shape[1]
    U = np.zeros((m, k))
    J = np.zeros(2 * sweeps) if history else None
    rs = np.zeros(m, dtype=np.int32); cs = np.zeros(n, dtype=np.int32)
    lib().orc_als(m, n, _p(row_ptr, _i64), _p(col, _i32), _p(val, _d), k, lam, sweeps,
                  _p(U, _d), _p(V, _d), _p(J, _d) if history else None, _p(rs, _i32),
                  _p(cs, _i32))
    return U, V, J, rs, cs


def als_dense(P, V0, lam, sweeps, history=False):
    P = _c(P, np.float64)
    V = np.array(V0, dtype=np.float64, copy=True, order="C")
    m, n = P.shape
    k = V.shape[1]
    U = np.zeros((m, k))
    J = np.zeros(2 * sweeps) if history else None
    lib().orc_als_dense(m, n, _p(P, _d), k, lam, sweeps, _p(U, _d), _p(V, _d),
                        _p(J, _d) if history else None)
    return U, V, J


def predict(U, V):
    U = _c(U, np.float64); V = _c(V, np.float64)
    T = np.zeros((U.shape[0], V.shape[0]))
    lib().orc_predict(U.shape[0], V.shape[0], U.shape[1], _p(U, _d), _p(V, _d), _p(T, _d))
    return T


def baseline_index(cpu_caps, gpu_caps):
    """Index of the (max CPU cap, max GPU cap) setting, CPU-major."""
    return int(np.argmax(cpu_caps)) * len(gpu_caps) + int(np.argmax(gpu_caps))


def select_f64(T, cpu_caps, gpu_caps, gamma, base=None):
    T = _c(T, np.float64)
    cpu = _c(cpu_caps, np.float64); gpu = _c(gpu_caps, np.float64)
    base = baseline_index(cpu, gpu) if base is None or base < 0 else int(base)
    m, n = T.shape
    best = np.zeros(m, dtype=np.int32); sav = np.zeros(m)
    lib().orc_select_f64(m, n, _p(T, _d), len(gpu), _p(cpu, _d), _p(gpu, _d), gamma, base,
                         _p(best, _i32), _p(sav, _d))
    return best, sav


def select_f32(T, cpu_caps, gpu_caps, gamma, base=None):
    T = _c(T, np.float32)
    cpu = _c(cpu_caps, np.float32); gpu = _c(gpu_caps, np.float32)
    base = baseline_index(cpu, gpu) if base is None or base < 0 else int(base)
    m, n = T.shape
    best = np.zeros(m, dtype=np.int32); sav = np.zeros(m, dtype=np.float32)
    lib().orc_select_f32(m, n, _p(T, _f), len(gpu), _p(cpu, _f), _p(gpu, _f),
                         np.float32(gamma), base, _p(best, _i32), _p(sav, _f))
    return best, sav


def mlp_forward(X, params):
    """params = [W1, b1, W2, b2, W3, b3] with W [in, out]; returns (Z1, Z2, Y)."""
    X = _c(X, np.float64)
    P = [_c(p, np.float64) for p in params]
    B, din = X.shape
    h1, h2, dout = P[0].shape[1], P[2].shape[1], P[4].shape[1]
    Z1 = np.zeros((B, h1)); Z2 = np.zeros((B, h2)); Y = np.zeros((B, dout))
    lib().orc_mlp_forward(B, din, h1, h2, dout, _p(X, _d), *[_p(p, _d) for p in P],
                          _p(Z1, _d), _p(Z2, _d), _p(Y, _d))
    return Z1, Z2, Y


def mlp_loss_grad(X, params, Ytgt, G):
    X = _c(X, np.float64)
    P = [_c(p, np.float64) for p in params]
    Ytgt = _c(Ytgt, np.float64); G = _c(G, np.float64)
    B, din = X.shape
    h1, h2, dout = P[0].shape[1], P[2].shape[1], P[4].shape[1]
    grads = [np.zeros_like(p) for p in P]
    L = lib().orc_mlp_loss_grad(B, din, h1, h2, dout, _p(X, _d), *[_p(p, _d) for p in P],
                                _p(Ytgt, _d), _p(G, _d), *[_p(g, _d) for g in grads])
    return float(L), grads


def adam(theta, g, m1, m2, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """In-place Adam step on flat FP64 arrays."""
    for a in (theta, g, m1, m2):
        assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    lib().orc_adam(theta.size, _p(theta, _d), _p(g, _d), _p(m1, _d), _p(m2, _d), int(t), lr,
                   beta1, beta2, eps)


def mlp_features(row_ptr, col, val, cpu_caps, gpu_caps, s_in=16):
    row_ptr = _c(row_ptr, np.int64); col = _c(col, np.int32); val = _c(val, np.float64)
    cpu = _c(cpu_caps, np.float64); gpu = _c(gpu_caps, np.float64)
    m = len(row_ptr) - 1
    X = np.zeros((m, 3 * s_in))
    lib().orc_mlp_features(m, _p(row_ptr, _i64), _p(col, _i32), _p(val, _d), len(cpu), len(gpu),
                           _p(cpu, _d), _p(gpu, _d), s_in, _p(X, _d))
    return X


def phase_detect(power, p_th=60.0, window=25, intervals=5):
    """Algorithm 1 on each row of `power` (float32 [traces, len]); returns the
    index of the sample at which a transition is first reported, or -1."""
    power = _c(np.atleast_2d(power), np.float32)
    n, L = power.shape
    first = np.zeros(n, dtype=np.int64)
    if window % intervals:
        intervals = 1
    lib().orc_phase_detect(n, L, L, _p(power, _f), np.float32(p_th), int(window), int(intervals),
                           _p(first, _i64))
    return first


def half_step_wr(row_ptr, col, val, F, lam):
    """Weighted-lambda (ALS-WR) half-step: row i solved with lambda * s_i."""
    row_ptr = _c(row_ptr, np.int64); col = _c(col, np.int32); val = _c(val, np.float64)
    F = _c(F, np.float64)
    m, k = len(row_ptr) - 1, F.shape[1]
    out = np.zeros((m, k)); st = np.zeros(m, dtype=np.int32)
    lib().orc_half_step_wr(m, _p(row_ptr, _i64), _p(col, _i32), _p(val, _d), _p(F, _d), k, lam,
                           _p(out, _d), _p(st, _i32))
    return out, st


def objective_wr(row_ptr, col, val, U, V, lam):
    row_ptr = _c(row_ptr, np.int64); col = _c(col, np.int32); val = _c(val, np.float64)
    U = _c(U, np.float64); V = _c(V, np.float64)
    return float(lib().orc_objective_wr(len(row_ptr) - 1, V.shape[0], _p(row_ptr, _i64),
                                        _p(col, _i32), _p(val, _d), _p(U, _d), _p(V, _d),
                                        U.shape[1], lam))


def als_wr(row_ptr, col, val, n, V0, lam, sweeps, history=False):
    """ALS-WR from V0; returns (U, V, J_hist or None)."""
    row_ptr = _c(row_ptr, np.int64); col = _c(col, np.int32); val = _c(val, np.float64)
    V = np.array(V0, dtype=np.float64, copy=True, order="C")
    m, k = len(row_ptr) - 1, V.shape[1]
    U = np.zeros((m, k))
    J = np.zeros(2 * sweeps) if history else None
    lib().orc_als_wr(m, n, _p(row_ptr, _i64), _p(col, _i32), _p(val, _d), k, lam, sweeps,
                     _p(U, _d), _p(V, _d), _p(J, _d) if history else None)
    return U, V, J


# ---------------------------------------------------------------- NCF
def ncf_net_size(d, h1, h2):
    return int(lib().orc_ncf_net_size(d, h1, h2))


def ncf_forward(ai, sj, Ea, Es, net, h1, h2, keep=False):
    """Predicted entries y[b] for the pairs (ai[b], sj[b]); with keep, also
    the pre-activations (Z1, Z2)."""
    ai = _c(ai, np.int32); sj = _c(sj, np.int32)
    Ea = _c(Ea, np.float64); Es = _c(Es, np.float64); net = _c(net, np.float64)
    B, d = len(ai), Ea.shape[1]
    assert net.size == ncf_net_size(d, h1, h2)
    y = np.zeros(B)
    Z1 = np.zeros((B, h1)) if keep else None
    Z2 = np.zeros((B, h2)) if keep else None
    lib().orc_ncf_forward(B, _p(ai, _i32), _p(sj, _i32), d, h1, h2, _p(Ea, _d), _p(Es, _d),
                          _p(net, _d), _p(y, _d), _p(Z1, _d) if keep else None,
                          _p(Z2, _d) if keep else None)
    return (y, Z1, Z2) if keep else y


def ncf_loss_grad(ai, sj, r, Ea, Es, net, h1, h2):
    """(L, g_net, gEa, gEs) of the batch's mean squared error."""
    ai = _c(ai, np.int32); sj = _c(sj, np.int32); r = _c(r, np.float64)
    Ea = _c(Ea, np.float64); Es = _c(Es, np.float64); net = _c(net, np.float64)
    (m, d), n = Ea.shape, Es.shape[0]
    g_net = np.zeros_like(net); gEa = np.zeros_like(Ea); gEs = np.zeros_like(Es)
    L = lib().orc_ncf_loss_grad(len(ai), _p(ai, _i32), _p(sj, _i32), _p(r, _d), m, n, d, h1, h2,
                                _p(Ea, _d), _p(Es, _d), _p(net, _d), _p(g_net, _d),
                                _p(gEa, _d), _p(gEs, _d))
    return float(L), g_net, gEa, gEs


def ncf_predict(Ea, Es, net, h1, h2):
    """The completed matrix T[i, j] = y(i, j) over every application and setting."""
    Ea = _c(Ea, np.float64); Es = _c(Es, np.float64); net = _c(net, np.float64)
    (m, d), n = Ea.shape, Es.shape[0]
    T = np.zeros((m, n))
    lib().orc_ncf_predict(m, n, d, h1, h2, _p(Ea, _d), _p(Es, _d), _p(net, _d), _p(T, _d))
    return T


def ncf_train(ai, sj, r, Ea, Es, net, h1, h2, perms, batch, lr, beta1=0.9, beta2=0.999,
              eps=1e-8):
    """Mini-batch Adam over the observed entries: epoch e visits them in the
    order perms[e] in consecutive batches of `batch` (the last one shorter);
    Adam runs on the packed vector [net, Ea, Es].  Returns (net, Ea, Es,
    per-step losses)."""
    ai = np.asarray(ai, np.int32); sj = np.asarray(sj, np.int32); r = np.asarray(r, np.float64)
    m, d = np.shape(Ea); n = np.shape(Es)[0]
    nn = np.asarray(net).size
    theta = np.concatenate([np.asarray(net, np.float64).ravel(),
                            np.asarray(Ea, np.float64).ravel(),
                            np.asarray(Es, np.float64).ravel()])
    m1 = np.zeros_like(theta); m2 = np.zeros_like(theta)
    losses = []
    t = 0
    for perm in perms:
        for b0 in range(0, len(perm), batch):
            sel = perm[b0:b0 + batch]
            net_, Ea_, Es_ = (theta[:nn], theta[nn:nn + m * d].reshape(m, d),
                              theta[nn + m * d:].reshape(n, d))
            L, gn, ga, gs = ncf_loss_grad(ai[sel], sj[sel], r[sel], Ea_, Es_, net_, h1, h2)
            g = np.concatenate([gn, ga.ravel(), gs.ravel()])
            t += 1
            adam(theta, g, m1, m2, t, lr, beta1, beta2, eps)
            losses.append(L)
    return (theta[:nn].copy(), theta[nn:nn + m * d].reshape(m, d).copy(),
            theta[nn + m * d:].reshape(n, d).copy(), np.array(losses))


# ---------------------------------------------------------------- streaming refit
class StreamState:
    """Per-setting sums of the V-half-step's normal equations over every row
    ingested so far (G [n, k, k], b [n, k], counts [n]) and the current V."""

    def __init__(self, n, k, lam, weighted=False):
        self.n, self.k, self.lam, self.weighted = n, k, float(lam), bool(weighted)
        self.G = np.zeros((n, k, k))
        self.b = np.zeros((n, k))
        self.cnt = np.zeros(n, dtype=np.int64)
        self.V = np.zeros((n, k))
        self.status = np.zeros(n, dtype=np.int32)

    def add(self, row_ptr, col, val, U):
        """Add the rank-one terms of rows with known factors U, then re-solve V."""
        row_ptr = _c(row_ptr, np.int64); col = _c(col, np.int32); val = _c(val, np.float64)
        U = _c(U, np.float64)
        lib().orc_stream_accumulate(len(row_ptr) - 1, _p(row_ptr, _i64), _p(col, _i32),
                                    _p(val, _d), _p(U, _d), self.k, _p(self.G, _d),
                                    _p(self.b, _d), _p(self.cnt, _i64))
        return self.solve()

    def solve(self):
        """V from the current sums (after they were changed from outside)."""
        lib().orc_stream_solve(self.n, self.k, _p(self.G, _d), _p(self.b, _d),
                               _p(self.cnt, _i64), self.lam, int(self.weighted), _p(self.V, _d),
                               _p(self.status, _i32))
        return self.V

    def ingest(self, row_ptr, col, val):
        """A batch of new applications: fold-in against the current V, then add."""
        fold = half_step_wr if self.weighted else half_step
        U, st = fold(row_ptr, col, val, self.V, self.lam)
        self.add(row_ptr, col, val, U)
        return U, st


# ---------------------------------------------------------------- performance predictor
def pred_unpack(params, n_features, h1=128, h2=64):
    """Packed [W1 (nf x h1), b1, W2 (h1 x h2), b2, w3, b3] -> the layer list of
    mlp_forward / mlp_loss_grad (output width 1)."""
    p = np.asarray(params, dtype=np.float64)
    o, out = 0, []
    for shape in [(n_features, h1), (h1,), (h1, h2), (h2,), (h2, 1), (1,)]:
        size = int(np.prod(shape))
        out.append(p[o:o + size].reshape(shape))
        o += size
    assert o == p.size
    return out


def pred_forward(X, params, n_features):
    return mlp_forward(X, pred_unpack(params, n_features))[2][:, 0]


def pred_loss_grad(X, y, params, n_features):
    """Mean squared error of the predictor on (X, y) and its packed gradient."""
    L, grads = mlp_loss_grad(X, pred_unpack(params, n_features), np.asarray(y)[:, None],
                             np.ones((1, 1)))
    return L, np.concatenate([g.ravel() for g in grads])


def pred_train(X, y, params, n_features, perms, batch, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """Mini-batch Adam over the samples in the orders perms[e]; returns
    (packed parameters, per-step losses)."""
    theta = np.array(params, dtype=np.float64, copy=True)
    m1 = np.zeros_like(theta); m2 = np.zeros_like(theta)
    X = np.asarray(X, np.float64); y = np.asarray(y, np.float64)
    losses, t = [], 0
    for perm in perms:
        for b0 in range(0, len(perm), batch):
            sel = perm[b0:b0 + batch]
            L, g = pred_loss_grad(X[sel], y[sel], theta, n_features)
            t += 1
            adam(theta, g, m1, m2, t, lr, beta1, beta2, eps)
            losses.append(L)
    return theta, np.array(losses)
