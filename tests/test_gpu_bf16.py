"""BF16-Gram path (Gram and right-hand side from BF16 copies of the factors on
tensor cores, FP32 accumulation, FP32 or FP64 Cholesky) against the FP64
oracle.  Gate: per-row relative error of the predicted runtimes t = u V^T,
|t_gpu - t_oracle| / |t_oracle| <= 2e-3, with the oracle fed the same FP32
V and observations (the BF16 rounding is the path's own approximation)."""
import numpy as np
import pytest
import torch

import synth

from gpu_util import DEV, csr_dev, dev, host, rounded

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2508_07605_b300 as ocf  # noqa: E402

TOL_T = 2e-3


def _pred_err(U_gpu, U_ref, V):
    Tg = np.asarray(U_gpu, np.float64) @ V.T
    Tr = np.asarray(U_ref, np.float64) @ V.T
    return np.linalg.norm(Tg - Tr, axis=1) / np.maximum(np.linalg.norm(Tr, axis=1), 1e-30)


@pytest.mark.parametrize("k,chol64", [(32, True), (32, False), (16, False), (8, True), (24, True),
                                       (17, True)])
def test_bf16_foldin_matches_oracle(orc, k, chol64):
    """Fold-in of new rows against a fixed V at the shape of the large
    workload (4096 settings, ~1 % observed), scaled down in rows."""
    prob = synth.make_sparse_problem(seed=k, m=3000, n_cpu=64, n_gpu=64, rank=k, density=0.01,
                                     k=k, lam=0.05, n_heldout=8)
    rng = np.random.default_rng(k)
    V = rounded(rng.standard_normal((prob.n, k)) / 2.0, torch.float32)
    val = rounded(prob.val, torch.float32)
    h = ocf.OpenCF(k=k, lam=prob.lam, precision="bf16_gram", cholesky_fp64=chol64)
    h.set_V(dev(V, torch.float32))
    U, st = h.complete_rows(*csr_dev(prob.row_ptr, prob.col, val, torch.float32))
    torch.cuda.synchronize()
    Uref, sref = orc.half_step(prob.row_ptr, prob.col, val, V, prob.lam)
    assert np.array_equal(host(st), sref)
    ok = np.diff(prob.row_ptr) > 0
    err = _pred_err(host(U), Uref, V)[ok]
    assert err.max() <= TOL_T, (err.max(), np.median(err))


def test_bf16_one_sweep_stepwise(orc):
    prob = synth.make_sparse_problem(seed=3, m=600, n_cpu=4, n_gpu=32, rank=16, density=0.1,
                                     k=16, lam=0.05, sweeps=1, n_heldout=8)
    val = rounded(prob.val, torch.float32)
    V0 = rounded(prob.V0, torch.float32)
    h = ocf.OpenCF(k=16, lam=prob.lam, sweeps=1, precision="bf16_gram")
    h.set_V(dev(V0, torch.float32))
    U1 = h.fit_csr(*csr_dev(prob.row_ptr, prob.col, val, torch.float32), prob.n)
    V1 = h.get_V()
    torch.cuda.synchronize()
    Uref, _ = orc.half_step(prob.row_ptr, prob.col, val, V0, prob.lam)
    assert _pred_err(host(U1), Uref, V0).max() <= TOL_T
    cptr, cidx, cval = orc.transpose(prob.row_ptr, prob.col, val, prob.n)
    U1d = host(U1).astype(np.float64)
    Vref, _ = orc.half_step(cptr, cidx, cval, U1d, prob.lam)
    assert _pred_err(host(V1), Vref, U1d).max() <= TOL_T


def test_bf16_fit_heldout_rmse(orc):
    prob = synth.make_sparse_problem(seed=5, m=800, n_cpu=4, n_gpu=64, rank=16, density=0.08,
                                     k=16, lam=0.05, sweeps=15, n_heldout=8192)
    val = rounded(prob.val, torch.float32)
    h = ocf.OpenCF(k=16, lam=prob.lam, sweeps=15, precision="bf16_gram")
    h.set_V(dev(prob.V0, torch.float32))
    U = h.fit_csr(*csr_dev(prob.row_ptr, prob.col, val, torch.float32), prob.n)
    V = h.get_V()
    torch.cuda.synchronize()
    Ur, Vr, _, _, _ = orc.als(prob.row_ptr, prob.col, val, prob.n, prob.V0, prob.lam, 15)
    def rmse(U_, V_):
        p = np.einsum("tk,tk->t", np.asarray(U_, np.float64)[prob.heldout_rows],
                      np.asarray(V_, np.float64)[prob.heldout_cols])
        return np.sqrt(np.mean((p - prob.heldout_truth) ** 2))
    assert rmse(host(U), host(V)) <= rmse(Ur, Vr) + 1e-3


def test_bf16_large_foldin_sampled(orc):
    """1M apps x 4096 settings, k=32, 1 % observed, FP64 Cholesky, in the
    configuration the large-workload benchmark times; the oracle re-solves a
    10k-row sample in FP64 from the identical V and observations."""
    prob = synth.make_large_foldin(seed=0, device=DEV)
    h = ocf.OpenCF(k=32, lam=prob.lam, precision="bf16_gram", cholesky_fp64=True)
    h.set_V(prob.V)
    U, st = h.complete_rows(prob.row_ptr, prob.col, prob.val)
    torch.cuda.synchronize()
    rng = np.random.default_rng(0)
    rows = np.sort(rng.choice(prob.m, 10000, replace=False))
    rp = host(prob.row_ptr)
    col = host(prob.col)
    val = host(prob.val).astype(np.float64)
    V = host(prob.V).astype(np.float64)
    sp = [0]; sc = []; sv = []
    for i in rows:
        sc.append(col[rp[i]:rp[i + 1]]); sv.append(val[rp[i]:rp[i + 1]])
        sp.append(sp[-1] + rp[i + 1] - rp[i])
    Uref, sref = orc.half_step(np.array(sp), np.concatenate(sc), np.concatenate(sv), V, prob.lam)
    assert np.array_equal(host(st)[rows], sref)
    err = _pred_err(host(U)[rows], Uref, V)
    ok = np.diff(np.array(sp)) > 0
    assert err[ok].max() <= TOL_T, (err[ok].max(), np.median(err[ok]))


def _pred_inputs(rng, m, n, k):
    U = rounded(rng.standard_normal((m, k)) * 0.3, torch.float32)
    V = rounded(rng.standard_normal((n, k)) * 0.3, torch.float32)
    U[:, 0] = np.abs(U[:, 0]) + 1.5          # most predicted runtimes positive
    V[:, 0] = np.abs(V[:, 0]) + 0.5
    return U, V


@pytest.mark.parametrize("m,n_cpu,n_gpu,baseline", [
    (1, 64, 64, -1),                # one row, 16 chunks of 256 settings
    (300, 20, 50, -1),              # ragged last chunk (1000 settings)
    (148 * 128 + 77, 16, 64, 700),  # more tiles than SMs, a ragged tile; baseline in chunk 2
    (517, 8, 15, 3),                # fewer settings than one chunk
])
@pytest.mark.parametrize("gamma", [0.0, 0.1])
def test_bf16_predict_select_tensor_cores(orc, m, n_cpu, n_gpu, baseline, gamma):
    """k = 32 in BF16-Gram mode: T = U V^T from split BF16 operands on the
    tensor cores.  T against the FP64 oracle within the BF16 gate; the
    selection bit for bit equal to the oracle's FP32 Algorithm 2 on the T the
    kernel wrote; the same decisions without the dense output."""
    rng = np.random.default_rng(m + n_cpu)
    k = 32
    n = n_cpu * n_gpu
    U, V = _pred_inputs(rng, m, n, k)
    if m > 5:
        U[5] = 0.0                          # a row whose baseline runtime is 0
    cpu, gpu = synth.cap_grid(n_cpu, n_gpu)
    h = ocf.OpenCF(k=k, lam=0.05, precision="bf16_gram", cpu_caps=cpu, gpu_caps=gpu)
    h.set_V(dev(V, torch.float32))
    T, best, sav = h.predict(dev(U, torch.float32), gamma=gamma, baseline=baseline)
    _, best2, sav2 = h.predict(dev(U, torch.float32), gamma=gamma, baseline=baseline,
                               want_T=False)
    torch.cuda.synchronize()
    Tg = host(T).astype(np.float64)
    Tr = orc.predict(U, V)
    ok = np.linalg.norm(Tr, axis=1) > 0
    err = np.linalg.norm(Tg - Tr, axis=1)[ok] / np.linalg.norm(Tr, axis=1)[ok]
    assert err.max() <= 1e-4, err.max()   # split BF16: ~2^-16 relative, well inside 2e-3
    b_or, s_or = orc.select_f32(host(T).astype(np.float32), cpu, gpu, gamma,
                                baseline if baseline >= 0 else -1)
    assert np.array_equal(host(best), b_or)
    assert np.array_equal(host(sav), s_or)
    assert torch.equal(best, best2) and torch.equal(sav, sav2)
    if m > 5:
        assert host(best)[5] == -1
