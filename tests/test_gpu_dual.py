"""Thin rows at rank 17..32: rows with at most 16 observations are solved from
the 16 x 16 dual system (u = S^T w, (S S^T + lambda I) w = r) when both rows of
a solver pair are thin, and from the k x k normal equations otherwise (FP32
mode adds one refinement step of the dual system).  Both branches against the
FP64 oracle's primal row solve on the same inputs."""
import numpy as np
import pytest
import torch

import synth

from gpu_util import TOL_FP32, csr_dev, dev, host, rounded, row_rel_err, solve_err

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2508_07605_b300 as ocf  # noqa: E402

TOL_T = 2e-3   # BF16-Gram path: per-row relative error of the predicted runtimes


def _thin_csr(rng, m, n, mix):
    """Every length 0..16 first (pairs of thin rows, a thin row beside an empty
    one), then random thin lengths, or (mix) thin and thick rows alternating in
    runs so that some pairs take the primal branch."""
    lens = list(range(17)) + [16, 16, 0, 1]
    while len(lens) < m:
        if mix and rng.random() < 0.3:
            lens += [int(rng.integers(17, 60))] * int(rng.integers(1, 4))
        else:
            lens.append(int(rng.integers(0, 17)))
    lens = lens[:m]
    ptr = [0]; cols = []
    for s in lens:
        c = np.sort(rng.choice(n, size=s, replace=False)).astype(np.int32)
        cols.append(c); ptr.append(ptr[-1] + s)
    return np.array(ptr, dtype=np.int64), np.concatenate(cols)


@pytest.mark.parametrize("k", [17, 24, 32])
@pytest.mark.parametrize("mix", [False, True])
@pytest.mark.parametrize("weighted", [False, True])
def test_dual_foldin_fp32(orc, k, mix, weighted):
    rng = np.random.default_rng(7 * k + mix + 2 * weighted)
    n, m, lam = 300, 611, 0.05
    ptr, col = _thin_csr(rng, m, n, mix)
    val = rounded(rng.random(len(col)) + 0.2, torch.float32)
    V = rounded(rng.standard_normal((n, k)) / np.sqrt(k), torch.float32)
    h = ocf.OpenCF(k=k, lam=lam, weighted_lambda=weighted)
    h.set_V(dev(V, torch.float32))
    U, st = h.complete_rows(*csr_dev(ptr, col, val, torch.float32))
    torch.cuda.synchronize()
    fold = orc.half_step_wr if weighted else orc.half_step
    Uref, sref = fold(ptr, col, val, V, lam)
    assert np.array_equal(host(st), sref)
    ok = np.diff(ptr) > 0
    assert np.abs(host(U)[~ok]).max(initial=0.0) == 0.0
    err = solve_err(host(U), Uref, V, ptr, col, val, lam, weighted=weighted)
    assert err[ok].max() <= TOL_FP32, (err[ok].max(), int(np.argmax(np.where(ok, err, 0))))
    plain = row_rel_err(host(U), Uref)[ok]
    assert np.median(plain) <= TOL_FP32


@pytest.mark.parametrize("k", [17, 32])
@pytest.mark.parametrize("mix", [False, True])
def test_dual_foldin_bf16(orc, k, mix):
    rng = np.random.default_rng(100 + k + mix)
    n, m, lam = 4096, 733, 0.05
    ptr, col = _thin_csr(rng, m, n, mix)
    val = rounded(rng.random(len(col)) + 0.2, torch.float32)
    V = rounded(rng.standard_normal((n, k)) / 2.0, torch.float32)
    h = ocf.OpenCF(k=k, lam=lam, precision="bf16_gram")
    h.set_V(dev(V, torch.float32))
    U, st = h.complete_rows(*csr_dev(ptr, col, val, torch.float32))
    torch.cuda.synchronize()
    Uref, sref = orc.half_step(ptr, col, val, V, lam)
    assert np.array_equal(host(st), sref)
    ok = np.diff(ptr) > 0
    assert np.abs(host(U)[~ok]).max(initial=0.0) == 0.0
    Tg, Tr = host(U).astype(np.float64) @ V.T, Uref @ V.T
    err = np.linalg.norm(Tg - Tr, axis=1) / np.maximum(np.linalg.norm(Tr, axis=1), 1e-30)
    assert err[ok].max() <= TOL_T, err[ok].max()


def test_dual_bf16_sweep_stepwise(orc):
    """A rank-32 BF16-Gram sweep on a matrix whose rows and columns are both
    thin (~10 observations each): the U-half and the V-half take the dual
    branch, and the V-half reads the split BF16 copy of U the U-half wrote."""
    prob = synth.make_sparse_problem(seed=9, m=512, n_cpu=8, n_gpu=64, rank=32, density=0.02,
                                     k=32, lam=0.05, sweeps=1, n_heldout=8)
    assert np.diff(prob.row_ptr).max() <= 30
    val = rounded(prob.val, torch.float32)
    V0 = rounded(prob.V0, torch.float32)
    h = ocf.OpenCF(k=32, lam=prob.lam, sweeps=1, precision="bf16_gram")
    h.set_V(dev(V0, torch.float32))
    U1 = h.fit_csr(*csr_dev(prob.row_ptr, prob.col, val, torch.float32), prob.n)
    V1 = h.get_V()
    torch.cuda.synchronize()

    def pred_err(Ug, Ur, F):
        Tg, Tr = np.asarray(Ug, np.float64) @ F.T, Ur @ F.T
        return np.linalg.norm(Tg - Tr, axis=1) / np.maximum(np.linalg.norm(Tr, axis=1), 1e-30)

    Uref, _ = orc.half_step(prob.row_ptr, prob.col, val, V0, prob.lam)
    ok = np.diff(prob.row_ptr) > 0
    assert pred_err(host(U1), Uref, V0)[ok].max() <= TOL_T
    cptr, cidx, cval = orc.transpose(prob.row_ptr, prob.col, val, prob.n)
    U1d = host(U1).astype(np.float64)
    Vref, _ = orc.half_step(cptr, cidx, cval, U1d, prob.lam)
    okc = np.diff(cptr) > 0
    assert pred_err(host(V1), Vref, U1d)[okc].max() <= TOL_T


@pytest.mark.parametrize("decay", [0.0, 3.0])
def test_dual_as_accurate_as_normal_equations(orc, decay):
    """FP32 mode, rank 32, 16 observations per row (the learned workload's
    rows).  V's singular values fall by 10^decay, so some rows' observed
    factor rows are nearly dependent and S^T w cancels; the dual branch (with
    its refinement step) must stay as accurate as the 32 x 32 normal-equation
    solve, which the checked fold-in runs on the same rows."""
    rng = np.random.default_rng(31 + int(decay))
    k, n, m, lam = 32, 4096, 4000, 0.05
    Q = np.linalg.qr(rng.standard_normal((n, k)))[0]
    V = rounded(Q * np.logspace(0, -decay, k) * np.sqrt(n / k) * 0.6, torch.float32)
    cols = np.stack([np.sort(rng.choice(n, 16, replace=False)) for _ in range(m)])
    ptr = np.arange(0, 16 * m + 1, 16, dtype=np.int64)
    col = cols.reshape(-1).astype(np.int32)
    val = rounded(rng.random(16 * m) * 0.5 + 0.2, torch.float32)
    h = ocf.OpenCF(k=k, lam=lam)
    h.set_V(dev(V, torch.float32))
    csr = csr_dev(ptr, col, val, torch.float32)
    Ud, _ = h.complete_rows(*csr)                            # dual systems
    Up, _, _ = h.complete_rows_checked(*csr, refine=False)   # normal equations
    torch.cuda.synchronize()
    Uref, _ = orc.half_step(ptr, col, val, V, lam)

    def pred(U):
        T, Tr = np.asarray(U, np.float64) @ V.T, Uref @ V.T
        return np.linalg.norm(T - Tr, axis=1) / np.linalg.norm(Tr, axis=1)

    ed, ep = pred(host(Ud)), pred(host(Up))
    print(f"decay {decay}: dual max {ed.max():.2e} median {np.median(ed):.2e}; "
          f"normal equations max {ep.max():.2e} median {np.median(ep):.2e}")
    assert ed.max() <= 2 * ep.max() + 1e-7
    assert np.median(ed) <= 2 * np.median(ep) + 1e-8
