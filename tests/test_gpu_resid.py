"""Rank-32 fold-in with the final residual check, one refinement step, and
the normal-equation residual of given factors (the a9 residual), through the
C ABI, against the FP64 oracle.

Tolerances:
  * factors: FP32 mode (3-pass TF32 Gram, FP32 Cholesky) the FP32 gate 1e-5
    on solve_err; BF16-Gram mode 2e-3 on the predicted rows u V^T;
  * the residual |A u - b| / (|A|_F |u| + |b|): the GPU forms A and b in the
    handle's Gram precision, the oracle in FP64, so the two values differ by
    at most about the Gram's relative accuracy (the numerator moves by
    |dA||u| + |db|, the denominator is |A||u| + |b|): 2e-6 for the 3-pass
    TF32 Gram (operands split to ~2^-21), 1e-4 for the split-BF16 Gram
    (~2^-16).  Planted perturbations make the residual ~1e-2, so these are
    tight relative checks;
  * a solved row's own residual: at most 1e-5 (an FP32 solve's backward
    error is ~k 2^-24 ~ 2e-6 of |A||u|)."""
import numpy as np
import pytest
import torch

import synth

from gpu_util import DEV, TOL_FP32, csr_dev, dev, host, rounded, solve_err

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2508_07605_b300 as ocf  # noqa: E402

TOL_T = 2e-3
TOL_RES = {"fp32": 2e-6, "bf16_gram": 1e-4}


def _ragged(seed, m, n, k):
    """Rows of 0, 1, 31, 32, 33, 64, 97 observations, then random 0..80."""
    rng = np.random.default_rng(seed)
    counts = rng.integers(0, 81, m)
    counts[:7] = [0, 1, 31, 32, 33, 64, 97]
    ptr = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    col = np.concatenate([np.sort(rng.choice(n, c, replace=False)) for c in counts]).astype(np.int32)
    val = rounded(rng.standard_normal(ptr[-1]), torch.float32)
    V = rounded(rng.standard_normal((n, k)) / np.sqrt(k), torch.float32)
    return ptr, col, val, V


def _pred_err(U, Uref, V):
    T, Tr = np.asarray(U, np.float64) @ V.T, Uref @ V.T
    return np.linalg.norm(T - Tr, axis=1) / np.maximum(np.linalg.norm(Tr, axis=1), 1e-30)


def _handle(k, lam, precision, V):
    h = ocf.OpenCF(k=k, lam=lam, precision=precision)
    h.set_V(dev(V, torch.float32))
    return h


@pytest.mark.parametrize("precision", ["fp32", "bf16_gram"])
@pytest.mark.parametrize("k", [20, 32])
def test_checked_foldin_matches_oracle(orc, precision, k):
    ptr, col, val, V = _ragged(k, 1500, 700, k)
    lam = 0.05
    h = _handle(k, lam, precision, V)
    csr = csr_dev(ptr, col, val, torch.float32)
    U0, st0 = h.complete_rows(*csr)
    U1, st1, r1 = h.complete_rows_checked(*csr, refine=False)
    U2, st2, r2 = h.complete_rows_checked(*csr, refine=True)
    torch.cuda.synchronize()
    Uref, sref = orc.half_step(ptr, col, val, V, lam)
    # the check alone changes nothing where the plain fold-in runs the same
    # solver: rows of more than 16 observations (the plain fold-in solves
    # thinner rows from the 16 x 16 dual system, the checked one from the
    # normal equations it checks; both against the oracle below)
    thick = torch.as_tensor(np.diff(ptr) > 16, device=DEV)
    assert torch.equal(U0[thick], U1[thick]) and torch.equal(st0, st1)
    for st in (st1, st2):
        assert np.array_equal(host(st), sref)
    ok = sref == 0
    for U in (U0, U1, U2):
        if precision == "fp32":
            err = solve_err(host(U), Uref, V, ptr, col, val, lam)[ok]
            assert err.max() <= TOL_FP32, err.max()
        else:
            err = _pred_err(host(U), Uref, V)[ok]
            assert err.max() <= TOL_T, err.max()
    for r in (r1, r2):
        r = host(r)
        assert (r[~ok] == -1).all()
        assert (r[ok] >= 0).all() and r[ok].max() <= 1e-5, r[ok].max()
    # the reported residual of the refined rows (the first residual updated by the
    # step taken) against the double-FP32 residual recomputed for the refined U:
    # the update's FP32 error is ~k kappa eps^2 |A||u| against a residual of
    # ~eps |A||u| (measured: within 1.2e-5 relative; gate 1e-3)
    rg = host(h.normal_residual(*csr, U2))
    r2h = host(r2)
    assert np.allclose(rg[ok], r2h[ok], rtol=0, atol=1e-7)
    rel = np.abs(rg[ok] - r2h[ok]) / np.maximum(rg[ok], 1e-12)
    print(f"refined residual vs recomputed: max rel diff {rel.max():.2e}, median {np.median(rel):.2e}")
    assert (np.abs(rg[ok] - r2h[ok]) <= 1e-3 * rg[ok] + 1e-12).all()


@pytest.mark.parametrize("precision", ["fp32", "bf16_gram"])
def test_normal_residual_matches_oracle(orc, precision):
    k, lam = 32, 0.05
    ptr, col, val, V = _ragged(40, 600, 500, k)
    h = _handle(k, lam, precision, V)
    csr = csr_dev(ptr, col, val, torch.float32)
    Uref, _ = orc.half_step(ptr, col, val, V, lam)
    rng = np.random.default_rng(41)
    scale = np.maximum(np.linalg.norm(Uref, axis=1, keepdims=True), 1e-3) / np.sqrt(k)
    for rel in (0.0, 1e-2):
        Ug = rounded(Uref + rel * scale * rng.standard_normal(Uref.shape), torch.float32)
        r = host(h.normal_residual(*csr, dev(Ug, torch.float32)))
        torch.cuda.synchronize()
        ro = np.array([orc.normal_residual(V, col[ptr[i]:ptr[i + 1]], val[ptr[i]:ptr[i + 1]],
                                           lam, Ug[i]) for i in range(len(ptr) - 1)])
        assert np.isfinite(r).all()
        assert np.abs(r - ro).max() <= TOL_RES[precision], np.abs(r - ro).max()
        if rel > 0:
            assert ro[np.diff(ptr) > 0].min() > 1e-4   # the planted error is visible


@pytest.mark.parametrize("precision", ["fp32", "bf16_gram"])
def test_refinement_on_ill_conditioned_rows(orc, precision):
    """Rows whose Gram the library forms EXACTLY (factor entries are multiples
    of 1/4 below 17, values multiples of 1/8, lambda = 2^-6: every product and
    partial sum fits FP32, and both BF16 and TF32 hold the entries exactly), so
    the only error left is the FP32 solve's, ~kappa 2^-24 with kappa ~1e5 here
    (a rank-4 structure plus small perturbations).  One refinement step with
    the double-FP32 residual removes most of it (prototype: 2.5e-6 -> 2.5e-8)."""
    k, n, m = 32, 400, 300
    lam = 2.0 ** -6
    rng = np.random.default_rng(7)
    B = rng.integers(-2, 3, (n, 4))
    C = rng.integers(-2, 3, (4, k))
    E = rng.integers(-1, 2, (n, k)) * (rng.random((n, k)) < 0.3)
    V = (B @ C + E / 4.0).astype(np.float64)
    counts = rng.integers(40, 90, m)
    ptr = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    col = np.concatenate([np.sort(rng.choice(n, c, replace=False)) for c in counts]).astype(np.int32)
    val = rng.integers(-64, 65, ptr[-1]) / 8.0
    h = _handle(k, lam, precision, V)
    csr = csr_dev(ptr, col, val, torch.float32)
    U1, _, r1 = h.complete_rows_checked(*csr, refine=False)
    U2, _, r2 = h.complete_rows_checked(*csr, refine=True)
    torch.cuda.synchronize()
    Uref, sref = orc.half_step(ptr, col, val, V, lam)
    assert (sref == 0).all()
    e1 = np.linalg.norm(host(U1) - Uref, axis=1) / np.linalg.norm(Uref, axis=1)
    e2 = np.linalg.norm(host(U2) - Uref, axis=1) / np.linalg.norm(Uref, axis=1)
    print(f"{precision} ill-conditioned fold-in: median error {np.median(e1):.2e} -> "
          f"{np.median(e2):.2e} refined; residual {np.median(host(r1)):.2e} -> "
          f"{np.median(host(r2)):.2e}")
    assert np.median(e1) > 3e-7                      # the FP32 solve's error is visible
    assert np.median(e2) < 0.1 * np.median(e1)
    assert e2.max() < 0.5 * e1.max()


def test_checked_foldin_rejects_unsupported():
    ptr, col, val, V = _ragged(3, 10, 128, 16)
    csr = csr_dev(ptr, col, val, torch.float32)
    h16 = _handle(16, 0.1, "fp32", V)
    with pytest.raises(ocf.OpenCFError) as e:
        h16.complete_rows_checked(*csr)
    assert e.value.code == ocf.UNSUPPORTED
    ptr, col, val, V = _ragged(4, 10, 128, 32)
    csr = csr_dev(ptr, col, val, torch.float32)
    hc = ocf.OpenCF(k=32, lam=0.1, precision="bf16_gram", cholesky_fp64=True)
    hc.set_V(dev(V, torch.float32))
    with pytest.raises(ocf.OpenCFError) as e:
        hc.complete_rows_checked(*csr)
    assert e.value.code == ocf.UNSUPPORTED
