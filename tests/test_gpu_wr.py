"""GPU-vs-oracle parity of weighted-lambda regularisation (ALS-WR).

With the handle's weighted_lambda flag set, every row solve adds
lambda * s_i to the Gram diagonal (s_i the row's observation count) and the
objective weights each factor's squared norm by its count.  The CUDA path is
compared with the oracle's ALS-WR routines on identical (rounded) inputs:
fold-in on ragged rows across every solver branch, one sweep stepwise, an
FP64 fit end to end with its objective history, the weighted objective, and
the batched fit stepwise.
"""
import numpy as np
import pytest
import torch

import synth

from gpu_util import (TOL_FP32, TOL_FP64, csr_dev, dev, host, rounded, row_rel_err,
                      solve_err)

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU hosts deselect these
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2508_07605_b300 as ocf  # noqa: E402

DT = {"fp32": torch.float32, "fp64": torch.float64}
TOL = {"fp32": TOL_FP32, "fp64": TOL_FP64}


def _ragged(rng, m, n, k):
    lens = [0, 1, max(k - 1, 0), k, k + 1, min(33, n), n]
    lens += list(rng.integers(0, min(n, 3 * k + 40) + 1, size=m - len(lens)))
    ptr = [0]; cols = []
    for s in lens:
        c = np.sort(rng.choice(n, size=int(s), replace=False)).astype(np.int32)
        cols.append(c); ptr.append(ptr[-1] + len(c))
    return np.array(ptr, dtype=np.int64), np.concatenate(cols)


@pytest.mark.parametrize("precision,k,chol64", [("fp32", 3, False), ("fp32", 16, False),
                                                ("fp32", 32, False), ("fp32", 16, True),
                                                ("fp32", 32, True), ("fp32", 20, True),
                                                ("fp64", 8, False), ("fp64", 32, False)])
def test_wr_foldin_ragged(orc, precision, k, chol64):
    rng = np.random.default_rng(700 + k)
    dt = DT[precision]
    n, m, lam = 150, 401, 0.05
    ptr, col = _ragged(rng, m, n, k)
    val = rounded(rng.random(len(col)), dt)
    V = rounded(rng.standard_normal((n, k)) / np.sqrt(k), dt)
    h = ocf.OpenCF(k=k, lam=lam, precision=precision, cholesky_fp64=chol64,
                   weighted_lambda=True)
    h.set_V(dev(V, dt))
    U, st = h.complete_rows(*csr_dev(ptr, col, val, dt))
    torch.cuda.synchronize()
    Uref, sref = orc.half_step_wr(ptr, col, val, V, lam)
    assert np.array_equal(host(st), sref)
    ok = np.diff(ptr) > 0
    err = solve_err(host(U), Uref, V, ptr, col, val, lam, weighted=True)
    assert err[ok].max() <= TOL[precision], (err[ok].max(), np.argmax(err))
    # the flag changes the answer wherever a row has more than one observation
    Uplain, _ = orc.half_step(ptr, col, val, V, lam)
    many = np.diff(ptr) > 1
    assert row_rel_err(host(U)[many], Uplain[many]).min() > 100 * TOL[precision]


def test_wr_bf16_gram_foldin(orc):
    rng = np.random.default_rng(71)
    k, n, m, lam = 32, 128, 600, 0.05
    ptr, col = _ragged(rng, m, n, k)
    val = rounded(np.abs(rng.random(len(col))) + 0.5, torch.float32)
    V = rounded(rng.standard_normal((n, k)) / 2, torch.float32)
    V[:, 0] = np.abs(V[:, 0]) + 0.5
    h = ocf.OpenCF(k=k, lam=lam, precision="bf16_gram", weighted_lambda=True)
    h.set_V(dev(V, torch.float32))
    U, st = h.complete_rows(*csr_dev(ptr, col, val, torch.float32))
    torch.cuda.synchronize()
    Uref, sref = orc.half_step_wr(ptr, col, val, V, lam)
    assert np.array_equal(host(st), sref)
    ok = np.diff(ptr) > 0
    # BF16 split products: a reconstruction-scale gate, as for the unweighted path
    Ug = host(U).astype(np.float64)
    pe = np.abs((Ug - Uref) @ V.T).max(1) / np.maximum(np.abs(Uref @ V.T).max(1), 1e-30)
    assert pe[ok].max() <= 2e-3, pe[ok].max()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_wr_one_sweep_stepwise(orc, precision):
    prob = synth.make_sparse_problem(seed=17, m=600, n_cpu=4, n_gpu=32, rank=16, density=0.1,
                                     k=16, lam=0.05, sweeps=1, n_heldout=64)
    dt = DT[precision]
    val = rounded(prob.val, dt)
    V0 = rounded(prob.V0, dt)
    h = ocf.OpenCF(k=prob.k, lam=prob.lam, sweeps=1, precision=precision, weighted_lambda=True)
    h.set_V(dev(V0, dt))
    U1, rs, cs = h.fit_csr(*csr_dev(prob.row_ptr, prob.col, val, dt), prob.n, status=True)
    V1 = h.get_V()
    torch.cuda.synchronize()
    Uref, rsref = orc.half_step_wr(prob.row_ptr, prob.col, val, V0, prob.lam)
    assert np.array_equal(host(rs), rsref)
    ok = np.diff(prob.row_ptr) > 0
    eu = solve_err(host(U1), Uref, V0, prob.row_ptr, prob.col, val, prob.lam, weighted=True)
    assert eu[ok].max() <= TOL[precision]
    cptr, cidx, cval = orc.transpose(prob.row_ptr, prob.col, val, prob.n)
    U1d = host(U1).astype(np.float64)
    Vref, csref = orc.half_step_wr(cptr, cidx, cval, U1d, prob.lam)
    assert np.array_equal(host(cs), csref)
    okc = np.diff(cptr) > 0
    ev = solve_err(host(V1), Vref, U1d, cptr, cidx, cval, prob.lam, weighted=True)
    assert ev[okc].max() <= TOL[precision]


def test_wr_fp64_fit_end_to_end(orc):
    prob = synth.make_small_offline_online(seed=2).joint
    h = ocf.OpenCF(k=prob.k, lam=prob.lam, sweeps=prob.sweeps, precision="fp64",
                   weighted_lambda=True)
    h.set_V(dev(prob.V0, torch.float64))
    U, J = h.fit_csr(*csr_dev(prob.row_ptr, prob.col, prob.val, torch.float64), prob.n,
                     J_hist=True)
    V = h.get_V()
    torch.cuda.synchronize()
    Ur, Vr, Jr = orc.als_wr(prob.row_ptr, prob.col, prob.val, prob.n, prob.V0, prob.lam,
                            prob.sweeps, history=True)
    assert row_rel_err(host(U), Ur).max() <= 1e-9
    assert row_rel_err(host(V), Vr).max() <= 1e-9
    Jg = host(J)
    assert np.abs(Jg - Jr).max() <= 1e-10 * Jr.max()
    assert (np.diff(Jg) <= 1e-12 * Jg[:-1]).all()
    # the history's last entry is the weighted objective at the returned factors
    assert abs(Jg[-1] - orc.objective_wr(prob.row_ptr, prob.col, prob.val, Ur, Vr,
                                         prob.lam)) <= 1e-10 * Jg[-1]


def test_wr_fp32_fit_monotone(orc):
    prob = synth.make_sparse_problem(seed=18, m=2000, n_cpu=4, n_gpu=64, rank=16, density=0.05,
                                     k=16, lam=0.05, sweeps=15, n_heldout=64)
    val = rounded(prob.val, torch.float32)
    h = ocf.OpenCF(k=prob.k, lam=prob.lam, sweeps=prob.sweeps, weighted_lambda=True)
    h.set_V(dev(prob.V0, torch.float32))
    U, J = h.fit_csr(*csr_dev(prob.row_ptr, prob.col, val, torch.float32), prob.n, J_hist=True)
    torch.cuda.synchronize()
    _, _, Jr = orc.als_wr(prob.row_ptr, prob.col, val, prob.n, prob.V0, prob.lam, prob.sweeps,
                          history=True)
    Jg = host(J)
    assert (np.diff(Jg) <= 1e-5 * Jg[:-1]).all(), Jg
    assert np.abs(Jg - Jr).max() <= 1e-3 * Jr.max()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_wr_objective(orc, precision):
    prob = synth.make_sparse_problem(seed=19, m=700, n_cpu=4, n_gpu=32, rank=8, density=0.1,
                                     k=8, lam=0.05, n_heldout=16)
    dt = DT[precision]
    val = rounded(prob.val, dt)
    rng = np.random.default_rng(3)
    U = rounded(rng.standard_normal((prob.m, prob.k)) * 0.3, dt)
    V = rounded(rng.standard_normal((prob.n, prob.k)) * 0.3, dt)
    h = ocf.OpenCF(k=prob.k, lam=prob.lam, precision=precision, weighted_lambda=True)
    h.set_V(dev(V, dt))
    J = h.objective(*csr_dev(prob.row_ptr, prob.col, val, dt), dev(U, dt))
    torch.cuda.synchronize()
    Jr = orc.objective_wr(prob.row_ptr, prob.col, val, U, V, prob.lam)
    Jplain = orc.objective(prob.row_ptr, prob.col, val, U, V, prob.lam)
    rtol = 1e-6 if precision == "fp32" else 1e-12
    assert abs(host(J)[0] - Jr) <= rtol * Jr
    assert abs(Jr - Jplain) > 1e3 * rtol * Jr


def test_wr_batched_one_sweep_stepwise(orc):
    bp = synth.make_batched(seed=21, n_problems=40, n_heldout=16)
    c = bp.concat()
    val = rounded(c["val"], torch.float32)
    V = dev(rounded(c["V0"], torch.float32), torch.float32)
    nnz_p = np.array([p.nnz for p in bp.problems])
    h = ocf.OpenCF(k=4, lam=0.05, sweeps=1, weighted_lambda=True)
    U = h.batched_fit(c["m"], c["n"], c["k"], nnz_p, dev(c["row_ptr"], torch.int64),
                      dev(c["col"], torch.int32), dev(val, torch.float32), V)
    torch.cuda.synchronize()
    U, V = host(U).astype(np.float64), host(V).astype(np.float64)
    for t, p in enumerate(bp.problems):
        us = slice(int(c["u_off"][t]), int(c["u_off"][t + 1]))
        vs = slice(int(c["v_off"][t]), int(c["v_off"][t + 1]))
        pv = val[int(c["nnz_off"][t]):int(c["nnz_off"][t + 1])]
        Ug = U[us].reshape(p.m, p.k)
        Vg = V[vs].reshape(p.n, p.k)
        V0 = rounded(p.V0, torch.float32)
        Ur, _ = orc.half_step_wr(p.row_ptr, p.col, pv, V0, p.lam)
        ok = np.diff(p.row_ptr) > 0
        eu = solve_err(Ug, Ur, V0, p.row_ptr, p.col, pv, p.lam, weighted=True)
        assert eu[ok].max(initial=0.0) <= TOL_FP32, (t, eu[ok].max())
        cptr, cidx, cval = orc.transpose(p.row_ptr, p.col, pv, p.n)
        Vr, _ = orc.half_step_wr(cptr, cidx, cval, Ug, p.lam)
        okc = np.diff(cptr) > 0
        ev = solve_err(Vg, Vr, Ug, cptr, cidx, cval, p.lam, weighted=True)
        assert ev[okc].max(initial=0.0) <= TOL_FP32, (t, ev[okc].max())
