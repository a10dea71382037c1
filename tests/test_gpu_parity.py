"""GPU-vs-oracle parity of the completion path through the C ABI.

Every case feeds the CUDA path and the FP64 oracle the same seeded inputs
(rounded to the kernel's storage precision) and compares element by element
within the stated tolerances.  Multi-sweep fits are checked stepwise (the
oracle re-runs a half-step from the GPU's own inputs), because independent
FP32 and FP64 ALS trajectories drift apart over sweeps; end-to-end FP64 fits
are compared directly.
"""
import json
import os

import numpy as np
import pytest
import torch

import oracle
import synth

from gpu_util import (DEV, TOL_FP32, TOL_FP64, csr_dev, dev, host, rounded, row_rel_err,
                      solve_err)

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU hosts deselect these
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2508_07605_b300 as ocf  # noqa: E402

DT = {"fp32": torch.float32, "fp64": torch.float64}
TOL = {"fp32": TOL_FP32, "fp64": TOL_FP64}
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _handle(k, lam, sweeps=15, precision="fp32", caps=None, chol64=False):
    cpu, gpu = caps if caps is not None else (None, None)
    return ocf.OpenCF(k=k, lam=lam, sweeps=sweeps, precision=precision, cholesky_fp64=chol64,
                      cpu_caps=cpu, gpu_caps=gpu)


# ---------------------------------------------------------------- fold-in
@pytest.mark.parametrize("precision,chol64", [("fp32", False), ("fp32", True), ("fp64", False)])
def test_foldin_small_offline_online(orc, precision, chol64):
    prob = synth.make_small_offline_online(seed=0)
    dt = DT[precision]
    _, V, _ = orc.als_dense(prob.offline, prob.new.V0, prob.new.lam, prob.new.sweeps)
    Vr = rounded(V, dt)
    h = _handle(prob.new.k, prob.new.lam, precision=precision, caps=prob.new.caps(),
                chol64=chol64)
    h.set_V(dev(Vr, dt))
    p, c, v = csr_dev(prob.new.row_ptr, prob.new.col, rounded(prob.new.val, dt), dt)
    U, st = h.complete_rows(p, c, v)
    torch.cuda.synchronize()
    Uref, sref = orc.half_step(prob.new.row_ptr, prob.new.col, rounded(prob.new.val, dt), Vr,
                               prob.new.lam)
    assert np.array_equal(host(st), sref)
    err = row_rel_err(host(U), Uref)
    assert err.max() <= TOL[precision], err.max()


def _ragged_csr(rng, m, n, k):
    """Rows of every interesting length: empty, 1, k-1, k, k+1, 33, n, random."""
    lens = [0, 1, max(k - 1, 0), k, k + 1, min(33, n), n]
    lens += list(rng.integers(0, min(n, 3 * k + 40) + 1, size=m - len(lens)))
    ptr = [0]; cols = []
    for s in lens:
        c = np.sort(rng.choice(n, size=int(s), replace=False)).astype(np.int32)
        cols.append(c); ptr.append(ptr[-1] + len(c))
    return np.array(ptr, dtype=np.int64), np.concatenate(cols)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("k", [1, 3, 8, 13, 16, 17, 32])
def test_foldin_ragged_rows_every_k(orc, precision, k):
    rng = np.random.default_rng(100 + k)
    dt = DT[precision]
    n, m, lam = 150, 333, 0.05
    ptr, col = _ragged_csr(rng, m, n, k)
    val = rounded(rng.random(len(col)), dt)
    V = rounded(rng.standard_normal((n, k)) / np.sqrt(k), dt)
    h = _handle(k, lam, precision=precision)
    h.set_V(dev(V, dt))
    U, st = h.complete_rows(*csr_dev(ptr, col, val, dt))
    torch.cuda.synchronize()
    Uref, sref = orc.half_step(ptr, col, val, V, lam)
    assert np.array_equal(host(st), sref)
    assert (host(st)[np.diff(ptr) == 0] == ocf.ROW_EMPTY).all()
    err = solve_err(host(U), Uref, V, ptr, col, val, lam)
    ok = np.diff(ptr) > 0
    assert err[ok].max() <= TOL[precision], (err[ok].max(), np.argmax(err))
    assert np.abs(host(U)[~ok]).max(initial=0.0) == 0.0
    # the plain relative error |u - u_or| / |u_or| beside it: rows above the gate
    # under that measure are those whose right-hand side cancels (solve_err)
    plain = row_rel_err(host(U), Uref)[ok]
    loose = int((plain > TOL[precision]).sum())
    print(f"k={k} {precision}: plain relative error max {plain.max():.2e} median "
          f"{np.median(plain):.2e}; {loose} of {ok.sum()} rows need the cancellation scale")
    assert np.median(plain) <= TOL[precision]


def test_foldin_bad_index_is_flagged_not_read(orc):
    rng = np.random.default_rng(5)
    n, k = 40, 8
    ptr = np.array([0, 3, 6, 9], dtype=np.int64)
    col = np.array([1, 5, 9, 2, 4, 400, 0, 1, 2], dtype=np.int32)   # row 1 has col 400 >= n
    val = rng.random(9).astype(np.float32).astype(np.float64)
    V = rounded(rng.standard_normal((n, k)), torch.float32)
    h = _handle(k, 0.1)
    h.set_V(dev(V, torch.float32))
    U, st = h.complete_rows(*csr_dev(ptr, col, val, torch.float32))
    torch.cuda.synchronize()
    s = host(st)
    assert list(s) == [ocf.ROW_OK, ocf.ROW_BAD_INPUT, ocf.ROW_OK]
    assert np.all(host(U)[1] == 0)
    keep = np.array([0, 2])
    Uref, _ = orc.half_step(np.array([0, 3, 6]), np.concatenate([col[:3], col[6:]]),
                            np.concatenate([val[:3], val[6:]]), V, 0.1)
    assert row_rel_err(host(U)[keep], Uref).max() <= TOL_FP32


def test_empty_inputs():
    h = _handle(8, 0.1)
    h.set_V(torch.zeros(10, 8, device=DEV))
    p = torch.zeros(1, dtype=torch.int64, device=DEV)
    c = torch.zeros(0, dtype=torch.int32, device=DEV)
    v = torch.zeros(0, dtype=torch.float32, device=DEV)
    U, st = h.complete_rows(p, c, v)
    torch.cuda.synchronize()
    assert U.shape == (0, 8)


# ---------------------------------------------------------------- CSR -> CSC
@pytest.mark.parametrize("m,n,density", [(500, 300, 0.05), (4096, 1024, 0.05), (37, 5, 0.9),
                                         (10000, 1000, 0.01)])
def test_csr_to_csc_bit_exact(orc, m, n, density):
    prob = synth.make_sparse_problem(seed=m, m=m, n_cpu=1, n_gpu=n, rank=4, density=density,
                                     k=4, n_heldout=8)
    val = rounded(prob.val, torch.float32)
    h = _handle(4, 0.1)
    cptr, ridx, cval = h.csr_to_csc(*csr_dev(prob.row_ptr, prob.col, val, torch.float32), n)
    torch.cuda.synchronize()
    rp, ri, rv = orc.transpose(prob.row_ptr, prob.col, val, n)
    assert np.array_equal(host(cptr), rp)
    assert np.array_equal(host(ridx), ri)
    assert np.array_equal(host(cval).astype(np.float64), rv)


# ---------------------------------------------------------------- sweeps
def _small_sparse(seed=3, m=600, n_gpu=32, n_cpu=4, k=16, density=0.1, sweeps=15):
    return synth.make_sparse_problem(seed=seed, m=m, n_cpu=n_cpu, n_gpu=n_gpu, rank=k,
                                     density=density, k=k, lam=0.05, sweeps=sweeps,
                                     n_heldout=4096)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_one_sweep_stepwise(orc, precision):
    prob = _small_sparse()
    dt = DT[precision]
    val = rounded(prob.val, dt)
    V0 = rounded(prob.V0, dt)
    h = _handle(prob.k, prob.lam, sweeps=1, precision=precision)
    h.set_V(dev(V0, dt))
    U1, rs, cs = h.fit_csr(*csr_dev(prob.row_ptr, prob.col, val, dt), prob.n, status=True)
    V1 = h.get_V()
    torch.cuda.synchronize()
    Uref, _ = orc.half_step(prob.row_ptr, prob.col, val, V0, prob.lam)
    assert row_rel_err(host(U1), Uref).max() <= TOL[precision]
    cptr, cidx, cval = orc.transpose(prob.row_ptr, prob.col, val, prob.n)
    Vref, csref = orc.half_step(cptr, cidx, cval, host(U1).astype(np.float64), prob.lam)
    assert row_rel_err(host(V1), Vref).max() <= TOL[precision]
    assert np.array_equal(host(cs), csref)


def test_fp64_fit_end_to_end_matches_oracle(orc):
    prob = synth.make_small_offline_online(seed=0).joint
    h = _handle(prob.k, prob.lam, sweeps=prob.sweeps, precision="fp64")
    h.set_V(dev(prob.V0, torch.float64))
    U, J = h.fit_csr(*csr_dev(prob.row_ptr, prob.col, prob.val, torch.float64), prob.n,
                     J_hist=True)
    V = h.get_V()
    torch.cuda.synchronize()
    Ur, Vr, Jr, _, _ = orc.als(prob.row_ptr, prob.col, prob.val, prob.n, prob.V0, prob.lam,
                               prob.sweeps, history=True)
    assert row_rel_err(host(U), Ur).max() <= 1e-9
    assert row_rel_err(host(V), Vr).max() <= 1e-9
    Jg = host(J)
    assert np.abs(Jg - Jr).max() <= 1e-10 * Jr.max()
    assert (np.diff(Jg) <= 1e-12 * Jg[:-1]).all()


def test_fp32_fit_heldout_rmse_and_monotone(orc):
    prob = _small_sparse(sweeps=15)
    val = rounded(prob.val, torch.float32)
    h = _handle(prob.k, prob.lam, sweeps=prob.sweeps)
    h.set_V(dev(prob.V0, torch.float32))
    U, J = h.fit_csr(*csr_dev(prob.row_ptr, prob.col, val, torch.float32), prob.n, J_hist=True)
    V = h.get_V()
    torch.cuda.synchronize()
    Ug, Vg = host(U).astype(np.float64), host(V).astype(np.float64)
    Ur, Vr, Jr, _, _ = orc.als(prob.row_ptr, prob.col, val, prob.n, prob.V0, prob.lam,
                               prob.sweeps, history=True)
    pred_g = np.einsum("tk,tk->t", Ug[prob.heldout_rows], Vg[prob.heldout_cols])
    pred_r = np.einsum("tk,tk->t", Ur[prob.heldout_rows], Vr[prob.heldout_cols])
    rmse_g = np.sqrt(np.mean((pred_g - prob.heldout_truth) ** 2))
    rmse_r = np.sqrt(np.mean((pred_r - prob.heldout_truth) ** 2))
    assert rmse_g <= rmse_r + 1e-3, (rmse_g, rmse_r)
    Jg = host(J)
    assert (np.diff(Jg) <= 1e-5 * Jg[:-1]).all(), Jg
    assert np.abs(Jg - Jr).max() <= 1e-3 * Jr.max()


def test_offline_fit_then_joint_refit_fp64(orc):
    prob = synth.make_small_offline_online(seed=1)
    new = prob.new
    h = _handle(new.k, new.lam, sweeps=new.sweeps, precision="fp64", caps=new.caps())
    h.set_V(dev(new.V0, torch.float64))
    Uoff, J = h.fit_offline(dev(prob.offline, torch.float64), J_hist=True)
    Voff = h.get_V()
    torch.cuda.synchronize()
    Uo_r, Vo_r, Jo_r = orc.als_dense(prob.offline, new.V0, new.lam, new.sweeps, history=True)
    assert row_rel_err(host(Uoff), Uo_r).max() <= 1e-9
    assert row_rel_err(host(Voff), Vo_r).max() <= 1e-9
    # joint refit over offline block + new rows, from the fitted V
    Unew, st = h.complete_rows(*csr_dev(new.row_ptr, new.col, new.val, torch.float64),
                               joint=True)
    Vj = h.get_V()
    torch.cuda.synchronize()
    joint = prob.joint
    Uj_r, Vj_r, _, _, _ = orc.als(joint.row_ptr, joint.col, joint.val, joint.n, Vo_r, new.lam,
                                  new.sweeps)
    assert row_rel_err(host(Unew), Uj_r[prob.m_off:]).max() <= 1e-9
    assert row_rel_err(host(Vj), Vj_r).max() <= 1e-9


def test_full_size_fit_sampled_parity(orc):
    """4096 x 1024, k=16, 15 sweeps, in the configuration the benchmark times:
    every sampled column of the final V must be the ridge solve of that column
    against the returned U, and a fold-in against the final V must match the
    oracle on sampled rows."""
    prob = synth.make_c2(seed=0)
    val = rounded(prob.val, torch.float32)
    h = _handle(prob.k, prob.lam, sweeps=prob.sweeps, caps=prob.caps())
    h.set_V(dev(prob.V0, torch.float32))
    p, c, v = csr_dev(prob.row_ptr, prob.col, val, torch.float32)
    U = h.fit_csr(p, c, v, prob.n)
    V = h.get_V()
    Uf, st = h.complete_rows(p, c, v)
    torch.cuda.synchronize()
    Ug, Vg = host(U).astype(np.float64), host(V).astype(np.float64)
    rng = np.random.default_rng(0)
    cptr, cidx, cval = orc.transpose(prob.row_ptr, prob.col, val, prob.n)
    cols = rng.choice(prob.n, 256, replace=False)
    for j in cols:
        s = slice(cptr[j], cptr[j + 1])
        vj, _ = orc.row_solve(Ug, cidx[s], cval[s], prob.lam)
        assert np.linalg.norm(Vg[j] - vj) <= TOL_FP32 * np.linalg.norm(vj)
    rows = rng.choice(prob.m, 512, replace=False)
    Ufg = host(Uf).astype(np.float64)
    for i in rows:
        s = slice(prob.row_ptr[i], prob.row_ptr[i + 1])
        ui, _ = orc.row_solve(Vg, prob.col[s], val[s], prob.lam)
        assert np.linalg.norm(Ufg[i] - ui) <= TOL_FP32 * np.linalg.norm(ui)


# ---------------------------------------------------------------- objective
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_objective_and_row_rmse(orc, precision):
    prob = _small_sparse(seed=8)
    dt = DT[precision]
    val = rounded(prob.val, dt)
    rng = np.random.default_rng(1)
    U = rounded(rng.standard_normal((prob.m, prob.k)) * 0.3, dt)
    V = rounded(rng.standard_normal((prob.n, prob.k)) * 0.3, dt)
    h = _handle(prob.k, prob.lam, precision=precision)
    h.set_V(dev(V, dt))
    J, rr = h.objective(*csr_dev(prob.row_ptr, prob.col, val, dt), dev(U, dt), row_rmse=True)
    torch.cuda.synchronize()
    Jr = orc.objective(prob.row_ptr, prob.col, val, U, V, prob.lam)
    rtol = 1e-6 if precision == "fp32" else 1e-12
    assert abs(host(J)[0] - Jr) <= rtol * Jr
    rr_ref = orc.row_rmse(prob.row_ptr, prob.col, val, U, V)
    assert np.abs(host(rr) - rr_ref).max() <= 1e-5 * rr_ref.max()


# ---------------------------------------------------------------- predict / Algorithm 2
def test_select_golden_tables():
    cases = json.load(open(os.path.join(GOLDEN, "alg2_tables.json")))["cases"]
    for c in cases:
        h = _handle(1, 0.1, caps=(c["cpu"], c["gpu"]))
        T = torch.tensor([c["t"]], dtype=torch.float32, device=DEV)
        best, sav = h.select(T, gamma=c["gamma"])
        torch.cuda.synchronize()
        assert int(host(best)[0]) == c["best"], c["name"]
        assert abs(float(host(sav)[0]) - c["saving"]) <= 1e-6, c["name"]


@pytest.mark.parametrize("precision,m", [("fp32", 300), ("fp64", 300), ("fp32", 20011)])
@pytest.mark.parametrize("gamma", [0.0, 0.05, 0.15])
def test_predict_and_select_parity(orc, precision, m, gamma):
    """Row tiles of 16 (few rows) and 64 (many rows), a ragged last tile."""
    prob = synth.make_small_offline_online(seed=2)
    dt = DT[precision]
    cpu, gpu = prob.new.caps()
    rng = np.random.default_rng(3)
    n, k = prob.new.n, 8
    U = rounded(rng.standard_normal((m, k)) * 0.4, dt)
    V = rounded(rng.standard_normal((n, k)) * 0.4, dt)
    U[:, 0] = np.abs(U[:, 0]) + 2.0      # keep most predicted runtimes positive
    V[:, 0] = np.abs(V[:, 0]) + 0.5
    U[7] = 0.0                           # a row whose baseline runtime is 0
    h = _handle(k, 0.1, precision=precision, caps=(cpu, gpu))
    h.set_V(dev(V, dt))
    T, best, sav = h.predict(dev(U, dt), gamma=gamma)
    torch.cuda.synchronize()
    Tr = orc.predict(U, V)
    tol = 1e-6 if precision == "fp32" else 1e-13
    assert np.abs(host(T) - Tr).max() <= tol * np.abs(Tr).max()
    # bit-exact: the kernel's decision equals the oracle's FP32 Algorithm 2 on the same T
    Tg32 = host(T).astype(np.float32)
    b_or, s_or = orc.select_f32(Tg32, cpu, gpu, gamma)
    assert np.array_equal(host(best), b_or)
    assert np.array_equal(host(sav), s_or)
    assert host(best)[7] == -1
    # the stand-alone select on the same matrix agrees bit for bit
    b2, s2 = h.select(dev(Tg32, torch.float32), gamma=gamma)
    assert np.array_equal(host(b2), b_or) and np.array_equal(host(s2), s_or)
    # against the FP64 oracle: the pick is valid and within 1e-5 of the best saving
    b64, s64 = orc.select_f64(Tr, cpu, gpu, gamma)
    bg = host(best)
    for i in range(0, m, max(1, m // 500)):
        if b64[i] < 0:
            continue
        j = bg[i]
        base = oracle.baseline_index(cpu, gpu)
        p = Tr[i, base] / Tr[i, j]
        assert 1 - p <= gamma + 1e-5
        cg = cpu[j // len(gpu)] + gpu[j % len(gpu)]
        Eb = cpu[base // len(gpu)] + gpu[base % len(gpu)]
        assert (Eb - cg / p) / Eb >= s64[i] - 1e-5


@pytest.mark.parametrize("gamma", [0.0, 1e-30, 0.05, 0.1, 0.3, 0.9999, 1.0, 2.0, -0.05, -3.0])
def test_select_loss_bound_edges(orc, gamma):
    """Runtimes a few units in the last place on either side of the loss
    bound t_b / (1 - gamma), for several baselines: the kernel's validity
    test (a largest valid runtime per row) must pick exactly the settings the
    oracle's per-element FP32 check keeps."""
    cpu, gpu = synth.cap_grid(4, 8)
    n = len(cpu) * len(gpu)
    base = oracle.baseline_index(cpu, gpu)
    rng = np.random.default_rng(11)
    tbs = np.array([1.0, 0.37, 3.0e-3, 7.25, 1.0e5, 0.999999, 2.0 ** -20], np.float32)
    rows = []
    for tb in tbs:
        g1 = np.float32(1.0) - np.float32(gamma)
        t0 = np.float32(tb / g1) if g1 > 0 else np.float32(tb * 4)
        for _ in range(3):
            steps = rng.integers(-6, 7, size=n).astype(np.int64)
            bits = np.int64(t0.view(np.int32)) + steps
            t = np.clip(bits, 1, 0x7f7fffff).astype(np.int32).view(np.float32)
            t[base] = tb
            rows.append(t)
    T = np.stack(rows).astype(np.float32)
    h = _handle(1, 0.1, caps=(cpu, gpu))
    b, s = h.select(dev(T, torch.float32), gamma=gamma)
    torch.cuda.synchronize()
    b_or, s_or = orc.select_f32(T, cpu, gpu, gamma)
    assert np.array_equal(host(b), b_or)
    assert np.array_equal(host(s), s_or)


def test_predict_without_dense_output_matches():
    rng = np.random.default_rng(4)
    cpu, gpu = synth.cap_grid(8, 15)
    U = rng.standard_normal((130, 8)).astype(np.float32); U[:, 0] = np.abs(U[:, 0]) + 2
    V = rng.standard_normal((120, 8)).astype(np.float32); V[:, 0] = np.abs(V[:, 0]) + 1
    h = _handle(8, 0.1, caps=(cpu, gpu))
    h.set_V(dev(V, torch.float32))
    _, b1, s1 = h.predict(dev(U, torch.float32), gamma=0.1, want_T=True)
    _, b2, s2 = h.predict(dev(U, torch.float32), gamma=0.1, want_T=False)
    torch.cuda.synchronize()
    assert torch.equal(b1, b2) and torch.equal(s1, s2)


# ---------------------------------------------------------------- validation
def test_validate_csr_reports_each_fault():
    h = _handle(4, 0.1)
    ptr = np.array([0, 2, 4], dtype=np.int64)
    col = np.array([0, 3, 1, 2], dtype=np.int32)
    val = np.array([0.1, 0.2, 0.3, 0.4])
    assert h.validate_csr(*csr_dev(ptr, col, val, torch.float32), 4) == 0
    bad_ptr = np.array([0, 5, 4], dtype=np.int64)
    assert h.validate_csr(*csr_dev(bad_ptr, col, val, torch.float32), 4) == 1
    assert h.validate_csr(*csr_dev(ptr, np.array([0, 4, 1, 2]), val, torch.float32), 4) == 2
    assert h.validate_csr(*csr_dev(ptr, np.array([3, 0, 1, 2]), val, torch.float32), 4) == 3
    assert h.validate_csr(*csr_dev(ptr, col, np.array([0.1, np.nan, 0.3, 0.4]),
                                   torch.float32), 4) == 4


def test_argument_errors_are_synchronous():
    h = _handle(4, 0.1)
    with pytest.raises(ocf.OpenCFError) as e:
        h.complete_rows(*csr_dev(np.array([0, 1]), np.array([0]), np.array([1.0]),
                                 torch.float32))
    assert e.value.code == ocf.NOT_FITTED
    with pytest.raises(ocf.OpenCFError) as e:
        ocf.OpenCF(k=33, lam=0.1)
    assert e.value.code == ocf.UNSUPPORTED
    with pytest.raises(ocf.OpenCFError) as e:
        ocf.OpenCF(k=4, lam=0.0)
    assert e.value.code == ocf.INVALID_ARG
