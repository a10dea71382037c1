"""The allocation-free CSR -> CSC entry point, through the C ABI.

Callers whose host framework owns all device memory, or whose latency path
cannot absorb cudaMalloc/cudaFree, use open_cf_csr_to_csc_noalloc: it keeps
its scratch in a fixed device array instead of allocating.  The transpose is
exact integer and copy work, so its output must equal the FP64 oracle's
stable counting sort bit for bit, and the handle-based open_cf_csr_to_csc
too, on two calls in a row with different inputs (a stale array left by the
first call would show up in the second).

The file name sorts last so that, in a run that stops at the first failure,
every other test has already run if this one fails; nothing here depends on
that order: the tests pass alone in a fresh process as well.
"""
import ctypes

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU hosts deselect these
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2508_07605_b300 as ocf  # noqa: E402

DEV = torch.device("cuda", 0)
MAX_N = 25000   # OPEN_CF_NOALLOC_MAX_COLUMNS


def _dev(a, dt):
    return torch.as_tensor(np.ascontiguousarray(a)).to(DEV, dt)


def _noalloc(m, n, row_ptr, col, val):
    nnz = 0 if col is None else col.numel()
    cptr = torch.full((n + 1,), -7, dtype=torch.int64, device=DEV)
    ridx = torch.full((max(nnz, 1),), -7, dtype=torch.int32, device=DEV)
    cval = torch.full((max(nnz, 1),), -7.0, dtype=torch.float32, device=DEV)
    stream = ctypes.c_void_p(torch.cuda.current_stream(DEV).cuda_stream)
    ptr = lambda t: ctypes.c_void_p(None if t is None else t.data_ptr())
    rc = ocf.lib().open_cf_csr_to_csc_noalloc(
        m, n, nnz, ptr(row_ptr), ptr(col), ptr(val), ptr(cptr), ptr(ridx), ptr(cval), stream)
    return rc, cptr, ridx[:nnz], cval[:nnz]


def _check_against_oracle(orc, row_ptr, col, val32, n, got):
    cptr_o, ridx_o, cval_o = orc.transpose(row_ptr, col, val32.astype(np.float64), n)
    assert np.array_equal(got[0].cpu().numpy(), cptr_o)
    assert np.array_equal(got[1].cpu().numpy(), ridx_o)
    assert np.array_equal(got[2].cpu().numpy().astype(np.float64), cval_o)


def test_noalloc_matches_oracle_and_handle_on_two_calls(orc):
    h = ocf.OpenCF(k=4, lam=0.1)
    cases = [dict(seed=1, m=4096, n_gpu=1024, density=0.05),   # the 4096 x 1024 fit's shape
             dict(seed=2, m=777, n_gpu=300, density=0.11)]     # smaller, ragged
    for c in cases:
        p = synth.make_sparse_problem(seed=c["seed"], m=c["m"], n_cpu=1, n_gpu=c["n_gpu"],
                                      rank=4, density=c["density"], k=4, n_heldout=8)
        val32 = p.val.astype(np.float32)
        rp, col, val = _dev(p.row_ptr, torch.int64), _dev(p.col, torch.int32), _dev(val32, torch.float32)
        rc, cptr, ridx, cval = _noalloc(p.m, p.n, rp, col, val)
        ref = h.csr_to_csc(rp, col, val, p.n)
        torch.cuda.synchronize()
        assert rc == ocf.OK
        _check_against_oracle(orc, p.row_ptr, p.col, val32, p.n, (cptr, ridx, cval))
        assert torch.equal(cptr, ref[0]) and torch.equal(ridx, ref[1]) and torch.equal(cval, ref[2])
    h.close()


def test_noalloc_widest_matrix(orc):
    # n at the limit: the column totals and the counters use the array's most
    # columns; a few rows, one of them touching the last column
    rng = np.random.default_rng(5)
    m, n = 300, MAX_N
    cols, ptr = [], [0]
    for i in range(m):
        c = np.sort(rng.choice(n, size=int(rng.integers(0, 40)), replace=False))
        if i == 7:
            c = np.union1d(c, [0, n - 1])
        cols.append(c); ptr.append(ptr[-1] + len(c))
    col = np.concatenate(cols).astype(np.int32)
    row_ptr = np.array(ptr, dtype=np.int64)
    val32 = rng.standard_normal(len(col)).astype(np.float32)
    got = _noalloc(m, n, _dev(row_ptr, torch.int64), _dev(col, torch.int32),
                   _dev(val32, torch.float32))
    torch.cuda.synchronize()
    assert got[0] == ocf.OK
    _check_against_oracle(orc, row_ptr, col, val32, n, got[1:])


def test_noalloc_empty_matrix():
    # m = 0 and nnz = 0: row_ptr may be NULL; every column pointer is 0
    rc, cptr, _, _ = _noalloc(0, 1000, None, None, None)
    torch.cuda.synchronize()
    assert rc == ocf.OK
    assert bool((cptr == 0).all())


def test_noalloc_rejects_too_many_columns():
    n = MAX_N + 1
    rp = torch.zeros(2, dtype=torch.int64, device=DEV)
    col = torch.zeros(0, dtype=torch.int32, device=DEV)
    val = torch.zeros(0, dtype=torch.float32, device=DEV)
    rc, cptr, _, _ = _noalloc(1, n, rp, col, val)
    torch.cuda.synchronize()
    assert rc == ocf.UNSUPPORTED
    assert bool((cptr == -7).all())            # outputs untouched
