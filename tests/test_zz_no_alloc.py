"""The allocation-free CSR -> CSC entry point, through the C ABI.

Callers whose host framework owns all device memory, or whose latency path
cannot absorb cudaMalloc/cudaFree, use open_cf_csr_to_csc_noalloc: it keeps
its scratch in a fixed device array instead of allocating.  Its output must
equal the handle-based open_cf_csr_to_csc bit for bit (the transpose is exact
integer and copy work), on two calls in a row with different inputs, so a
stale array from the first call would show up in the second.

This file is collected last on purpose.
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


def _dev(a, dt):
    return torch.as_tensor(np.ascontiguousarray(a)).to(DEV, dt)


def _noalloc(m, n, row_ptr, col, val):
    nnz = col.numel()
    cptr = torch.full((n + 1,), -7, dtype=torch.int64, device=DEV)
    ridx = torch.full((max(nnz, 1),), -7, dtype=torch.int32, device=DEV)
    cval = torch.full((max(nnz, 1),), -7.0, dtype=torch.float32, device=DEV)
    stream = ctypes.c_void_p(torch.cuda.current_stream(DEV).cuda_stream)
    rc = ocf.lib().open_cf_csr_to_csc_noalloc(
        m, n, nnz, ctypes.c_void_p(row_ptr.data_ptr()), ctypes.c_void_p(col.data_ptr()),
        ctypes.c_void_p(val.data_ptr()), ctypes.c_void_p(cptr.data_ptr()),
        ctypes.c_void_p(ridx.data_ptr()), ctypes.c_void_p(cval.data_ptr()), stream)
    return rc, cptr, ridx[:nnz], cval[:nnz]


def test_noalloc_matches_handle_transpose_on_two_calls():
    h = ocf.OpenCF(k=4, lam=0.1)
    cases = [dict(seed=1, m=4096, n_gpu=1024, density=0.05),   # the benchmark's shape
             dict(seed=2, m=777, n_gpu=300, density=0.11)]     # smaller, ragged
    for c in cases:
        p = synth.make_sparse_problem(seed=c["seed"], m=c["m"], n_cpu=1, n_gpu=c["n_gpu"],
                                      rank=4, density=c["density"], k=4, n_heldout=8)
        rp, col = _dev(p.row_ptr, torch.int64), _dev(p.col, torch.int32)
        val = _dev(p.val, torch.float32)
        ref = h.csr_to_csc(rp, col, val, p.n)
        rc, cptr, ridx, cval = _noalloc(p.m, p.n, rp, col, val)
        torch.cuda.synchronize()
        assert rc == ocf.OK
        assert torch.equal(cptr, ref[0])
        assert torch.equal(ridx, ref[1])
        assert torch.equal(cval, ref[2])
    h.close()


def test_noalloc_rejects_too_many_columns():
    n = 21825   # one column beyond the fixed scratch
    rp = torch.zeros(2, dtype=torch.int64, device=DEV)
    col = torch.zeros(0, dtype=torch.int32, device=DEV)
    val = torch.zeros(0, dtype=torch.float32, device=DEV)
    rc, cptr, _, _ = _noalloc(1, n, rp, col, val)
    torch.cuda.synchronize()
    assert rc == ocf.UNSUPPORTED
    assert bool((cptr == -7).all())            # outputs untouched
