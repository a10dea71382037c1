"""The online phase from host memory (open_cf_complete_select_host): the CSR
in pinned host memory is copied chunk by chunk on the handle's copy stream
while earlier chunks are solved, and the decisions come back to host memory.
Each chunk is solved as its own CSR, so the results must equal, bit for bit,
those of the device-memory calls on the whole batch (fold-in, then
reconstruction + Algorithm 2), which the other parity tests hold to the
oracle; a sample is also checked against the oracle's FP32 selection on the
GPU's own predicted runtimes."""
import numpy as np
import pytest
import torch

import synth

from gpu_util import DEV, dev, host, rounded

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2508_07605_b300 as ocf  # noqa: E402


def _problem(m, seed):
    prob = synth.make_large_foldin(seed=seed, m=m, device=DEV)
    cpu, gpu = synth.cap_grid(prob.n_cpu, prob.n_gpu)
    return prob, cpu, gpu


def _pinned(t):
    return t.cpu().pin_memory()


@pytest.mark.parametrize("precision,check,chunk,col16", [
    ("bf16_gram", 2, 4096, False),   # the default line's configuration, 13 chunks (ragged last)
    ("bf16_gram", 2, 4096, True),    # the same with 16-bit setting indices
    ("bf16_gram", 1, 0, False),      # default chunking
    ("fp32", 0, 2560, True),         # plain fold-in, FP32 mode
])
def test_host_pipeline_equals_device_calls(orc, precision, check, chunk, col16):
    m = 50_001
    prob, cpu, gpu = _problem(m, seed=3)
    h = ocf.OpenCF(k=prob.k, lam=prob.lam, precision=precision, cpu_caps=cpu, gpu_caps=gpu)
    h.set_V(prob.V.contiguous())
    # reference: device-memory calls on the whole batch
    if check > 0:
        U, st, res = h.complete_rows_checked(prob.row_ptr, prob.col, prob.val, refine=check == 2)
    else:
        U, st = h.complete_rows(prob.row_ptr, prob.col, prob.val)
        res = None
    T, best, sav = h.predict(U, gamma=0.05)
    torch.cuda.synchronize()
    # the same from pinned host memory, in chunks
    hp, hv = _pinned(prob.row_ptr), _pinned(prob.val)
    hc = (prob.col.cpu().to(torch.uint16) if col16 else prob.col.cpu()).pin_memory()
    st_h = torch.empty(m, dtype=torch.int32).pin_memory()
    res_h = torch.empty(m, dtype=torch.float32).pin_memory() if check > 0 else None
    for _ in range(2):   # twice: the second call reuses the handle's device copies
        b_h, s_h, _, _ = h.complete_select_host(hp, hc, hv, check=check, gamma=0.05,
                                                status=st_h, resid=res_h, chunk_rows=chunk)
        torch.cuda.synchronize()
        assert torch.equal(b_h, best.cpu())
        assert torch.equal(s_h, sav.cpu())
        assert torch.equal(st_h, st.cpu())
        if check > 0:
            assert torch.equal(res_h, res.cpu())
    # a sample of the decisions against the oracle's FP32 selection on the GPU's T
    rows = np.arange(0, m, 997)
    b_or, s_or = orc.select_f32(host(T)[rows].astype(np.float32), cpu, gpu, 0.05)
    assert np.array_equal(b_h.numpy()[rows], b_or)
    assert np.array_equal(s_h.numpy()[rows], s_or)


def test_host_pipeline_pageable_and_errors():
    m = 3000
    prob, cpu, gpu = _problem(m, seed=4)
    h = ocf.OpenCF(k=prob.k, lam=prob.lam, precision="bf16_gram", cpu_caps=cpu, gpu_caps=gpu)
    h.set_V(prob.V.contiguous())
    U, st, _ = h.complete_rows_checked(prob.row_ptr, prob.col, prob.val, refine=True)
    _, best, sav = h.predict(U, gamma=0.1, want_T=False)
    torch.cuda.synchronize()
    hp, hc, hv = prob.row_ptr.cpu(), prob.col.cpu(), prob.val.cpu()   # pageable memory
    b_h, s_h, _, _ = h.complete_select_host(hp, hc, hv, check=2, gamma=0.1, chunk_rows=256)
    torch.cuda.synchronize()
    assert torch.equal(b_h, best.cpu()) and torch.equal(s_h, sav.cpu())
    # rows with an out-of-range setting index: the same BAD_INPUT status and the same
    # decisions as the device-memory calls, whichever chunk the row falls in
    cb = hc.clone()
    cb[int(hp[5])] = -3
    cb[int(hp[2000])] = prob.n + 7
    cbd = cb.to(DEV)
    Ub, stb, _ = h.complete_rows_checked(prob.row_ptr, cbd, prob.val, refine=True)
    _, bb, sb = h.predict(Ub, gamma=0.1, want_T=False)
    torch.cuda.synchronize()
    assert int(stb[5]) == ocf.ROW_BAD_INPUT and int(stb[2000]) == ocf.ROW_BAD_INPUT
    st_h = torch.empty(m, dtype=torch.int32)
    b_h, s_h, _, _ = h.complete_select_host(hp, cb, hv, check=2, gamma=0.1, status=st_h,
                                            chunk_rows=512)
    torch.cuda.synchronize()
    assert torch.equal(st_h, stb.cpu())
    assert torch.equal(b_h, bb.cpu()) and torch.equal(s_h, sb.cpu())
    # an empty batch does nothing
    e = torch.zeros(1, dtype=torch.int64)
    b0, _, _, _ = h.complete_select_host(e, hc[:0], hv[:0])
    assert b0.numel() == 0
    # a row_ptr that does not end at nnz is refused before anything is queued
    bad = hp.clone()
    bad[-1] -= 1
    with pytest.raises(ocf.OpenCFError) as ei:
        h.complete_select_host(bad, hc, hv)
    assert ei.value.code == ocf.INVALID_ARG
    # a decreasing chunk boundary is refused as well
    bad = hp.clone()
    bad[256] = bad[512] + 1
    with pytest.raises(ocf.OpenCFError) as ei:
        h.complete_select_host(bad, hc, hv, chunk_rows=256)
    assert ei.value.code == ocf.INVALID_ARG
    # the FP64 handle has no host path
    h64 = ocf.OpenCF(k=8, lam=0.1, precision="fp64", cpu_caps=cpu, gpu_caps=gpu)
    h64.set_V(torch.randn(prob.n, 8, dtype=torch.float64, device=DEV))
    with pytest.raises(ocf.OpenCFError) as ei:
        h64.complete_select_host(hp, hc, hv, check=0)
    assert ei.value.code == ocf.UNSUPPORTED
