"""The rank-32 row solver's work split: each warp solves a contiguous range of
row pairs and then claims the remaining pairs one at a time from a counter of
the handle.  Every row must be solved exactly once whatever the batch size
(fewer pairs than warps, the boundary where the contiguous ranges start, many
pairs per warp), and a row's result must not depend on which warp solved it:
the same rows solved as a smaller batch give the same bits."""
import pytest
import torch

import synth

from gpu_util import DEV

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2508_07605_b300 as ocf  # noqa: E402


@pytest.mark.parametrize("m", [1, 2, 3, 4735, 4737, 5415, 6001, 20001, 120001])
def test_every_row_solved_once_and_independent_of_the_split(m):
    prob = synth.make_large_foldin(seed=31, m=m, device=DEV)
    cpu, gpu = synth.cap_grid(prob.n_cpu, prob.n_gpu)
    h = ocf.OpenCF(k=prob.k, lam=prob.lam, precision="bf16_gram", cpu_caps=cpu, gpu_caps=gpu)
    h.set_V(prob.V.contiguous())
    nan = float("nan")
    U = torch.full((m, prob.k), nan, device=DEV)
    st = torch.full((m,), -7, dtype=torch.int32, device=DEV)
    res = torch.full((m,), nan, device=DEV)
    h.complete_rows_checked(prob.row_ptr, prob.col, prob.val, refine=True, U=U, st=st, resid=res)
    torch.cuda.synchronize()
    assert torch.isfinite(U).all() and torch.isfinite(res).all()
    assert (st != -7).all()
    # the first rows again, as a batch of their own (another split of the work)
    q = max(1, m // 3)
    e = int(prob.row_ptr[q])
    Uq = torch.full((q, prob.k), nan, device=DEV)
    stq = torch.full((q,), -7, dtype=torch.int32, device=DEV)
    resq = torch.full((q,), nan, device=DEV)
    h.complete_rows_checked(prob.row_ptr[:q + 1].contiguous(), prob.col[:e].contiguous(),
                            prob.val[:e].contiguous(), refine=True, U=Uq, st=stq, resid=resq)
    torch.cuda.synchronize()
    assert torch.equal(Uq, U[:q]) and torch.equal(stq, st[:q]) and torch.equal(resq, res[:q])
    # and the plain fold-in (the same split) leaves no row unsolved either
    Up, stp = h.complete_rows(prob.row_ptr, prob.col, prob.val)
    torch.cuda.synchronize()
    assert torch.isfinite(Up).all() and (stp == ocf.ROW_OK).all()
