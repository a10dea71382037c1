"""The tensor-core pipelines' watchdog, tested without a fault: with the wait
bound set to 0 polls every mbarrier wait gives up at once (as if the phase it
waits for never completed), so each kernel takes its timeout path: it sets
the device flag, stops issuing, drains the copies it already issued, frees its
tensor memory and returns.  The host reads the flag through check() (TIMEOUT,
then cleared), the outputs are what the header promises for that kernel, and
with the default bound restored the same handle gives the results of a run
that never timed out, bit for bit (the context stayed usable)."""
import numpy as np
import pytest
import torch

import synth

from gpu_util import DEV, csr_dev, dev, host

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2508_07605_b300 as ocf  # noqa: E402

K = 32


def _timeout_reported(h):
    with pytest.raises(ocf.OpenCFError) as ei:
        h.check()
    assert ei.value.code == ocf.TIMEOUT
    h.check()   # cleared


def test_reconstruction_timeout_is_reported_and_recovers():
    prob = synth.make_large_foldin(seed=12, m=5000, device=DEV)
    cpu, gpu = synth.cap_grid(prob.n_cpu, prob.n_gpu)
    h = ocf.OpenCF(k=prob.k, lam=prob.lam, precision="bf16_gram", cpu_caps=cpu, gpu_caps=gpu)
    h.set_V(prob.V.contiguous())
    U, _ = h.complete_rows(prob.row_ptr, prob.col, prob.val)
    T0, b0, s0 = h.predict(U, gamma=0.05)
    torch.cuda.synchronize()
    h.check()
    h.set_wait_limit(0)
    h.predict(U, gamma=0.05)
    _timeout_reported(h)
    # the host pipeline's reconstruction launches report it the same way
    hp, hc, hv = prob.row_ptr.cpu(), prob.col.cpu(), prob.val.cpu()
    h.complete_select_host(hp, hc, hv, check=0, gamma=0.05, chunk_rows=1024)
    _timeout_reported(h)
    h.set_wait_limit(-1)
    T1, b1, s1 = h.predict(U, gamma=0.05)
    bh, sh, _, _ = h.complete_select_host(hp, hc, hv, check=0, gamma=0.05, chunk_rows=1024)
    torch.cuda.synchronize()
    h.check()
    assert torch.equal(T1, T0) and torch.equal(b1, b0) and torch.equal(s1, s0)
    assert torch.equal(bh, b0.cpu()) and torch.equal(sh, s0.cpu())
    with pytest.raises(ocf.OpenCFError) as ei:
        h.set_wait_limit(-2)
    assert ei.value.code == ocf.INVALID_ARG


def _mlp_problem(seed, m):
    rng = np.random.default_rng(seed)
    cpu, gpu = synth.cap_grid(8, 8)
    n = 64
    counts = rng.integers(0, 25, m)
    counts[:2] = [0, 24]
    ptr = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    col = np.concatenate([np.sort(rng.choice(n, c, replace=False)) for c in counts]).astype(
        np.int32)
    val = rng.uniform(0.05, 1.0, ptr[-1])
    V = (rng.standard_normal((n, K)) / 4).astype(np.float32)
    flat = np.concatenate([np.asarray(p, np.float32).reshape(-1)
                           for p in synth.mlp_init(rng, (48, 256, 256, K))])
    return csr_dev(ptr, col, val, torch.float32), V, flat, cpu, gpu, rng


def _mlp_handle(V, flat, cpu, gpu):
    h = ocf.OpenCF(k=K, lam=0.05, cpu_caps=cpu, gpu_caps=gpu, mlp_fallback_threshold=1e30)
    h.set_V(dev(V, torch.float32))
    h.mlp_set_params(dev(flat, torch.float32))
    return h


def test_learned_inference_timeout_falls_back_to_als():
    csr, V, flat, cpu, gpu, _ = _mlp_problem(3, 700)
    h = _mlp_handle(V, flat, cpu, gpu)
    U0, st0 = h.mlp_infer(*csr)
    Uf, stf = h.complete_rows(*csr)
    torch.cuda.synchronize()
    h.check()
    h.set_wait_limit(0)
    U1, st1 = h.mlp_infer(*csr)
    torch.cuda.synchronize()
    _timeout_reported(h)
    # every tile gave up: every row is the fold-in's, flagged as a fallback
    assert torch.equal(U1, Uf)
    stf = host(stf)
    assert np.array_equal(host(st1), np.where(stf == 0, ocf.ROW_FALLBACK_USED, stf))
    h.set_wait_limit(-1)
    U2, st2 = h.mlp_infer(*csr)
    torch.cuda.synchronize()
    h.check()
    assert torch.equal(U2, U0) and torch.equal(st2, st0)


@pytest.mark.parametrize("B", [512, 128 * 90])   # cluster-pair kernel; one CTA per tile
def test_learned_training_timeout_changes_nothing(B):
    csr, V, flat, cpu, gpu, rng = _mlp_problem(4, B)
    tgt = dev(rng.standard_normal((B, K)) / 8, torch.float32)
    ha = _mlp_handle(V, flat, cpu, gpu)
    hb = _mlp_handle(V, flat, cpu, gpu)
    ha.mlp_train_step(*csr, tgt, lr=1e-3)
    p1 = ha.mlp_get_params()
    torch.cuda.synchronize()
    ha.set_wait_limit(0)
    loss = torch.zeros(1, dtype=torch.float64, device=DEV)
    ha.mlp_train_step(*csr, tgt, lr=1e-3, loss=loss)
    torch.cuda.synchronize()
    assert torch.isnan(loss).all()
    assert torch.equal(ha.mlp_get_params(), p1)   # the step changed nothing
    _timeout_reported(ha)
    ha.set_wait_limit(-1)
    ha.mlp_train_step(*csr, tgt, lr=1e-3)
    # the same two steps on a handle that never timed out
    hb.mlp_train_step(*csr, tgt, lr=1e-3)
    hb.mlp_train_step(*csr, tgt, lr=1e-3)
    torch.cuda.synchronize()
    ha.check()
    assert torch.equal(ha.mlp_get_params(), hb.mlp_get_params())


def test_ncf_completion_timeout_is_reported_and_recovers():
    m, ncpu, ngpu = 300, 8, 16
    n = ncpu * ngpu
    rng = np.random.default_rng(6)
    net, Ea, Es = synth.ncf_init(rng, m, n, emb_scale=0.5, out_scale=0.3)
    net = net + 0.05 * rng.standard_normal(net.shape)
    cpu, gpu = synth.cap_grid(ncpu, ngpu)
    h = ocf.NCF(m, cpu, gpu, batch=256)
    h.set_params(dev(net, torch.float32), dev(Ea, torch.float32), dev(Es, torch.float32))
    T0, _, _ = h.predict(gamma=0.05)
    torch.cuda.synchronize()
    h.check()
    h.set_wait_limit(0)
    T1, _, _ = h.predict(gamma=0.05, select=False)
    torch.cuda.synchronize()
    with pytest.raises(ocf.OpenCFError) as ei:
        h.check()
    assert ei.value.code == ocf.TIMEOUT
    h.check()
    assert torch.isnan(T1).all()   # tiles that could not be computed are NaN
    h.set_wait_limit(-1)
    T2, _, _ = h.predict(gamma=0.05)
    torch.cuda.synchronize()
    h.check()
    assert torch.equal(T2, T0)
    h.close()
