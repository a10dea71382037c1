"""Checkpoint and resume (open_cf_save / open_cf_load): a fit, the learned
path's training and the streaming refit stopped half-way, saved, restored into
a fresh handle and continued must give the same bits as the uninterrupted
run; a damaged or mismatched checkpoint is refused and leaves the handle as it
was."""
import math

import numpy as np
import pytest
import torch

import synth

from gpu_util import DEV, csr_dev, dev, rounded

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2508_07605_b300 as ocf  # noqa: E402


@pytest.mark.parametrize("precision,k", [("fp32", 16), ("bf16_gram", 32), ("fp64", 8)])
def test_fit_resumed_from_checkpoint_is_bit_identical(precision, k):
    prob = synth.make_sparse_problem(seed=21, m=700, n_cpu=4, n_gpu=64, rank=k, density=0.08,
                                     k=k, lam=0.05, n_heldout=8)
    dt = torch.float64 if precision == "fp64" else torch.float32
    csr = csr_dev(prob.row_ptr, prob.col, rounded(prob.val, dt), dt)
    V0 = dev(rounded(prob.V0, dt), dt)
    cpu, gpu = synth.cap_grid(prob.n_cpu, prob.n_gpu)

    def handle(sweeps):
        return ocf.OpenCF(k=k, lam=prob.lam, sweeps=sweeps, precision=precision, cpu_caps=cpu,
                          gpu_caps=gpu)

    ha = handle(6)
    ha.set_V(V0.clone())
    ha.fit_csr(*csr, prob.n)
    ck = ha.save()
    hb = handle(9)
    hb.load(ck)
    Ub = hb.fit_csr(*csr, prob.n)
    Vb = hb.get_V()
    hc = handle(15)
    hc.set_V(V0.clone())
    Uc = hc.fit_csr(*csr, prob.n)
    Vc = hc.get_V()
    torch.cuda.synchronize()
    assert torch.equal(Ub, Uc) and torch.equal(Vb, Vc)
    # and the resumed handle's predictions and decisions are the uninterrupted one's
    Tb, bb, sb = hb.predict(Ub, gamma=0.05)
    Tc, bc, sc = hc.predict(Uc, gamma=0.05)
    torch.cuda.synchronize()
    assert torch.equal(Tb, Tc) and torch.equal(bb, bc) and torch.equal(sb, sc)


def test_learned_training_resumed_is_bit_identical():
    rng = np.random.default_rng(5)
    cpu, gpu = synth.cap_grid(8, 8)
    n, K, B = 64, 32, 512
    V = dev(rounded(rng.standard_normal((n, K)) / 4, torch.float32), torch.float32)
    flat = np.concatenate([np.asarray(p, np.float32).reshape(-1)
                           for p in synth.mlp_init(rng, (48, 256, 256, 32), out_scale=0.1)])
    counts = np.full(B, 16)
    ptr = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    col = np.concatenate([np.sort(rng.choice(n, 16, replace=False)) for _ in range(B)]).astype(np.int32)
    val = rng.uniform(0.1, 1.0, ptr[-1])
    csr = csr_dev(ptr, col, rounded(val, torch.float32), torch.float32)
    tgt = dev(rng.standard_normal((B, K)) / 8, torch.float32)

    def handle():
        h = ocf.OpenCF(k=K, lam=0.05, cpu_caps=cpu, gpu_caps=gpu)
        h.set_V(V)
        return h

    def train(h, steps, s0):
        for s in range(s0, s0 + steps):
            h.mlp_train_step(*csr, tgt, lr=1e-3 * 0.5 * (1 + math.cos(math.pi * s / 40)))

    ha = handle()
    ha.mlp_set_params(dev(flat, torch.float32))
    train(ha, 20, 0)
    ck = ha.save()
    hb = handle()
    hb.load(ck)
    train(hb, 20, 20)
    hc = handle()
    hc.mlp_set_params(dev(flat, torch.float32))
    train(hc, 40, 0)
    torch.cuda.synchronize()
    assert torch.equal(hb.mlp_get_params(), hc.mlp_get_params())
    assert torch.equal(hb.mlp_infer(*csr)[0], hc.mlp_infer(*csr)[0])


def test_streaming_refit_resumed_is_bit_identical():
    sp = synth.make_sparse_problem(seed=7, m=1200, n_cpu=2, n_gpu=32, rank=8, density=0.2, k=8,
                                   lam=0.05, n_heldout=8)
    vals = rounded(sp.val, torch.float32)
    rng = np.random.default_rng(8)
    U0 = dev(rounded(rng.standard_normal((300, 8)) / 3, torch.float32), torch.float32)

    def part(a, b):
        e0, e1 = int(sp.row_ptr[a]), int(sp.row_ptr[b])
        return csr_dev(sp.row_ptr[a:b + 1] - e0, sp.col[e0:e1], vals[e0:e1], torch.float32)

    def begin():
        h = ocf.OpenCF(k=8, lam=0.05)
        h.set_V(torch.zeros(sp.n, 8, device=DEV))
        h.stream_begin(*part(0, 300), U0)
        return h

    ha = begin()
    ha.stream_ingest(*part(300, 600))
    ck = ha.save()
    hb = ocf.OpenCF(k=8, lam=0.05)
    hb.load(ck)
    Ub = [hb.stream_ingest(*part(a, b))[0] for a, b in ((600, 900), (900, 1200))]
    hc = begin()
    hc.stream_ingest(*part(300, 600))
    Uc = [hc.stream_ingest(*part(a, b))[0] for a, b in ((600, 900), (900, 1200))]
    torch.cuda.synchronize()
    assert all(torch.equal(x, y) for x, y in zip(Ub, Uc))
    assert torch.equal(hb.get_V(), hc.get_V())


def test_damaged_or_mismatched_checkpoint_is_refused():
    cpu, gpu = synth.cap_grid(4, 8)
    rng = np.random.default_rng(9)
    V = dev(rounded(rng.standard_normal((32, 16)), torch.float32), torch.float32)
    ha = ocf.OpenCF(k=16, lam=0.05, cpu_caps=cpu, gpu_caps=gpu)
    ha.set_V(V)
    ck = bytearray(ha.save())
    hb = ocf.OpenCF(k=16, lam=0.05, cpu_caps=cpu, gpu_caps=gpu)
    V2 = dev(rounded(rng.standard_normal((32, 16)), torch.float32), torch.float32)
    hb.set_V(V2)
    for bad in (bytes(ck[:-1]), bytes(ck[:100]), b"x" * len(ck)):
        with pytest.raises(ocf.OpenCFError) as ei:
            hb.load(bad)
        assert ei.value.code == ocf.INVALID_ARG
    flipped = bytearray(ck)
    flipped[200] ^= 1          # a bit of V: the checksum catches it
    with pytest.raises(ocf.OpenCFError):
        hb.load(bytes(flipped))
    torch.cuda.synchronize()
    assert torch.equal(hb.get_V(), V2)     # unchanged
    for other in (ocf.OpenCF(k=8, lam=0.05, cpu_caps=cpu, gpu_caps=gpu),
                  ocf.OpenCF(k=16, lam=0.1, cpu_caps=cpu, gpu_caps=gpu),
                  ocf.OpenCF(k=16, lam=0.05, precision="bf16_gram", cpu_caps=cpu, gpu_caps=gpu),
                  ocf.OpenCF(k=16, lam=0.05, cpu_caps=cpu[::-1].copy(), gpu_caps=gpu)):
        with pytest.raises(ocf.OpenCFError) as ei:
            other.load(bytes(ck))
        assert ei.value.code == ocf.INVALID_ARG
    hb.load(bytes(ck))
    torch.cuda.synchronize()
    assert torch.equal(hb.get_V(), V)
