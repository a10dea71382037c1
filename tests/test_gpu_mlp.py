"""Learned warm start: MLP 48 -> 256 -> 256 -> 32 (SELU) on BF16 tensor cores
with FP32 accumulation, trained by the library's own forward/backward/Adam
kernels, with the ALS fold-in as fallback.

Against the FP64 oracle fed the same FP32 inputs:
  * loss and gradients (per-tensor relative Frobenius error <= 2e-2, the BF16
    rounding of features, weights and activations: unit roundoff 2^-8 per
    operand, accumulated over three layers);
  * forward output per row (same bound) on random-init weights; with a
    trained network on 2^20 rows, each row's predicted runtimes within
    2e-3 of the last contraction's magnitude (see the test);
  * the Adam update given the kernel's own gradient (FP32 vs FP64, 1e-6);
  * the fallback: rows whose observed-entry RMSE is above the threshold carry
    the fold-in's factor bit for bit;
and a training run that shows what the network gains over the fold-in from
the same 16 observations."""
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
TOL_BF16 = 2e-2
SIZES = (48, 256, 256, K)


def _flat(params):
    return np.concatenate([np.asarray(p, np.float32).reshape(-1) for p in params])


def _split(flat):
    out, o = [], 0
    for a, b in zip(SIZES[:-1], SIZES[1:]):
        out.append(flat[o:o + a * b].reshape(a, b)); o += a * b
        out.append(flat[o:o + b]); o += b
    assert o == flat.size
    return out


def _small(seed, m=200, n_cpu=8, n_gpu=8):
    """Ragged rows: one empty, one with exactly 16 observations, one with more
    than 16 (only the first 16 enter the features), the rest 0..24."""
    rng = np.random.default_rng(seed)
    n = n_cpu * n_gpu
    counts = rng.integers(0, 25, m)
    counts[:3] = [0, 16, 24][:min(3, m)]
    ptr = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    col = np.concatenate([np.sort(rng.choice(n, c, replace=False)) for c in counts]).astype(
        np.int32)
    val = rng.uniform(0.05, 1.0, ptr[-1]).astype(np.float32).astype(np.float64)
    V = (rng.standard_normal((n, K)) / 4).astype(np.float32).astype(np.float64)
    cpu, gpu = synth.cap_grid(n_cpu, n_gpu)
    params = [np.asarray(p, np.float32).astype(np.float64)
              for p in synth.mlp_init(rng, SIZES)]
    return ptr, col, val, V, cpu, gpu, params


def _handle(V, cpu, gpu, params, thr=1e30, precision="fp32"):
    h = ocf.OpenCF(k=K, lam=0.05, cpu_caps=cpu, gpu_caps=gpu, mlp_fallback_threshold=thr,
                   precision=precision)
    h.set_V(dev(V, torch.float32))
    h.mlp_set_params(dev(_flat(params), torch.float32))
    return h


def _rel(a, b):
    return np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-30)


@pytest.mark.parametrize("seed", [0, 1])
def test_mlp_loss_and_gradients_match_oracle(orc, seed):
    ptr, col, val, V, cpu, gpu, params = _small(seed)
    m = len(ptr) - 1
    rng = np.random.default_rng(100 + seed)
    Yt = (rng.standard_normal((m, K)) / 2).astype(np.float32).astype(np.float64)
    h = _handle(V, cpu, gpu, params)
    loss = torch.zeros(1, dtype=torch.float64, device=DEV)
    g = h.mlp_train_step(*csr_dev(ptr, col, val, torch.float32), dev(Yt, torch.float32),
                         loss=loss, grads=True)
    torch.cuda.synchronize()
    X = orc.mlp_features(ptr, col, val, cpu, gpu)
    L, gref = orc.mlp_loss_grad(X, params, Yt, V.T @ V)
    assert abs(float(host(loss)[0]) - L) <= TOL_BF16 * abs(L)
    gg = _split(host(g).astype(np.float64))
    for name, a, b in zip(("W1", "b1", "W2", "b2", "W3", "b3"), gg, gref):
        assert _rel(a, b) <= TOL_BF16, (name, _rel(a, b))
    # parameters untouched by a gradient-only call
    assert np.array_equal(host(h.mlp_get_params()), _flat(params))


@pytest.mark.parametrize("m", [1, 74 * 128, 75 * 128 + 5, 148 * 128 + 300])
def test_mlp_gradients_over_tiles_match_oracle(orc, m):
    """The fused training step at one row; at 74 tiles (the largest batch the
    cluster-pair kernel takes: one pair of CTAs per tile); at 75 tiles (the
    one-CTA-per-tile kernel); and with more tiles than SMs (CTAs add a second
    tile into their partial sums).  The gradient is bit-reproducible from
    call to call."""
    ptr, col, val, V, cpu, gpu, params = _small(20 + m % 5, m=m)
    rng = np.random.default_rng(200 + m)
    Yt = (rng.standard_normal((m, K)) / 2).astype(np.float32).astype(np.float64)
    h = _handle(V, cpu, gpu, params)
    csr = csr_dev(ptr, col, val, torch.float32)
    loss = torch.zeros(1, dtype=torch.float64, device=DEV)
    g1 = h.mlp_train_step(*csr, dev(Yt, torch.float32), loss=loss, grads=True)
    g2 = h.mlp_train_step(*csr, dev(Yt, torch.float32), grads=True)
    torch.cuda.synchronize()
    assert torch.equal(g1, g2)
    X = orc.mlp_features(ptr, col, val, cpu, gpu)
    L, gref = orc.mlp_loss_grad(X, params, Yt, V.T @ V)
    assert abs(float(host(loss)[0]) - L) <= TOL_BF16 * abs(L)
    for name, a, b in zip(("W1", "b1", "W2", "b2", "W3", "b3"), _split(host(g1).astype(np.float64)),
                          gref):
        assert _rel(a, b) <= TOL_BF16, (name, _rel(a, b))


def test_mlp_gradient_follows_V(orc):
    """The loss matrix G = V^T V is kept between steps while V is unchanged;
    a new V (set_V) gives the gradient of the new loss."""
    ptr, col, val, V, cpu, gpu, params = _small(30, m=300)
    m = len(ptr) - 1
    Yt = (np.random.default_rng(31).standard_normal((m, K)) / 2).astype(np.float32).astype(np.float64)
    h = _handle(V, cpu, gpu, params)
    csr = csr_dev(ptr, col, val, torch.float32)
    X = orc.mlp_features(ptr, col, val, cpu, gpu)
    V2 = (np.random.default_rng(32).standard_normal(V.shape) / 2).astype(np.float32).astype(np.float64)
    for Vk in (V, V2):
        h.set_V(dev(Vk, torch.float32))
        loss = torch.zeros(1, dtype=torch.float64, device=DEV)
        g = h.mlp_train_step(*csr, dev(Yt, torch.float32), loss=loss, grads=True)
        torch.cuda.synchronize()
        L, gref = orc.mlp_loss_grad(X, params, Yt, Vk.T @ Vk)
        assert abs(float(host(loss)[0]) - L) <= TOL_BF16 * abs(L)
        for name, a, b in zip(("W1", "b1", "W2", "b2", "W3", "b3"),
                              _split(host(g).astype(np.float64)), gref):
            assert _rel(a, b) <= TOL_BF16, (name, _rel(a, b))


def test_mlp_forward_and_residual_match_oracle(orc):
    ptr, col, val, V, cpu, gpu, params = _small(2, m=333)
    h = _handle(V, cpu, gpu, params)
    U, st, rr = h.mlp_infer(*csr_dev(ptr, col, val, torch.float32), row_rmse=True)
    torch.cuda.synchronize()
    X = orc.mlp_features(ptr, col, val, cpu, gpu)
    _, _, Y = orc.mlp_forward(X, params)
    Ug = host(U).astype(np.float64)
    err = np.linalg.norm(Ug - Y, axis=1) / np.maximum(np.linalg.norm(Y, axis=1), 1e-30)
    assert err.max() <= TOL_BF16, err.max()
    assert (host(st) == 0).all()
    rref = orc.row_rmse(ptr, col, val, Ug, V)
    assert np.allclose(host(rr), rref, rtol=1e-4, atol=1e-6)


@pytest.mark.parametrize("m", [1, 128, 129, 148 * 128 * 2 + 77])
def test_mlp_forward_tiles_match_oracle(orc, m):
    """The fused tensor-core forward pass over 128-row tiles: one row, one
    full tile, a ragged second tile, and more tiles than SMs (each CTA loops
    over two or three tiles, the last one ragged)."""
    ptr, col, val, V, cpu, gpu, params = _small(10 + m % 7, m=m)
    h = _handle(V, cpu, gpu, params)
    U, st = h.mlp_infer(*csr_dev(ptr, col, val, torch.float32))
    torch.cuda.synchronize()
    X = orc.mlp_features(ptr, col, val, cpu, gpu)
    _, _, Y = orc.mlp_forward(X, params)
    Ug = host(U).astype(np.float64)
    assert np.isfinite(Ug).all()
    err = np.linalg.norm(Ug - Y, axis=1) / np.maximum(np.linalg.norm(Y, axis=1), 1e-30)
    assert err.max() <= TOL_BF16, (err.max(), int(err.argmax()))
    assert (host(st) == 0).all()


@pytest.mark.parametrize("precision", ["fp32", "bf16_gram"])
def test_mlp_fallback_everywhere_is_the_foldin(precision):
    """Threshold below every residual: each row is re-solved by the fold-in
    and must equal open_cf_complete_rows bit for bit."""
    ptr, col, val, V, cpu, gpu, params = _small(3, m=300)
    h = _handle(V, cpu, gpu, params, thr=-1.0, precision=precision)
    csr = csr_dev(ptr, col, val, torch.float32)
    U, st = h.mlp_infer(*csr)
    Uf, stf = h.complete_rows(*csr)
    torch.cuda.synchronize()
    assert torch.equal(U, Uf)
    stf = host(stf)
    assert np.array_equal(host(st), np.where(stf == 0, 3, stf))
    assert (stf[np.diff(ptr) == 0] == 2).all()


def test_mlp_fallback_by_threshold():
    ptr, col, val, V, cpu, gpu, params = _small(4, m=400)
    csr = csr_dev(ptr, col, val, torch.float32)
    h = _handle(V, cpu, gpu, params)
    Um, _, rr = h.mlp_infer(*csr, row_rmse=True)
    Uf, stf = h.complete_rows(*csr)
    rr = host(rr)
    thr = float(np.median(rr[rr > 0]))
    h2 = _handle(V, cpu, gpu, params, thr=thr)
    U2, st2 = h2.mlp_infer(*csr)
    torch.cuda.synchronize()
    keep = rr <= np.float32(thr)
    assert 0 < keep.sum() < len(keep)
    assert torch.equal(U2[torch.as_tensor(keep, device=DEV)], Um[torch.as_tensor(keep, device=DEV)])
    fb = torch.as_tensor(~keep, device=DEV)
    assert torch.equal(U2[fb], Uf[fb])
    st2 = host(st2)
    assert (st2[keep] == 0).all()
    stf = host(stf)
    assert np.array_equal(st2[~keep], np.where(stf[~keep] == 0, 3, stf[~keep]))


def test_mlp_adam_steps_match_oracle(orc):
    ptr, col, val, V, cpu, gpu, params = _small(5)
    m = len(ptr) - 1
    Yt = np.random.default_rng(7).standard_normal((m, K)) / 2
    h = _handle(V, cpu, gpu, params)
    csr = csr_dev(ptr, col, val, torch.float32)
    T = dev(Yt, torch.float32)
    theta = _flat(params).astype(np.float64)
    m1 = np.zeros_like(theta); m2 = np.zeros_like(theta)
    for t, lr in ((1, 1e-3), (2, 3e-4)):
        g = host(h.mlp_train_step(*csr, T, grads=True)).astype(np.float64)
        h.mlp_train_step(*csr, T, lr=lr)
        got = host(h.mlp_get_params()).astype(np.float64)
        orc.adam(theta, g, m1, m2, t, lr=lr)
        assert np.allclose(got, theta, rtol=1e-6, atol=1e-7), np.abs(got - theta).max()
        theta = got.copy()


def test_mlp_rejects_bad_use():
    ptr, col, val, V, cpu, gpu, params = _small(6, m=8)
    csr = csr_dev(ptr, col, val, torch.float32)
    h = ocf.OpenCF(k=K, lam=0.05, cpu_caps=cpu, gpu_caps=gpu)
    h.set_V(dev(V, torch.float32))
    with pytest.raises(ocf.OpenCFError):      # no parameters yet
        h.mlp_infer(*csr)
    h16 = ocf.OpenCF(k=16, lam=0.05, cpu_caps=cpu, gpu_caps=gpu)
    with pytest.raises(ocf.OpenCFError):      # the network's output is k = 32
        h16.mlp_set_params(dev(_flat(params), torch.float32))
    hn = ocf.OpenCF(k=K, lam=0.05)
    hn.set_V(dev(V, torch.float32))
    hn.mlp_set_params(dev(_flat(params), torch.float32))
    with pytest.raises(ocf.OpenCFError):      # features need the cap grid
        hn.mlp_infer(*csr)
    hf = ocf.OpenCF(k=K, lam=0.05, cpu_caps=cpu, gpu_caps=gpu, precision="fp64")
    hf.set_V(dev(V, torch.float64))
    with pytest.raises(ocf.OpenCFError):      # FP32 modes only
        hf.mlp_set_params(dev(_flat(params), torch.float32))


def _heldout_rmse(U, V, clean):
    return float(torch.sqrt(torch.mean((U @ V.T - clean) ** 2)).item())


def test_mlp_training_gain():
    """Train on factors the plain method produces (fold-in of each training
    app's full 4096-setting profile; a pool of 2^20 apps), then complete new
    apps from 16 observed settings: the network's rows are closer to the
    noiseless truth than the fold-in's from the same 16 entries, and so are
    the rows of the network with the 0.02 residual fallback.

    V here is the synthetic model's own setting factors, which carry nothing
    about how applications are distributed; the fold-in's isotropic ridge
    prior cannot use the applications' shared traits, the network learns
    them from the training pool.  (With V fitted offline on apps of the same
    population the fold-in already exploits that structure; the learned
    workload of the benchmark reports that case.)"""
    wl = synth.make_learned(seed=0, device=DEV)
    cpu, gpu = synth.cap_grid(wl.n_cpu, wl.n_gpu)
    V = wl.V_fixed()
    h = ocf.OpenCF(k=K, lam=wl.lam, cpu_caps=cpu, gpu_caps=gpu, mlp_fallback_threshold=1e30)
    h.set_V(V)
    rng = np.random.default_rng(0)
    h.mlp_set_params(dev(_flat(synth.mlp_init(rng, SIZES, out_scale=0.1)), torch.float32))
    noisy_t, clean_t, obs_t = wl.draw_apps(4096)
    csr_t = synth.observed_csr(noisy_t, obs_t)
    Uf, _ = h.complete_rows(*csr_t)
    rmse_fold = _heldout_rmse(Uf, V, clean_t)
    pool = 1 << 20
    pc, pv, pt = synth.learned_pool(wl, h, pool)
    B, steps, lr0 = 4096, 20000, 2e-3
    rp = torch.arange(0, (B + 1) * wl.s_obs, wl.s_obs, dtype=torch.int64, device=DEV)
    cb = torch.empty(B, wl.s_obs, dtype=torch.int32, device=DEV)
    vb = torch.empty(B, wl.s_obs, dtype=torch.float32, device=DEV)
    tb = torch.empty(B, K, dtype=torch.float32, device=DEV)
    gen = torch.Generator(device=DEV)
    gen.manual_seed(1)
    pos = pool
    for step in range(steps):
        if pos + B > pool:
            perm = torch.randperm(pool, generator=gen, device=DEV)
            pos = 0
        idx = perm[pos:pos + B]
        pos += B
        torch.index_select(pc, 0, idx, out=cb)
        torch.index_select(pv, 0, idx, out=vb)
        torch.index_select(pt, 0, idx, out=tb)
        h.mlp_train_step(rp, cb.view(-1), vb.view(-1), tb,
                         lr=lr0 * 0.5 * (1 + np.cos(np.pi * step / steps)))
    Um, _ = h.mlp_infer(*csr_t)
    rmse_mlp = _heldout_rmse(Um, V, clean_t)
    h2 = ocf.OpenCF(k=K, lam=wl.lam, cpu_caps=cpu, gpu_caps=gpu, mlp_fallback_threshold=0.02)
    h2.set_V(V)
    h2.mlp_set_params(h.mlp_get_params())
    Ufb, st = h2.mlp_infer(*csr_t)
    rmse_fb = _heldout_rmse(Ufb, V, clean_t)
    torch.cuda.synchronize()
    print(f"held-out RMSE: fold-in {rmse_fold:.5f}, trained {rmse_mlp:.5f}, "
          f"trained+fallback {rmse_fb:.5f} ({float((st == 3).float().mean()):.3f} fell back)")
    assert rmse_mlp < 0.85 * rmse_fold
    assert rmse_fb < rmse_fold


def _selu(z):
    return np.where(z > 0, 1.0507009873554805 * z,
                    1.0507009873554805 * 1.6732632423543772 * np.expm1(np.minimum(z, 0.0)))


def test_trained_network_full_size_rows(orc):
    """The fused tensor-core forward pass with a TRAINED network on 2^20 rows
    (8192 tiles of 128 rows: each persistent CTA walks 55 or 56 tiles),
    against the FP64 oracle's forward pass with the same weights, on 4096
    rows sampled over every tile position.

    Bound per row: the BF16 operands (features, weights, hidden activations;
    unit roundoff 2^-8) give an error in u that scales with the magnitude of
    the last contraction, S_c = sum_d |W3[d, c] h2_d| + |b3_c|, not with |u|:
    a row whose predicted runtimes nearly cancel (small |u V^T|) has a large
    relative error with no defect anywhere.  So the test bounds
        |(u_gpu - u_or) V^T| <= 2e-3 * |S |V|^T|   (about u/2 of BF16)
    for every sampled row, and keeps the plain relative error's median within
    the BF16 gate of 2e-2.  A wrong tile, row or weight gives errors of the
    size of |u V^T| itself, about 1e-2 of |S |V|^T| here."""
    import math
    wl = synth.make_learned(seed=0, device=DEV)
    cpu, gpu = synth.cap_grid(wl.n_cpu, wl.n_gpu)
    S = wl.s_obs
    h = ocf.OpenCF(k=K, lam=wl.lam, sweeps=15, cpu_caps=cpu, gpu_caps=gpu,
                   mlp_fallback_threshold=1e30)
    off, _, _ = wl.draw_apps(4096)
    g0 = torch.Generator(device=DEV)
    g0.manual_seed(7)
    h.set_V(torch.randn(wl.n, K, generator=g0, device=DEV) / math.sqrt(K))
    h.fit_offline(off)
    V = h.get_V()
    del off
    pool = 1 << 19
    pc, pv, pt = synth.learned_pool(wl, h, pool)
    rng = np.random.default_rng(0)
    h.mlp_set_params(dev(_flat(synth.mlp_init(rng, SIZES, out_scale=0.1)), torch.float32))
    B, steps, lr0 = 4096, 8000, 2e-3
    rp = torch.arange(0, (B + 1) * S, S, dtype=torch.int64, device=DEV)
    gen = torch.Generator(device=DEV)
    gen.manual_seed(1)
    pos = pool
    for step in range(steps):
        if pos + B > pool:
            perm = torch.randperm(pool, generator=gen, device=DEV)
            pos = 0
        idx = perm[pos:pos + B]
        pos += B
        h.mlp_train_step(rp, pc[idx].reshape(-1).contiguous(), pv[idx].reshape(-1).contiguous(),
                         pt[idx].contiguous(), lr=lr0 * 0.5 * (1 + math.cos(math.pi * step / steps)))
    del pc, pv, pt
    M = 1 << 20
    cols, vals = [], []
    for _ in range(M // 65536):
        noisy, _, obs = wl.draw_apps(65536)
        cols.append(obs.reshape(-1))
        vals.append(torch.gather(noisy, 1, obs.to(torch.int64)).reshape(-1))
        del noisy
    col, val = torch.cat(cols).contiguous(), torch.cat(vals).contiguous()
    row_ptr = torch.arange(0, (M + 1) * S, S, dtype=torch.int64, device=DEV)
    U, st = h.mlp_infer(row_ptr, col, val)
    torch.cuda.synchronize()
    assert bool((st == 0).all())
    # 4096 sampled rows: every position in a tile, tiles from first to last
    sample = np.unique(np.concatenate([np.random.default_rng(3).choice(M, 3968, replace=False),
                                       np.arange(M - 128, M)]))
    si = torch.as_tensor(sample, device=DEV)
    sc = host(col.view(M, S)[si]).reshape(-1)
    sv = host(val.view(M, S)[si]).astype(np.float64).reshape(-1)
    sp = np.arange(0, (len(sample) + 1) * S, S, dtype=np.int64)
    params = _split(host(h.mlp_get_params()).astype(np.float64))
    X = orc.mlp_features(sp, sc, sv, cpu, gpu)
    _, Z2, Y = orc.mlp_forward(X, params)
    mag = np.abs(_selu(Z2)) @ np.abs(params[4]) + np.abs(params[5])
    Vd = host(V).astype(np.float64)
    Ug = host(U[si]).astype(np.float64)
    err = np.linalg.norm((Ug - Y) @ Vd.T, axis=1)
    scale = np.linalg.norm(mag @ np.abs(Vd).T, axis=1)
    rel = err / np.linalg.norm(Y @ Vd.T, axis=1)
    worst = int(np.argmax(err / scale))
    print(f"trained network, 2^20 rows: |dT|/|S|V|^T| max {float((err / scale).max()):.2e}, "
          f"relative error median {float(np.median(rel)):.2e}, max {float(rel.max()):.2e}")
    assert (err <= 2e-3 * scale).all(), (int(sample[worst]), float(err[worst] / scale[worst]))
    assert float(np.median(rel)) <= TOL_BF16
